"""Rounding floors of the parity tolerances (test infrastructure).

Momentum over a hydrostatic background.  Both the CUDA path and the oracle
form the pressure perturbation p' = p - pbar(z) by cancelling values of the
size of the background pressure (p0 = 1e5 Pa): each forms p' with a rounding
error of a few units in the last place of p0, independently.  That error
enters the momentum update through the face lifting, whose largest
coefficient is (|phi_i(0)| + |phi_i(1)|) / (h w_i) <= 2 / (h w_min), once per
step and direction.  Over `steps` steps of size dt the momentum of the two
implementations may therefore differ per node by about

    steps * dt * (2 / w_min) * 2 ulp(p0) / h,

and by sqrt(nodes) times that in the L2 norm over all nodes -- independent
of the momentum itself, which starts at zero in a fluid at rest.  Measured
differences of the FP64 path against the oracle sit 8-40x below this floor
(warm bubble 81x81, 2 steps: 4.8e-12 against 4.3e-11); a planted momentum
error of ten times the floor fails the tests.  Without gravity the
background is zero and the floor is zero.
"""
import math

import numpy as np


def momentum_floor(cfg, dt, steps, nodes):
    """L2 floor of the momentum difference of two correct FP64 implementations."""
    if not cfg.gravity:
        return 0.0
    _, w = np.polynomial.legendre.leggauss(cfg.degree + 1)
    w_min = 0.5 * w.min()
    h = min(cfg.Lx / cfg.nx, cfg.Ly / cfg.ny)
    ulp = np.spacing(cfg.p0)
    return steps * dt * (2.0 / w_min) * 2.0 * ulp / h * math.sqrt(nodes)
