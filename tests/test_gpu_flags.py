"""Refinement flags at the thresholds (Eq. 7): the device decides
TV >= mean + T_r sigma and TV < mean + T_c sigma exactly as the oracle does,
including TV values one unit in the last place either side of a threshold,
thresholds at or below zero, NaN, and the sigma = 0 case (reading F1)."""
import ctypes
import math

import numpy as np
import pytest
import torch

from paper_1905_05524_gb300 import _lib as L
from paper_1905_05524_gb300.solver import Mesh, steady_manufactured_config
from oracle import indicator as oind

pytestmark = pytest.mark.gpu


def device_flags(m, tv, count, mean, m2, T_r, T_c):
    tv_d = tv.to("cuda").contiguous()
    fl = torch.empty(tv.numel(), dtype=torch.int8, device="cuda")
    L.check(m._lib.adg_tv_flags(m.h, ctypes.c_void_p(tv_d.data_ptr()), float(count), float(mean), float(m2),
                                float(T_r), float(T_c), ctypes.c_void_p(fl.data_ptr()), None))
    return fl.cpu()


def border_values(thr, rng, k):
    vals = [thr, np.nextafter(thr, np.inf), np.nextafter(thr, -np.inf), 0.0]
    vals += list(np.abs(rng.normal(thr, abs(thr) + 1.0, k)))
    return [v for v in vals if v >= 0.0]


@pytest.mark.parametrize("mean,sigma,T_r,T_c", [(1.0, 0.5, 1.5, -0.5), (0.1, 0.3, 1.7, -0.3),
                                                 (2.5e-3, 7.1e-4, 2.5, -0.5), (1.0, 0.2, 1.5, -7.0)])
def test_flags_at_thresholds_match_oracle(mean, sigma, T_r, T_c):
    m = Mesh(steady_manufactured_config(degree=1, nx=16, ny=16))
    cells = m.leaves
    count = 1000.0
    m2 = count * sigma * sigma
    sig = math.sqrt(m2 / count)  # what both sides use
    rng = np.random.default_rng(7)
    vals = border_values(mean + T_r * sig, rng, 40) + border_values(mean + T_c * sig, rng, 40)
    vals += list(np.abs(rng.normal(mean, sigma, cells)))
    tv = torch.tensor(vals[:cells], dtype=torch.float64)
    got = device_flags(m, tv, count, mean, m2, T_r, T_c)
    want = oind.flags(tv, mean, sig, T_r, T_c)
    assert torch.equal(got, want), (got - want).nonzero()
    assert (got == 1).any() and (got == 0).any()


def test_flags_flat_and_nan():
    m = Mesh(steady_manufactured_config(degree=1, nx=4, ny=4))
    tv = torch.full((16,), 0.5, dtype=torch.float64)
    assert (device_flags(m, tv, 16.0, 0.5, 0.0, 1.5, -0.5) == 0).all()  # sigma = 0: keep all
    tv[3] = float("nan")
    tv[5] = 10.0
    got = device_flags(m, tv, 16.0, 0.5, 16.0 * 0.01, 1.5, -0.5)
    assert got[3] == 0 and got[5] == 1 and got[0] == 0
