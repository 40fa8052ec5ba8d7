"""The paper's time-dependent manufactured solution (Sec. 4.1, Eq. 8) on the
GPU FP64 path against the oracle, whose source is built by automatic
differentiation of the field and of its flux function (an independent
derivation from the device's dual-number evaluation).

Tolerance: relative L2 per variable <= 1e-11, as for the other FP64 parity
tests."""
import math

import pytest
import torch

from paper_1905_05524_gb300 import _lib as L
from paper_1905_05524_gb300 import inputs
from paper_1905_05524_gb300.solver import Mesh, paper_manufactured_config
from tests.oracle_bridge import oracle_for, paper_field

pytestmark = pytest.mark.gpu

TOL = 1e-11


def assert_close(a, b, tol=TOL, what=""):
    a = a.detach().cpu().double()
    b = b.detach().cpu().double()
    for v in range(4):
        d = torch.linalg.vector_norm(a[:, v] - b[:, v]).item()
        nb = torch.linalg.vector_norm(b[:, v]).item()
        assert d <= tol * nb, f"{what} var {v}: rel={d / nb:.3e}"


def test_init_paper_field_matches_oracle():
    cfg = paper_manufactured_config(degree=4, nx=7, ny=6)
    m = Mesh(cfg)
    m.init_scenario(L.ADG_SCEN_PAPER)
    assert_close(m.get_state(), paper_field(oracle_for(cfg), 0.0), 1e-14, "init")


@pytest.mark.parametrize("degree", [1, 2, 3, 4, 5, 6, 7])
def test_paper_source_steps_match_oracle(degree):
    """Three steps from t0 = 0.3 (the source's time dependence enters every
    time node) on a perturbed Eq. 8 field; ragged 7x5 periodic grid."""
    cfg = paper_manufactured_config(degree=degree, nx=7, ny=5)
    o = oracle_for(cfg)
    t0 = 0.3
    u0 = paper_field(o, t0)
    u0 = u0 + torch.from_numpy(inputs.perturbation(tuple(u0.shape), seed=degree, scale=1e-3))
    dt = 0.5 * o.stable_dt(u0, 0.5)
    m = Mesh(cfg)
    m.set_state(u0.to("cuda").contiguous())
    m.time = t0
    uo, t = u0.clone(), t0
    for _ in range(3):
        uo = o.step(uo, dt, t)
        t += dt
    m.step(dt, 3)
    torch.cuda.synchronize()
    assert abs(m.time - t) < 1e-15
    assert_close(m.get_state(), uo, TOL, f"N={degree}")


def test_paper_source_time_offset_matters():
    """The same state stepped from two start times differs by the source's
    time dependence: the device does not evaluate the source at t = 0."""
    cfg = paper_manufactured_config(degree=3, nx=6, ny=6)
    o = oracle_for(cfg)
    u0 = paper_field(o, 0.0)
    dt = o.stable_dt(u0, 0.5)
    outs = []
    for t0 in (0.0, 0.25):
        m = Mesh(cfg)
        m.set_state(u0.to("cuda").contiguous())
        m.time = t0
        m.step(dt, 1)
        outs.append(m.get_state().cpu())
        uo = o.step(u0.clone(), dt, t0)
        assert_close(outs[-1], uo, TOL, f"t0={t0}")
    assert (outs[0] - outs[1]).abs().max().item() > 1e-4


def test_paper_manufactured_convergence_gpu():
    """Degree 3 on 8^2, 16^2, 32^2 cells to t = 0.1: the error against the
    exact Eq. 8 field falls at high order (the oracle reaches >= 2.5 on the
    first pair, the same bound as its own pin)."""
    errs = []
    for nc in (8, 16, 32):
        cfg = paper_manufactured_config(degree=3, nx=nc, ny=nc)
        o = oracle_for(cfg)
        m = Mesh(cfg)
        m.init_scenario(L.ADG_SCEN_PAPER)
        T = 0.1
        dt0 = m.stable_dt(0.5)
        steps = math.ceil(T / dt0)
        m.step(T / steps, steps)
        torch.cuda.synchronize()
        errs.append(o.l2_error(m.get_state().cpu(), paper_field(o, T))[0].item())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert orders[0] >= 2.5 and orders[1] >= 2.5, (errs, orders)


def test_paper_source_rejected_where_unsupported():
    for kw in (dict(precision=L.ADG_PREC_MIXED), dict(max_levels=2), dict(gravity=1)):
        cfg = paper_manufactured_config(degree=2, nx=4, ny=4)
        for k, v in kw.items():
            setattr(cfg, k, v)
        with pytest.raises(RuntimeError):
            Mesh(cfg)
    m = Mesh(paper_manufactured_config(degree=2, nx=4, ny=4))
    u = m.get_state()
    lam = torch.ones_like(u)
    with pytest.raises(RuntimeError):
        from paper_1905_05524_gb300.adjoint import step_adjoint
        step_adjoint(m, 0.01, u, lam)
