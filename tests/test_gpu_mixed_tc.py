"""The tensor-core precisions: the mixed-precision predictor with its
derivative contractions as warp MMAs with FP32 accumulation --
ADG_PREC_MIXED_TF32 (TF32 operands split in two, three products) and
ADG_PREC_MIXED_BF16X3 (BF16 operands split in three, six products) --
against the FP64 oracle at the mixed path's stated bound (relative L2 of
theta' <= 1e-6), on ragged walled bubble meshes with momentum everywhere,
without gravity, at full size over 400 steps, and the cases they refuse."""
import pytest
import torch

from paper_1905_05524_gb300 import _lib as L
from paper_1905_05524_gb300 import inputs
from paper_1905_05524_gb300.solver import Mesh, atmosphere_config, steady_manufactured_config
from tests.oracle_bridge import oracle_for, cosine_field, steady_field
from tests.test_gpu_mixed import rel_theta_err, THETA_TOL

pytestmark = pytest.mark.gpu

TC = [L.ADG_PREC_MIXED_TF32, L.ADG_PREC_MIXED_BF16X3]


@pytest.mark.parametrize("prec", TC)
@pytest.mark.parametrize("degree", [3, 5, 7])
def test_tc_bubble_vs_oracle(degree, prec):
    """Ragged 7x6 walled bubble with seeded momentum (every flux term active),
    10 steps at CFL 0.25: theta' within 1e-6, rho within 1e-9."""
    cfg = atmosphere_config(degree=degree, nx=7, ny=6, precision=prec)
    o = oracle_for(cfg)
    u0 = cosine_field(o)
    u0[:, 1:3] += torch.from_numpy(inputs.perturbation(tuple(u0[:, 1:3].shape), seed=degree, scale=0.5)) * u0[:, 0:1]
    dt = o.stable_dt(u0, 0.25)
    m = Mesh(cfg)
    m.set_state(u0.cuda().contiguous())
    m.step(dt, 10)
    uo = u0
    for _ in range(10):
        uo = o.step(uo, dt)
    a = m.get_state().cpu()
    err = rel_theta_err(o, a, uo)
    assert err <= THETA_TOL, (degree, err)
    rho = (torch.linalg.vector_norm(a[:, 0] - uo[:, 0]) / torch.linalg.vector_norm(uo[:, 0])).item()
    assert rho <= 1e-9, (degree, rho)
    for v in (1, 2):
        r = (torch.linalg.vector_norm(a[:, v] - uo[:, v]) / torch.linalg.vector_norm(uo[:, v])).item()
        assert r <= 1e-6, (degree, v, r)


@pytest.mark.parametrize("prec", TC)
@pytest.mark.parametrize("degree", [3, 5, 7])
def test_tc_manufactured_vs_oracle(degree, prec):
    """Periodic steady manufactured field without gravity: the tensor-core
    contractions carry the full state; FP32-level error per variable."""
    cfg = steady_manufactured_config(degree=degree, nx=5, ny=4, precision=prec)
    o = oracle_for(cfg)
    u0 = steady_field(o, cfg)
    dt = o.stable_dt(u0, 0.25)
    m = Mesh(cfg)
    m.set_state(u0.cuda().contiguous())
    m.step(dt, 5)
    uo = u0
    for _ in range(5):
        uo = o.step(uo, dt)
    a = m.get_state().cpu()
    for v in range(4):
        r = (torch.linalg.vector_norm(a[:, v] - uo[:, v]) / torch.linalg.vector_norm(uo[:, v])).item()
        assert r <= 1e-6, (degree, v, r)


@pytest.mark.parametrize("tc", TC)
def test_tc_warm_bubble_81x81_400_steps_vs_fp64(tc):
    """The bench workload (degree 5, 81x81, CFL 0.45), 400 steps of the
    tensor-core form against the FP64 GPU path: theta' within 1e-6."""
    res = {}
    for prec in (L.ADG_PREC_FP64, tc):
        m = Mesh(atmosphere_config(degree=5, nx=81, ny=81, precision=prec))
        m.init_scenario(L.ADG_SCEN_COSINE, A=0.5, a=250.0, xc=500.0, zc=350.0)
        if prec == L.ADG_PREC_FP64:
            dt = m.stable_dt(0.45)
        for _ in range(8):
            m.step(dt, 50)
            m.check_finite()
        res[prec] = m.get_state().cpu()
    o = oracle_for(atmosphere_config(degree=5, nx=81, ny=81))
    err = rel_theta_err(o, res[tc], res[L.ADG_PREC_FP64])
    print(f"tensor-core form, 400 steps: theta' relative L2 vs FP64 = {err:.3e}")
    assert err <= THETA_TOL, err


@pytest.mark.parametrize("prec", TC)
def test_tc_refuses_unsupported(prec):
    for cfg in (atmosphere_config(degree=4, nx=3, ny=3, precision=prec),
                atmosphere_config(degree=5, nx=3, ny=3, precision=prec)):
        if cfg.degree == 5:
            cfg.max_levels = 1
        with pytest.raises(L.AdgError) as e:
            Mesh(cfg)
        assert e.value.code == L.ADG_EUNSUPPORTED
