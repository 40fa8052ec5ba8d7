"""Pins of the oracle's TV indicator and refinement rule (Sec. 3, Eqs. 6-8)."""
import numpy as np
import pytest
import torch

from oracle.aderdg import Mesh, Solver
from oracle import indicator as ind
from oracle import physics as ph
from paper_1905_05524_gb300 import inputs


@pytest.mark.parametrize("N", [1, 3, 5])
def test_tv_of_linear_field_exact(N):
    """f = a x + b y: TV = |a| + |b| on every cell (reading T1)."""
    s = Solver(Mesh(4, 3, Lx=2.0, Ly=6.0), ph.cfd_params(N, source="none"))
    a, b = -0.7, 1.9
    f = a * s.X + b * s.Y
    tv = ind.total_variation(s, f)
    assert torch.allclose(tv, torch.full_like(tv, abs(a) + abs(b)), rtol=1e-12)


def test_tv_of_constant_is_zero_and_flags_keep():
    s = Solver(Mesh(5, 5), ph.cfd_params(3, source="none"))
    u = torch.zeros(25, 4, 4, 4, dtype=torch.float64)
    u[:, 0], u[:, 3] = 1.0, 2.5
    tv, fl, mean, std = ind.tv_indicator(s, u, "rho", 2.5, -0.5)
    assert tv.abs().max().item() < 1e-14
    assert std == 0.0 and bool((fl == 0).all())  # reading F1


def test_mean_std_match_numpy():
    x = torch.from_numpy(inputs.uniform_values(1000, seed=7, lo=0.0, hi=3.0) ** 3)
    mean, std = ind.mean_std(x)
    assert abs(mean - np.mean(x.numpy())) <= 1e-14 * abs(mean)
    assert abs(std - np.std(x.numpy())) <= 1e-13 * std


@pytest.mark.parametrize("T_r,T_c", [(2.5, -0.5), (1.5, -0.5), (1.0, 0.0)])
def test_flags_obey_cantelli_bound(T_r, T_c):
    """One-sided Chebyshev (Cantelli): the refine fraction is at most
    1/(1 + T_r^2); the coarsen fraction at most 1/(1 + T_c^2) for T_c < 0."""
    for seed in range(5):
        x = inputs.uniform_values(4000, seed=seed, lo=0.0, hi=1.0)
        tv = torch.from_numpy(np.exp(8.0 * x))  # heavy right tail
        mean, std = ind.mean_std(tv)
        fl = ind.flags(tv, mean, std, T_r, T_c)
        frac_r = (fl == 1).double().mean().item()
        assert frac_r <= 1.0 / (1.0 + T_r ** 2) + 1e-12
        if T_c < 0:
            assert (fl == -1).double().mean().item() <= 1.0 / (1.0 + T_c ** 2) + 1e-12
        assert not bool((fl == 1).all()) and not bool((fl == -1).all())


def test_flag_rule_inequalities():
    """Eq. 7 exactly: >= for refine, < for coarsen, refine wins."""
    tv = torch.tensor([0.0, 1.0, 2.0, 3.0, 4.0], dtype=torch.float64)
    mean, std = ind.mean_std(tv)      # 2, sqrt(2)
    fl = ind.flags(tv, mean, std, 2.0 / std, -1.0 / std)   # thresholds 4 and 1
    assert fl.tolist() == [-1, 0, 0, 0, 1]
