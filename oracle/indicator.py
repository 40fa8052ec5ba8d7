"""Total-variation refinement indicator (oracle), Sec. 3 of the paper.

* Eq. 6 (TV): TV[f] = || int_C |grad f| dx ||_1, integral by Gaussian
  quadrature over the collocated nodes.  Reading T1: the component-wise
  absolute physical gradient is integrated with the quadrature of the
  reference cell (weights summing to 1) and the L1 norm sums the
  components, TV = sum_ij w_i w_j (|df/dx| + |df/dy|).  Integrating over the
  physical cell instead (a factor hx hy) makes a child's TV 1/9 of its
  parent's for the same gradient, so refinement stops after one level --
  contrary to the three cell sizes of the paper's two-level runs (Sec. 4.2).
* mean and population standard deviation of TV over all (leaf) cells --
  here their plain two-pass definition, which Chan et al.'s parallel update
  (cited by the paper) reaches up to rounding.
* Eq. 7: refine if TV >= mu + T_r sigma, coarsen if TV < mu + T_c sigma,
  keep otherwise (refine wins if both hold).  Codes: +1 refine, -1 coarsen,
  0 keep.
* Eq. 8 (Chebyshev): not all cells can be flagged (reading F1: sigma = 0
  keeps every cell).

The indicator variable f is the potential temperature theta for the
stratified scenarios and the density for the CFD scenarios (reading).

Pins: tests/test_oracle_indicator.py (TV of a linear field is exact, TV of a
constant is zero, flags obey the Chebyshev/Cantelli bound, sigma = 0 flags
nothing).  The cell-size scaling of reading T1 is a recorded choice (parity
unpinned for that factor).
"""
import torch

from . import DTYPE
from . import physics as ph


def indicator_field(solver, u, var):
    """Nodal indicator values f[c, j, i]: 'theta' or 'rho'."""
    if var == "rho":
        return u[:, 0]
    if var == "theta":
        return ph.theta(u.unbind(1), solver.Y, solver.P)
    raise ValueError(var)


def total_variation(solver, f):
    """TV per cell of nodal data f[c, j, i]."""
    D, w = solver.b.D, solver.b.w
    hx, hy = solver.m.hx, solver.m.hy
    fx = torch.einsum("ip,cjp->cji", D, f) / hx
    fy = torch.einsum("jp,cpi->cji", D, f) / hy
    return torch.einsum("j,i,cji->c", w, w, fx.abs() + fy.abs())


def mean_std(tv):
    """Mean and population standard deviation (two-pass definition)."""
    n = tv.numel()
    mean = tv.sum() / n
    var = ((tv - mean) ** 2).sum() / n
    return float(mean), float(torch.sqrt(var))


def flags(tv, mean, std, T_r, T_c):
    """Eq. 7 refinement decision per cell.  Reading F1: with sigma = 0 (all
    cells share one TV, up to rounding: sigma <= 1e-12 |mu|) every cell is
    kept -- the literal rule would refine all of them, which the Chebyshev
    argument of Eq. 8 is meant to exclude."""
    out = torch.zeros(tv.shape, dtype=torch.int8)
    if std <= 1e-12 * abs(mean):
        return out
    refine = tv >= mean + T_r * std
    coarsen = tv < mean + T_c * std
    out[coarsen] = -1
    out[refine] = 1
    return out


def tv_indicator(solver, u, var, T_r, T_c):
    f = indicator_field(solver, u, var)
    tv = total_variation(solver, f)
    mean, std = mean_std(tv)
    return tv, flags(tv, mean, std, T_r, T_c), mean, std
