"""Nodal Gauss-Legendre basis on the reference interval [0, 1] (oracle).

The paper evaluates all cell integrals "with Gaussian quadrature over the
collocated quadrature points" (Sec. 3, after Eq. 6) and uses the ADER-DG
scheme of Dumbser et al. (Sec. 1, Sec. 3), whose space-time predictor is a
nodal Lagrange polynomial in space and in time on the same Gauss-Legendre
nodes.  This module builds, from first principles:

* Gauss-Legendre nodes and weights (Newton iteration on the Legendre
  three-term recurrence), mapped to [0, 1] so that sum(w) = 1;
* Lagrange basis values phi_j(x) by the product formula;
* the derivative matrix D[i, j] = phi_j'(xi_i) (barycentric form);
* the time-stiffness matrix K1[l, k] = phi_l(1) phi_k(1) - w_k D[k, l]
  (integration by parts in time of int_0^1 phi_l dq/dtau, with the
  upwind value u^n entering through F0[l] = phi_l(0)).

Pins (tests/test_oracle_basis.py): closed-form nodes for n = 2, 3, sum of
weights, exactness of int_0^1 x^k for k <= 2n-1 and inexactness at 2n,
D applied to monomials, K1 @ 1 = F0.
"""
import math

import torch

from . import DTYPE


def gauss_legendre(n):
    """n Gauss-Legendre nodes xi (ascending) and weights w on [0, 1]."""
    xs, ws = [], []
    for i in range(n):
        # Tricomi-style initial guess for the i-th root of P_n on [-1, 1]
        x = math.cos(math.pi * (i + 0.75) / (n + 0.5))
        for _ in range(100):
            p0, p1 = 1.0, x  # P_0, P_1
            for m in range(2, n + 1):
                p0, p1 = p1, ((2 * m - 1) * x * p1 - (m - 1) * p0) / m
            if n == 1:
                pn, pnm1 = x, 1.0
            else:
                pn, pnm1 = p1, p0
            dpn = n * (x * pn - pnm1) / (x * x - 1.0)
            dx = pn / dpn
            x -= dx
            if abs(dx) < 1e-16:
                break
        # final derivative at the converged root
        p0, p1 = 1.0, x
        for m in range(2, n + 1):
            p0, p1 = p1, ((2 * m - 1) * x * p1 - (m - 1) * p0) / m
        pn, pnm1 = (x, 1.0) if n == 1 else (p1, p0)
        dpn = n * (x * pn - pnm1) / (x * x - 1.0)
        w = 2.0 / ((1.0 - x * x) * dpn * dpn)
        xs.append(0.5 * (x + 1.0))
        ws.append(0.5 * w)
    order = sorted(range(n), key=lambda k: xs[k])
    xi = torch.tensor([xs[k] for k in order], dtype=DTYPE)
    w = torch.tensor([ws[k] for k in order], dtype=DTYPE)
    return xi, w


def lagrange_values(xi, x):
    """L[a, j] = phi_j(x[a]) for the Lagrange basis on nodes xi."""
    x = torch.as_tensor(x, dtype=DTYPE).reshape(-1)
    n = xi.numel()
    L = torch.ones(x.numel(), n, dtype=DTYPE)
    for j in range(n):
        for m in range(n):
            if m != j:
                L[:, j] = L[:, j] * (x - xi[m]) / (xi[j] - xi[m])
    return L


def derivative_matrix(xi):
    """D[i, j] = phi_j'(xi_i), barycentric formula (Berrut & Trefethen 2004)."""
    n = xi.numel()
    lam = torch.ones(n, dtype=DTYPE)
    for j in range(n):
        for m in range(n):
            if m != j:
                lam[j] = lam[j] / (xi[j] - xi[m])
    D = torch.zeros(n, n, dtype=DTYPE)
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = (lam[j] / lam[i]) / (xi[i] - xi[j])
        D[i, i] = -sum(D[i, j] for j in range(n) if j != i)
    return D


class Basis:
    """All one-dimensional operators of a degree-N nodal GL basis on [0, 1]."""

    def __init__(self, N):
        self.N = N
        self.n = n = N + 1
        self.xi, self.w = gauss_legendre(n)
        self.D = derivative_matrix(self.xi)
        self.phi0 = lagrange_values(self.xi, [0.0])[0]  # phi_j(0)
        self.phi1 = lagrange_values(self.xi, [1.0])[0]  # phi_j(1)
        # time stiffness (Dumbser et al. 2008): K1 q = F0 u^n + dt * W R(q)
        self.K1 = torch.outer(self.phi1, self.phi1) - (self.w[:, None] * self.D).T
        self.F0 = self.phi0.clone()
        self.K1inv = torch.linalg.inv(self.K1)
