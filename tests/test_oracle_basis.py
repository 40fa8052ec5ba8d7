"""Pins of the oracle's nodal Gauss-Legendre basis against closed forms,
exactness properties and a library routine (numpy's leggauss)."""
import math

import numpy as np
import pytest
import torch

from oracle.basis import Basis, gauss_legendre, lagrange_values, derivative_matrix


def test_closed_form_nodes_n2_n3():
    xi, w = gauss_legendre(2)
    assert torch.allclose(xi, torch.tensor([0.5 - math.sqrt(3) / 6, 0.5 + math.sqrt(3) / 6], dtype=torch.float64), atol=1e-15)
    assert torch.allclose(w, torch.tensor([0.5, 0.5], dtype=torch.float64), atol=1e-15)
    xi, w = gauss_legendre(3)
    r = math.sqrt(15) / 10
    assert torch.allclose(xi, torch.tensor([0.5 - r, 0.5, 0.5 + r], dtype=torch.float64), atol=1e-15)
    assert torch.allclose(w, torch.tensor([5 / 18, 8 / 18, 5 / 18], dtype=torch.float64), atol=1e-15)


@pytest.mark.parametrize("n", range(1, 9))
def test_nodes_match_numpy_leggauss(n):
    x, w = np.polynomial.legendre.leggauss(n)
    xi, ww = gauss_legendre(n)
    assert np.allclose(xi.numpy(), 0.5 * (x + 1), atol=1e-14)
    assert np.allclose(ww.numpy(), 0.5 * w, atol=1e-14)


@pytest.mark.parametrize("n", range(1, 9))
def test_quadrature_exact_to_degree_2n_minus_1(n):
    xi, w = gauss_legendre(n)
    assert abs(float(w.sum()) - 1.0) < 1e-14
    for k in range(2 * n):
        assert abs(float((w * xi ** k).sum()) - 1.0 / (k + 1)) < 1e-14
    # not exact at degree 2n
    assert abs(float((w * xi ** (2 * n)).sum()) - 1.0 / (2 * n + 1)) > 1e-12


@pytest.mark.parametrize("N", range(1, 8))
def test_derivative_matrix_exact_on_polynomials(N):
    b = Basis(N)
    for k in range(N + 1):
        f = b.xi ** k
        df = k * b.xi ** (k - 1) if k > 0 else torch.zeros_like(b.xi)
        assert torch.allclose(b.D @ f, df, atol=1e-11 * max(1, k * N))
    assert torch.allclose(b.D @ torch.ones_like(b.xi), torch.zeros_like(b.xi), atol=1e-12)


@pytest.mark.parametrize("N", range(1, 8))
def test_lagrange_and_time_matrices(N):
    b = Basis(N)
    n = N + 1
    L = lagrange_values(b.xi, b.xi)
    assert torch.allclose(L, torch.eye(n, dtype=torch.float64), atol=1e-13)
    x = torch.linspace(0, 1, 17, dtype=torch.float64)
    assert torch.allclose(lagrange_values(b.xi, x).sum(1), torch.ones(17, dtype=torch.float64), atol=1e-12)
    # K1 1 = F0 (integration by parts of d/dtau of a constant)
    assert torch.allclose(b.K1 @ torch.ones(n, dtype=torch.float64), b.F0, atol=1e-12)
    assert torch.allclose(b.K1 @ b.K1inv, torch.eye(n, dtype=torch.float64), atol=1e-11)
    # K1 applied to the nodal values of tau^m equals int phi_l dtau^m/dtau + phi_l(0) 0^m
    for m in range(1, n):
        lhs = b.K1 @ (b.xi ** m)
        # int_0^1 phi_l m tau^{m-1} dtau by quadrature (exact: degree N + m - 1 <= 2n-1)
        rhs = b.w * m * b.xi ** (m - 1)
        assert torch.allclose(lhs, rhs, atol=1e-12)
