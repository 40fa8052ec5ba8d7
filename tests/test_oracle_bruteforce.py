"""Brute-force pin of the oracle's whole ADER-DG step (Sec. 3) on tiny
periodic meshes.

The oracle's step (``oracle.aderdg.Solver.step``) is compared with a second,
independent statement of the same discrete equations, assembled here as dense
global operators over every degree of freedom of the mesh:

* the one-dimensional basis comes from exact polynomial algebra (numpy's
  Gauss-Legendre rule, Lagrange polynomials as coefficient vectors, the time
  matrices K1 = phi(1) phi(1)^T - int phi' phi^T and M = int phi phi^T by exact
  integration of polynomial products) instead of the oracle's Newton
  iteration, product formula and barycentric derivative;
* gradients, face extrapolation, neighbour exchange, volume and lifting terms
  are explicit (cells * n^2)-sized matrices built entry by entry from the
  weak form, applied as matrix-vector products (the oracle contracts per cell
  with einsum);
* the space-time update solves K1 q = F0 u + dt M R with a linear solve per
  node instead of applying a stored inverse;
* the point-wise Navier-Stokes fluxes (Eqs. 1-7) are written in primitive
  variables (stress tensor tau = -sigma, grad T = grad p/(rho R) -
  p grad rho/(rho^2 R)), not in the oracle's arrangement.

Both must agree to rounding on 1x1, 2x2 and 3x3 periodic meshes at degrees 1
and 2, viscous, with and without gravity.  Planted mistakes in the oracle (a
transposed derivative, a halved Rusanov penalty, a flipped lifting sign, a
dropped heat flux) each fail the comparison.
"""
import math

import numpy as np
import numpy.polynomial.polynomial as npp
import pytest
import torch

from oracle.aderdg import Mesh, Solver
from oracle import physics as ph


# ------------------------------------------------------------------ basis
class PolyBasis:
    """Degree-N nodal basis on [0, 1] from exact polynomial algebra."""

    def __init__(self, N):
        n = N + 1
        x, w = np.polynomial.legendre.leggauss(n)
        self.xi = 0.5 * (x + 1.0)
        self.w = 0.5 * w
        self.n = n
        # Lagrange polynomials as coefficient vectors (ascending powers)
        self.L = []
        for j in range(n):
            others = [self.xi[m] for m in range(n) if m != j]
            c = npp.polyfromroots(others)
            self.L.append(c / npp.polyval(self.xi[j], c))
        dL = [npp.polyder(c) for c in self.L]
        self.D = np.array([[npp.polyval(self.xi[i], dL[j]) for j in range(n)] for i in range(n)])
        self.phi0 = np.array([npp.polyval(0.0, c) for c in self.L])
        self.phi1 = np.array([npp.polyval(1.0, c) for c in self.L])

        def integral01(c):
            ci = npp.polyint(c)
            return npp.polyval(1.0, ci) - npp.polyval(0.0, ci)

        # K1[l, k] = phi_l(1) phi_k(1) - int_0^1 phi_l'(t) phi_k(t) dt
        self.K1 = np.array([[self.phi1[l] * self.phi1[k] - integral01(npp.polymul(dL[l], self.L[k]))
                             for k in range(n)] for l in range(n)])
        # M[l, k] = int_0^1 phi_l phi_k dt (diagonal = w for Gauss-Legendre nodes)
        self.M = np.array([[integral01(npp.polymul(self.L[l], self.L[k])) for k in range(n)] for l in range(n)])


# --------------------------------------------------------- point-wise physics
def background(z, P):
    """Isentropic atmosphere of constant potential temperature theta0."""
    if not P.gravity:
        return np.zeros_like(z), np.zeros_like(z)
    cp = P.gamma * P.R / (P.gamma - 1.0)
    T = P.theta0 - P.g * z / cp
    p = P.p0 * (T / P.theta0) ** (cp / P.R)
    return p, p / (P.R * T)


def physics(Q, Qx, Qy, z, P):
    """F, G, S of the compressible Navier-Stokes system at points (arrays of
    shape [4, ...]), primitive-variable form."""
    g = P.g if P.gravity else 0.0
    rho, mx, my, E = Q
    u, v = mx / rho, my / rho
    p = (P.gamma - 1.0) * (E - 0.5 * rho * (u * u + v * v) - rho * g * z)
    pbar, rhobar = background(z, P)
    T = p / (rho * P.R)
    du = [(Qx[1] - u * Qx[0]) / rho, (Qy[1] - u * Qy[0]) / rho]   # d/dx, d/dy of u
    dv = [(Qx[2] - v * Qx[0]) / rho, (Qy[2] - v * Qy[0]) / rho]
    dp = []
    for a, dz in ((0, 0.0), (1, 1.0)):
        Qa = Qx if a == 0 else Qy
        dkin = 0.5 * (u * u + v * v) * Qa[0] + rho * (u * du[a] + v * dv[a])
        dp.append((P.gamma - 1.0) * (Qa[3] - dkin - g * z * Qa[0] - rho * g * dz))
    dT = [dp[a] / (rho * P.R) - p * (Qx if a == 0 else Qy)[0] / (rho * rho * P.R) for a in (0, 1)]
    div = du[0] + dv[1]
    txx = P.mu * (2.0 * du[0] - (2.0 / 3.0) * div)
    tyy = P.mu * (2.0 * dv[1] - (2.0 / 3.0) * div)
    txy = P.mu * (du[1] + dv[0])
    kappa = P.mu * P.gamma * P.R / (P.Pr * (P.gamma - 1.0))
    H = E + p
    F = np.stack([mx, mx * u + (p - pbar) - txx, my * u - txy, u * H - (u * txx + v * txy) - kappa * dT[0]])
    G = np.stack([my, mx * v - txy, my * v + (p - pbar) - tyy, v * H - (u * txy + v * tyy) - kappa * dT[1]])
    zero = np.zeros_like(rho)
    S = np.stack([zero, zero, -g * (rho - rhobar), zero])
    return F, G, S


def speed(Q, z, normal_x, h, P):
    """Rusanov speed |v.n| + c + 2 eta lambda_v of face states Q[4, ...]."""
    g = P.g if P.gravity else 0.0
    rho, mx, my, E = Q
    p = (P.gamma - 1.0) * (E - 0.5 * (mx * mx + my * my) / rho - rho * g * z)
    vn = np.abs((mx if normal_x else my) / rho)
    lam_v = max(4.0 / 3.0, P.gamma / P.Pr) * P.mu / rho
    eta = (2 * P.N + 1) / (h * math.sqrt(0.5 * math.pi))
    return vn + np.sqrt(P.gamma * p / rho) + 2.0 * eta * lam_v


# ------------------------------------------------------------ dense scheme
class DenseStep:
    """One ADER-DG step on a periodic nx x ny mesh as dense global operators.
    Global node index g(c, j, i) = (c n + j) n + i, c = iy nx + ix."""

    def __init__(self, nx, ny, Lx, Ly, P):
        self.P = P
        b = PolyBasis(P.N)
        self.b = b
        n = b.n
        C = nx * ny
        self.C, self.n = C, n
        hx, hy = Lx / nx, Ly / ny
        self.hx, self.hy = hx, hy
        G = C * n * n
        g = lambda c, j, i: (c * n + j) * n + i
        cell = lambda ix, iy: (iy % ny) * nx + (ix % nx)
        self.GX = np.zeros((G, G))
        self.GY = np.zeros((G, G))
        self.VX = np.zeros((G, G))
        self.VY = np.zeros((G, G))
        for c in range(C):
            for j in range(n):
                for i in range(n):
                    for p in range(n):
                        self.GX[g(c, j, i), g(c, j, p)] = b.D[i, p] / hx
                        self.GY[g(c, j, i), g(c, p, i)] = b.D[j, p] / hy
                        # weak volume term: int dphi/dx F over the cell / mass
                        self.VX[g(c, j, i), g(c, j, p)] = b.w[p] * b.D[p, i] / (b.w[i] * hx)
                        self.VY[g(c, j, i), g(c, p, i)] = b.w[p] * b.D[p, j] / (b.w[j] * hy)
        # face extrapolation (face index f(c, m) = c n + m) and lifting
        F = C * n
        self.XE, self.XW, self.YN, self.YS = (np.zeros((F, G)) for _ in range(4))
        self.LE, self.LW, self.LN, self.LS = (np.zeros((G, F)) for _ in range(4))
        for c in range(C):
            for m in range(n):
                for a in range(n):
                    self.XE[c * n + m, g(c, m, a)] = b.phi1[a]
                    self.XW[c * n + m, g(c, m, a)] = b.phi0[a]
                    self.YN[c * n + m, g(c, a, m)] = b.phi1[a]
                    self.YS[c * n + m, g(c, a, m)] = b.phi0[a]
                    self.LE[g(c, m, a), c * n + m] = b.phi1[a] / (hx * b.w[a])
                    self.LW[g(c, m, a), c * n + m] = b.phi0[a] / (hx * b.w[a])
                    self.LN[g(c, a, m), c * n + m] = b.phi1[a] / (hy * b.w[a])
                    self.LS[g(c, a, m), c * n + m] = b.phi0[a] / (hy * b.w[a])
        # neighbour permutations: (PE f)[c] = f[east(c)], (PWs f)[c] = f[west(c)], ...
        self.PE, self.PW, self.PN, self.PS = (np.zeros((F, F)) for _ in range(4))
        for iy in range(ny):
            for ix in range(nx):
                c = cell(ix, iy)
                for m in range(n):
                    self.PE[c * n + m, cell(ix + 1, iy) * n + m] = 1.0
                    self.PW[c * n + m, cell(ix - 1, iy) * n + m] = 1.0
                    self.PN[c * n + m, cell(ix, iy + 1) * n + m] = 1.0
                    self.PS[c * n + m, cell(ix, iy - 1) * n + m] = 1.0
        # heights of volume nodes and of the faces
        self.z = np.zeros(G)
        self.zx = np.zeros(F)      # x-faces: node heights
        self.zN = np.zeros(F)
        for iy in range(ny):
            for ix in range(nx):
                c = cell(ix, iy)
                for j in range(n):
                    self.zx[c * n + j] = (iy + b.xi[j]) * hy
                    for i in range(n):
                        self.z[g(c, j, i)] = (iy + b.xi[j]) * hy
                self.zN[c * n:(c + 1) * n] = (iy + 1) * hy

    def step(self, U, dt):
        """U[4, G] -> U[4, G] after one predictor + corrector step."""
        P, b, n = self.P, self.b, self.n
        # predictor: n Picard sweeps on q[k][4, G], then the final evaluation
        q = [U.copy() for _ in range(n)]
        rhs0 = np.einsum("l,vg->lvg", b.phi0, U)  # F0 u
        for sweep in range(n + 1):
            Fs, Gs, Ss, Qxs, Qys = [], [], [], [], []
            for k in range(n):
                Qx = np.stack([self.GX @ q[k][v] for v in range(4)])
                Qy = np.stack([self.GY @ q[k][v] for v in range(4)])
                Fk, Gk, Sk = physics(q[k], Qx, Qy, self.z, P)
                Fs.append(Fk), Gs.append(Gk), Ss.append(Sk), Qxs.append(Qx), Qys.append(Qy)
            if sweep == n:
                break
            R = np.stack([np.stack([-(self.GX @ Fs[k][v]) - self.GY @ Gs[k][v] + Ss[k][v] for v in range(4)])
                          for k in range(n)])                      # [k, v, G]
            rhs = rhs0 + dt * np.einsum("lk,kvg->lvg", b.M, R)
            sol = np.linalg.solve(b.K1, rhs.reshape(n, -1)).reshape(n, 4, -1)
            q = [sol[l] for l in range(n)]
        avg = lambda xs: sum(b.w[k] * xs[k] for k in range(n))
        qb, Fb, Gb, Sb = avg(q), avg(Fs), avg(Gs), avg(Ss)
        # faces: F* on the east face of every cell and G* on the north face
        qE = np.stack([self.XE @ qb[v] for v in range(4)])
        qWn = np.stack([self.PE @ (self.XW @ qb[v]) for v in range(4)])
        fE = np.stack([self.XE @ Fb[v] for v in range(4)])
        fWn = np.stack([self.PE @ (self.XW @ Fb[v]) for v in range(4)])
        s = np.maximum(speed(qE, self.zx, True, self.hx, P), speed(qWn, self.zx, True, self.hx, P))
        FE = 0.5 * (fE + fWn) - 0.5 * s * (qWn - qE)
        qN = np.stack([self.YN @ qb[v] for v in range(4)])
        qSn = np.stack([self.PN @ (self.YS @ qb[v]) for v in range(4)])
        gN = np.stack([self.YN @ Gb[v] for v in range(4)])
        gSn = np.stack([self.PN @ (self.YS @ Gb[v]) for v in range(4)])
        s = np.maximum(speed(qN, self.zN, False, self.hy, P), speed(qSn, self.zN, False, self.hy, P))
        GN = 0.5 * (gN + gSn) - 0.5 * s * (qSn - qN)
        out = np.empty_like(U)
        for v in range(4):
            FW = self.PW @ FE[v]
            GS = self.PS @ GN[v]
            du = (self.VX @ Fb[v] + self.VY @ Gb[v]
                  - (self.LE @ FE[v] - self.LW @ FW) - (self.LN @ GN[v] - self.LS @ GS) + Sb[v])
            out[v] = U[v] + dt * du
        return out


# ------------------------------------------------------------------ cases
def _state(nx, ny, P, L, seed):
    """Smooth-plus-noise state with positive density and pressure, nodal
    [cells, 4, n, n] (oracle layout)."""
    rng = np.random.default_rng(seed)
    n = P.N + 1
    C = nx * ny
    b = PolyBasis(P.N)
    ix = np.arange(C) % nx
    iy = np.arange(C) // nx
    x = (ix[:, None, None] + b.xi[None, None, :]) * (L / nx) + 0 * b.xi[None, :, None]
    y = (iy[:, None, None] + b.xi[None, :, None]) * (L / ny) + 0 * b.xi[None, None, :]
    if P.gravity:
        pbar, rhobar = background(y, P)
        rho = rhobar * (1.0 + 0.01 * rng.uniform(-1, 1, (C, n, n)))
        u = 2.0 * rng.uniform(-1, 1, (C, n, n))
        v = 2.0 * rng.uniform(-1, 1, (C, n, n))
        p = pbar * (1.0 + 0.001 * rng.uniform(-1, 1, (C, n, n)))
        E = p / (P.gamma - 1.0) + 0.5 * rho * (u * u + v * v) + rho * P.g * y
    else:
        rho = 1.0 + 0.2 * np.sin(2 * math.pi * (x + 2 * y) / L) + 0.05 * rng.uniform(-1, 1, (C, n, n))
        u = 0.3 + 0.1 * rng.uniform(-1, 1, (C, n, n))
        v = -0.2 + 0.1 * rng.uniform(-1, 1, (C, n, n))
        p = 1.0 + 0.1 * np.cos(2 * math.pi * x / L) + 0.05 * rng.uniform(-1, 1, (C, n, n))
        E = p / (P.gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return np.stack([rho, rho * u, rho * v, E], 1)


CASES = [(nc, N, grav) for nc in (1, 2, 3) for N in (1, 2) for grav in (False, True)]


def _params(N, grav):
    if grav:
        P = ph.atmosphere_params(N, mu=5.0)
    else:
        P = ph.cfd_params(N, mu=0.05, source="none")
    return P


def _compare(nc, N, grav, seed=7):
    P = _params(N, grav)
    L = 900.0 if grav else 3.0
    u = _state(nc, nc, P, L, seed)
    s = Solver(Mesh(nc, nc, Lx=L, Ly=L), P)
    ut = torch.from_numpy(u)
    dt = s.stable_dt(ut, 0.5)
    uo = s.step(ut, dt).numpy()
    d = DenseStep(nc, nc, L, L, P)
    n = N + 1
    U = u.transpose(1, 0, 2, 3).reshape(4, -1)          # [v, (c, j, i)]
    ub = d.step(U, dt).reshape(4, nc * nc, n, n).transpose(1, 0, 2, 3)
    return u, uo, ub, dt, L / nc


@pytest.mark.parametrize("nc,N,grav", CASES)
def test_step_equals_dense_assembly(nc, N, grav):
    """Oracle step = dense global assembly of the same discrete equations,
    to rounding: the state within 1e-14 of its magnitude per variable (plus,
    with gravity, the rounding of the 1e5 Pa background that p' = p - pbar
    carries through one lifting) and the increment u^{n+1} - u^n within 1e-12
    of its own magnitude (measured: 3e-14 at worst)."""
    u, uo, ub, dt, h = _compare(nc, N, grav)
    b = PolyBasis(N)
    P = _params(N, grav)
    # rounding of the background pressure (p' = p - pbar) carried through one
    # lifting into the momentum and energy updates
    floor = 4.0 * dt * np.finfo(float).eps * (P.p0 if grav else 0.0) / (h * b.w.min())
    for v in range(4):
        scale = np.abs(u[:, v]).max()
        assert np.abs(uo[:, v] - ub[:, v]).max() <= 1e-14 * scale + floor, v
        du_o, du_b = uo[:, v] - u[:, v], ub[:, v] - u[:, v]
        tol = 1e-12 * np.abs(du_b).max()
        assert np.abs(du_o - du_b).max() <= tol, (v, np.abs(du_o - du_b).max(), np.abs(du_b).max())


@pytest.mark.parametrize("mistake", ["transposed_D_y", "half_penalty", "lift_sign", "no_heat_flux"])
def test_planted_mistakes_fail(monkeypatch, mistake):
    """Each plausible slip in the oracle's scheme changes the step far beyond
    rounding, so the dense-assembly comparison would catch it."""
    import oracle.aderdg as ad
    if mistake == "transposed_D_y":
        orig = ad.Solver.grad

        def grad(self, q):
            qx, _ = orig(self, q)
            qy = torch.einsum("pj,...pi->...ji", self.b.D, q) / self.m.hy
            return qx, qy
        monkeypatch.setattr(ad.Solver, "grad", grad)
    elif mistake == "half_penalty":
        def riemann(self, qL, fL, qR, fR, zL, zR, nrm, h):
            sL = ph.wave_speed(qL.unbind(1), zL, nrm[0], nrm[1], h, self.P)
            sR = ph.wave_speed(qR.unbind(1), zR, nrm[0], nrm[1], h, self.P)
            return 0.5 * (fL + fR) - 0.25 * torch.maximum(sL, sR)[:, None] * (qR - qL)
        monkeypatch.setattr(ad.Solver, "riemann", riemann)
    elif mistake == "lift_sign":
        orig_ff = ad.Solver.face_fluxes

        def face_fluxes(self, tr, halo=None, t=0.0, dt=0.0):
            FE, FW, GN, GS = orig_ff(self, tr, halo, t, dt)
            return FE, -FW, GN, GS
        monkeypatch.setattr(ad.Solver, "face_fluxes", face_fluxes)
    elif mistake == "no_heat_flux":
        orig_fl = ph.fluxes

        def fluxes(q, qx, qy, z, P, heat_override=None):
            z0 = torch.zeros_like(q[0])
            return orig_fl(q, qx, qy, z, P, heat_override=(z0, z0))
        monkeypatch.setattr(ad.ph, "fluxes", fluxes)
    u, uo, ub, _, _ = _compare(2, 2, False)
    worst = max(np.abs(uo[:, v] - ub[:, v]).max() / np.abs(ub[:, v] - u[:, v]).max() for v in range(4))
    assert worst > 1e-6, worst


def test_polybasis_agrees_with_closed_forms():
    """The independent basis itself: K1 1 = F0, M = diag(w), D exact on x^k."""
    for N in (1, 2, 3):
        b = PolyBasis(N)
        assert np.allclose(b.K1 @ np.ones(b.n), b.phi0, atol=1e-14)
        assert np.allclose(b.M, np.diag(b.w), atol=1e-13)
        for k in range(N + 1):
            assert np.allclose(b.D @ b.xi ** k, k * b.xi ** max(k - 1, 0) if k else 0.0, atol=1e-13)
