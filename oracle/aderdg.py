"""ADER-DG space-time predictor and corrector on a uniform 2D mesh (oracle).

The paper uses the ADER-DG scheme of Dumbser et al. 2008 (Sec. 1, Sec. 3):
an element-local space-time predictor followed by a corrector with one face
exchange per step, and a Rusanov-type numerical flux adapted to viscous terms
(Gassner et al. 2008, used with ADER-DG in Dumbser 2010; Sec. 3).  The paper
does not print the scheme, so the steps below are the standard ADER-DG
predictor/corrector written from the mathematics, with these readings:

P1  the Picard iteration of the predictor runs a fixed n = N+1 sweeps;
P2  after the last sweep grad q, F, G and S are evaluated once more on the
    final iterate; their time averages feed the corrector;
B1  face data are the boundary extrapolation of the time-averaged nodal
    quantities (q-bar, F-bar, G-bar, grad q-bar), i.e. of the predictor's
    nodal interpolants;
R6  Rusanov speed s = |v.n| + c + 2 eta lambda_v on the extrapolated
    time-averaged face state, F* = (F_L + F_R)/2 - max(s_L, s_R)(q_R - q_L)/2;
R8  slip wall: ghost rho and rhoE from the background, momentum reflected,
    ghost gradient = interior gradient, the ghost's heat flux replaced by the
    background value -kappa dTbar/dz n_z (Eq. 10);
R12 no-slip wall moving tangentially with velocity v_w: ghost rho and p of
    the interior, ghost velocity 2 v_w - v, ghost gradient = interior
    gradient, adiabatic ghost heat flux (zero);
R13 analytic (Dirichlet) boundary: the ghost is the analytic field at the
    face node, averaged over the step at the Gauss-Legendre time nodes like
    the interior traces: q-bar = sum_k w_k Q(t + xi_k dt), normal flux
    sum_k w_k F(Q_k, grad Q_k) with the analytic gradient.

Layout: u[c, v, j, i] with c = iy * nx + ix, v in (rho, rho u, rho v, rho E),
j the y-node and i the x-node.  Space-time tensors carry a time index k in
front of v: q[c, k, v, j, i].

Pins: tests/test_oracle_scheme.py (constant state, conservation, linear
predictor vs a dense space-time solve, convergence order on the paper's
manufactured solution, hydrostatic balance, mirror symmetry).
"""
import math
from dataclasses import dataclass

import torch

from . import DTYPE
from .basis import Basis
from . import physics as ph


@dataclass
class Mesh:
    nx: int
    ny: int
    x0: float = 0.0
    y0: float = 0.0
    Lx: float = 10.0
    Ly: float = 10.0
    bc_x: str = "periodic"   # "periodic" | "wall" | "noslip" | "dirichlet"
    bc_y: str = "periodic"   # also "halo", "wall_halo", "halo_wall": strip of a larger mesh
                             # (south/north side takes the neighbour strip's traces)
    lid_u: float = 0.0       # x-velocity of the north wall (no-slip)
    dirichlet: object = None  # analytic field fn(x, y, t, P) of the "dirichlet" sides

    @property
    def hx(self):
        return self.Lx / self.nx

    @property
    def hy(self):
        return self.Ly / self.ny

    @property
    def cells(self):
        return self.nx * self.ny


class Solver:
    """Plain FP64 ADER-DG for the 2D compressible Navier-Stokes equations."""

    def __init__(self, mesh, params):
        self.m = mesh
        self.P = params
        self.b = Basis(params.N)
        n = self.b.n
        ix = torch.arange(mesh.nx, dtype=DTYPE)
        iy = torch.arange(mesh.ny, dtype=DTYPE)
        xi = self.b.xi
        # node coordinates X[c, j, i], Y[c, j, i]
        xc = mesh.x0 + (ix[:, None] + xi[None, :]) * mesh.hx      # [nx, n(i)]
        yc = mesh.y0 + (iy[:, None] + xi[None, :]) * mesh.hy      # [ny, n(j)]
        self.X = xc[None, :, None, :].expand(mesh.ny, mesh.nx, n, n).reshape(-1, n, n)
        self.Y = yc[:, None, :, None].expand(mesh.ny, mesh.nx, n, n).reshape(-1, n, n)
        # face coordinates: east/west faces carry y-nodes, north/south x-nodes
        self.Yface_x = yc[:, None, :].expand(mesh.ny, mesh.nx, n).reshape(-1, n)  # y at nodes j
        self.y_south = (mesh.y0 + iy * mesh.hy)[:, None].expand(mesh.ny, mesh.nx).reshape(-1)
        self.y_north = self.y_south + mesh.hy
        self.Xface_y = xc[None, :, :].expand(mesh.ny, mesh.nx, n).reshape(-1, n)  # x at nodes i
        self.x_west = (mesh.x0 + ix * mesh.hx)[None, :].expand(mesh.ny, mesh.nx).reshape(-1)
        self.x_east = self.x_west + mesh.hx
        # Lagrange weights folded into the time update: K1^{-1} diag(w)
        self.Kw = self.b.K1inv * self.b.w[None, :]

    # ------------------------------------------------------------ helpers
    def grad(self, q):
        """x- and y-derivatives of nodal data q[..., v, j, i]."""
        D = self.b.D
        qx = torch.einsum("ip,...jp->...ji", D, q) / self.m.hx
        qy = torch.einsum("jp,...pi->...ji", D, q) / self.m.hy
        return qx, qy

    def manufactured(self, t):
        """Manufactured source at the nodes at time t (zero if none)."""
        if self.P.source == "none":
            return None
        S = ph.manufactured_source(self.X, self.Y, t, self.P)
        return torch.stack(S, dim=1)  # [c, v, j, i]

    def evaluate(self, q, Sman):
        """F, G, S (and the gradients) of a space-time iterate q[c, k, v, j, i]."""
        qx, qy = self.grad(q)
        Y = self.Y[:, None]  # broadcast over k
        F, G, S = ph.fluxes(q.unbind(2), qx.unbind(2), qy.unbind(2), Y, self.P)
        F = torch.stack(F, 2)
        G = torch.stack(G, 2)
        S = torch.stack(S, 2)
        if Sman is not None:
            S = S + Sman
        return F, G, S, qx, qy

    # ------------------------------------------------------------ predictor
    def predictor(self, u, dt, t=0.0, sweeps=None):
        """Element-local space-time predictor (Picard iteration).

        q_l = u + dt * sum_k (K1^{-1})_{lk} w_k R_k with
        R = -dF/dx - dG/dy + S evaluated at the space-time nodes.
        Returns the final iterate q and the time averages needed by the
        corrector: qbar, Fbar, Gbar, Sbar, qxbar, qybar (each [c, v, j, i]).
        """
        b = self.b
        n = b.n
        sweeps = n if sweeps is None else sweeps
        if self.P.source != "none":
            Sman = torch.stack([self.manufactured(t + float(b.xi[k]) * dt) for k in range(n)], 1)
        else:
            Sman = None
        q = u[:, None].expand(-1, n, -1, -1, -1).clone()
        for _ in range(sweeps):
            F, G, S, _, _ = self.evaluate(q, Sman)
            Fx, _ = self.grad(F)
            _, Gy = self.grad(G)
            R = -Fx - Gy + S
            q = u[:, None] + dt * torch.einsum("lk,ck...->cl...", self.Kw, R)
        F, G, S, qx, qy = self.evaluate(q, Sman)
        w = b.w
        avg = lambda a: torch.einsum("k,ck...->c...", w, a)
        return q, dict(qbar=avg(q), Fbar=avg(F), Gbar=avg(G), Sbar=avg(S),
                       qxbar=avg(qx), qybar=avg(qy))

    # ------------------------------------------------------------ faces
    def face_traces(self, tavg):
        """Boundary extrapolation of time-averaged data to the 4 faces."""
        p0, p1 = self.b.phi0, self.b.phi1
        ex = lambda a, phi: torch.einsum("i,cvji->cvj", phi, a)  # to x = const faces
        ey = lambda a, phi: torch.einsum("j,cvji->cvi", phi, a)  # to y = const faces
        tr = {}
        for name, phi in (("E", p1), ("W", p0)):
            tr[name] = dict(q=ex(tavg["qbar"], phi), f=ex(tavg["Fbar"], phi),
                            qx=ex(tavg["qxbar"], phi), qy=ex(tavg["qybar"], phi))
        for name, phi in (("N", p1), ("S", p0)):
            tr[name] = dict(q=ey(tavg["qbar"], phi), f=ey(tavg["Gbar"], phi),
                            qx=ey(tavg["qxbar"], phi), qy=ey(tavg["qybar"], phi))
        return tr

    def _ghost(self, tr, nrm, z):
        """Ghost (q, normal flux) for a slip wall from the interior trace tr."""
        P = self.P
        nx, ny = nrm
        q = tr["q"].unbind(1)
        rho, mx, my, E = q
        mn = mx * nx + my * ny
        gmx = mx - 2.0 * mn * nx
        gmy = my - 2.0 * mn * ny
        if P.gravity:
            pbar, rhobar, _ = ph.background(z, P)
            grho = rhobar + 0.0 * rho
            gE = pbar / (P.gamma - 1.0) + rhobar * P.g * z + 0.0 * rho
        else:
            grho, gE = rho, E
        gq = [grho, gmx, gmy, gE]
        Tz = ph.dTbar_dz(P)
        zero = torch.zeros_like(rho)
        F, G, _ = ph.fluxes(gq, tr["qx"].unbind(1), tr["qy"].unbind(1), z, P,
                            heat_override=(zero, zero + Tz))
        f = torch.stack(F if nx != 0.0 else G, 1)  # the x- or y-flux
        return torch.stack(gq, 1), f

    def _ghost_noslip(self, tr, nrm, wall_u):
        """Ghost (q, normal flux) of a no-slip wall moving with velocity
        (wall_u, 0) (reading R12)."""
        P = self.P
        nx, ny = nrm
        rho, mx, my, E = tr["q"].unbind(1)
        gmx = 2.0 * rho * wall_u - mx
        gmy = -my
        # same density and pressure: only the kinetic energy changes
        gE = E - 0.5 * (mx * mx + my * my) / rho + 0.5 * (gmx * gmx + gmy * gmy) / rho
        gq = [rho, gmx, gmy, gE]
        zero = torch.zeros_like(rho)
        F, G, _ = ph.fluxes(gq, tr["qx"].unbind(1), tr["qy"].unbind(1), 0.0 * rho, P,
                            heat_override=(zero, zero))
        f = torch.stack(F if nx != 0.0 else G, 1)
        return torch.stack(gq, 1), f

    def _ghost_dirichlet(self, x, y, nrm, t, dt):
        """Ghost (q-bar, normal flux) from the analytic field at face nodes
        (x, y), averaged over [t, t + dt] at the time nodes (reading R13)."""
        P = self.P
        nx, ny = nrm
        b = self.b
        qbar, fbar = 0.0, 0.0
        for k in range(b.n):
            Q, Qx, Qy = ph.field_with_gradient(self.m.dirichlet, x, y, t + float(b.xi[k]) * dt, P)
            F, G, _ = ph.fluxes(Q, Qx, Qy, y, P)
            qbar = qbar + float(b.w[k]) * torch.stack(Q, 1)
            fbar = fbar + float(b.w[k]) * torch.stack(F if nx != 0.0 else G, 1)
        return qbar, fbar

    def _boundary(self, kind, side, tr, x, y, t, dt):
        """Ghost (q, f) of a boundary of the given kind on side E, W, N or S."""
        nrm = {"E": (1.0, 0.0), "W": (-1.0, 0.0), "N": (0.0, 1.0), "S": (0.0, -1.0)}[side]
        if kind == "wall":
            return self._ghost(tr, nrm, y)
        if kind == "noslip":
            return self._ghost_noslip(tr, nrm, self.m.lid_u if side == "N" else 0.0)
        if kind == "dirichlet":
            return self._ghost_dirichlet(x, y, nrm, t, dt)
        raise ValueError(kind)

    def riemann(self, qL, fL, qR, fR, zL, zR, nrm, h):
        """Rusanov-type viscous flux at face nodes (x- or y-component)."""
        P = self.P
        nx, ny = nrm
        sL = ph.wave_speed(qL.unbind(1), zL, nx, ny, h, P)
        sR = ph.wave_speed(qR.unbind(1), zR, nx, ny, h, P)
        s = torch.maximum(sL, sR)[:, None]
        return 0.5 * (fL + fR) - 0.5 * s * (qR - qL)

    def face_fluxes(self, tr, halo=None, t=0.0, dt=0.0):
        """F*_E, F*_W (x-fluxes along j) and G*_N, G*_S (y-fluxes along i).
        halo = {"S": (q, f), "N": (q, f)} with [nx, 4, n] face data of the
        strips below and above (strip decomposition, bc_y "halo*"); t, dt:
        the step, for analytic boundary data."""
        m = self.m
        nxc, nyc = m.nx, m.ny
        C = m.cells
        n = self.b.n
        idx = torch.arange(C).reshape(nyc, nxc)
        east = idx.roll(-1, dims=1).reshape(-1)   # neighbour at ix+1 (periodic wrap)
        north = idx.roll(-1, dims=0).reshape(-1)  # neighbour at iy+1
        zx = self.Yface_x                          # [c, n] y of the nodes on x-faces
        # ---- x-faces: face between c (L) and east[c] (R)
        qL, fL = tr["E"]["q"], tr["E"]["f"]
        qR, fR = tr["W"]["q"][east], tr["W"]["f"][east]
        Fx = self.riemann(qL, fL, qR, fR, zx, zx, (1.0, 0.0), m.hx)  # flux on c's east face
        FE = Fx.clone()
        FW = Fx[idx.roll(1, dims=1).reshape(-1)].clone()           # west face = east face of ix-1
        if m.bc_x in ("wall", "noslip", "dirichlet"):
            ix = torch.arange(C) % nxc
            last = ix == nxc - 1
            first = ix == 0
            xe = self.x_east[:, None].expand(C, n)
            xw = self.x_west[:, None].expand(C, n)
            gq, gf = self._boundary(m.bc_x, "E", tr["E"], xe, zx, t, dt)
            FE_w = self.riemann(tr["E"]["q"], tr["E"]["f"], gq, gf, zx, zx, (1.0, 0.0), m.hx)
            FE[last] = FE_w[last]
            gq, gf = self._boundary(m.bc_x, "W", tr["W"], xw, zx, t, dt)
            FW_w = self.riemann(gq, gf, tr["W"]["q"], tr["W"]["f"], zx, zx, (1.0, 0.0), m.hx)
            FW[first] = FW_w[first]
        # ---- y-faces: face between c (below) and north[c] (above)
        zN = self.y_north[:, None].expand(C, n)
        zS = self.y_south[:, None].expand(C, n)
        qL, fL = tr["N"]["q"], tr["N"]["f"]
        qR, fR = tr["S"]["q"][north], tr["S"]["f"][north]
        Gy = self.riemann(qL, fL, qR, fR, zN, zN, (0.0, 1.0), m.hy)
        GN = Gy.clone()
        GS = Gy[idx.roll(1, dims=0).reshape(-1)].clone()
        iy = torch.arange(C) // nxc
        top = iy == nyc - 1
        bot = iy == 0
        north = {"wall": "wall", "halo": "halo", "wall_halo": "halo", "halo_wall": "wall",
                 "noslip": "noslip", "dirichlet": "dirichlet"}.get(m.bc_y)
        south = {"wall": "wall", "halo": "halo", "wall_halo": "wall", "halo_wall": "halo",
                 "noslip": "noslip", "dirichlet": "dirichlet"}.get(m.bc_y)
        if north in ("wall", "noslip", "dirichlet"):
            gq, gf = self._boundary(north, "N", tr["N"], self.Xface_y, zN, t, dt)
            GN_w = self.riemann(tr["N"]["q"], tr["N"]["f"], gq, gf, zN, zN, (0.0, 1.0), m.hy)
            GN[top] = GN_w[top]
        if south in ("wall", "noslip", "dirichlet"):
            gq, gf = self._boundary(south, "S", tr["S"], self.Xface_y, zS, t, dt)
            GS_w = self.riemann(gq, gf, tr["S"]["q"], tr["S"]["f"], zS, zS, (0.0, 1.0), m.hy)
            GS[bot] = GS_w[bot]
        if north == "halo":
            hq, hf = halo["N"]
            GN[top] = self.riemann(tr["N"]["q"][top], tr["N"]["f"][top], hq, hf, zN[top], zN[top], (0.0, 1.0), m.hy)
        if south == "halo":
            hq, hf = halo["S"]
            GS[bot] = self.riemann(hq, hf, tr["S"]["q"][bot], tr["S"]["f"][bot], zS[bot], zS[bot], (0.0, 1.0), m.hy)
        return FE, FW, GN, GS

    # ------------------------------------------------------------ corrector
    def corrector(self, u, dt, tavg, halo=None, t=0.0):
        """u^{n+1} = u + dt (volume - face + Sbar), weak form with GL collocation."""
        b = self.b
        m = self.m
        w, D, p0, p1 = b.w, b.D, b.phi0, b.phi1
        tr = self.face_traces(tavg)
        FE, FW, GN, GS = self.face_fluxes(tr, halo, t, dt)
        # volume: (1/hx) sum_p (w_p/w_i) D[p,i] Fbar[p,j] + (1/hy) sum_p (w_p/w_j) D[p,j] Gbar[i,p]
        Vx = (w[:, None] * D) / w[None, :]   # Vx[p, i] = w_p D[p,i] / w_i
        vol = (torch.einsum("pi,cvjp->cvji", Vx, tavg["Fbar"]) / m.hx
               + torch.einsum("pj,cvpi->cvji", Vx, tavg["Gbar"]) / m.hy)
        face = ((p1[None, None, None, :] * FE[:, :, :, None] - p0[None, None, None, :] * FW[:, :, :, None])
                / (m.hx * w[None, None, None, :])
                + (p1[None, None, :, None] * GN[:, :, None, :] - p0[None, None, :, None] * GS[:, :, None, :])
                / (m.hy * w[None, None, :, None]))
        return u + dt * (vol - face + tavg["Sbar"])

    def step(self, u, dt, t=0.0):
        _, tavg = self.predictor(u, dt, t)
        return self.corrector(u, dt, tavg, t=t)

    # ------------------------------------------------------------ utilities
    def interpolate(self, fn, t=0.0):
        """Nodal interpolation of an analytic field fn(x, y, t) -> 4 tensors."""
        return torch.stack(fn(self.X, self.Y, torch.as_tensor(t, dtype=DTYPE), self.P), 1)

    def integral(self, u):
        """Per-variable integral sum_c hx hy sum_ij w_i w_j u."""
        w = self.b.w
        return torch.einsum("j,i,cvji->v", w, w, u) * self.m.hx * self.m.hy

    def l2_error(self, u, uex):
        """Quadrature-weighted L2 norm of (u - uex) per variable."""
        w = self.b.w
        d = (u - uex) ** 2
        return torch.sqrt(torch.einsum("j,i,cvji->v", w, w, d) * self.m.hx * self.m.hy)

    def stable_dt(self, u, cfl):
        """dt = CFL min(h) / (d (2N+1) max(|v| + c + 2 eta lambda_v)) over the
        nodes (reading R11: the paper gives no time-step rule)."""
        P = self.P
        q = u.unbind(1)
        h = min(self.m.hx, self.m.hy)
        rho, mx, my, E = q
        p = ph.pressure(q, self.Y, P)
        c = torch.sqrt(P.gamma * p / rho)
        vel = torch.sqrt(mx * mx + my * my) / rho
        lam_v = max(4.0 / 3.0, P.gamma / P.Pr) * P.mu / rho
        eta = (2 * P.N + 1) / (h * math.sqrt(math.pi / 2.0))
        lam = (vel + c + 2.0 * eta * lam_v).max()
        return float(cfl * h / (2 * (2 * P.N + 1) * lam))
