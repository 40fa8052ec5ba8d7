"""ADER-DG space-time predictor and corrector on a uniform 3D mesh (oracle).

The 2D scheme of aderdg.py in three dimensions (Sec. 3; the paper's 3D runs
are the ABC flow of Sec. 4.1 and the 3D cosine bubble of Sec. 4.2), with the
same readings P1, P2, B1, R6, R8 and R13:

P1  n = N+1 Picard sweeps q_l = u + dt sum_k (K1^{-1})_{lk} w_k R_k with
    R = -dF/dx - dG/dy - dH/dz + S;
P2  grad q, F, G, H, S once more on the final iterate, averaged in time;
B1  face data: boundary extrapolation of the time averages (q, normal flux,
    grad q);
R6  Rusanov speed |v.n| + c + 2 eta lambda_v, F* = (F_L + F_R)/2
    - max(s_L, s_R)(q_R - q_L)/2;
R8  slip wall: ghost rho and rhoE from the background at the face (the
    interior ones without gravity), momentum reflected, interior gradient,
    heat flux of the background temperature gradient (Eq. 10);
R13 analytic boundary: the analytic field and flux at the face nodes,
    averaged over the step at the Gauss-Legendre time nodes;
R11 dt = CFL h / (3 (2N+1) max(|v| + c + 2 eta lambda_v)) (d = 3).

Layout: u[c, v, l, j, i] with c = (iz ny + iy) nx + ix, v in (rho, rho u,
rho v, rho w, rho E), l the z-node, j the y-node, i the x-node.  Space-time
iterates carry the time index in front of v: q[c, k, v, l, j, i].

Pins: tests/test_oracle_3d.py.
"""
import math
from dataclasses import dataclass

import torch

from . import DTYPE
from .basis import Basis
from . import physics as ph
from . import physics3d as p3

FACES = ("E", "W", "N", "S", "T", "B")          # +x, -x, +y, -y, +z, -z
NORMAL = {"E": (1.0, 0.0, 0.0), "W": (-1.0, 0.0, 0.0), "N": (0.0, 1.0, 0.0),
          "S": (0.0, -1.0, 0.0), "T": (0.0, 0.0, 1.0), "B": (0.0, 0.0, -1.0)}


@dataclass
class Mesh3:
    nx: int
    ny: int
    nz: int
    x0: float = 0.0
    y0: float = 0.0
    z0: float = 0.0
    Lx: float = 1000.0
    Ly: float = 1000.0
    Lz: float = 1000.0
    bc_x: str = "periodic"   # "periodic" | "wall" | "dirichlet"
    bc_y: str = "periodic"
    bc_z: str = "periodic"
    dirichlet: object = None  # analytic field fn(x, y, z, t, P) of the "dirichlet" sides

    @property
    def h(self):
        return (self.Lx / self.nx, self.Ly / self.ny, self.Lz / self.nz)

    @property
    def cells(self):
        return self.nx * self.ny * self.nz


class Solver3:
    """Plain FP64 ADER-DG for the 3D compressible Navier-Stokes equations."""

    def __init__(self, mesh, params):
        self.m = mesh
        self.P = params
        self.b = Basis(params.N)
        n = self.b.n
        m = mesh
        hx, hy, hz = m.h
        xi = self.b.xi
        ix = torch.arange(m.nx, dtype=DTYPE)
        iy = torch.arange(m.ny, dtype=DTYPE)
        iz = torch.arange(m.nz, dtype=DTYPE)
        xn = m.x0 + (ix[:, None] + xi[None, :]) * hx   # [nx, n]
        yn = m.y0 + (iy[:, None] + xi[None, :]) * hy
        zn = m.z0 + (iz[:, None] + xi[None, :]) * hz
        shp = (m.nz, m.ny, m.nx, n, n, n)
        # node coordinates [c, l, j, i]
        self.X = xn[None, None, :, None, None, :].expand(shp).reshape(-1, n, n, n)
        self.Y = yn[None, :, None, None, :, None].expand(shp).reshape(-1, n, n, n)
        self.Z = zn[:, None, None, :, None, None].expand(shp).reshape(-1, n, n, n)
        self.Kw = self.b.K1inv * self.b.w[None, :]
        idx = torch.arange(m.cells).reshape(m.nz, m.ny, m.nx)
        self.idx = idx
        self.iz = torch.arange(m.cells) // (m.nx * m.ny)
        self.iy = (torch.arange(m.cells) // m.nx) % m.ny
        self.ix = torch.arange(m.cells) % m.nx

    # ------------------------------------------------------------ helpers
    def grad(self, q):
        """x-, y- and z-derivatives of nodal data q[..., l, j, i]."""
        D = self.b.D
        hx, hy, hz = self.m.h
        qx = torch.einsum("ip,...ljp->...lji", D, q) / hx
        qy = torch.einsum("jp,...lpi->...lji", D, q) / hy
        qz = torch.einsum("lp,...pji->...lji", D, q) / hz
        return qx, qy, qz

    def evaluate(self, q):
        """F, G, H, S and the gradients of a space-time iterate q[c, k, v, l, j, i]."""
        qx, qy, qz = self.grad(q)
        Z = self.Z[:, None]
        F, G, H, S = p3.fluxes(q.unbind(2), qx.unbind(2), qy.unbind(2), qz.unbind(2), Z, self.P)
        st = lambda a: torch.stack(a, 2)
        return st(F), st(G), st(H), st(S), qx, qy, qz

    # ------------------------------------------------------------ predictor
    def predictor(self, u, dt):
        """Picard iteration (P1, P2); returns the time averages."""
        n = self.b.n
        q = u[:, None].expand(-1, n, -1, -1, -1, -1).clone()
        for _ in range(n):
            F, G, H, S, _, _, _ = self.evaluate(q)
            Fx, _, _ = self.grad(F)
            _, Gy, _ = self.grad(G)
            _, _, Hz = self.grad(H)
            R = -Fx - Gy - Hz + S
            q = u[:, None] + dt * torch.einsum("ab,cb...->ca...", self.Kw, R)
        F, G, H, S, qx, qy, qz = self.evaluate(q)
        w = self.b.w
        avg = lambda a: torch.einsum("k,ck...->c...", w, a)
        return dict(qbar=avg(q), Fbar=avg(F), Gbar=avg(G), Hbar=avg(H), Sbar=avg(S),
                    qxbar=avg(qx), qybar=avg(qy), qzbar=avg(qz))

    # ------------------------------------------------------------ faces
    def face_traces(self, tavg):
        """Boundary extrapolation (B1) of the time averages to the 6 faces.
        x-faces carry [c, v, l, j], y-faces [c, v, l, i], z-faces [c, v, j, i]."""
        p0, p1 = self.b.phi0, self.b.phi1
        ext = {"x": lambda a, phi: torch.einsum("i,cvlji->cvlj", phi, a),
               "y": lambda a, phi: torch.einsum("j,cvlji->cvli", phi, a),
               "z": lambda a, phi: torch.einsum("l,cvlji->cvji", phi, a)}
        flux = {"x": "Fbar", "y": "Gbar", "z": "Hbar"}
        tr = {}
        for name, d, phi in (("E", "x", p1), ("W", "x", p0), ("N", "y", p1), ("S", "y", p0),
                             ("T", "z", p1), ("B", "z", p0)):
            e = ext[d]
            tr[name] = dict(q=e(tavg["qbar"], phi), f=e(tavg[flux[d]], phi), qx=e(tavg["qxbar"], phi),
                            qy=e(tavg["qybar"], phi), qz=e(tavg["qzbar"], phi))
        return tr

    def face_coords(self, name):
        """(x, y, z) of the nodes of face `name` of every cell, shaped like its
        trace's node grid."""
        hx, hy, hz = self.m.h
        if name in ("E", "W"):
            x = self.X[:, :, :, 0] - self.b.xi[0] * hx + (hx if name == "E" else 0.0)
            return x, self.Y[:, :, :, 0], self.Z[:, :, :, 0]
        if name in ("N", "S"):
            y = self.Y[:, :, 0, :] - self.b.xi[0] * hy + (hy if name == "N" else 0.0)
            return self.X[:, :, 0, :], y, self.Z[:, :, 0, :]
        z = self.Z[:, 0, :, :] - self.b.xi[0] * hz + (hz if name == "T" else 0.0)
        return self.X[:, 0, :, :], self.Y[:, 0, :, :], z

    def _ghost_wall(self, tr, nrm, z):
        P = self.P
        rho, mx, my, mz, E = tr["q"].unbind(1)
        mn = mx * nrm[0] + my * nrm[1] + mz * nrm[2]
        gm = [mx - 2.0 * mn * nrm[0], my - 2.0 * mn * nrm[1], mz - 2.0 * mn * nrm[2]]
        if P.gravity:
            pbar, rhobar, _ = ph.background(z, P)
            grho = rhobar + 0.0 * rho
            gE = pbar / (P.gamma - 1.0) + rhobar * P.g * z + 0.0 * rho
        else:
            grho, gE = rho, E
        gq = [grho] + gm + [gE]
        zero = torch.zeros_like(rho)
        F, G, H, _ = p3.fluxes(gq, tr["qx"].unbind(1), tr["qy"].unbind(1), tr["qz"].unbind(1), z, P,
                               heat_override=(zero, zero, zero + ph.dTbar_dz(P)))
        f = F if nrm[0] != 0.0 else (G if nrm[1] != 0.0 else H)
        return torch.stack(gq, 1), torch.stack(f, 1)

    def _ghost_dirichlet(self, x, y, z, nrm, t, dt):
        P = self.P
        qbar, fbar = 0.0, 0.0
        for k in range(self.b.n):
            Q, Qx, Qy, Qz = p3.field_with_gradient(self.m.dirichlet, x, y, z, t + float(self.b.xi[k]) * dt, P)
            F, G, H, _ = p3.fluxes(Q, Qx, Qy, Qz, z, P)
            f = F if nrm[0] != 0.0 else (G if nrm[1] != 0.0 else H)
            wk = float(self.b.w[k])
            qbar = qbar + wk * torch.stack(Q, 1)
            fbar = fbar + wk * torch.stack(f, 1)
        return qbar, fbar

    def riemann(self, qL, fL, qR, fR, z, nrm, h):
        P = self.P
        sL = p3.wave_speed(qL.unbind(1), z, nrm, h, P)
        sR = p3.wave_speed(qR.unbind(1), z, nrm, h, P)
        s = torch.maximum(sL, sR)[:, None]
        return 0.5 * (fL + fR) - 0.5 * s * (qR - qL)

    def face_fluxes(self, tr, t=0.0, dt=0.0):
        """Numerical fluxes on the 6 faces of every cell (own-face node grids)."""
        m = self.m
        hx, hy, hz = m.h
        idx = self.idx
        out = {}
        for plus, minus, dim, bc, h, first, last in (
                ("E", "W", 2, m.bc_x, hx, self.ix == 0, self.ix == m.nx - 1),
                ("N", "S", 1, m.bc_y, hy, self.iy == 0, self.iy == m.ny - 1),
                ("T", "B", 0, m.bc_z, hz, self.iz == 0, self.iz == m.nz - 1)):
            nrm = NORMAL[plus]
            nb = idx.roll(-1, dims=dim).reshape(-1)     # neighbour on the + side
            _, _, zp = self.face_coords(plus)
            _, _, zm = self.face_coords(minus)
            Fp = self.riemann(tr[plus]["q"], tr[plus]["f"], tr[minus]["q"][nb], tr[minus]["f"][nb], zp, nrm, h)
            Fm = Fp[idx.roll(1, dims=dim).reshape(-1)].clone()
            Fp = Fp.clone()
            if bc == "wall":
                gq, gf = self._ghost_wall(tr[plus], nrm, zp)
                Fp[last] = self.riemann(tr[plus]["q"], tr[plus]["f"], gq, gf, zp, nrm, h)[last]
                gq, gf = self._ghost_wall(tr[minus], NORMAL[minus], zm)
                Fm[first] = self.riemann(gq, gf, tr[minus]["q"], tr[minus]["f"], zm, nrm, h)[first]
            elif bc == "dirichlet":
                xp, yp, zp_ = self.face_coords(plus)
                gq, gf = self._ghost_dirichlet(xp[last], yp[last], zp_[last], nrm, t, dt)
                Fp[last] = self.riemann(tr[plus]["q"][last], tr[plus]["f"][last], gq, gf, zp[last], nrm, h)
                xm, ym, zm_ = self.face_coords(minus)
                gq, gf = self._ghost_dirichlet(xm[first], ym[first], zm_[first], nrm, t, dt)
                Fm[first] = self.riemann(gq, gf, tr[minus]["q"][first], tr[minus]["f"][first], zm[first], nrm, h)
            out[plus], out[minus] = Fp, Fm
        return out

    # ------------------------------------------------------------ corrector
    def corrector(self, u, dt, tavg, t=0.0):
        """u^{n+1} = u + dt (volume - face + Sbar), weak form with GL collocation."""
        b = self.b
        w, D, p0, p1 = b.w, b.D, b.phi0, b.phi1
        hx, hy, hz = self.m.h
        fl = self.face_fluxes(self.face_traces(tavg), t, dt)
        V = (w[:, None] * D) / w[None, :]        # V[p, i] = w_p D[p, i] / w_i
        vol = (torch.einsum("pi,cvljp->cvlji", V, tavg["Fbar"]) / hx
               + torch.einsum("pj,cvlpi->cvlji", V, tavg["Gbar"]) / hy
               + torch.einsum("pl,cvpji->cvlji", V, tavg["Hbar"]) / hz)
        face = ((p1[None, None, None, None, :] * fl["E"][..., None] - p0[None, None, None, None, :] * fl["W"][..., None])
                / (hx * w[None, None, None, None, :])
                + (p1[None, None, None, :, None] * fl["N"][:, :, :, None, :]
                   - p0[None, None, None, :, None] * fl["S"][:, :, :, None, :]) / (hy * w[None, None, None, :, None])
                + (p1[None, None, :, None, None] * fl["T"][:, :, None] - p0[None, None, :, None, None] * fl["B"][:, :, None])
                / (hz * w[None, None, :, None, None]))
        return u + dt * (vol - face + tavg["Sbar"])

    def step(self, u, dt, t=0.0):
        return self.corrector(u, dt, self.predictor(u, dt), t)

    # ------------------------------------------------------------ utilities
    def interpolate(self, fn, t=0.0):
        return torch.stack(fn(self.X, self.Y, self.Z, torch.as_tensor(t, dtype=DTYPE), self.P), 1)

    def integral(self, u):
        w = self.b.w
        hx, hy, hz = self.m.h
        return torch.einsum("l,j,i,cvlji->v", w, w, w, u) * hx * hy * hz

    def l2_error(self, u, uex):
        w = self.b.w
        hx, hy, hz = self.m.h
        return torch.sqrt(torch.einsum("l,j,i,cvlji->v", w, w, w, (u - uex) ** 2) * hx * hy * hz)

    def stable_dt(self, u, cfl):
        """Reading R11 with d = 3."""
        P = self.P
        q = u.unbind(1)
        h = min(self.m.h)
        rho, mx, my, mz, E = q
        p = p3.pressure(q, self.Z, P)
        c = torch.sqrt(P.gamma * p / rho)
        vel = torch.sqrt(mx * mx + my * my + mz * mz) / rho
        lam_v = max(4.0 / 3.0, P.gamma / P.Pr) * P.mu / rho
        eta = (2 * P.N + 1) / (h * math.sqrt(math.pi / 2.0))
        lam = (vel + c + 2.0 * eta * lam_v).max()
        return float(cfl * h / (3 * (2 * P.N + 1) * lam))
