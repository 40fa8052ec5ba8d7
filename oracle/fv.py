"""MUSCL-Hancock finite-volume scheme with the van Albada limiter (oracle).

The paper's engine also offers a MUSCL-Hancock finite-volume method,
stabilised with the van Albada limiter (Sec. 3), run without viscosity on
the colliding-bubbles scenario (Sec. 4.2: "as we use limiting, we do not
need any viscosity").  The paper does not print the scheme; these are the
readings (the standard unsplit MUSCL-Hancock method):

FV1 cell averages of the conserved variables (rho, rho u, rho v, rho E) on a
    uniform grid, reconstructed as perturbations of the hydrostatic
    background Ubar(z) (zero without gravity): U' = U - Ubar(z_centre),
    slopes of U' per direction and variable from the van Albada limiter of
    the one-sided differences a, b: slope = a b (a + b) / (a^2 + b^2) where
    a b > 0, else 0; face states Ubar(z_face) + U' +- slope/2, so the
    background at rest is reproduced exactly at every face (well-balanced,
    in the spirit of Eq. 7's perturbation form); cells next to a wall take
    zero slopes in the wall's direction;
FV2 Hancock predictor: the four face-extrapolated states U +- slope/2 and
    the cell mean are advanced by dt/2 with the cell's own flux differences
    F(U_E) - F(U_W), G(U_N) - G(U_S) and the source at the cell mean;
FV3 Rusanov flux on the evolved face states with s = max(|v.n| + c);
    update U - dt/hx (F*_E - F*_W) - dt/hy (G*_N - G*_S) + dt S(U-mean at
    the half step);
FV4 the perturbation form of the paper (Eq. 7): momentum flux with
    p' = p - pbar(z) at the height where the flux is evaluated (cell centre
    for x-fluxes, face height for y-fluxes), source -g rho' with rhobar at
    the cell centre;
FV5 slip wall: the ghost face state has the background rho and rhoE at the
    face height (the interior ones without gravity) and the momentum
    reflected, as reading R8 of the DG scheme.

Layout: U[v, iy, ix] (structure of arrays, cells row-major).
Pins: tests/test_oracle_fv.py.
"""
import torch

from . import DTYPE
from . import physics as ph


def van_albada(a, b):
    """Limited slope from the one-sided differences a and b (FV1)."""
    ab = a * b
    den = a * a + b * b
    return torch.where(ab > 0.0, ab * (a + b) / torch.where(den > 0.0, den, torch.ones_like(den)),
                       torch.zeros_like(a))


class MusclHancock:
    def __init__(self, nx, ny, Lx, Ly, P, bc_x="periodic", bc_y="periodic", x0=0.0, y0=0.0):
        assert P.mu == 0.0, "the finite-volume scheme is inviscid"
        self.nx, self.ny, self.P = nx, ny, P
        self.hx, self.hy = Lx / nx, Ly / ny
        self.bc_x, self.bc_y = bc_x, bc_y
        iy = torch.arange(ny, dtype=DTYPE)
        ix = torch.arange(nx, dtype=DTYPE)
        self.zc = (y0 + (iy + 0.5) * self.hy)[:, None].expand(ny, nx)        # cell centres
        self.xc = (x0 + (ix + 0.5) * self.hx)[None, :].expand(ny, nx)
        self.zN = self.zc + 0.5 * self.hy
        self.zS = self.zc - 0.5 * self.hy

    # ------------------------------------------------------------ pieces
    def _flux(self, U, z, xdir):
        q = list(U.unbind(0))
        zero = [torch.zeros_like(q[0])] * 4
        F, G, _ = ph.fluxes(q, zero, zero, z, self.P)
        return torch.stack(F if xdir else G, 0)

    def _source(self, U, z):
        P = self.P
        if not P.gravity:
            return torch.zeros_like(U)
        _, rhobar, _ = ph.background(z, P)
        S = torch.zeros_like(U)
        S[2] = -P.g * (U[0] - rhobar)
        return S

    def _slopes(self, U, dim, wall):
        a = U - U.roll(1, dims=dim)
        b = U.roll(-1, dims=dim) - U
        s = van_albada(a, b)
        if wall:
            n = U.shape[dim]
            idx = torch.tensor([0, n - 1])
            s.index_fill_(dim, idx, 0.0)
        return s

    def _speed(self, U, z, xdir):
        q = list(U.unbind(0))
        return ph.wave_speed(q, z, 1.0 if xdir else 0.0, 0.0 if xdir else 1.0, 1.0, self.P)

    def _rusanov(self, UL, UR, zL, zR, xdir):
        FL, FR = self._flux(UL, zL, xdir), self._flux(UR, zR, xdir)
        s = torch.maximum(self._speed(UL, zL, xdir), self._speed(UR, zR, xdir))
        return 0.5 * (FL + FR) - 0.5 * s * (UR - UL)

    def _wall_ghost(self, Ub, z, nrm):
        P = self.P
        nx, ny = nrm
        rho, mx, my, E = Ub.unbind(0)
        mn = mx * nx + my * ny
        g = [rho, mx - 2.0 * mn * nx, my - 2.0 * mn * ny, E]
        if P.gravity:
            pbar, rhobar, _ = ph.background(z, P)
            g[0] = rhobar + 0.0 * rho
            g[3] = pbar / (P.gamma - 1.0) + rhobar * P.g * z + 0.0 * rho
        return torch.stack(g, 0)

    # ------------------------------------------------------------ step
    def background_state(self, z):
        """Ubar(z) = (rhobar, 0, 0, pbar/(gamma-1) + rhobar g z); zero without gravity."""
        P = self.P
        pbar, rhobar, _ = ph.background(z, P)
        zero = torch.zeros_like(pbar)
        E = pbar / (P.gamma - 1.0) + (rhobar * P.g * z if P.gravity else zero)
        return torch.stack([rhobar, zero, zero, E], 0)

    def half_step(self, U, dt):
        """FV1-FV2: slopes, face states and their half-step evolution.
        Returns (UE, UW, UN, US, Um) at t + dt/2."""
        P = self.P
        Bc = self.background_state(self.zc)
        Up = U - Bc
        sx = self._slopes(Up, 2, self.bc_x == "wall")
        sy = self._slopes(Up, 1, self.bc_y == "wall")
        UE, UW = U + 0.5 * sx, U - 0.5 * sx
        UN = self.background_state(self.zN) + Up + 0.5 * sy
        US = self.background_state(self.zS) + Up - 0.5 * sy
        dF = self._flux(UE, self.zc, True) - self._flux(UW, self.zc, True)
        dG = self._flux(UN, self.zN, False) - self._flux(US, self.zS, False)
        d = -0.5 * dt / self.hx * dF - 0.5 * dt / self.hy * dG + 0.5 * dt * self._source(U, self.zc)
        return UE + d, UW + d, UN + d, US + d, U + d

    def face_fluxes(self, UE, UW, UN, US):
        """FV3/FV5: Rusanov fluxes on the four faces of every cell."""
        FE = self._rusanov(UE, UW.roll(-1, dims=2), self.zc, self.zc, True)   # east face of (iy, ix)
        FW = FE.roll(1, dims=2)
        GN = self._rusanov(UN, US.roll(-1, dims=1), self.zN, self.zN, False)  # north face
        GS = GN.roll(1, dims=1)
        if self.bc_x == "wall":
            gE = self._wall_ghost(UE[:, :, -1], self.zc[:, -1], (1.0, 0.0))
            FE[:, :, -1] = self._rusanov(UE[:, :, -1], gE, self.zc[:, -1], self.zc[:, -1], True)
            gW = self._wall_ghost(UW[:, :, 0], self.zc[:, 0], (-1.0, 0.0))
            FW[:, :, 0] = self._rusanov(gW, UW[:, :, 0], self.zc[:, 0], self.zc[:, 0], True)
        if self.bc_y == "wall":
            gN = self._wall_ghost(UN[:, -1, :], self.zN[-1, :], (0.0, 1.0))
            GN[:, -1, :] = self._rusanov(UN[:, -1, :], gN, self.zN[-1, :], self.zN[-1, :], False)
            gS = self._wall_ghost(US[:, 0, :], self.zS[0, :], (0.0, -1.0))
            GS[:, 0, :] = self._rusanov(gS, US[:, 0, :], self.zS[0, :], self.zS[0, :], False)
        return FE, FW, GN, GS

    def step(self, U, dt):
        UE, UW, UN, US, Um = self.half_step(U, dt)
        FE, FW, GN, GS = self.face_fluxes(UE, UW, UN, US)
        return (U - dt / self.hx * (FE - FW) - dt / self.hy * (GN - GS)
                + dt * self._source(Um, self.zc))

    def stable_dt(self, U, cfl):
        """cfl / (max(|u| + c)/hx + max(|v| + c)/hy) (a reading; the paper is silent)."""
        sx = self._speed(U, self.zc, True).max().item()
        sy = self._speed(U, self.zc, False).max().item()
        return cfl / (sx / self.hx + sy / self.hy)

    def integral(self, U):
        return U.sum(dim=(1, 2)) * self.hx * self.hy
