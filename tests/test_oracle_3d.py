"""Pins of the 3D oracle (oracle/aderdg3d.py, oracle/physics3d.py).

The 3D scheme has no printed worked example; it is pinned to the 2D oracle
(itself pinned in test_oracle_scheme.py) and to symmetries:

* data invariant along y (no y-momentum, periodic in y) evolve exactly as
  the 2D scheme on the (x, z) plane; invariant along x as the 2D scheme on
  (y, z); invariant along z (no gravity) as the 2D scheme on (x, y).  Each
  direction's fluxes, faces, boundaries and the gravity terms are exercised
  by at least one of them; a dropped term, a wrong sign or a transposed
  stress component in that direction breaks the 1e-12 agreement;
* a cyclic permutation of the axes (x, y, z) -> (y, z, x) commutes with a
  step on a cubic periodic mesh (fully 3D data: cross terms that vanish in
  the reductions);
* conservation on a periodic mesh, the atmosphere at rest with walls;
* the ABC field is divergence free and a Beltrami field (curl v = v).
"""
import math

import torch

from paper_1905_05524_gb300 import inputs
from oracle import physics as ph
from oracle import physics3d as p3
from oracle.aderdg import Mesh, Solver
from oracle.aderdg3d import Mesh3, Solver3

TOL = 1e-12


def smooth_momentum(X, Y, L1, L2, seed, amp=1.0):
    """Two seeded smooth periodic velocity components on a 2D node grid."""
    a = inputs.smooth_perturbation((6,), seed, 1.0)
    u = amp * (a[0] * torch.sin(2 * math.pi * X / L1 + a[1]) * torch.cos(2 * math.pi * Y / L2 + a[2]))
    v = amp * (a[3] * torch.cos(2 * math.pi * X / L1 + a[4]) * torch.sin(2 * math.pi * Y / L2 + a[5]))
    return u, v


def stirred_2d(s, seed, bubble=True):
    """2D state: the cosine bubble (with gravity) or a smooth density field
    (without), plus smooth momentum."""
    P = s.P
    m = s.m
    if P.gravity:
        th = ph.cosine_bubble(s.X, s.Y, 0.5, 250.0, 500.0, 350.0) if bubble else 0.0 * s.X
        q = ph.bubble_state(s.X, s.Y, th, P)
    else:
        rho = 1.0 + 0.2 * torch.sin(2 * math.pi * s.X / m.Lx) * torch.cos(2 * math.pi * s.Y / m.Ly)
        zero = torch.zeros_like(rho)
        q = [rho, zero, zero, 2.5 + 0.1 * torch.cos(2 * math.pi * (s.X / m.Lx + s.Y / m.Ly))]
    u, v = smooth_momentum(s.X, s.Y, m.Lx, m.Ly, seed)
    rho = q[0]
    E = q[3] + 0.5 * rho * (u * u + v * v)
    return torch.stack([rho, rho * u, rho * v, E], 1)


def lift(u2, shape3, axis, n):
    """Map a 2D state to the 3D layout, constant along `axis` ('x', 'y', 'z')."""
    nz, ny, nx = shape3
    if axis == "y":      # 2D (x, y2) = 3D (x, z); 2D cell c2 = iz nx + ix, nodes (l, i)
        U = u2.reshape(nz, nx, 4, n, n)
        U = U[:, None, :, :, :, None, :].expand(nz, ny, nx, 4, n, n, n)
        comps = [U[:, :, :, 0], U[:, :, :, 1], torch.zeros_like(U[:, :, :, 0]), U[:, :, :, 2], U[:, :, :, 3]]
    elif axis == "x":    # 2D (x2, y2) = 3D (y, z); c2 = iz ny + iy, nodes (l, j)
        U = u2.reshape(nz, ny, 4, n, n)
        U = U[:, :, None, :, :, :, None].expand(nz, ny, nx, 4, n, n, n)
        comps = [U[:, :, :, 0], torch.zeros_like(U[:, :, :, 0]), U[:, :, :, 1], U[:, :, :, 2], U[:, :, :, 3]]
    else:                # 2D (x, y) = 3D (x, y); c2 = iy nx + ix, nodes (j, i)
        U = u2.reshape(ny, nx, 4, n, n)
        U = U[None, :, :, :, None, :, :].expand(nz, ny, nx, 4, n, n, n)
        comps = [U[:, :, :, 0], U[:, :, :, 1], U[:, :, :, 2], torch.zeros_like(U[:, :, :, 0]), U[:, :, :, 3]]
    return torch.stack(comps, 3).reshape(nz * ny * nx, 5, n, n, n).contiguous()


def assert_close(a, b, tol=TOL, what=""):
    for v in range(5):
        d = torch.linalg.vector_norm(a[:, v] - b[:, v]).item()
        nb = max(torch.linalg.vector_norm(b[:, v]).item(), torch.linalg.vector_norm(b[:, 0]).item())
        assert d <= tol * nb, f"{what} var {v}: {d / nb:.3e}"


def run_pair(P, m2, m3, axis, seed, steps=2, bubble=True):
    s2, s3 = Solver(m2, P), Solver3(m3, P)
    u2 = stirred_2d(s2, seed, bubble)
    n = P.N + 1
    u3 = lift(u2, (m3.nz, m3.ny, m3.nx), axis, n)
    dt = 0.5 * s3.stable_dt(u3, 0.5)
    for _ in range(steps):
        u2 = s2.step(u2, dt)
        u3 = s3.step(u3, dt)
    assert_close(u3, lift(u2, (m3.nz, m3.ny, m3.nx), axis, n), TOL, f"reduction along {axis}")


def atm(N, mu=0.5):
    return ph.atmosphere_params(N, mu=mu)


def test_y_invariant_equals_2d_xz_with_gravity_and_walls():
    """Walls in x and z, gravity, viscosity, the cosine bubble plus smooth
    momentum; degree 2, 3 x 2 x 4 cells."""
    P = atm(2)
    m2 = Mesh(3, 4, 0.0, 0.0, 1000.0, 1000.0, "wall", "wall")
    m3 = Mesh3(3, 2, 4, bc_x="wall", bc_y="periodic", bc_z="wall")
    run_pair(P, m2, m3, "y", 11)


def test_x_invariant_equals_2d_yz_with_gravity_and_walls():
    P = atm(3)
    m2 = Mesh(3, 3, 0.0, 0.0, 1000.0, 1000.0, "wall", "wall")
    m3 = Mesh3(2, 3, 3, bc_x="periodic", bc_y="wall", bc_z="wall")
    run_pair(P, m2, m3, "x", 12)


def test_z_invariant_equals_2d_xy_without_gravity():
    """Periodic in x, walls in y; degree 1 and 2."""
    for N in (1, 2):
        P = ph.cfd_params(N, mu=0.1, source="none")
        m2 = Mesh(4, 3, 0.0, 0.0, 10.0, 8.0, "periodic", "wall")
        m3 = Mesh3(4, 3, 2, Lx=10.0, Ly=8.0, Lz=5.0, bc_x="periodic", bc_y="wall", bc_z="periodic")
        run_pair(P, m2, m3, "z", 13 + N)


def test_reductions_detect_a_planted_error():
    """An error confined to the y-z plane (the z-momentum y-flux without its
    shear stress) fails the y-z reduction: the pins see a dropped term."""
    orig = p3.fluxes

    def planted(q, gx, gy, gz, z, P, heat_override=None):
        F, G, H, S = orig(q, gx, gy, gz, z, P, heat_override)
        # an error confined to the y-z plane: the z-momentum y-flux loses its stress
        rho, mx, my, mz, E = q
        G = list(G)
        G[3] = mz * my / rho
        return F, G, H, S

    P = atm(2)
    m2 = Mesh(3, 3, 0.0, 0.0, 1000.0, 1000.0, "wall", "wall")
    m3 = Mesh3(2, 3, 3, bc_x="periodic", bc_y="wall", bc_z="wall")
    p3.fluxes = planted
    try:
        failed = False
        try:
            run_pair(P, m2, m3, "x", 12)
        except AssertionError:
            failed = True
    finally:
        p3.fluxes = orig
    assert failed


def rotate(u, nc):
    """Field after the rotation (x, y, z) -> (y, z, x) on a cubic mesh of nc^3
    cells: B(x', y', z') = M A(z', x', y'), momentum components cycled."""
    n = u.shape[-1]
    A = u.reshape(nc, nc, nc, 5, n, n, n)
    B = A.permute(2, 0, 1, 3, 6, 4, 5)
    B = B[:, :, :, [0, 2, 3, 1, 4]]
    return B.reshape(nc ** 3, 5, n, n, n).contiguous()


def smooth_3d(s, seed):
    a = inputs.smooth_perturbation((12,), seed, 1.0)
    L = s.m.Lx
    k = 2 * math.pi / L
    X, Y, Z = s.X, s.Y, s.Z
    rho = 1.0 + 0.2 * torch.sin(k * X + a[0]) * torch.cos(k * Y + a[1]) * torch.sin(k * Z + a[2])
    u = a[3] * torch.sin(k * Y + a[4]) + 0.3 * torch.cos(k * Z + a[5])
    v = a[6] * torch.sin(k * Z + a[7]) * torch.cos(k * X)
    w = a[8] * torch.cos(k * X + a[9]) + 0.2 * torch.sin(k * Y + a[10]) * torch.sin(k * Z)
    p = 2.0 + 0.1 * torch.cos(k * (X + Y + Z) + a[11])
    E = p / (s.P.gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return torch.stack([rho, rho * u, rho * v, rho * w, E], 1)


def test_cyclic_axis_permutation_commutes_with_a_step():
    for bc in ("periodic", "wall"):
        P = ph.cfd_params(2, mu=0.1, source="none")
        m = Mesh3(3, 3, 3, Lx=6.0, Ly=6.0, Lz=6.0, bc_x=bc, bc_y=bc, bc_z=bc)
        s = Solver3(m, P)
        u = smooth_3d(s, 21)
        dt = 0.5 * s.stable_dt(u, 0.5)
        a = rotate(s.step(u, dt), 3)
        b = s.step(rotate(u, 3), dt)
        assert_close(a, b, TOL, f"rotation {bc}")


def test_conservation_periodic():
    P = ph.cfd_params(2, mu=0.1, source="none")
    m = Mesh3(3, 4, 2, Lx=6.0, Ly=6.0, Lz=6.0)
    s = Solver3(m, P)
    u = smooth_3d(s, 22)
    I0 = s.integral(u)
    dt = 0.5 * s.stable_dt(u, 0.5)
    for _ in range(3):
        u = s.step(u, dt)
    I1 = s.integral(u)
    assert ((I1 - I0).abs() <= 1e-13 * I0.abs().clamp(min=1.0)).all(), I1 - I0


def test_atmosphere_at_rest_with_walls():
    """Degree 3 on 111 m cells: the background's interpolation error leaves
    velocities of 2e-11 m/s after 10 steps (degree 2 on 250 m cells: 2e-6,
    the same as the 2D scheme, which the reductions above tie it to)."""
    P = ph.atmosphere_params(3, mu=0.005)
    m = Mesh3(2, 2, 9, bc_x="wall", bc_y="wall", bc_z="wall")
    s = Solver3(m, P)
    u = torch.stack(p3.bubble_state(s.Z, 0.0 * s.Z, P), 1)
    dt = s.stable_dt(u, 0.5)
    for _ in range(10):
        u = s.step(u, dt)
    vel = (u[:, 1:4] / u[:, 0:1]).abs().max().item()
    th = (p3.theta(u.unbind(1), s.Z, P) - P.theta0).abs().max().item()
    assert vel < 1e-9 and th < 1e-9, (vel, th)


def test_abc_field_is_divergence_free_beltrami():
    P = ph.cfd_params(2, mu=0.01, source="none")
    g = torch.Generator().manual_seed(3)
    x, y, z = [(torch.rand(50, generator=g, dtype=torch.float64) * 2 - 1) * math.pi for _ in range(3)]
    Q, Qx, Qy, Qz = p3.field_with_gradient(p3.abc_flow, x, y, z, 0.3, P)
    div = Qx[1] + Qy[2] + Qz[3]        # rho = 1: momentum = velocity
    assert div.abs().max().item() < 1e-14
    curl = [Qy[3] - Qz[2], Qz[1] - Qx[3], Qx[2] - Qy[1]]
    for c in range(3):
        assert (curl[c] - Q[1 + c]).abs().max().item() < 1e-14


def test_abc_flow_short_run_tracks_the_analytic_field():
    """Degree 2 on 6^3 cells with analytic boundaries to t = 0.02: the
    compressible solution stays within 1e-2 (relative L2 of the velocity) of
    the incompressible ABC field (the paper: qualitative agreement)."""
    P = ph.cfd_params(2, mu=0.01, source="none")
    m = Mesh3(6, 6, 6, x0=-math.pi, y0=-math.pi, z0=-math.pi, Lx=2 * math.pi, Ly=2 * math.pi, Lz=2 * math.pi,
              bc_x="dirichlet", bc_y="dirichlet", bc_z="dirichlet", dirichlet=p3.abc_flow)
    s = Solver3(m, P)
    u = s.interpolate(p3.abc_flow, 0.0)
    dt = s.stable_dt(u, 0.5)
    T = 0.02
    steps = math.ceil(T / dt)
    dt = T / steps
    t = 0.0
    for _ in range(steps):
        u = s.step(u, dt, t)
        t += dt
    ue = s.interpolate(p3.abc_flow, T)
    err = s.l2_error(u, ue)
    nrm = s.l2_error(0.0 * ue, ue)
    assert (err[1:4] / nrm[1:4]).max().item() < 1e-2, err / nrm
