"""Thin Python front end of the C ABI (include/aderdg.h).

PyTorch supplies device memory and the CUDA stream; every step of the method
runs in libaderdg.so.  The functions here only build the C descriptors, pass
pointers and turn status codes into exceptions.
"""
import ctypes
import math
from dataclasses import dataclass

import torch

from . import _lib as L


@dataclass
class MeshConfig:
    """Python mirror of adg_mesh_desc (defaults: the CFD constants of Sec. 4.1)."""
    degree: int = 3
    nx: int = 9
    ny: int = 9
    x0: float = 0.0
    y0: float = 0.0
    Lx: float = 10.0
    Ly: float = 10.0
    bc_x: int = L.ADG_BC_PERIODIC
    bc_y: int = L.ADG_BC_PERIODIC
    gamma: float = 1.4
    Pr: float = 0.7
    R: float = 0.4
    mu: float = 0.1
    gravity: int = 0
    g: float = 9.81
    p0: float = 1e5
    theta0: float = 300.0
    source: int = L.ADG_SRC_NONE
    src_a: float = 0.1
    src_L: float = 10.0
    src_U: float = 0.5
    src_p: float = 1.0
    precision: int = L.ADG_PREC_FP64
    device: int = 0
    max_levels: int = 0
    lid_u: float = 0.0
    bc_field: int = L.ADG_FIELD_NONE

    def to_c(self):
        return L.MeshDesc(**{f: getattr(self, f) for f, _ in L.MeshDesc._fields_})

    @property
    def n(self):
        return self.degree + 1

    @property
    def cells(self):
        return self.nx * self.ny


def steady_manufactured_config(degree=3, nx=9, ny=9, precision=L.ADG_PREC_FP64, device=0):
    """Periodic [0,10]^2, gamma 1.4, Pr 0.7, c_v 1, mu 0.1, steady manufactured
    solution rho = 1 + 0.1 sin(2 pi (x+y)/10), u = v = 0.5, p = 1 with its source."""
    return MeshConfig(degree=degree, nx=nx, ny=ny, source=L.ADG_SRC_STEADY,
                      precision=precision, device=device)


def paper_manufactured_config(degree=3, nx=9, ny=9, mu=0.1, device=0):
    """Periodic [0,10]^2, gamma 1.4, Pr 0.7, c_v 1, with the time-dependent
    manufactured solution of Sec. 4.1 (Eq. 8) and its source (FP64)."""
    return MeshConfig(degree=degree, nx=nx, ny=ny, mu=mu, source=L.ADG_SRC_PAPER, device=device)


def taylor_green_config(degree=4, nx=25, ny=25, device=0):
    """Taylor-Green vortex (Sec. 4.1): [0, 2pi]^2, gamma 1.4, Pr 0.7, c_v 1,
    mu = 0.1, the analytic field imposed on every boundary."""
    two_pi = 2.0 * 3.141592653589793
    return MeshConfig(degree=degree, nx=nx, ny=ny, Lx=two_pi, Ly=two_pi, mu=0.1,
                      bc_x=L.ADG_BC_ANALYTIC, bc_y=L.ADG_BC_ANALYTIC, bc_field=L.ADG_FIELD_TAYLOR_GREEN,
                      device=device)


def cavity_config(degree=2, nx=27, ny=27, mu=0.01, lid_u=1.0, device=0):
    """Lid-driven cavity (Sec. 4.1): [0, 1]^2 m with no-slip walls, the lid
    (north wall) moving at lid_u; gamma 1.4, Pr 0.7, c_v 1; mu = 0.01
    (Reynolds number 100 at rho = 1, the paper does not state mu)."""
    return MeshConfig(degree=degree, nx=nx, ny=ny, Lx=1.0, Ly=1.0, mu=mu,
                      bc_x=L.ADG_BC_NOSLIP, bc_y=L.ADG_BC_NOSLIP, lid_u=lid_u, device=device)


def atmosphere_config(degree=5, nx=81, ny=81, mu=0.01, precision=L.ADG_PREC_FP64, device=0):
    """[0,1000]^2 m with slip walls, gamma 1.4, Pr 0.71, R 287.058, p0 1e5 Pa,
    g 9.81, theta0 300 K isentropic background (Sec. 4.2)."""
    return MeshConfig(degree=degree, nx=nx, ny=ny, Lx=1000.0, Ly=1000.0,
                      bc_x=L.ADG_BC_WALL, bc_y=L.ADG_BC_WALL, gamma=1.4, Pr=0.71,
                      R=287.058, mu=mu, gravity=1, g=9.81, p0=1e5, theta0=300.0,
                      precision=precision, device=device)


def _device_view(ptr, numel, device):
    """A float64 tensor aliasing `numel` doubles of device memory at `ptr`."""
    class _Iface:
        __cuda_array_interface__ = {"shape": (numel,), "typestr": "<f8", "data": (ptr, False), "version": 3}
    return torch.as_tensor(_Iface(), device=device)


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Mesh:
    """Owns one adg_mesh handle."""

    def __init__(self, cfg: MeshConfig):
        self.cfg = cfg
        self._lib = L.lib()
        h = ctypes.c_void_p()
        L.check(self._lib.adg_create_mesh(ctypes.byref(cfg.to_c()), ctypes.byref(h)))
        self.h = h
        self.count = self._lib.adg_state_count(self.h)
        self.device = torch.device("cuda", cfg.device)

    def close(self):
        if getattr(self, "h", None):
            self._lib.adg_destroy_mesh(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        n = self.cfg.n
        return (self.cfg.cells, 4, n, n)

    # --------------------------------------------------------------- state
    def set_state(self, u: torch.Tensor, stream=None):
        assert u.dtype == torch.float64 and u.is_contiguous() and u.numel() == self.count
        on_dev = 1 if u.is_cuda else 0
        L.check(self._lib.adg_set_state(self.h, ctypes.c_void_p(u.data_ptr()), self.count,
                                        on_dev, _stream_ptr(stream)))

    def get_state(self, out: torch.Tensor = None, stream=None):
        if out is None:
            out = torch.empty(self.state_shape, dtype=torch.float64, device=self.device)
        assert out.dtype == torch.float64 and out.is_contiguous() and out.numel() == self.count
        L.check(self._lib.adg_get_state(self.h, ctypes.c_void_p(out.data_ptr()), self.count,
                                        1 if out.is_cuda else 0, _stream_ptr(stream)))
        return out

    def state_view(self):
        """Zero-copy torch view of the mesh's device state (borrowed: valid until
        close() or adapt())."""
        ptr = self._lib.adg_state_ptr(self.h)
        n = self.cfg.n
        size = self.leaves * 4 * n * n
        return _device_view(ptr, size, self.device).view(self.state_shape)

    @property
    def time(self):
        return self._lib.adg_get_time(self.h)

    @time.setter
    def time(self, t):
        L.check(self._lib.adg_set_time(self.h, float(t)))

    def init_scenario(self, kind, A=0.5, a=250.0, xc=500.0, zc=350.0, stream=None):
        sc = L.Scenario(kind=kind, A=A, a=a, xc=xc, zc=zc)
        L.check(self._lib.adg_init_scenario(self.h, ctypes.byref(sc), _stream_ptr(stream)))

    # --------------------------------------------------------------- method
    def predictor(self, dt, stream=None):
        L.check(self._lib.adg_predictor(self.h, float(dt), _stream_ptr(stream)))

    def corrector(self, dt, stream=None):
        L.check(self._lib.adg_corrector(self.h, float(dt), _stream_ptr(stream)))

    def step(self, dt, nsteps=1, stream=None):
        sp = _stream_ptr(stream)
        for _ in range(nsteps):
            L.check(self._lib.adg_step(self.h, float(dt), sp))

    def step_lts(self, dt, stream=None):
        """One local-time-stepping cycle of an adaptive FP64 mesh (adg_step_lts);
        returns the cycle length."""
        c = ctypes.c_double()
        L.check(self._lib.adg_step_lts(self.h, float(dt), ctypes.byref(c), _stream_ptr(stream)))
        return c.value

    def stable_dt(self, cfl, stream=None):
        dt = ctypes.c_double()
        L.check(self._lib.adg_stable_dt(self.h, float(cfl), ctypes.byref(dt), _stream_ptr(stream)))
        return dt.value

    def tv_indicator(self, var, T_r, T_c, want_stats=True, stream=None):
        C = self.leaves
        tv = torch.empty(C, dtype=torch.float64, device=self.device)
        flags = torch.empty(C, dtype=torch.int8, device=self.device)
        stats = (ctypes.c_double * 2)()
        L.check(self._lib.adg_tv_indicator(
            self.h, int(var), float(T_r), float(T_c), ctypes.c_void_p(tv.data_ptr()),
            ctypes.c_void_p(flags.data_ptr()), stats if want_stats else None,
            _stream_ptr(stream)))
        return tv, flags, (stats[0], stats[1])

    def step_tv(self, dt, var, T_r, T_c, want_stats=True, stream=None):
        """One step, then the TV indicator of the new state (adg_step_tv)."""
        C = self.leaves
        tv = torch.empty(C, dtype=torch.float64, device=self.device)
        flags = torch.empty(C, dtype=torch.int8, device=self.device)
        stats = (ctypes.c_double * 2)()
        L.check(self._lib.adg_step_tv(
            self.h, float(dt), int(var), float(T_r), float(T_c), ctypes.c_void_p(tv.data_ptr()),
            ctypes.c_void_p(flags.data_ptr()), stats if want_stats else None, _stream_ptr(stream)))
        return tv, flags, (stats[0], stats[1])

    def check_finite(self, stream=None):
        L.check(self._lib.adg_check_finite(self.h, _stream_ptr(stream)))

    # --------------------------------------------------------------- adaptive mesh
    @property
    def leaves(self):
        return int(self._lib.adg_leaf_count(self.h))

    def leaf_info(self):
        n = self.leaves
        buf = (ctypes.c_int * (3 * n))()
        L.check(self._lib.adg_leaf_info(self.h, buf, 3 * n))
        return [tuple(buf[3 * k:3 * k + 3]) for k in range(n)]

    def adapt(self, flags: torch.Tensor, stream=None):
        assert flags.dtype == torch.int8 and flags.is_cuda and flags.numel() == self.leaves
        out = ctypes.c_int()
        L.check(self._lib.adg_adapt(self.h, ctypes.c_void_p(flags.data_ptr()), ctypes.byref(out),
                                    _stream_ptr(stream)))
        self.count = self._lib.adg_state_count(self.h)
        return out.value

    @property
    def state_shape(self):
        n = self.cfg.n
        return (self.leaves, 4, n, n)


class Batch:
    """Owns one adg_batch handle over a list of Mesh objects (kept alive here)."""

    def __init__(self, meshes):
        self.meshes = list(meshes)
        self._lib = L.lib()
        arr = (ctypes.c_void_p * len(self.meshes))(*[m.h.value for m in self.meshes])
        h = ctypes.c_void_p()
        L.check(self._lib.adg_batch_create(arr, len(self.meshes), ctypes.byref(h)))
        self.h = h

    def step(self, dts, nsteps=1, stream=None):
        arr = (ctypes.c_double * len(self.meshes))(*[float(d) for d in dts])
        L.check(self._lib.adg_batch_step(self.h, arr, int(nsteps), _stream_ptr(stream)))

    def set_candidate(self, cand):
        """Pin the predictor's candidate (0, 1, 2: tile sizes; 3: node pairs) instead of the timed choice."""
        L.check(self._lib.adg_batch_set_candidate(self.h, int(cand)))

    def info(self):
        buf = (ctypes.c_int * 13)()
        L.check(self._lib.adg_batch_info(self.h, buf, 13))
        keys = ["tiles_pred", "cpb_pred", "grid_pred", "tiles_corr", "cpb_corr", "grid_corr",
                "tune_ns_0", "tune_ns_1", "tune_ns_2", "candidate", "tune_source", "adaptive_instances",
                "tune_ns_3"]
        return dict(zip(keys, list(buf)))

    def close(self):
        if getattr(self, "h", None):
            self._lib.adg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fv_bubble_config(nx=630, ny=630, device=0):
    """MUSCL-Hancock colliding bubbles (Sec. 4.2): [0,1000]^2 m, slip walls,
    the atmosphere of Eq. 11 without viscosity (the paper: 7^2 patches of
    90^2 finite volumes = 630^2 cells)."""
    return MeshConfig(degree=1, nx=nx, ny=ny, Lx=1000.0, Ly=1000.0, bc_x=L.ADG_BC_WALL, bc_y=L.ADG_BC_WALL,
                      gamma=1.4, Pr=0.71, R=287.058, mu=0.0, gravity=1, g=9.81, p0=1e5, theta0=300.0,
                      device=device)


class FvMesh:
    """MUSCL-Hancock finite volumes (adg_fv_*): state tensor [4, ny, nx]."""

    def __init__(self, cfg: MeshConfig):
        self.cfg = cfg
        self._lib = L.lib()
        self.device = torch.device("cuda", cfg.device)
        h = ctypes.c_void_p()
        L.check(self._lib.adg_fv_create(ctypes.byref(cfg.to_c()), ctypes.byref(h)))
        self.h = h
        self.count = self._lib.adg_fv_state_count(self.h)

    def close(self):
        if getattr(self, "h", None):
            self._lib.adg_fv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        return (4, self.cfg.ny, self.cfg.nx)

    def set_state(self, u: torch.Tensor, stream=None):
        u = u.to(self.device, torch.float64).contiguous()
        L.check(self._lib.adg_fv_set_state(self.h, ctypes.c_void_p(u.data_ptr()), self.count, 1, _stream_ptr(stream)))

    def get_state(self, stream=None):
        out = torch.empty(self.shape, dtype=torch.float64, device=self.device)
        L.check(self._lib.adg_fv_get_state(self.h, ctypes.c_void_p(out.data_ptr()), self.count, 1,
                                           _stream_ptr(stream)))
        return out

    def init_scenario(self, kind, A=0.5, a=250.0, xc=500.0, zc=350.0, stream=None):
        sc = L.Scenario(kind=kind, A=A, a=a, xc=xc, zc=zc)
        L.check(self._lib.adg_fv_init_scenario(self.h, ctypes.byref(sc), _stream_ptr(stream)))

    def step(self, dt, nsteps=1, stream=None):
        for _ in range(nsteps):
            L.check(self._lib.adg_fv_step(self.h, float(dt), _stream_ptr(stream)))

    def stable_dt(self, cfl, stream=None):
        dt = ctypes.c_double()
        L.check(self._lib.adg_fv_stable_dt(self.h, float(cfl), ctypes.byref(dt), _stream_ptr(stream)))
        return dt.value



@dataclass
class Mesh3Config(MeshConfig):
    """A 3D mesh: the 2D descriptor's x and y plus the vertical z (gravity,
    background and perturbation split along z)."""
    nz: int = 9
    z0: float = 0.0
    Lz: float = 10.0
    bc_z: int = L.ADG_BC_PERIODIC

    @property
    def cells(self):
        return self.nx * self.ny * self.nz


def bubble3d_config(degree=2, n=25, mu=0.005, device=0):
    """The 3D cosine bubble of Sec. 4.2: [0,1000]^3 m, 40 m cells (25^3),
    order 3 (degree 2), mu = 0.005, slip walls, the atmosphere of Eq. 11."""
    return Mesh3Config(degree=degree, nx=n, ny=n, Lx=1000.0, Ly=1000.0, bc_x=L.ADG_BC_WALL, bc_y=L.ADG_BC_WALL,
                       gamma=1.4, Pr=0.71, R=287.058, mu=mu, gravity=1, g=9.81, p0=1e5, theta0=300.0,
                       device=device, nz=n, z0=0.0, Lz=1000.0, bc_z=L.ADG_BC_WALL)


def abc_config(degree=2, n=27, mu=0.01, device=0):
    """The ABC flow of Sec. 4.1: [-pi, pi]^3, 27^3 cells, order 3 (degree 2),
    mu = 0.01, analytic boundaries, gamma 1.4, Pr 0.7, c_v 1."""
    return Mesh3Config(degree=degree, nx=n, ny=n, x0=-math.pi, y0=-math.pi, Lx=2 * math.pi, Ly=2 * math.pi,
                       bc_x=L.ADG_BC_ANALYTIC, bc_y=L.ADG_BC_ANALYTIC, mu=mu, bc_field=L.ADG_FIELD_ABC,
                       device=device, nz=n, z0=-math.pi, Lz=2 * math.pi, bc_z=L.ADG_BC_ANALYTIC)


class Mesh3:
    """A 3D FP64 mesh (adg3_*): state tensor [cells, 5, n, n, n]."""

    def __init__(self, cfg: Mesh3Config):
        self.cfg = cfg
        self._lib = L.lib()
        self.device = torch.device("cuda", cfg.device)
        h = ctypes.c_void_p()
        L.check(self._lib.adg3_create(ctypes.byref(cfg.to_c()), cfg.nz, float(cfg.z0), float(cfg.Lz), cfg.bc_z,
                                      ctypes.byref(h)))
        self.h = h
        self.count = self._lib.adg3_state_count(self.h)

    def close(self):
        if getattr(self, "h", None):
            self._lib.adg3_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        n = self.cfg.n
        return (self.cfg.cells, 5, n, n, n)

    @property
    def time(self):
        return self._lib.adg3_get_time(self.h)

    @time.setter
    def time(self, t):
        L.check(self._lib.adg3_set_time(self.h, float(t)))

    def set_state(self, u: torch.Tensor, stream=None):
        u = u.to(self.device, torch.float64).contiguous()
        L.check(self._lib.adg3_set_state(self.h, ctypes.c_void_p(u.data_ptr()), self.count, 1, _stream_ptr(stream)))

    def get_state(self, stream=None):
        out = torch.empty(self.shape, dtype=torch.float64, device=self.device)
        L.check(self._lib.adg3_get_state(self.h, ctypes.c_void_p(out.data_ptr()), self.count, 1,
                                         _stream_ptr(stream)))
        return out

    def init_scenario(self, kind, A=0.5, a=250.0, xc=500.0, zc=350.0, stream=None):
        sc = L.Scenario(kind=kind, A=A, a=a, xc=xc, zc=zc)
        L.check(self._lib.adg3_init_scenario(self.h, ctypes.byref(sc), _stream_ptr(stream)))

    def step(self, dt, nsteps=1, stream=None):
        L.check(self._lib.adg3_step(self.h, float(dt), int(nsteps), _stream_ptr(stream)))

    def stable_dt(self, cfl, stream=None):
        dt = ctypes.c_double()
        L.check(self._lib.adg3_stable_dt(self.h, float(cfl), ctypes.byref(dt), _stream_ptr(stream)))
        return dt.value
