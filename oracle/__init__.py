"""FP64 CPU oracle of the coupled TSLB + conservative Allen-Cahn step (arXiv 2501.00846).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this package.  The
product path (``paper_2501_00846_b300``) never imports it, and this package imports nothing
from the product except the seeded input generators, which hold none of the method's
arithmetic.

The arithmetic lives in ``tslb_oracle.c`` (plain C, FP64, literal loops).  This module
marshals numpy arrays into it and adds the FP64 diagnostics (sums, centroids) used by the
tests.  Array layout: populations ``g[27, nz, ny, nx]``, velocity ``u[3, nz, ny, nx]``,
scalars ``[nz, ny, nx]``; velocity index i = 9 (cz+1) + 3 (cy+1) + (cx+1).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os

import numpy as np

from .build import build as _build, library_path

Q = 27
CS2 = 1.0 / 3.0

_lib = None


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("wall_z", ctypes.c_int),
        ("rho_l", ctypes.c_double), ("rho_g", ctypes.c_double),
        ("mu_l", ctypes.c_double), ("mu_g", ctypes.c_double),
        ("sigma", ctypes.c_double), ("width", ctypes.c_double), ("mobility", ctypes.c_double),
        ("gravity", ctypes.c_double * 3),
        ("rho_ref", ctypes.c_double),
        ("body", ctypes.c_double * 3),
        ("advect", ctypes.c_int),
        ("literal_weight", ctypes.c_int),
        ("storage16", ctypes.c_int),
    ]


@dataclasses.dataclass
class Params:
    """Physical and grid parameters (lattice units, dx = dt = 1)."""
    nx: int
    ny: int
    nz: int
    wall_z: int = 0
    rho_l: float = 1.0
    rho_g: float = 0.1
    mu_l: float = 0.1
    mu_g: float = 0.01
    sigma: float = 0.01
    width: float = 4.0
    mobility: float = 0.1
    gravity: tuple = (0.0, 0.0, 0.0)
    rho_ref: float = 1.0
    body: tuple = (0.0, 0.0, 0.0)
    advect: int = 0          # 0: flux form div(ubar phi) (reading R4); 1: literal ubar . grad(phi)
    literal_weight: int = 0  # 0: sharpening weight max(phi (1 - phi), 0) (reading R15); 1: phi (1 - phi)
    storage16: int = 0       # 0: FP64 populations; 1 / 2: the library's BF16 / FP16 deviation storage, emulated;
                             # 3 / 4: its BF16 / FP16 deviation-moment storage, emulated

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def n(self):
        return self.nx * self.ny * self.nz

    def c_struct(self) -> _Params:
        p = _Params()
        p.nx, p.ny, p.nz, p.wall_z = self.nx, self.ny, self.nz, self.wall_z
        p.rho_l, p.rho_g, p.mu_l, p.mu_g = self.rho_l, self.rho_g, self.mu_l, self.mu_g
        p.sigma, p.width, p.mobility = self.sigma, self.width, self.mobility
        p.gravity[:] = list(self.gravity)
        p.rho_ref = self.rho_ref
        p.body[:] = list(self.body)
        p.advect = int(self.advect)
        p.literal_weight = int(self.literal_weight)
        p.storage16 = int(self.storage16)
        return p


def lib():
    global _lib
    if _lib is None:
        path = library_path()
        src = os.path.join(os.path.dirname(__file__), "tslb_oracle.c")
        if not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(src):
            _build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(_Params)
        L.oracle_lattice.argtypes = [ctypes.POINTER(ctypes.c_int), dp]
        L.oracle_set_threads.argtypes = [ctypes.c_int]
        L.oracle_get_threads.restype = ctypes.c_int
        for name in ("oracle_grad", "oracle_lap", "oracle_div"):
            getattr(L, name).argtypes = [pp, dp, dp]
        L.oracle_equilibrium.argtypes = [ctypes.c_double, dp, dp]
        L.oracle_guo_source.argtypes = [dp, dp, dp]
        L.oracle_nonequilibrium.argtypes = [dp, dp, dp]
        L.oracle_collide_node.argtypes = [dp, dp, ctypes.c_double, dp, dp, dp]
        L.oracle_force_node.argtypes = [pp, dp, ctypes.c_double, dp, ctypes.c_double, dp, dp]
        L.oracle_ac_update.argtypes = [pp, dp, dp, dp]
        L.oracle_step.argtypes = [pp, dp, dp, dp, dp, dp, dp]
        L.oracle_init.argtypes = [pp, dp, dp, dp, dp, dp, dp]
        L.oracle_run.argtypes = [pp, ctypes.c_int, dp, dp, dp]
        L.oracle_pressure.argtypes = [pp, dp, dp, dp]
        L.oracle_store16_node.argtypes = [ctypes.c_int, dp, dp, dp, dp, dp]
        L.oracle_mom_extract.argtypes = [dp, dp, dp, dp, dp]
        L.oracle_mom_rebuild.argtypes = [ctypes.c_double, dp, dp, dp, dp]
        L.oracle_store_mom16_node.argtypes = [ctypes.c_int, dp, dp, dp, dp]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(lib().oracle_get_threads())


def lattice():
    """Velocities c[27, 3] (int) and weights w[27] as the oracle builds them."""
    c = np.zeros((Q, 3), dtype=np.int32)
    w = np.zeros(Q, dtype=np.float64)
    lib().oracle_lattice(c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _p(w))
    return c.astype(np.int64), w


def grad(P: Params, psi):
    psi = _f64(psi)
    out = np.zeros((3,) + P.shape)
    lib().oracle_grad(ctypes.byref(P.c_struct()), _p(psi), _p(out))
    return out


def lap(P: Params, psi):
    psi = _f64(psi)
    out = np.zeros(P.shape)
    lib().oracle_lap(ctypes.byref(P.c_struct()), _p(psi), _p(out))
    return out


def div(P: Params, V):
    V = _f64(V)
    out = np.zeros(P.shape)
    lib().oracle_div(ctypes.byref(P.c_struct()), _p(V), _p(out))
    return out


def equilibrium(pstar: float, u):
    u = _f64(u)
    out = np.zeros(Q)
    lib().oracle_equilibrium(float(pstar), _p(u), _p(out))
    return out


def guo_source(u, a):
    u, a = _f64(u), _f64(a)
    out = np.zeros(Q)
    lib().oracle_guo_source(_p(u), _p(a), _p(out))
    return out


def nonequilibrium(A, u):
    A, u = _f64(np.asarray(A).reshape(9)), _f64(u)
    out = np.zeros(Q)
    lib().oracle_nonequilibrium(_p(A), _p(u), _p(out))
    return out


def collide_node(f, acc, omega: float):
    """Returns (g[27], u[3], A[3,3]) for one node."""
    f, acc = _f64(f), _f64(acc)
    g = np.zeros(Q)
    u = np.zeros(3)
    A = np.zeros(9)
    lib().oracle_collide_node(_p(f), _p(acc), float(omega), _p(g), _p(u), _p(A))
    return g, u, A.reshape(3, 3)


def store16_node(fmt: int, g, u):
    """The library's 16-bit storage of one node (fmt 1 BF16, 2 FP16): the stored P, the rounded
    deviations hr [27] and the populations w_i (P + e_i(u) + hr_i) they represent."""
    g, u = _f64(g), _f64(u)
    P_out = ctypes.c_double()
    hr, gout = np.zeros(Q), np.zeros(Q)
    lib().oracle_store16_node(int(fmt), _p(g), _p(u), ctypes.byref(P_out), _p(hr), _p(gout))
    return P_out.value, hr, gout


def mom_extract(g, u):
    """(p*, a[3], B[3,3]) of one node's populations g with velocity u (the moment storage's set)."""
    g, u = _f64(g), _f64(u)
    ps = ctypes.c_double()
    a, B = np.zeros(3), np.zeros(9)
    lib().oracle_mom_extract(_p(g), _p(u), ctypes.byref(ps), _p(a), _p(B))
    return ps.value, a, B.reshape(3, 3)


def mom_rebuild(ps: float, u, a, B):
    """The populations [27] of the moment set (p*, u, a, B)."""
    u, a, B = _f64(u), _f64(a), _f64(np.asarray(B).reshape(9))
    g = np.zeros(Q)
    lib().oracle_mom_rebuild(float(ps), _p(u), _p(a), _p(B), _p(g))
    return g


def store_mom16_node(fmt: int, g, u):
    """The library's 16-bit moment storage of one node (fmt 1 BF16, 2 FP16): the rounded
    (a_x, a_y, a_z, B_xx, B_yy, B_zz, B_xy, B_xz, B_yz) and the populations they represent."""
    g, u = _f64(g), _f64(u)
    ab, gout = np.zeros(9), np.zeros(Q)
    lib().oracle_store_mom16_node(int(fmt), _p(g), _p(u), _p(ab), _p(gout))
    return ab, gout


def force_node(P: Params, f, phi: float, gphi, lphi: float, ubar):
    f, gphi, ubar = _f64(f), _f64(gphi), _f64(ubar)
    F = np.zeros(3)
    lib().oracle_force_node(ctypes.byref(P.c_struct()), _p(f), float(phi), _p(gphi), float(lphi),
                            _p(ubar), _p(F))
    return F


def ac_update(P: Params, phi, ubar):
    phi, ubar = _f64(phi), _f64(ubar)
    out = np.zeros(P.shape)
    lib().oracle_ac_update(ctypes.byref(P.c_struct()), _p(phi), _p(ubar), _p(out))
    return out


@dataclasses.dataclass
class State:
    """(g, phi, ubar) after a step; see the state convention in tslb_oracle.c."""
    g: np.ndarray
    phi: np.ndarray
    u: np.ndarray
    step: int = 0

    def copy(self):
        return State(self.g.copy(), self.phi.copy(), self.u.copy(), self.step)


def init(P: Params, phi0, u0, pstar0=None) -> State:
    phi0, u0 = _f64(phi0), _f64(u0)
    g = np.zeros((Q,) + P.shape)
    phi = np.zeros(P.shape)
    u = np.zeros((3,) + P.shape)
    ps_arr = _f64(pstar0) if pstar0 is not None else None
    ps = _p(ps_arr) if ps_arr is not None else None
    lib().oracle_init(ctypes.byref(P.c_struct()), _p(phi0), _p(u0), ps, _p(g), _p(phi), _p(u))
    return State(g, phi, u, 0)


def step(P: Params, s: State) -> State:
    out = State(np.zeros_like(s.g), np.zeros_like(s.phi), np.zeros_like(s.u), s.step + 1)
    lib().oracle_step(ctypes.byref(P.c_struct()), _p(s.g), _p(s.phi), _p(s.u),
                      _p(out.g), _p(out.phi), _p(out.u))
    return out


def run(P: Params, s: State, nsteps: int) -> State:
    out = s.copy()
    lib().oracle_run(ctypes.byref(P.c_struct()), int(nsteps), _p(out.g), _p(out.phi), _p(out.u))
    out.step = s.step + nsteps
    return out


def pressure(P: Params, s: State):
    """p = p* rho cs^2, p* = sum_i g_i."""
    out = np.zeros(P.shape)
    lib().oracle_pressure(ctypes.byref(P.c_struct()), _p(s.g), _p(s.phi), _p(out))
    return out


def pstar(s: State):
    return s.g.sum(axis=0)


def density(P: Params, phi):
    return P.rho_l * phi + (1.0 - phi) * P.rho_g


def observables(P: Params, s: State) -> dict:
    """FP64 integral diagnostics of a state (the quantities the device reduction reports)."""
    phi = s.phi
    rho = density(P, phi)
    ps = pstar(s)
    p = ps * rho * CS2
    z, y, x = np.meshgrid(np.arange(P.nz), np.arange(P.ny), np.arange(P.nx), indexing="ij")
    coords = (x, y, z)
    sphi = phi.sum()
    sgas = (1.0 - phi).sum()
    liq = phi > 0.999
    gas = phi < 0.001
    umag = np.sqrt((s.u ** 2).sum(axis=0))
    return {
        "step": s.step,
        "sum_phi": sphi,
        "mass": rho.sum(),
        "sum_pstar": ps.sum(),
        "momentum": [float((rho * s.u[a]).sum()) for a in range(3)],
        "centroid_liq": [float((phi * coords[a]).sum() / sphi) for a in range(3)],
        "centroid_gas": [float(((1.0 - phi) * coords[a]).sum() / sgas) for a in range(3)],
        "vel_liq": [float((phi * s.u[a]).sum() / sphi) for a in range(3)],
        "vel_gas": [float(((1.0 - phi) * s.u[a]).sum() / sgas) for a in range(3)],
        "p_liq": float(p[liq].mean()) if liq.any() else float("nan"),
        "p_gas": float(p[gas].mean()) if gas.any() else float("nan"),
        "umax": float(umag.max()),
        "phi_min": float(phi.min()),
        "phi_max": float(phi.max()),
        "n_nonfinite": int((~np.isfinite(s.g)).sum() + (~np.isfinite(phi)).sum() + (~np.isfinite(s.u)).sum()),
    }
