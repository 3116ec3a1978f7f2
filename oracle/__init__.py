"""CPU oracle for the linear MHS multigrid path (test infrastructure only).

Only the tests, the smoke check and the CPU-baseline leg of the benchmark
use this package.  It shares no code with the GPU library and never imports
it.  Arrays are float64 numpy arrays in [nz][ny][nx] order (x fastest).

The numerical work lives in ``mhs_oracle.c`` (plain C, FP64, optional OpenMP
over z-planes), compiled on first use by :func:`build`.  ``exact.py`` holds two
further, independent solvers (separable sine-transform + tridiagonal, and a
direct sparse solve of a Kronecker-assembled matrix) used to pin the
multigrid oracle.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mhs_oracle.c")
_LIB = os.path.join(_HERE, "libmhs_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (-O2, OpenMP) into oracle/libmhs_oracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Problem(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("Lx", ctypes.c_double), ("Ly", ctypes.c_double), ("Lz", ctypes.c_double),
                ("alpha", ctypes.c_double), ("xi_kind", ctypes.c_int),
                ("xi_a", ctypes.c_double), ("xi_kappa", ctypes.c_double),
                ("xi_b", ctypes.c_double), ("xi_omega", ctypes.c_double),
                ("g", ctypes.c_double), ("mu0", ctypes.c_double), ("T_cor", ctypes.c_double),
                ("z1", ctypes.c_double), ("z2", ctypes.c_double)]


class Info(ctypes.Structure):
    _fields_ = [("cycles_2d", ctypes.c_int), ("cycles_3d", ctypes.c_int),
                ("rel_res_2d", ctypes.c_double), ("rel_res_3d", ctypes.c_double),
                ("conv_factor_3d", ctypes.c_double)]


_D = ctypes.POINTER(ctypes.c_double)
_PP = ctypes.POINTER(Problem)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # MHS_ORACLE_LIB points the oracle at another build of mhs_oracle.c
            # (the mutation tests compile deliberately broken copies).
            lib = ctypes.CDLL(os.environ.get("MHS_ORACLE_LIB") or build())
            sig = {
                "orc_set_threads": (None, [ctypes.c_int]),
                "orc_max_threads": (ctypes.c_int, []),
                "orc_coeffs": (None, [_PP, _D, _D, _D, _D]),
                "orc_residual3d": (None, [_PP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D, _D]),
                "orc_rbgs3d": (None, [_PP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D, ctypes.c_int]),
                "orc_rbgs3d_colour": (None, [_PP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D, ctypes.c_int]),
                "orc_zline3d": (None, [_PP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D, ctypes.c_int]),
                "orc_zline3d_colour": (None, [_PP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D, ctypes.c_int]),
                "orc_residual2d": (None, [_PP, ctypes.c_int, ctypes.c_int, _D, _D, _D]),
                "orc_rbgs2d": (None, [_PP, ctypes.c_int, ctypes.c_int, _D, _D, ctypes.c_int]),
                "orc_restrict": (None, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D]),
                "orc_prolong_add": (None, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D]),
                "orc_solve2d": (ctypes.c_int, [_PP, _D, _D, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_int, _D, _D]),
                "orc_solve3d": (ctypes.c_int, [_PP, _D, _D, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_int, _D, _D, _D]),
                "orc_solve3d_s": (ctypes.c_int, [_PP, _D, _D, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_int, ctypes.c_int, _D, _D, _D]),
                "orc_solve": (ctypes.c_int, [_PP, _D, _D, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_int, ctypes.POINTER(Info)]),
                "orc_solve_s": (ctypes.c_int, [_PP, _D, _D, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                               ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Info)]),
                "orc_num_levels": (ctypes.c_int, [_PP, ctypes.c_int]),
                "orc_vcycle": (None, [_PP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D,
                                      ctypes.c_int, ctypes.c_int]),
                "orc_vcycle_s": (None, [_PP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int]),
                "orc_vcycle_x": (None, [_PP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
                "orc_fields": (None, [_PP, _D, _D, _D, _D, _D, _D, ctypes.c_int]),
                "orc_profiles": (None, [_PP, _D, _D, _D, _D, _D]),
                "orc_current": (None, [_PP, _D, _D, _D, _D, _D, _D, _D, _D]),
                "orc_trace": (None, [_PP, _D, _D, _D, _D, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                     ctypes.c_double, _D, ctypes.POINTER(ctypes.c_int)]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _prob(pr) -> Problem:
    if isinstance(pr, Problem):
        return pr
    return Problem(**{k: pr[k] for k, _ in Problem._fields_})


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def max_threads() -> int:
    return int(_load().orc_max_threads())


def coeffs(pr):
    """Per-plane (cx, cy, diag) arrays and the scalar cz of the 3D operator."""
    p = _prob(pr)
    cx, cy, dg = (np.zeros(p.nz) for _ in range(3))
    cz = ctypes.c_double()
    _load().orc_coeffs(ctypes.byref(p), _ptr(cx), _ptr(cy), ctypes.byref(cz), _ptr(dg))
    return cx, cy, cz.value, dg


def profiles(pr):
    """xi, dxi/dz, p_b, rho_b, T_b on the node heights of the problem."""
    p = _prob(pr)
    out = [np.zeros(p.nz) for _ in range(5)]
    _load().orc_profiles(ctypes.byref(p), *[_ptr(a) for a in out])
    return dict(zip(["xi", "dxi", "pb", "rhob", "Tb"], out))


def residual3d(pr, u, f=None):
    u = _f64(u); f = _f64(f)
    nz, ny, nx = u.shape
    r = np.zeros_like(u)
    p = _prob(pr)
    _load().orc_residual3d(ctypes.byref(p), nx, ny, nz, _ptr(u), _ptr(f), _ptr(r))
    return r


def rbgs3d(pr, u, f=None, sweeps=1):
    u = _f64(u).copy(); f = _f64(f)
    nz, ny, nx = u.shape
    p = _prob(pr)
    _load().orc_rbgs3d(ctypes.byref(p), nx, ny, nz, _ptr(u), _ptr(f), int(sweeps))
    return u


def rbgs3d_colour(pr, u, f=None, colour=0):
    u = _f64(u).copy(); f = _f64(f)
    nz, ny, nx = u.shape
    p = _prob(pr)
    _load().orc_rbgs3d_colour(ctypes.byref(p), nx, ny, nz, _ptr(u), _ptr(f), int(colour))
    return u


def zline3d(pr, u, f=None, sweeps=1):
    """Zebra z-line Gauss-Seidel sweeps (columns with i + j even, then odd,
    each solved exactly along z); returns the new u."""
    u = _f64(u).copy(); f = _f64(f)
    nz, ny, nx = u.shape
    p = _prob(pr)
    _load().orc_zline3d(ctypes.byref(p), nx, ny, nz, _ptr(u), _ptr(f), int(sweeps))
    return u


def zline3d_colour(pr, u, f=None, colour=0):
    u = _f64(u).copy(); f = _f64(f)
    nz, ny, nx = u.shape
    p = _prob(pr)
    _load().orc_zline3d_colour(ctypes.byref(p), nx, ny, nz, _ptr(u), _ptr(f), int(colour))
    return u


SMOOTHERS = {"point": 0, "zline": 1}


def residual2d(pr, u, f=None):
    u = _f64(u); f = _f64(f)
    ny, nx = u.shape
    r = np.zeros_like(u)
    p = _prob(pr)
    _load().orc_residual2d(ctypes.byref(p), nx, ny, _ptr(u), _ptr(f), _ptr(r))
    return r


def rbgs2d(pr, u, f=None, sweeps=1):
    u = _f64(u).copy(); f = _f64(f)
    ny, nx = u.shape
    p = _prob(pr)
    _load().orc_rbgs2d(ctypes.byref(p), nx, ny, _ptr(u), _ptr(f), int(sweeps))
    return u


def coarse_shape(shape):
    return tuple((n - 1) // 2 + 1 for n in shape)


def restrict(rf):
    """Full-weighting restriction of a 2D [ny][nx] or 3D [nz][ny][nx] array."""
    rf = _f64(rf)
    if rf.ndim == 2:
        ny, nx = rf.shape; nz = 1
        fc = np.zeros(coarse_shape(rf.shape))
    else:
        nz, ny, nx = rf.shape
        fc = np.zeros(coarse_shape(rf.shape))
    _load().orc_restrict(nx, ny, nz, _ptr(rf), _ptr(fc))
    return fc


def prolong_add(ec, uf):
    """uf + I ec ((bi/tri)linear interpolation added at fine interior nodes)."""
    ec = _f64(ec); uf = _f64(uf).copy()
    if uf.ndim == 2:
        ny, nx = uf.shape; nz = 1
    else:
        nz, ny, nx = uf.shape
    assert ec.shape == coarse_shape(uf.shape)
    _load().orc_prolong_add(nx, ny, nz, _ptr(ec), _ptr(uf))
    return uf


def solve2d(pr, bz, tol=1e-12, max_cycles=200, nu1=2, nu2=2, P0=None):
    """Multigrid solve of eq. (lower_bound).  Returns (P0, cycles, rel, history)."""
    p = _prob(pr)
    bz = _f64(bz)
    P0 = np.zeros((p.ny, p.nx)) if P0 is None else _f64(P0).copy()
    rel = ctypes.c_double()
    hist = np.zeros(max_cycles + 1)
    c = _load().orc_solve2d(ctypes.byref(p), _ptr(bz), _ptr(P0), tol, max_cycles, nu1, nu2,
                            ctypes.byref(rel), _ptr(hist))
    return P0, c, rel.value, hist[: c + 1]


def solve3d(pr, P, f=None, tol=1e-12, max_cycles=200, nu1=2, nu2=2, smoother="point"):
    """Multigrid solve of eq. (scalar_pot) with Dirichlet data in P's boundary
    entries and optional right-hand side f.  Returns (P, cycles, rel, history, conv)."""
    p = _prob(pr)
    P = _f64(P).copy(); f = _f64(f)
    rel = ctypes.c_double(); conv = ctypes.c_double()
    hist = np.zeros(max_cycles + 1)
    c = _load().orc_solve3d_s(ctypes.byref(p), _ptr(P), _ptr(f), tol, max_cycles, nu1, nu2, SMOOTHERS[smoother],
                              ctypes.byref(rel), _ptr(hist), ctypes.byref(conv))
    return P, c, rel.value, hist[: c + 1], conv.value


def solve(pr, bz, tol2d=1e-12, tol3d=1e-12, max_cycles=200, nu1=2, nu2=2, smoother="point"):
    """The three-step procedure of Sect. 2.2.  Returns (P, info dict)."""
    p = _prob(pr)
    bz = _f64(bz)
    assert bz.shape == (p.ny, p.nx)
    P = np.zeros((p.nz, p.ny, p.nx))
    info = Info()
    status = _load().orc_solve_s(ctypes.byref(p), _ptr(bz), _ptr(P), tol2d, tol3d, max_cycles, nu1, nu2,
                                 SMOOTHERS[smoother], ctypes.byref(info))
    return P, dict(status=status, cycles_2d=info.cycles_2d, cycles_3d=info.cycles_3d,
                   rel_res_2d=info.rel_res_2d, rel_res_3d=info.rel_res_3d,
                   conv_factor_3d=info.conv_factor_3d)


def vcycle(pr, u, f=None, nu1=2, nu2=2, smoother="point", exact_level=-1):
    """One V-cycle on the grid of u (2D [ny][nx] or 3D [nz][ny][nx]); returns the new u.

    exact_level >= 1: the cycle stops at that level and solves its
    coarse-grid system to rounding (the coarse-grid solve of multigrid
    theory) instead of descending further."""
    u = _f64(u).copy(); f = _f64(f)
    p = _prob(pr)
    sm = SMOOTHERS[smoother]
    if u.ndim == 2:
        ny, nx = u.shape
        _load().orc_vcycle_x(ctypes.byref(p), 2, nx, ny, 1, _ptr(u), _ptr(f), nu1, nu2, sm, exact_level)
    else:
        nz, ny, nx = u.shape
        _load().orc_vcycle_x(ctypes.byref(p), 3, nx, ny, nz, _ptr(u), _ptr(f), nu1, nu2, sm, exact_level)
    return u


def num_levels(pr, dim=3) -> int:
    p = _prob(pr)
    return int(_load().orc_num_levels(ctypes.byref(p), dim))


def fields(pr, P, bz_mode=0):
    """B_x, B_y, B_z, p, rho from P (Sect. 2.2, eqs. pressure and density)."""
    p = _prob(pr)
    P = _f64(P)
    out = [np.zeros_like(P) for _ in range(5)]
    _load().orc_fields(ctypes.byref(p), _ptr(P), *[_ptr(a) for a in out], int(bz_mode))
    return dict(zip(["Bx", "By", "Bz", "p", "rho"], out))


def current(pr, Bx, By, Bz):
    """j = curl B / mu0 (the field-recovery difference operators), |j| and |B|."""
    p = _prob(pr)
    Bx, By, Bz = _f64(Bx), _f64(By), _f64(Bz)
    out = [np.zeros_like(Bx) for _ in range(5)]
    _load().orc_current(ctypes.byref(p), _ptr(Bx), _ptr(By), _ptr(Bz), *[_ptr(a) for a in out])
    return dict(zip(["jx", "jy", "jz", "jmag", "bmag"], out))


def trace(pr, Bx, By, Bz, seeds, ds, max_steps, direction=1):
    """RK4 field lines along direction * B/|B| from seeds [n][3] (x, y, z).
    Returns (points [n][max_steps+1][3], lengths [n])."""
    p = _prob(pr)
    Bx, By, Bz = _f64(Bx), _f64(By), _f64(Bz)
    seeds = np.ascontiguousarray(seeds, dtype=np.float64).reshape(-1, 3)
    n = seeds.shape[0]
    pts = np.zeros((n, max_steps + 1, 3))
    lens = np.zeros(n, dtype=np.int32)
    _load().orc_trace(ctypes.byref(p), _ptr(Bx), _ptr(By), _ptr(Bz), _ptr(seeds), n, float(ds), int(max_steps),
                      float(direction), _ptr(pts), lens.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return pts, lens
