"""ctypes binding of libmhs (include/mhs.h): argument marshalling only.

Every function of the C ABI is exposed under its own name.  Array arguments
may be torch tensors (device or host, float64, contiguous) or numpy float64
arrays; their data pointers are passed straight through.  Every step of the
solver runs in the library's CUDA kernels; there is no fallback: if the
library is missing or cannot be loaded, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmhs.so")

MHS_OK = 0
STATUS_NAMES = ["MHS_OK", "MHS_ERR_INVALID_ARG", "MHS_ERR_NOT_ELLIPTIC", "MHS_ERR_OUT_OF_MEMORY", "MHS_ERR_CUDA",
                "MHS_ERR_NO_CONVERGENCE", "MHS_ERR_NONFINITE", "MHS_ERR_BAD_STATE", "MHS_ERR_TIMEOUT",
                "MHS_ERR_REJECTED"]
(MHS_ERR_INVALID_ARG, MHS_ERR_NOT_ELLIPTIC, MHS_ERR_OUT_OF_MEMORY, MHS_ERR_CUDA, MHS_ERR_NO_CONVERGENCE,
 MHS_ERR_NONFINITE, MHS_ERR_BAD_STATE, MHS_ERR_TIMEOUT, MHS_ERR_REJECTED) = range(1, 10)
MHS_XI_NONE, MHS_XI_EXP, MHS_XI_EXP_SIN = 0, 1, 2
MHS_FP64, MHS_MIXED = 0, 1
MHS_FLAG_WARM, MHS_FLAG_BZ_MIMETIC, MHS_FLAG_NO_GRAPH, MHS_FLAG_FUSED_SWEEP64, MHS_FLAG_NO_TMA, MHS_FLAG_NO_FMG = \
    1, 2, 4, 8, 16, 32
MHS_FLAG_ZLINE, MHS_FLAG_POINT, MHS_FLAG_SEPARABLE, MHS_FLAG_LOWER_FP64 = 64, 128, 256, 512
MHS_FLAG_STAGED_TRANSFORMS = 1024
MHS_FIELD_U, MHS_FIELD_F, MHS_FIELD_R = 0, 1, 2
(MHS_OP_SMOOTH, MHS_OP_RESIDUAL, MHS_OP_RESTRICT, MHS_OP_PROLONG, MHS_OP_COARSE, MHS_OP_VCYCLE, MHS_OP_EXACT,
 MHS_OP_RESID_RESTRICT, MHS_OP_RESTRICT_RED) = range(9)


class XiParams(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("a", ctypes.c_double), ("kappa", ctypes.c_double),
                ("b", ctypes.c_double), ("omega", ctypes.c_double)]


class AtmosParams(ctypes.Structure):
    _fields_ = [("g", ctypes.c_double), ("mu0", ctypes.c_double), ("T_cor", ctypes.c_double),
                ("z1", ctypes.c_double), ("z2", ctypes.c_double)]


class SolverOpts(ctypes.Structure):
    _fields_ = [("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("max_cycles", ctypes.c_int),
                ("inner_cycles", ctypes.c_int), ("flags", ctypes.c_int), ("cut64", ctypes.c_int),
                ("cut32", ctypes.c_int), ("fused_min", ctypes.c_int), ("sep_coarse", ctypes.c_int),
                ("tile", ctypes.c_int),
                ("tma_rows", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("cycles_2d", ctypes.c_int), ("cycles_3d", ctypes.c_int), ("rel_res_2d", ctypes.c_double),
                ("rel_res_3d", ctypes.c_double), ("conv_factor", ctypes.c_double), ("ms", ctypes.c_double),
                ("outer_iters_2d", ctypes.c_int), ("outer_iters_3d", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TuneResult(ctypes.Structure):
    _fields_ = [("opts", SolverOpts), ("ms", ctypes.c_double), ("ms_start", ctypes.c_double),
                ("candidates", ctypes.c_int), ("aniso_class", ctypes.c_int)]

    def as_dict(self):
        o = self.opts
        return {"opts": {k: getattr(o, k) for k, _ in SolverOpts._fields_}, "ms": self.ms,
                "ms_start": self.ms_start, "candidates": self.candidates, "aniso_class": self.aniso_class}


class Request(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("Lx", ctypes.c_double), ("Ly", ctypes.c_double), ("Lz", ctypes.c_double),
                ("alpha", ctypes.c_double), ("xi", XiParams), ("atm", AtmosParams),
                ("tol", ctypes.c_double), ("mode", ctypes.c_int), ("bz", ctypes.c_void_p),
                ("phi", ctypes.c_void_p), ("Bx", ctypes.c_void_p), ("By", ctypes.c_void_p),
                ("Bz", ctypes.c_void_p), ("p", ctypes.c_void_p), ("rho", ctypes.c_void_p)]


class ServerStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_longlong), ("rejected", ctypes.c_longlong), ("queued", ctypes.c_longlong),
                ("running", ctypes.c_longlong), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("mean_ms", ctypes.c_double), ("solves_per_s", ctypes.c_double), ("device_bytes", ctypes.c_size_t),
                ("resident_hierarchies", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class MhsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {msg}")


_H = ctypes.c_void_p
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_SIGS = {
    "mhs_create": [_I, _I, _I, _D, _D, _D, _D, ctypes.POINTER(XiParams), ctypes.POINTER(AtmosParams),
                   ctypes.POINTER(_H)],
    "mhs_destroy": [_H],
    "mhs_set_stream": [_H, _P],
    "mhs_set_options": [_H, ctypes.POINTER(SolverOpts)],
    "mhs_set_params": [_H, _D, ctypes.POINTER(XiParams), ctypes.POINTER(AtmosParams)],
    "mhs_set_lower_bz": [_H, _P],
    "mhs_solve": [_H, _D, _I, ctypes.POINTER(SolveInfo)],
    "mhs_batch_solve": [ctypes.POINTER(_H), _I, _D, _I, ctypes.POINTER(SolveInfo), ctypes.POINTER(_I)],
    "mhs_group_create": [ctypes.POINTER(_H), _I, _I, ctypes.c_size_t, _I, ctypes.POINTER(_H)],
    "mhs_group_solve": [_H, _D, ctypes.POINTER(SolveInfo), ctypes.POINTER(_I)],
    "mhs_group_destroy": [_H],
    "mhs_group_set_eager": [_H, _I],
    "mhs_autotune": [_H, _D, _I, _I, ctypes.POINTER(TuneResult)],
    "mhs_tune_lookup": [_H, _I, ctypes.POINTER(SolverOpts), ctypes.POINTER(_I)],
    "mhs_tune_clear": [],
    "mhs_get_phi": [_H, _P],
    "mhs_current": [_H, _P, _P, _P, _P, _P],
    "mhs_trace": [_H, _P, _I, _D, _I, _I, _P, _P],
    "mhs_trace_field": [_I, _I, _I, _D, _D, _D, _P, _P, _P, _P, _I, _D, _I, _I, _P, _P, _P],
    "mhs_fields": [_H, _P, _P, _P, _P, _P],
    "mhs_num_levels": [_H, _I, ctypes.POINTER(_I)],
    "mhs_level_shape": [_H, _I, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)],
    "mhs_level_write": [_H, _I, _I, _I, _I, _P],
    "mhs_level_read": [_H, _I, _I, _I, _I, _P],
    "mhs_level_op": [_H, _I, _I, _I, _I],
    "mhs_set_kernel_timing": [_H, _I],
    "mhs_kernel_timing": [_H, _I, ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(_D),
                          ctypes.POINTER(_D)],
    "mhs_kernel_timing_finest": [_H, _I, ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(_D),
                                 ctypes.POINTER(_D)],
    "mhs_kernel_timing_reset": [_H],
    "mhs_kernel_kind_name": [_I],
    "mhs_kernel_launches": [],
    "mhs_probe_fma_rate": [_I, _P, ctypes.POINTER(_D)],
    "mhs_interior_residual_noalloc": [_I, _I, _I, _D, _D, _D, _D, ctypes.POINTER(XiParams), _P, _P, _P],
    "mhs_server_create": [ctypes.c_size_t, _I, ctypes.POINTER(_H)],
    "mhs_server_submit": [_H, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_longlong)],
    "mhs_server_poll": [_H, ctypes.c_longlong, ctypes.POINTER(_I), ctypes.POINTER(SolveInfo), ctypes.POINTER(_I),
                        ctypes.POINTER(_D)],
    "mhs_server_wait": [_H, ctypes.c_longlong, _D, ctypes.POINTER(SolveInfo), ctypes.POINTER(_I), ctypes.POINTER(_D)],
    "mhs_server_stats": [_H, ctypes.POINTER(ServerStats)],
    "mhs_server_destroy": [_H],
    "mhs_status_string": [_I],
    "mhs_last_error": [],
    "mhs_version": [],
}


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libmhs not built ({path} missing): run __graft_entry__.build() "
                          "or python paper_1307_6720_gb300/build.py")
    lib = ctypes.CDLL(path)
    for name, args in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        if name in ("mhs_destroy", "mhs_server_destroy", "mhs_tune_clear", "mhs_group_destroy"):
            fn.restype = None
        elif name in ("mhs_status_string", "mhs_last_error", "mhs_version", "mhs_kernel_kind_name"):
            fn.restype = ctypes.c_char_p
        elif name == "mhs_kernel_launches":
            fn.restype = ctypes.c_longlong
        else:
            fn.restype = ctypes.c_int
    return lib


LIB = load()


def _check(status: int) -> None:
    if status != MHS_OK:
        raise MhsError(status, LIB.mhs_last_error().decode())


def ptr(a) -> int | None:
    """Data pointer of a torch tensor or numpy array (None passes NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        import torch
        assert a.dtype == torch.float64 and a.is_contiguous(), "expected a contiguous float64 tensor"
        return a.data_ptr()
    import numpy as np
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "expected a contiguous float64 array"
    return a.ctypes.data


def iptr(a) -> int | None:
    """Data pointer of a contiguous int32 torch tensor or numpy array."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        import torch
        assert a.dtype == torch.int32 and a.is_contiguous(), "expected a contiguous int32 tensor"
        return a.data_ptr()
    import numpy as np
    assert a.dtype == np.int32 and a.flags["C_CONTIGUOUS"], "expected a contiguous int32 array"
    return a.ctypes.data


def _stream_ptr(stream):
    if stream is not None and hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return stream


def xi_params(kind=MHS_XI_NONE, a=0.0, kappa=0.0, b=0.0, omega=0.0) -> XiParams:
    return XiParams(kind, a, kappa, b, omega)


def atmos_params(g=1.0, mu0=0.5, T_cor=150.0, z1=5.0, z2=10.0) -> AtmosParams:
    return AtmosParams(g, mu0, T_cor, z1, z2)


# ---- one wrapper per C entry point, same names ----

def mhs_create(nx, ny, nz, Lx, Ly, Lz, alpha, xi: XiParams | None = None, atm: AtmosParams | None = None) -> int:
    h = _H()
    _check(LIB.mhs_create(nx, ny, nz, Lx, Ly, Lz, alpha, ctypes.byref(xi) if xi is not None else None,
                          ctypes.byref(atm) if atm is not None else None, ctypes.byref(h)))
    return h.value


def mhs_destroy(h) -> None:
    LIB.mhs_destroy(h)


def mhs_set_stream(h, stream) -> None:
    """stream: a torch.cuda.Stream, an integer cudaStream_t, or None (legacy default)."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    _check(LIB.mhs_set_stream(h, stream))


def mhs_set_options(h, nu1=0, nu2=0, max_cycles=0, inner_cycles=0, flags=0, cut64=0, cut32=0, fused_min=0,
                    sep_coarse=0, tile=0, tma_rows=0) -> None:
    o = SolverOpts(nu1, nu2, max_cycles, inner_cycles, flags, cut64, cut32, fused_min, sep_coarse, tile, tma_rows)
    _check(LIB.mhs_set_options(h, ctypes.byref(o)))


def mhs_set_params(h, alpha, xi: XiParams | None = None, atm: AtmosParams | None = None) -> None:
    _check(LIB.mhs_set_params(h, alpha, ctypes.byref(xi) if xi is not None else None,
                              ctypes.byref(atm) if atm is not None else None))


def mhs_set_lower_bz(h, bz) -> None:
    _check(LIB.mhs_set_lower_bz(h, ptr(bz)))


def mhs_solve(h, tol, mode=MHS_FP64) -> dict:
    info = SolveInfo()
    st = LIB.mhs_solve(h, tol, mode, ctypes.byref(info))
    if st != MHS_OK:
        err = MhsError(st, LIB.mhs_last_error().decode())
        err.info = info.as_dict()
        raise err
    return info.as_dict()


def mhs_batch_solve(handles, tol, mode=MHS_FP64):
    """Solve several handles concurrently; returns (per-instance info dicts, per-instance statuses)."""
    n = len(handles)
    arr = (_H * n)(*handles)
    infos = (SolveInfo * n)()
    sts = (_I * n)()
    st = LIB.mhs_batch_solve(arr, n, tol, mode, infos, sts)
    if st not in (MHS_OK, MHS_ERR_NO_CONVERGENCE, MHS_ERR_NONFINITE):
        _check(st)
    return [i.as_dict() for i in infos], list(sts)


def mhs_group_create(handles, mode=MHS_MIXED, part_bytes=0, nstreams=0) -> int:
    """A grouped solver over the handles: parts of at most part_bytes cycle working set (0: half the
    L2; ctypes.c_size_t(-1).value: one part), one launch per operation and level per part, parts
    launched round-robin on nstreams streams (0: 16)."""
    n = len(handles)
    arr = (_H * n)(*handles)
    g = _H()
    _check(LIB.mhs_group_create(arr, n, mode, part_bytes, nstreams, ctypes.byref(g)))
    return g.value


def mhs_group_solve(g, n, tol):
    """Solve the group's n instances; returns (per-instance info dicts, per-instance statuses)."""
    infos = (SolveInfo * n)()
    sts = (_I * n)()
    st = LIB.mhs_group_solve(g, tol, infos, sts)
    if st not in (MHS_OK, MHS_ERR_NO_CONVERGENCE, MHS_ERR_NONFINITE):
        _check(st)
    return [i.as_dict() for i in infos], list(sts)


def mhs_group_set_eager(g, eager=True) -> None:
    _check(LIB.mhs_group_set_eager(g, 1 if eager else 0))


def mhs_group_destroy(g) -> None:
    LIB.mhs_group_destroy(g)


def mhs_autotune(h, tol, mode=MHS_FP64, repeats=2) -> dict:
    """Time candidate option sets on h's problem, apply and store the fastest."""
    r = TuneResult()
    _check(LIB.mhs_autotune(h, tol, mode, repeats, ctypes.byref(r)))
    return r.as_dict()


def mhs_tune_lookup(h, mode=MHS_FP64):
    """Stored options (a dict of SolverOpts fields) for h's problem class, or None."""
    o = SolverOpts()
    found = _I()
    _check(LIB.mhs_tune_lookup(h, mode, ctypes.byref(o), ctypes.byref(found)))
    return {k: getattr(o, k) for k, _ in SolverOpts._fields_} if found.value else None


def mhs_tune_clear() -> None:
    LIB.mhs_tune_clear()


def mhs_get_phi(h, phi) -> None:
    _check(LIB.mhs_get_phi(h, ptr(phi)))


def mhs_fields(h, Bx=None, By=None, Bz=None, p=None, rho=None) -> None:
    _check(LIB.mhs_fields(h, ptr(Bx), ptr(By), ptr(Bz), ptr(p), ptr(rho)))


def mhs_current(h, jx=None, jy=None, jz=None, jmag=None, bmag=None) -> None:
    _check(LIB.mhs_current(h, ptr(jx), ptr(jy), ptr(jz), ptr(jmag), ptr(bmag)))


def mhs_trace(h, seeds, ds, max_steps, direction=1, points=None, lengths=None):
    """Field lines from seeds [n][3]; returns (points [n][max_steps+1][3], lengths [n]).
    points/lengths may be given (host numpy or device torch buffers)."""
    import numpy as np
    n = int(seeds.shape[0])
    if points is None:
        points = np.zeros((n, max_steps + 1, 3))
    if lengths is None:
        lengths = np.zeros(n, dtype=np.int32)
    _check(LIB.mhs_trace(h, ptr(seeds), n, float(ds), int(max_steps), int(direction), ptr(points), iptr(lengths)))
    return points, lengths


def mhs_trace_field(shape, box, Bx, By, Bz, seeds, ds, max_steps, direction=1, points=None, lengths=None,
                    stream=None):
    """The tracer on device arrays Bx, By, Bz [nz][ny][nx] of the box (Lx, Ly, Lz)."""
    nz, ny, nx = shape
    n = int(seeds.shape[0])
    _check(LIB.mhs_trace_field(nx, ny, nz, box[0], box[1], box[2], ptr(Bx), ptr(By), ptr(Bz), ptr(seeds), n,
                               float(ds), int(max_steps), int(direction), ptr(points), iptr(lengths),
                               _stream_ptr(stream)))
    return points, lengths


def mhs_num_levels(h, dim=3) -> int:
    n = _I()
    _check(LIB.mhs_num_levels(h, dim, ctypes.byref(n)))
    return n.value


def mhs_level_shape(h, dim, level):
    nx, ny, nz = _I(), _I(), _I()
    _check(LIB.mhs_level_shape(h, dim, level, ctypes.byref(nx), ctypes.byref(ny), ctypes.byref(nz)))
    return nx.value, ny.value, nz.value


def mhs_level_write(h, dim, level, field, prec, src) -> None:
    _check(LIB.mhs_level_write(h, dim, level, field, prec, ptr(src)))


def mhs_level_read(h, dim, level, field, prec, dst) -> None:
    _check(LIB.mhs_level_read(h, dim, level, field, prec, ptr(dst)))


def mhs_level_op(h, dim, level, op, prec) -> None:
    _check(LIB.mhs_level_op(h, dim, level, op, prec))


MHS_KT_COUNT = 15


def mhs_set_kernel_timing(h, enable: bool) -> None:
    _check(LIB.mhs_set_kernel_timing(h, 1 if enable else 0))


def mhs_kernel_timing(h, kind: int) -> dict:
    ms, n, b, f = _D(), ctypes.c_longlong(), _D(), _D()
    _check(LIB.mhs_kernel_timing(h, kind, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(b), ctypes.byref(f)))
    return dict(name=mhs_kernel_kind_name(kind), ms=ms.value, launches=n.value, bytes=b.value, flops=f.value)


def mhs_kernel_timing_finest(h, kind: int) -> dict:
    ms, n, b, f = _D(), ctypes.c_longlong(), _D(), _D()
    _check(LIB.mhs_kernel_timing_finest(h, kind, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(b), ctypes.byref(f)))
    return dict(name=mhs_kernel_kind_name(kind), ms=ms.value, launches=n.value, bytes=b.value, flops=f.value)


def mhs_kernel_timing_reset(h) -> None:
    _check(LIB.mhs_kernel_timing_reset(h))


def mhs_kernel_kind_name(kind: int) -> str:
    return LIB.mhs_kernel_kind_name(kind).decode()


def mhs_kernel_launches() -> int:
    return int(LIB.mhs_kernel_launches())


def mhs_probe_fma_rate(precision, stream=None) -> float:
    """Sustained FMA rate of the device in flop/s (FP64 for MHS_FP64, FP32 for MHS_MIXED)."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    r = _D()
    _check(LIB.mhs_probe_fma_rate(precision, stream, ctypes.byref(r)))
    return r.value


def mhs_interior_residual_noalloc(nx, ny, nz, Lx, Ly, Lz, alpha, xi: XiParams | None, P, out, stream=None) -> None:
    """Allocation-free residual check: out (3 device doubles) <- ||b - A P||, ||b||, their ratio."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    _check(LIB.mhs_interior_residual_noalloc(nx, ny, nz, Lx, Ly, Lz, alpha,
                                             ctypes.byref(xi) if xi is not None else None, ptr(P), ptr(out), stream))


def mhs_server_create(budget_bytes: int, max_inflight: int = 16) -> int:
    h = _H()
    _check(LIB.mhs_server_create(budget_bytes, max_inflight, ctypes.byref(h)))
    return h.value


def mhs_server_submit(server, nx, ny, nz, Lx, Ly, Lz, alpha, xi: XiParams | None, bz, tol=1e-10, mode=MHS_MIXED,
                      atm: AtmosParams | None = None, phi=None, Bx=None, By=None, Bz=None, p=None, rho=None) -> int:
    r = Request(nx, ny, nz, Lx, Ly, Lz, alpha, xi if xi is not None else XiParams(), atm if atm is not None else
                AtmosParams(), tol, mode, ptr(bz), ptr(phi), ptr(Bx), ptr(By), ptr(Bz), ptr(p), ptr(rho))
    t = ctypes.c_longlong()
    _check(LIB.mhs_server_submit(server, ctypes.byref(r), ctypes.byref(t)))
    return t.value


def mhs_server_poll(server, ticket):
    """Returns None while running, else (info dict, status, latency_ms)."""
    done, info, st, lat = _I(), SolveInfo(), _I(), _D()
    _check(LIB.mhs_server_poll(server, ticket, ctypes.byref(done), ctypes.byref(info), ctypes.byref(st),
                               ctypes.byref(lat)))
    return (info.as_dict(), st.value, lat.value) if done.value else None


def mhs_server_wait(server, ticket, timeout_s=0.0):
    info, st, lat = SolveInfo(), _I(), _D()
    _check(LIB.mhs_server_wait(server, ticket, timeout_s, ctypes.byref(info), ctypes.byref(st), ctypes.byref(lat)))
    return info.as_dict(), st.value, lat.value


def mhs_server_stats(server) -> dict:
    s = ServerStats()
    _check(LIB.mhs_server_stats(server, ctypes.byref(s)))
    return s.as_dict()


def mhs_server_destroy(server) -> None:
    LIB.mhs_server_destroy(server)


def mhs_status_string(s: int) -> str:
    return LIB.mhs_status_string(s).decode()


def mhs_last_error() -> str:
    return LIB.mhs_last_error().decode()


def mhs_version() -> str:
    return LIB.mhs_version().decode()


class Solver:
    """Owns one handle; device buffers come from torch (memory and streams only)."""

    def __init__(self, nx, ny, nz, Lx=1.0, Ly=1.0, Lz=1.0, alpha=0.0, xi: XiParams | None = None,
                 atm: AtmosParams | None = None, stream=None):
        self.shape = (nz, ny, nx)
        self.h = mhs_create(nx, ny, nz, Lx, Ly, Lz, alpha, xi, atm)
        if stream is not None:
            mhs_set_stream(self.h, stream)

    def close(self):
        if self.h:
            mhs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_options(self, **kw):
        mhs_set_options(self.h, **kw)

    def set_lower_bz(self, bz):
        mhs_set_lower_bz(self.h, bz)

    def solve(self, tol=1e-10, mode=MHS_FP64) -> dict:
        return mhs_solve(self.h, tol, mode)

    def phi(self, device="cuda"):
        import torch
        out = torch.empty(self.shape, dtype=torch.float64, device=device)
        mhs_get_phi(self.h, out)
        return out

    def fields(self, device="cuda"):
        import torch
        outs = [torch.empty(self.shape, dtype=torch.float64, device=device) for _ in range(5)]
        mhs_fields(self.h, *outs)
        return dict(zip(["Bx", "By", "Bz", "p", "rho"], outs))
