"""Thin ctypes binding of libcpm (include/cpm.h).

Argument marshalling only: every step runs in the CUDA library.  Functions
carry the C names (cpm_band_build, cpm_apply, oras_setup, oras_apply,
cpm_solve, cpm_solve_adjoint, ...); the classes Band and Schwarz own the
handles.  Vectors are torch tensors on the CUDA device; the current torch
stream is passed to every call unless a stream is given.

There is no fallback: if libcpm.so is missing or no CUDA device is present,
the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcpm.so")
_lib = None

CPM_OK, CPM_ERR_ARG, CPM_ERR_CUDA, CPM_ERR_OOM, CPM_ERR_BAND = 0, 1, 2, 3, 4
CPM_ERR_NOT_CONVERGED, CPM_ERR_BREAKDOWN, CPM_ERR_NAN, CPM_ERR_TIMEOUT = 5, 6, 7, 8
CPM_F64, CPM_F32, CPM_BF16 = 0, 1, 2
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_OOM", 4: "ERR_BAND", 5: "ERR_NOT_CONVERGED",
                6: "ERR_BREAKDOWN", 7: "ERR_NAN", 8: "ERR_TIMEOUT"}


class cpm_surface(C.Structure):
    _fields_ = [("kind", C.c_int32), ("param", C.c_double * 8)]


class oras_params(C.Structure):
    _fields_ = [("nparts", C.c_int32), ("overlap", C.c_int32), ("robin", C.c_int32), ("alpha", C.c_double),
                ("alpha_cross", C.c_double), ("store", C.c_int32), ("order", C.c_int32), ("coarse", C.c_int32)]


class oras_tuning(C.Structure):
    _fields_ = [("xplace", C.c_int32), ("lanes", C.c_int32), ("schedule", C.c_int32), ("ctas", C.c_int32),
                ("probe_timeout", C.c_int32), ("wait_polls", C.c_int64)]


class cpm_solve_params(C.Structure):
    _fields_ = [("restart", C.c_int32), ("maxit", C.c_int32), ("rtol", C.c_double), ("mixed", C.c_int32),
                ("reorth", C.c_int32), ("inner_rtol", C.c_double), ("timing", C.c_int32)]


class cpm_solve_info(C.Structure):
    _fields_ = [("iters", C.c_int32), ("restarts", C.c_int32), ("ir_steps", C.c_int32),
                ("rel_residual", C.c_double), ("status", C.c_int32), ("ms_precond", C.c_double),
                ("ms_operator", C.c_double), ("n_precond", C.c_int32), ("n_operator", C.c_int32)]


class cpm_schnakenberg(C.Structure):
    _fields_ = [("delta1", C.c_double), ("delta2", C.c_double), ("lambda_", C.c_double), ("Du", C.c_double),
                ("Dv", C.c_double), ("dt", C.c_double), ("model", C.c_int32)]


class CpmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def lib():
    """Load libcpm.so (built in-tree by paper_2110_06322_gb300.build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2110_06322_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, f64 = C.c_void_p, C.c_int, C.c_int64, C.c_double
    P = C.POINTER
    sig = {
        "cpm_last_error": (C.c_char_p, []),
        "cpm_band_build": (i32, [P(cpm_surface), f64, i32, vp, P(vp)]),
        "cpm_band_info": (i32, [vp, P(C.c_int64), P(C.c_int64), P(C.c_int64)]),
        "cpm_band_export": (i32, [vp, vp, vp, vp, vp, vp, vp]),
        "cpm_band_weights": (i32, [vp, vp, vp]),
        "cpm_apply": (i32, [vp, P(C.c_double), vp, vp, i32, i32, i32, vp]),
        "oras_setup": (i32, [vp, P(oras_params), f64, vp, P(vp)]),
        "oras_apply": (i32, [vp, vp, vp, i32, i32, i32, vp]),
        "oras_info": (i32, [vp, P(C.c_int32), P(C.c_int64), P(C.c_int64), P(C.c_int32)]),
        "oras_set_tuning": (i32, [vp, P(oras_tuning)]),
        "oras_get_tuning": (i32, [vp, P(oras_tuning)]),
        "oras_autotune": (i32, [vp, i32, i32, vp, P(oras_tuning), P(C.c_double)]),
        "cpm_device_allocations": (C.c_int64, []),
        "oras_export": (i32, [vp, vp, vp, vp, vp]),
        "cpm_solve": (i32, [vp, vp, f64, vp, vp, P(cpm_solve_params), P(cpm_solve_info), vp]),
        "cpm_solve_adjoint": (i32, [vp, vp, f64, vp, vp, P(cpm_solve_params), P(cpm_solve_info), vp]),
        "cpm_band_free": (None, [vp]),
        "oras_free": (None, [vp]),
        "cpm_kernel_launches": (C.c_int64, []),
        "cpm_apply_noalloc": (i32, [vp, P(C.c_double), vp, vp, i32, i32, vp]),
        "cpm_imex_rhs": (i32, [vp, P(cpm_schnakenberg), vp, vp, vp, vp, vp]),
        "cpm_imex_rhs_adjoint": (i32, [vp, P(cpm_schnakenberg), vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]),
        "cpm_imex2_rhs": (i32, [vp, P(cpm_schnakenberg), i32, vp, vp, vp, vp, vp, vp, vp]),
        "cpm_dot": (i32, [vp, vp, vp, vp, vp]),
        "cpm_solve_batch": (i32, [i32, vp, vp, P(C.c_double), P(C.c_int32), vp, vp, P(cpm_solve_params),
                                  P(cpm_solve_info), i32, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


EXPORTED = ["cpm_last_error", "cpm_band_build", "cpm_band_info", "cpm_band_export", "cpm_band_weights", "cpm_apply",
            "oras_setup", "oras_apply", "oras_info", "oras_set_tuning", "oras_get_tuning", "oras_autotune",
            "oras_export", "cpm_solve",
            "cpm_solve_adjoint", "cpm_band_free", "oras_free", "cpm_kernel_launches", "cpm_device_allocations",
            "cpm_apply_noalloc", "cpm_imex_rhs", "cpm_imex_rhs_adjoint", "cpm_imex2_rhs", "cpm_dot",
            "cpm_solve_batch"]


def _check(st):
    if st != CPM_OK:
        raise CpmError(st, lib().cpm_last_error().decode())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _dtype_code(t):
    if t.dtype == torch.float64:
        return CPM_F64
    if t.dtype == torch.float32:
        return CPM_F32
    raise TypeError("vectors must be float64 or float32 CUDA tensors")


# ------------------------------------------------------------------ C names
def cpm_band_build(kind, params, h, p=3, stream=None):
    surf = cpm_surface()
    surf.kind = int(kind)
    for q, v in enumerate(params):
        surf.param[q] = float(v)
    out = C.c_void_p()
    _check(lib().cpm_band_build(C.byref(surf), float(h), int(p), _stream(stream), C.byref(out)))
    return out


def _apply_args(band, c, x, y):
    """nrhs and the host array of shifts of an operator apply, after checking
    that x and y are matching device vectors of whole right-hand sides."""
    n = Band.n_active_of(band)
    code = _dtype_code(x)
    if x.numel() == 0 or x.numel() % n != 0:
        raise ValueError(f"x holds {x.numel()} values, not a whole number of {n}-node vectors")
    nrhs = x.numel() // n
    if y.numel() != x.numel() or y.dtype != x.dtype or y.device != x.device:
        raise ValueError("y must match x in size, dtype and device")
    if not (x.is_contiguous() and y.is_contiguous()):
        raise ValueError("x and y must be contiguous")
    cl = [float(c)] * nrhs if not hasattr(c, "__len__") else [float(v) for v in c]
    if len(cl) != nrhs:
        raise ValueError(f"{len(cl)} shifts given for {nrhs} right-hand sides")
    return nrhs, code, (C.c_double * nrhs)(*cl)


def cpm_apply(band, c, x, y, transpose=False, stream=None):
    nrhs, code, cs = _apply_args(band, c, x, y)
    _check(lib().cpm_apply(band, cs, _ptr(x), _ptr(y), code, nrhs, int(bool(transpose)), _stream(stream)))
    return y


def cpm_apply_noalloc(band, c, x, y, stream=None):
    """y = M x through the entry point that allocates nothing (fixed library scratch)."""
    nrhs, code, cs = _apply_args(band, c, x, y)
    _check(lib().cpm_apply_noalloc(band, cs, _ptr(x), _ptr(y), code, nrhs, _stream(stream)))
    return y


def cpm_device_allocations():
    return lib().cpm_device_allocations()


def oras_set_tuning(pc, xplace=0, lanes=0, schedule=0, probe_timeout=0, wait_polls=0, ctas=0):
    t = oras_tuning(int(xplace), int(lanes), int(schedule), int(ctas), int(probe_timeout), int(wait_polls))
    _check(lib().oras_set_tuning(pc, C.byref(t)))


def _tuning_dict(t):
    return {"xplace": t.xplace, "lanes": t.lanes, "schedule": t.schedule, "ctas": t.ctas,
            "probe_timeout": t.probe_timeout, "wait_polls": t.wait_polls}


def oras_get_tuning(pc):
    t = oras_tuning()
    _check(lib().oras_get_tuning(pc, C.byref(t)))
    return _tuning_dict(t)


def oras_autotune(pc, dtype=CPM_F32, reps=3, stream=None):
    """Time the equivalent apply kernels and keep the fastest; returns
    (setting, milliseconds per apply)."""
    t, ms = oras_tuning(), C.c_double()
    _check(lib().oras_autotune(pc, int(dtype), int(reps), _stream(stream), C.byref(t), C.byref(ms)))
    return _tuning_dict(t), ms.value


def _rx(prm):
    return cpm_schnakenberg(float(prm["delta1"]), float(prm["delta2"]), float(prm["lambda"]), float(prm["Du"]),
                            float(prm["Dv"]), float(prm["dt"]), int(prm.get("model", 0)))


def cpm_imex2_rhs(band, prm, stage, u, v, u2, v2, bu, bv, stream=None):
    """Right-hand sides of ARS(2,2,2) stage 2 (u2, v2 unused) or 3."""
    _check(lib().cpm_imex2_rhs(band, C.byref(_rx(prm)), int(stage), _ptr(u), _ptr(v), _ptr(u2), _ptr(v2), _ptr(bu),
                               _ptr(bv), _stream(stream)))
    return bu, bv


def cpm_imex_rhs(band, prm, u, v, bu, bv, stream=None):
    """bu = c_u (u + dt f(u, v)), bv = c_v (v + dt g(u, v)); prm: dict with
    delta1, delta2, lambda, Du, Dv, dt."""
    _check(lib().cpm_imex_rhs(band, C.byref(_rx(prm)), _ptr(u), _ptr(v), _ptr(bu), _ptr(bv), _stream(stream)))
    return bu, bv


def cpm_imex_rhs_adjoint(band, prm, u, v, u1, v1, lu, lv, ubar, vbar, dc, stream=None):
    _check(lib().cpm_imex_rhs_adjoint(band, C.byref(_rx(prm)), _ptr(u), _ptr(v), _ptr(u1), _ptr(v1), _ptr(lu),
                                      _ptr(lv), _ptr(ubar), _ptr(vbar), _ptr(dc), _stream(stream)))
    return ubar, vbar, dc


def cpm_dot(band, a, b, out, stream=None):
    _check(lib().cpm_dot(band, _ptr(a), _ptr(b), _ptr(out), _stream(stream)))
    return out


def oras_setup(band, c, nparts, overlap, robin=False, alpha=4.0, alpha_cross=20.0, store=CPM_F32, order=0,
               coarse=False, stream=None):
    prm = oras_params(int(nparts), int(overlap), int(bool(robin)), float(alpha), float(alpha_cross), int(store),
                      int(order), int(bool(coarse)))
    out = C.c_void_p()
    _check(lib().oras_setup(band, C.byref(prm), float(c), _stream(stream), C.byref(out)))
    return out


def oras_apply(pc, r, z, n_active, transpose=False, stream=None):
    nrhs = r.numel() // n_active
    _check(lib().oras_apply(pc, _ptr(r), _ptr(z), _dtype_code(r), nrhs, int(bool(transpose)), _stream(stream)))
    return z


def cpm_solve(band, pc, c, f, u, restart=30, maxit=10000, rtol=1e-8, mixed=False, reorth=0, inner_rtol=1e-4,
              adjoint=False, timing=False, stream=None):
    """reorth: 0 one classical Gram-Schmidt pass (default, the PETSc GMRES
    default that the paper's solver runs with), 1 a second pass when the first
    shrank the vector below 1/sqrt(2) of its norm, 2 always two passes."""
    prm = cpm_solve_params(int(restart), int(maxit), float(rtol), int(bool(mixed)), int(reorth),
                           float(inner_rtol), int(bool(timing)))
    info = cpm_solve_info()
    fn = lib().cpm_solve_adjoint if adjoint else lib().cpm_solve
    st = fn(band, pc, float(c), _ptr(f), _ptr(u), C.byref(prm), C.byref(info), _stream(stream))
    if st not in (CPM_OK, CPM_ERR_NOT_CONVERGED):
        _check(st)
    return {"status": st, "iters": info.iters, "restarts": info.restarts, "ir_steps": info.ir_steps,
            "rel_residual": info.rel_residual, "ms_precond": info.ms_precond, "ms_operator": info.ms_operator,
            "n_precond": info.n_precond, "n_operator": info.n_operator}


def _info_dict(st, info):
    return {"status": st, "iters": info.iters, "restarts": info.restarts, "ir_steps": info.ir_steps,
            "rel_residual": info.rel_residual, "ms_precond": info.ms_precond, "ms_operator": info.ms_operator,
            "n_precond": info.n_precond, "n_operator": info.n_operator}


def cpm_solve_batch(bands, pcs, c, nrhs, f, u, restart=30, maxit=10000, rtol=1e-8, mixed=False, inner_rtol=1e-4,
                    adjoint=False, stream=None):
    """Lockstep GMRES over len(bands) problems (band handles, preconditioner
    handles or None, shifts, right-hand-side counts); f, u: concatenated
    device vectors.  Returns (status, [info per system])."""
    P = len(bands)
    hb = (C.c_void_p * P)(*[b.value if isinstance(b, C.c_void_p) else b for b in bands])
    hp = (C.c_void_p * P)(*[(q.value if isinstance(q, C.c_void_p) else q) if q is not None else None for q in pcs])
    hc = (C.c_double * P)(*[float(x) for x in c])
    hn = (C.c_int32 * P)(*[int(x) for x in nrhs])
    S = sum(int(x) for x in nrhs)
    infos = (cpm_solve_info * S)()
    prm = cpm_solve_params(int(restart), int(maxit), float(rtol), int(bool(mixed)), 0, float(inner_rtol), 0)
    st = lib().cpm_solve_batch(P, hb, hp, hc, hn, _ptr(f), _ptr(u), C.byref(prm), infos, int(bool(adjoint)),
                               _stream(stream))
    if st not in (CPM_OK, CPM_ERR_NOT_CONVERGED):
        _check(st)
    return st, [_info_dict(infos[q].status, infos[q]) for q in range(S)]


def cpm_kernel_launches():
    return lib().cpm_kernel_launches()


def cpm_solve_adjoint(band, pc, c, g, lam, **kw):
    return cpm_solve(band, pc, c, g, lam, adjoint=True, **kw)


# ------------------------------------------------------------------ owning classes
class Band:
    """Computational band around a sphere (kind 0) or torus (kind 1)."""

    _sizes = {}

    def __init__(self, kind, params, h, p=3, stream=None):
        self.kind, self.params, self.h, self.p = int(kind), tuple(params), float(h), int(p)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.handle = cpm_band_build(kind, params, h, p, stream)
        nA, nG, nT = C.c_int64(), C.c_int64(), C.c_int64()
        _check(lib().cpm_band_info(self.handle, C.byref(nA), C.byref(nG), C.byref(nT)))
        self.n_active, self.n_ghost, self.n_tube = nA.value, nG.value, nT.value
        self.n_rows = self.n_active + self.n_ghost
        Band._sizes[self.handle.value] = self.n_active

    @staticmethod
    def n_active_of(handle):
        return Band._sizes[handle.value]

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _lib is not None:
            Band._sizes.pop(h.value, None)
            _lib.cpm_band_free(h)
            self.handle = None

    def export(self, stream=None):
        d = self.device
        ijkA = torch.empty((self.n_active, 3), dtype=torch.int32, device=d)
        ijkG = torch.empty((max(self.n_ghost, 1), 3), dtype=torch.int32, device=d)
        base = torch.empty((self.n_rows, 3), dtype=torch.int32, device=d)
        cp = torch.empty((self.n_rows, 3), dtype=torch.float64, device=d)
        perm = torch.empty(self.n_active, dtype=torch.int64, device=d)
        _check(lib().cpm_band_export(self.handle, _ptr(ijkA), _ptr(ijkG), _ptr(base), _ptr(cp), _ptr(perm),
                                     _stream(stream)))
        return ijkA, ijkG[: self.n_ghost], base, cp, perm

    def weights(self, stream=None):
        w = torch.empty((self.n_rows, 3, self.p + 1), dtype=torch.float64, device=self.device)
        _check(lib().cpm_band_weights(self.handle, _ptr(w), _stream(stream)))
        return w

    def apply(self, c, x, transpose=False, out=None, stream=None):
        y = torch.empty_like(x) if out is None else out
        return cpm_apply(self.handle, c, x, y, transpose, stream)


class Schwarz:
    """(O)RAS preconditioner over a Band (Section 2.2)."""

    def __init__(self, band, c, nparts, overlap, robin=False, alpha=4.0, alpha_cross=20.0, store=CPM_F32, order=0,
                 coarse=False, stream=None):
        self.band = band
        self.c = float(c)
        self.coarse = bool(coarse)
        self.handle = oras_setup(band.handle, c, nparts, overlap, robin, alpha, alpha_cross, store, order, coarse,
                                 stream)
        npt, rows, nnz, lev = C.c_int32(), C.c_int64(), C.c_int64(), C.c_int32()
        _check(lib().oras_info(self.handle, C.byref(npt), C.byref(rows), C.byref(nnz), C.byref(lev)))
        self.nparts, self.total_rows, self.total_nnz, self.max_levels = npt.value, rows.value, nnz.value, lev.value

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _lib is not None:
            _lib.oras_free(h)
            self.handle = None

    def apply(self, r, transpose=False, out=None, stream=None):
        z = torch.empty_like(r) if out is None else out
        return oras_apply(self.handle, r, z, self.band.n_active, transpose, stream)

    def set_tuning(self, xplace=0, lanes=0, schedule=0, probe_timeout=0, wait_polls=0, ctas=0):
        """Run-time settings of the apply (oras_set_tuning): local-vector
        placement (0 shared memory when it fits, 1 global slice, 2 and 3 an
        FP16 local vector in shared memory for FP32 applies whose FP32 one
        does not fit), lanes per factor row, subdomain schedule, CTAs per SM
        for global slices, the failure-path probe and the wait bound."""
        oras_set_tuning(self.handle, xplace, lanes, schedule, probe_timeout, wait_polls, ctas)

    def tuning(self):
        return oras_get_tuning(self.handle)

    def autotune(self, dtype=CPM_F32, reps=3, stream=None):
        return oras_autotune(self.handle, dtype, reps, stream)

    def export(self, stream=None):
        d = self.band.device
        part = torch.empty(self.band.n_active, dtype=torch.int32, device=d)
        sptr = torch.empty(self.nparts + 1, dtype=torch.int64, device=d)
        nodes = torch.empty(max(self.total_rows, 1), dtype=torch.int32, device=d)
        _check(lib().oras_export(self.handle, _ptr(part), _ptr(sptr), _ptr(nodes), _stream(stream)))
        return part, sptr, nodes[: self.total_rows]


def solve_batch(problems, rhs, u0=None, adjoint=False, **kw):
    """Solve a batch: problems is a list of (Band, Schwarz or None, c); rhs a
    list of FP64 CUDA tensors, one per problem, of shape (N_A,) or
    (nrhs, N_A).  Returns (solutions shaped like rhs, [info per system])."""
    shapes = [t.shape for t in rhs]
    nrhs = [1 if t.dim() == 1 else t.shape[0] for t in rhs]
    f = torch.cat([t.reshape(-1) for t in rhs]).contiguous()
    u = torch.zeros_like(f) if u0 is None else torch.cat([t.reshape(-1) for t in u0]).contiguous()
    bands = [b.handle for b, _, _ in problems]
    pcs = [p.handle if p is not None else None for _, p, _ in problems]
    cs = [float(c) for _, _, c in problems]
    st, infos = cpm_solve_batch(bands, pcs, cs, nrhs, f, u, adjoint=adjoint, **kw)
    out, o = [], 0
    for sh in shapes:
        k = 1
        for d in sh:
            k *= d
        out.append(u[o:o + k].reshape(sh))
        o += k
    return out, infos


def solve(band, f, pc=None, c=None, u0=None, adjoint=False, **kw):
    """Solve M u = f (or M^T u = f) on the device; returns (u, info)."""
    c = pc.c if c is None else float(c)
    u = torch.zeros_like(f) if u0 is None else u0.clone()
    info = cpm_solve(band.handle, pc.handle if pc is not None else None, c, f, u, adjoint=adjoint, **kw)
    return u, info
