"""FP64 CPU oracle for the closest point method solver (test infrastructure).

This package is TEST INFRASTRUCTURE.  Only the tests, the smoke check and the
CPU-baseline leg of the benchmark may import it; the product library
(``paper_2110_06322_gb300``) never does.  It wraps ``cpm_oracle.cpp`` (plain
C++, FP64, ``-ffp-contract=off``) through ctypes and shares no code with the
CUDA path.

Paper: May, Haynes & Ruuth, arXiv 2110.06322.  Section 2.1 (closest point
function eq. cpFunc, extension E, stabilised Laplace-Beltrami eq. lapBel),
Section 2.2 (RAS / ORAS), Section 4.1.1 (GMRES + ILU(0) local solves).

Parity unpinned: the Robin (P-ORAS) diagonal term, whose discretisation the
paper defers to other work; only "alpha -> infinity gives RAS" and "GMRES with
P-ORAS reaches the direct solution" pin it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cpm_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

SPHERE, TORUS = 0, 1

_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (FP64, no contraction, single thread)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", _LIB + ".tmp", _SRC]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is not None:
        return _lib
    build()
    L = C.CDLL(_LIB)
    vp, i32, i64, f64 = C.c_void_p, C.c_int, C.c_int64, C.c_double
    pi32 = C.POINTER(C.c_int)
    pi64 = C.POINTER(C.c_int64)
    pf64 = C.POINTER(C.c_double)
    sig = {
        "orc_last_error": (C.c_char_p, []),
        "orc_cp_dist": (i32, [i32, _f64p, _f64p, _f64p, pf64]),
        "orc_band_lambda": (f64, [f64, i32]),
        "orc_reach": (f64, [i32, _f64p]),
        "orc_weights1d": (None, [i32, f64, _f64p]),
        "orc_band_build": (vp, [i32, _f64p, f64, i32, pi32]),
        "orc_band_free": (None, [vp]),
        "orc_band_counts": (None, [vp, pi64, pi64, pi64]),
        "orc_band_export": (None, [vp, _i32p, _i32p, _i32p, _f64p]),
        "orc_band_active_index": (i64, [vp, i32, i32, i32]),
        "orc_band_row_index": (i64, [vp, i32, i32, i32]),
        "orc_erow_weights": (None, [vp, i64, _f64p]),
        "orc_E": (vp, [vp]),
        "orc_M": (vp, [vp, f64]),
        "orc_transpose": (vp, [vp]),
        "orc_csr_free": (None, [vp]),
        "orc_csr_info": (None, [vp, pi64, pi64, pi64]),
        "orc_csr_export": (None, [vp, _i64p, _i32p, _f64p]),
        "orc_csr_matvec": (None, [vp, _f64p, _f64p]),
        "orc_apply_rows": (None, [vp, f64, _f64p, i64, _i64p, _f64p]),
        "orc_apply_T_cols": (None, [vp, f64, _f64p, i64, _i64p, _f64p]),
        "orc_dense_solve": (i32, [i64, _f64p, _f64p, _f64p, i32]),
        "orc_oras_setup": (vp, [vp, vp, i32, i32, i32, f64, f64, i32, i32, i32, pi32]),
        "orc_oras_coarse_matrix": (None, [vp, _f64p]),
        "orc_oras_free": (None, [vp]),
        "orc_oras_partition": (None, [vp, _i32p]),
        "orc_oras_sub_size": (i64, [vp, i32]),
        "orc_oras_sub_nodes": (None, [vp, i32, _i32p]),
        "orc_oras_sub_matrix": (vp, [vp, i32]),
        "orc_oras_depth": (i32, [vp, i32, i32]),
        "orc_oras_sub_matrix_unfactored": (vp, [vp, vp, vp, i32]),
        "orc_oras_apply": (None, [vp, _f64p, _f64p, i32]),
        "orc_gmres": (i32, [vp, vp, i32, _f64p, _f64p, i32, i32, f64, i32, pi32, pf64]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _surf_params(kind, params):
    prm = np.zeros(8, dtype=np.float64)
    prm[: len(params)] = params
    return prm


def cp_dist(kind, params, x):
    """Closest point and unsigned distance of one point (eq. cpFunc)."""
    cp = np.zeros(3)
    d = C.c_double()
    st = lib().orc_cp_dist(kind, _surf_params(kind, params), np.ascontiguousarray(x, dtype=np.float64), cp,
                           C.byref(d))
    return st, cp, d.value


def band_lambda(h, p):
    return lib().orc_band_lambda(h, p)


def weights1d(p, s):
    out = np.zeros(p + 1)
    lib().orc_weights1d(p, float(s), out)
    return out


class CSR:
    """Owned oracle CSR matrix."""

    def __init__(self, ptr):
        if not ptr:
            raise RuntimeError("oracle matrix construction failed")
        self._p = C.c_void_p(ptr)

    def __del__(self):
        if getattr(self, "_p", None) and _lib is not None:
            _lib.orc_csr_free(self._p)
            self._p = None

    @property
    def shape(self):
        nr, nc, nnz = C.c_int64(), C.c_int64(), C.c_int64()
        lib().orc_csr_info(self._p, C.byref(nr), C.byref(nc), C.byref(nnz))
        return nr.value, nc.value, nnz.value

    def arrays(self):
        nr, nc, nnz = self.shape
        ptr = np.zeros(nr + 1, dtype=np.int64)
        col = np.zeros(max(nnz, 1), dtype=np.int32)
        val = np.zeros(max(nnz, 1), dtype=np.float64)
        lib().orc_csr_export(self._p, ptr, col, val)
        return ptr, col[:nnz], val[:nnz]

    def to_scipy(self):
        import scipy.sparse as sp
        nr, nc, _ = self.shape
        ptr, col, val = self.arrays()
        return sp.csr_matrix((val, col, ptr), shape=(nr, nc))

    def matvec(self, x):
        nr, nc, _ = self.shape
        y = np.zeros(nr)
        lib().orc_csr_matvec(self._p, np.ascontiguousarray(x, dtype=np.float64), y)
        return y

    def transpose(self):
        return CSR(lib().orc_transpose(self._p))


class Band:
    """Narrow band Sigma_A / Sigma_G with its E rows (Section 2.1)."""

    def __init__(self, kind, params, h, p=3):
        st = C.c_int()
        self.kind, self.params, self.h, self.p = kind, tuple(params), float(h), int(p)
        ptr = lib().orc_band_build(kind, _surf_params(kind, params), float(h), int(p), C.byref(st))
        self.status = st.value
        self._p = C.c_void_p(ptr) if ptr else None
        if self._p is None:
            raise BandError(self.status)
        nT, nA, nG = C.c_int64(), C.c_int64(), C.c_int64()
        lib().orc_band_counts(self._p, C.byref(nT), C.byref(nA), C.byref(nG))
        self.n_tube, self.n_active, self.n_ghost = nT.value, nA.value, nG.value
        self.n_rows = self.n_active + self.n_ghost
        self._export = None

    def __del__(self):
        if getattr(self, "_p", None) and _lib is not None:
            _lib.orc_band_free(self._p)
            self._p = None

    def export(self):
        """(ijk_active[N_A,3], ijk_ghost[N_G,3], erow_base[N_C,3], erow_cp[N_C,3])."""
        if self._export is None:
            a = np.zeros((max(self.n_active, 1), 3), dtype=np.int32)
            g = np.zeros((max(self.n_ghost, 1), 3), dtype=np.int32)
            b = np.zeros((max(self.n_rows, 1), 3), dtype=np.int32)
            c = np.zeros((max(self.n_rows, 1), 3), dtype=np.float64)
            lib().orc_band_export(self._p, a, g, b, c)
            self._export = (a[: self.n_active], g[: self.n_ghost], b[: self.n_rows], c[: self.n_rows])
        return self._export

    def active_index(self, i, j, k):
        return lib().orc_band_active_index(self._p, int(i), int(j), int(k))

    def row_index(self, i, j, k):
        return lib().orc_band_row_index(self._p, int(i), int(j), int(k))

    def erow_weights(self, r):
        W = np.zeros((self.p + 1) ** 3)
        lib().orc_erow_weights(self._p, int(r), W)
        return W

    def E(self):
        return CSR(lib().orc_E(self._p))

    def M(self, c):
        return CSR(lib().orc_M(self._p, float(c)))

    def apply_rows(self, c, x, rows):
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        out = np.zeros(len(rows))
        lib().orc_apply_rows(self._p, float(c), np.ascontiguousarray(x, dtype=np.float64), len(rows), rows, out)
        return out

    def apply_T_cols(self, c, x, cols):
        cols = np.ascontiguousarray(cols, dtype=np.int64)
        out = np.zeros(len(cols))
        lib().orc_apply_T_cols(self._p, float(c), np.ascontiguousarray(x, dtype=np.float64), len(cols), cols, out)
        return out


class BandError(RuntimeError):
    def __init__(self, status):
        super().__init__(f"oracle band build failed with status {status}")
        self.status = status


class ORAS:
    """(O)RAS preconditioner (Section 2.2) over an oracle band and matrix."""

    LOCAL_CANONICAL, LOCAL_DISTANCE, LOCAL_SHELLS = 0, 1, 2

    def __init__(self, band, M, nparts, overlap, robin=False, alpha=4.0, alpha_cross=20.0, exact=False,
                 order=LOCAL_DISTANCE, coarse=False):
        """coarse=True: the two-level variant, a coarse correction on one
        constant per disjoint part applied before the one-level apply
        (z = q + P_RAS (r - M q), q = Z (Z^T M Z)^{-1} Z^T r)."""
        st = C.c_int()
        ptr = lib().orc_oras_setup(band._p, M._p, int(nparts), int(overlap), int(bool(robin)), float(alpha),
                                   float(alpha_cross), int(bool(exact)), int(order), int(bool(coarse)),
                                   C.byref(st))
        if not ptr:
            raise RuntimeError(f"oracle ORAS setup failed with status {st.value}")
        self._p = C.c_void_p(ptr)
        self.band, self.M, self.nparts = band, M, int(nparts)
        self.n = band.n_active

    def __del__(self):
        if getattr(self, "_p", None) and _lib is not None:
            _lib.orc_oras_free(self._p)
            self._p = None

    def partition(self):
        part = np.zeros(self.n, dtype=np.int32)
        lib().orc_oras_partition(self._p, part)
        return part

    def sub_nodes(self, j):
        n = lib().orc_oras_sub_size(self._p, j)
        out = np.zeros(max(n, 1), dtype=np.int32)
        lib().orc_oras_sub_nodes(self._p, j, out)
        return out[:n]

    def sub_factors(self, j):
        return CSR(lib().orc_oras_sub_matrix(self._p, j))

    def depth(self, j, lower=True):
        """Number of dependency levels of subdomain j's lower (or upper)
        triangular sweep in its local order."""
        return int(lib().orc_oras_depth(self._p, int(j), int(bool(lower))))

    def sub_matrix(self, j):
        return CSR(lib().orc_oras_sub_matrix_unfactored(self.band._p, self.M._p, self._p, j))

    def coarse_matrix(self):
        """E0 = Z^T M Z of the two-level variant (np x np)."""
        E = np.zeros((self.nparts, self.nparts))
        lib().orc_oras_coarse_matrix(self._p, E)
        return E

    def apply(self, r, transpose=False):
        z = np.zeros(self.n)
        lib().orc_oras_apply(self._p, np.ascontiguousarray(r, dtype=np.float64), z, int(bool(transpose)))
        return z


def gmres(M, f, P=None, transpose=False, x0=None, restart=30, maxit=10000, rtol=1e-10, reorth=True):
    """Right-preconditioned restarted GMRES.  For the adjoint pass M^T (a CSR)
    and transpose=True so that P^T is used."""
    n = M.shape[0]
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    it, rr = C.c_int(), C.c_double()
    st = lib().orc_gmres(M._p, P._p if P is not None else None, int(bool(transpose)),
                         np.ascontiguousarray(f, dtype=np.float64), x, int(restart), int(maxit), float(rtol),
                         int(bool(reorth)), C.byref(it), C.byref(rr))
    return x, {"status": st, "iters": it.value, "relres": rr.value}


def dense_solve(A, b, transpose=False):
    A = np.ascontiguousarray(A, dtype=np.float64)
    x = np.zeros(A.shape[0])
    st = lib().orc_dense_solve(A.shape[0], A, np.ascontiguousarray(b, dtype=np.float64), x, int(bool(transpose)))
    if st:
        raise RuntimeError("singular dense system")
    return x
