"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This module holds NO arithmetic of the method (no closest points, no
interpolation, no operator): only random numbers and the synthetic surface
functions that play the role of the right-hand side f.  Both sides receive the
same arrays from here.

Random numbers come from SplitMix64 (Steele, Lea & Flood 2014), written here
from its published definition and used counter-style (output i is the mix of
seed + (i + 1) * golden-gamma), so any element can be drawn independently.
Normals use the Box-Muller transform.

Workloads (shapes of the paper's shifted-Poisson benchmarks, Section 4.1.1 and
Section 5; the paper's torus input file and meshes are not available, so
analytic surfaces stand in):
  * SPHERE_H01   unit sphere, h = 0.1, p = 3, c = 1, f = (c + 12) Y at cp with
                 Y = (x^2 - y^2) z (a degree-3 spherical harmonic, eigenvalue -12)
  * TORUS_H004   torus R = 1, r = 0.4, h = 0.004, c = 10, 20 random Fourier modes
  * TORUS_H002   same torus at h = 0.002 (mixed-precision workload)
  * TORUS_H0125, TORUS_H025   the same torus at h = 0.0125 / 0.025 with 64 / 16
                 parts (same rows per subdomain), small cases for profiling
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Outputs start .. start+n-1 of the SplitMix64 stream seeded with `seed`."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits."""
    return (splitmix64(seed, n, start) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Standard normals by Box-Muller from consecutive uniform pairs."""
    u = uniform(seed, 2 * n, 2 * start)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


# ---------------------------------------------------------------- surfaces
SPHERE, TORUS = 0, 1


def surface_params(kind: int, center=(0.0, 0.0, 0.0), a: float = 1.0, b: float = 0.0):
    """Surface parameter vector as the C ABI takes it: sphere (c, rho), torus (c, R, r)."""
    if kind == SPHERE:
        return (float(center[0]), float(center[1]), float(center[2]), float(a))
    return (float(center[0]), float(center[1]), float(center[2]), float(a), float(b))


# Each workload: surface, spacing h, degree p, shift c, right-hand side, Schwarz
# preconditioner (parts, overlap, Robin or not, ILU(0) local order) and GMRES
# settings; solve_rtol is the relative residual the benchmark solves to.
WORKLOADS = {
    "sphere_h0.1": dict(kind=SPHERE, params=surface_params(SPHERE, a=1.0), h=0.1, p=3, c=1.0,
                        rhs="y32", nparts=8, overlap=2, robin=False, restart=30, rtol=1e-10),
    "torus_h0.004": dict(kind=TORUS, params=surface_params(TORUS, a=1.0, b=0.4), h=0.004, p=3, c=10.0,
                         rhs="modes", seed=2, nparts=512, overlap=2, robin=False, alpha=4.0, alpha_cross=20.0,
                         restart=30, rtol=1e-8, solve_rtol=1e-8, order=2),
    "torus_h0.0125": dict(kind=TORUS, params=surface_params(TORUS, a=1.0, b=0.4), h=0.0125, p=3, c=10.0,
                          rhs="modes", seed=2, nparts=64, overlap=2, robin=False, restart=30, rtol=1e-8,
                          solve_rtol=1e-8, order=2),
    "torus_h0.025": dict(kind=TORUS, params=surface_params(TORUS, a=1.0, b=0.4), h=0.025, p=3, c=10.0,
                         rhs="modes", seed=2, nparts=16, overlap=2, robin=False, restart=30, rtol=1e-8,
                         solve_rtol=1e-8, order=2),
    # xplace 3: the subdomains (~58k rows) hold their local vectors in FP16 in shared memory
    "torus_h0.002": dict(kind=TORUS, params=surface_params(TORUS, a=1.0, b=0.4), h=0.002, p=3, c=10.0,
                         rhs="modes", seed=3, nparts=512, overlap=2, robin=False, alpha=4.0, alpha_cross=20.0,
                         restart=30, rtol=1e-8, solve_rtol=1e-8, order=2, xplace=3),
    # differentiable Schnakenberg run (eq. schnack): D = (1e-3, 1e-1), dt = 0.01, 500 steps, state
    # checkpoints every 25 steps; initial state (u*, v*) (1 + 0.01 U[-1, 1]) from seed 7 (u) and 8 (v)
    "schnakenberg_torus_h0.005": dict(kind=TORUS, params=surface_params(TORUS, a=1.0, b=0.4), h=0.005, p=3,
                                      Du=1e-3, Dv=1e-1, dt=0.01, steps=500, checkpoint=25, seed=7, nparts=256,
                                      overlap=2, robin=False, restart=30, rtol=1e-10),
}


# ---------------------------------------------------------------- right-hand sides
def y32(cp: np.ndarray, center=(0.0, 0.0, 0.0), rho: float = 1.0) -> np.ndarray:
    """Y = (x^2 - y^2) z on the sphere of radius rho (unnormalised degree-3,
    order-2 real spherical harmonic of the unit direction)."""
    d = (np.asarray(cp, dtype=np.float64) - np.asarray(center)) / rho
    return (d[:, 0] ** 2 - d[:, 1] ** 2) * d[:, 2]


def torus_modes(seed: int, n_modes: int = 20, max_freq: int = 8):
    """Random Fourier modes in the torus angles: amplitudes N(0,1), integer
    frequencies m, n in [0, max_freq], phases U[0, 2 pi)."""
    a = normal(seed, n_modes)
    u = uniform(seed ^ 0x5DEECE66D, 3 * n_modes)
    m = np.floor(u[0::3] * (max_freq + 1)).astype(np.int64)
    n = np.floor(u[1::3] * (max_freq + 1)).astype(np.int64)
    psi = 2.0 * math.pi * u[2::3]
    return a, m, n, psi


def torus_rhs(cp: np.ndarray, modes, center=(0.0, 0.0, 0.0), R: float = 1.0) -> np.ndarray:
    """f = sum_k a_k cos(m_k theta + n_k phi + psi_k) with phi = atan2(y, x)
    and theta = atan2(z, rho_xy - R), evaluated at the given surface points."""
    d = np.asarray(cp, dtype=np.float64) - np.asarray(center)
    phi = np.arctan2(d[:, 1], d[:, 0])
    theta = np.arctan2(d[:, 2], np.hypot(d[:, 0], d[:, 1]) - R)
    a, m, n, psi = modes
    f = np.zeros(len(d))
    for k in range(len(a)):
        f += a[k] * np.cos(m[k] * theta + n[k] * phi + psi[k])
    return f


def gaussian_vector(seed: int, n: int) -> np.ndarray:
    """i.i.d. N(0,1) per node in canonical order."""
    return normal(seed, n)
