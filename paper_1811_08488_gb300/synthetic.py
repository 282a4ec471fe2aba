"""Seeded synthetic inputs: SU(3) gauge fields and Gaussian sources.

This module only draws random inputs. It holds none of the solver's or the
operator's arithmetic, so both the CPU oracle and the CUDA path may use it.

Random numbers come from a counter-based splitmix64 stream (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): draw i
of stream `seed` is mix(seed + (i + 1) * 0x9E3779B97F4A7C15). Normal deviates
come from the Box-Muller transform applied to consecutive pairs of uniforms.

Layouts (all complex128, C order):

* gauge field  U[t][z][y][x][mu][a][b], mu = 0..3 for x, y, z, t; U_mu(x) is the
  3x3 matrix on the link from x to x + mu.
* parity half field  psi[s][t][z][y][xh][spin][colour], where the site of row
  (y, z, t) and half index xh is x = 2*xh + ((parity + y + z + t) % 2).
"""
from __future__ import annotations

import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Draws offset .. offset+count-1 of the splitmix64 stream `seed` (uint64)."""
    i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform deviates in the open interval (0, 1) from the top 53 bits
    (draws offset .. offset+count-1 of the stream)."""
    z = splitmix64(seed, count, offset)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normal(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Standard normal deviates by Box-Muller on pairs (u1, u2): deviates
    offset .. offset+count-1 of stream `seed` (offset even, so that a slice
    starts on a pair)."""
    if offset % 2:
        raise ValueError("normal(): offset must be even")
    n2 = (count + 1) // 2
    u = uniform(seed, 2 * n2, offset).reshape(n2, 2)
    rad = np.sqrt(-2.0 * np.log(u[:, 0]))
    ang = 2.0 * np.pi * u[:, 1]
    out = np.empty((n2, 2))
    out[:, 0] = rad * np.cos(ang)
    out[:, 1] = rad * np.sin(ang)
    return out.reshape(-1)[:count]


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices lambda_1..lambda_8 as an (8, 3, 3) array."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1], lam[1][1, 0] = -1j, 1j
    lam[2][0, 0], lam[2][1, 1] = 1, -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2], lam[4][2, 0] = -1j, 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2], lam[6][2, 1] = -1j, 1j
    lam[7] = np.diag([1, 1, -2]) / np.sqrt(3.0)
    return lam


def su3_exp(h: np.ndarray, eps: float) -> np.ndarray:
    """exp(i*eps*H) for H = sum_a h_a lambda_a / 2, over a batch of h (..., 8).

    H is Hermitian and traceless, so the result is in SU(3). The exponential
    is taken through the eigendecomposition of H and then re-unitarised by a
    polar step (one Newton iteration of U <- (U + U^-dagger)/2 suffices at
    machine precision; it is kept so the links are unitary to ~1e-16).
    """
    lam = gell_mann()
    H = np.einsum("...a,aij->...ij", h, lam) * 0.5
    w, v = np.linalg.eigh(H)
    ph = np.exp(1j * eps * w)
    U = np.einsum("...ik,...k,...jk->...ij", v, ph, v.conj())
    Uinv_dag = np.linalg.inv(U).conj().swapaxes(-1, -2)
    U = 0.5 * (U + Uinv_dag)
    # fix the overall phase so det U = 1 exactly up to rounding
    det = np.linalg.det(U)
    U = U * (det.conj() ** (1.0 / 3.0) / np.abs(det) ** (1.0 / 3.0))[..., None, None]
    return U


# Large fields are drawn in slabs by a pool of worker processes (started with
# "spawn", so a process that already uses a GPU can call this safely). Every
# slab reads its own part of the counter-based stream, so the result is the
# same array as the serial draw.
PARALLEL_MIN = 1 << 24  # deviates; smaller draws stay in this process


def _pool_workers() -> int:
    return max(1, min(16, os.cpu_count() or 1))


def _gauge_slab(dims, eps, seed, t):
    Lx, Ly, Lz, Lt = dims
    per = Lx * Ly * Lz * 4 * 8
    h = normal(seed, per, t * per).reshape(1, Lz, Ly, Lx, 4, 8)
    return su3_exp(h, eps)


def _normal_slab(seed, count, offset):
    return normal(seed, count, offset)


def gauge_field(dims, eps: float, seed: int, parallel_min: int = PARALLEL_MIN) -> np.ndarray:
    """Synthetic SU(3) links U = exp(i eps H), H Gaussian traceless Hermitian.

    dims = (Lx, Ly, Lz, Lt). Returns U[t][z][y][x][mu][3][3] complex128.
    Draw order: site (lexicographic, x fastest), then mu, then a = 1..8.
    """
    Lx, Ly, Lz, Lt = dims
    n = Lx * Ly * Lz * Lt * 4 * 8
    if n < parallel_min or _pool_workers() == 1 or Lt == 1:
        h = normal(seed, n).reshape(Lt, Lz, Ly, Lx, 4, 8)
        return su3_exp(h, eps)
    with cf.ProcessPoolExecutor(_pool_workers(), mp_context=mp.get_context("spawn")) as ex:
        slabs = list(ex.map(_gauge_slab, [dims] * Lt, [eps] * Lt, [seed] * Lt, range(Lt)))
    return np.concatenate(slabs, axis=0)


def unit_gauge(dims) -> np.ndarray:
    Lx, Ly, Lz, Lt = dims
    U = np.zeros((Lt, Lz, Ly, Lx, 4, 3, 3), dtype=np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1
    return U


def random_su3(shape, seed: int) -> np.ndarray:
    """Haar-ish random SU(3) matrices (used for gauge transformations)."""
    n = int(np.prod(shape)) * 8
    h = normal(seed, n).reshape(tuple(shape) + (8,))
    return su3_exp(h, 2.0)


def half_field(dims, Ls: int, seed: int, parallel_min: int = PARALLEL_MIN) -> np.ndarray:
    """Gaussian complex parity half field psi[s][t][z][y][xh][4][3].

    Real and imaginary parts are independent N(0,1); they are drawn as
    consecutive pairs (re, im) in the C order of the array.
    """
    Lx, Ly, Lz, Lt = dims
    shape = (Ls, Lt, Lz, Ly, Lx // 2, 4, 3)
    n = int(np.prod(shape))
    if 2 * n < parallel_min or _pool_workers() == 1:
        z = normal(seed, 2 * n).reshape(n, 2)
        return (z[:, 0] + 1j * z[:, 1]).reshape(shape)
    per = 2 * n // Ls  # deviates of one s slice
    with cf.ProcessPoolExecutor(_pool_workers(), mp_context=mp.get_context("spawn")) as ex:
        parts = list(ex.map(_normal_slab, [seed] * Ls, [per] * Ls, [s * per for s in range(Ls)]))
    out = np.empty(shape, dtype=np.complex128)
    for s, z in enumerate(parts):
        z = z.reshape(-1, 2)
        out[s] = (z[:, 0] + 1j * z[:, 1]).reshape(shape[1:])
    return out


def log_spaced_masses(lo: float, hi: float, n: int) -> np.ndarray:
    """n quark masses log-spaced over [lo, hi]."""
    if n == 1:
        return np.array([lo])
    return np.exp(np.linspace(np.log(lo), np.log(hi), n))


# Workloads: the lattices and actions the solver is measured on. Seeds follow
# gauge = 1000 + workload, source = 2000 + workload + rhs.
WORKLOADS = {
    "shamir_8^4x8": dict(dims=(8, 8, 8, 8), Ls=8, b=1.0, c=0.0, M5=1.8, mf=[0.1],
                         eps=0.3, id=0, block=(4, 4, 4, 4)),
    "mobius_16^3x32x12": dict(dims=(16, 16, 16, 32), Ls=12, b=1.5, c=0.5, M5=1.8,
                              mf=[0.01], eps=0.4, id=1, block=(8, 8, 8, 16)),
    "mobius_24^3x64x16": dict(dims=(24, 24, 24, 64), Ls=16, b=1.5, c=0.5, M5=1.8,
                              mf=[0.003], eps=0.45, id=2, block=(12, 12, 12, 16)),
    "mobius_16^3x32x12_16rhs": dict(dims=(16, 16, 16, 32), Ls=12, b=1.5, c=0.5, M5=1.8,
                                    mf=list(log_spaced_masses(0.001, 0.05, 16)),
                                    eps=0.4, id=3, block=(8, 8, 8, 16)),
    "mobius_32^3x64x12_4rhs": dict(dims=(32, 32, 32, 64), Ls=12, b=1.5, c=0.5, M5=1.8,
                                   mf=[0.0008] * 4, eps=0.5, id=4, block=(8, 8, 8, 16)),
}


def workload_inputs(name: str, nrhs: int | None = None):
    """Gauge field and sources (canonical layouts) for a named workload."""
    w = WORKLOADS[name]
    U = gauge_field(w["dims"], w["eps"], 1000 + w["id"])
    n = len(w["mf"]) if nrhs is None else nrhs
    srcs = [half_field(w["dims"], w["Ls"], 2000 + w["id"] + r) for r in range(n)]
    return U, srcs
