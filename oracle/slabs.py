"""A = D_PC^dag D_PC on lattices too large for one full-array evaluation.

Test infrastructure only (see oracle/__init__.py).

A couples sites at most four apart: D_PC = M_5 - M^4_eo M_5^-1 M^4_oe moves a
field by at most one site in each of its two hops, and A = D_PC^dag D_PC
applies it twice (paper Sec. 2.2, eq. (dirac_equation) and eq. (DdagD)); M_5
and M_5^-1 act in s only. So A x on a slab of time slices is exact when it is
computed on a small lattice that holds the slab plus four time slices on each
side: the small lattice's own periodic wrap in t only changes sites within four
slices of its ends, which are dropped. Its x, y and z extents are the full
periodic extents, so those directions need no halo. The antiperiodic sign of
the links that leave t = Lt - 1 is folded into those links, and the small
lattice is periodic.

The slabs are independent, so a pool of worker processes (started with
"spawn") evaluates them side by side with the oracle's own op.mdagm.
"""
from __future__ import annotations

import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np

from . import dwf_operator as op


def _slab_rows(Lt: int, t0: int, n: int, halo: int):
    """Global t of the rows of the small lattice for slab [t0, t0 + n)."""
    return [(t0 - halo + i) % Lt for i in range(n + 2 * halo)]


def _apply_on_slab(act_kw, U_rows, x_rows, mf, t_rows, Lt, antiperiodic, halo):
    """A x on the small lattice built from the given rows; returns the half
    field of the inner rows (even parity, canonical layout)."""
    dims = tuple(act_kw["dims"][:3]) + (len(t_rows),)
    box = op.Action(dims=dims, Ls=act_kw["Ls"], M5=act_kw["M5"], b=act_kw["b"], c=act_kw["c"],
                    antiperiodic=False)
    U = op.gauge_to_mu_major(U_rows)
    if antiperiodic:
        last = np.array(t_rows) == Lt - 1
        U[3, last] *= -1.0
    # the first row has even global t (slab and halo are even), so local
    # parity equals global parity
    x = op.half_to_full(x_rows, 0)
    y = op.full_to_half(op.mdagm(box, U, x, mf), 0)
    return y[:, halo:len(t_rows) - halo]


def mdagm_half(act: op.Action, U_canon: np.ndarray, x_half: np.ndarray, mf: float,
               slab: int = 4, workers: int | None = None) -> np.ndarray:
    """A x for an even half field x (canonical layout [s][t][z][y][xh][4][3])
    and canonical links U[t][z][y][x][mu][3][3], evaluated in t slabs of
    `slab` rows (slab even, dividing Lt) by worker processes. Returns A x in
    the canonical half layout."""
    Lt = act.dims[3]
    halo = 4
    if slab % 2 or Lt % slab:
        raise ValueError("slab must be even and divide Lt")
    if Lt <= slab + 2 * halo:
        return op.full_to_half(op.mdagm(act, op.gauge_to_mu_major(U_canon),
                                        op.half_to_full(x_half, 0), mf), 0)
    kw = dict(dims=act.dims, Ls=act.Ls, M5=act.M5, b=act.b, c=act.c)
    starts = list(range(0, Lt, slab))
    rows = [_slab_rows(Lt, t0, slab, halo) for t0 in starts]
    out = np.empty_like(x_half)
    nw = workers or max(1, min(16, os.cpu_count() or 1, len(starts)))
    with cf.ProcessPoolExecutor(nw, mp_context=mp.get_context("spawn")) as ex:
        futs = [ex.submit(_apply_on_slab, kw, U_canon[r], x_half[:, r], mf, r, Lt,
                          act.antiperiodic, halo) for r in rows]
        for t0, f in zip(starts, futs):
            out[:, t0:t0 + slab] = f.result()
    return out
