"""CG, the multisplitting block operator and MSPCG in plain numpy (FP64).

Test infrastructure only (see oracle/__init__.py).

Paper references:
* Sec. 2.1, eqs. (local) and (eq:ms): A x = b split on one sub-lattice s as
  A_s x_s + A_l x_l + A_r x_r = b_s; A_s is the part of A that couples the
  sub-lattice to itself.
* Sec. 2.3: A_s is taken from the whole 4-hop normal operator D_PC^dag D_PC with
  Dirichlet boundaries, so "snake" paths that leave the sub-lattice and come
  back are kept: A_s = P_s A P_s. Enforcing the boundary on each hop instead
  drops them (the truncated operator).
* Algorithm 1 (preconditioned CG) and Sec. 2.4: with a zero guess and one
  multisplitting sweep the preconditioner is M = (+)_s A_s; each A_s z_s = r_s
  is solved by a fixed number k of plain CG iterations (Sec. 3).

Readings where the paper is silent (they are listed in the design notes too):
x_0 = 0; convergence is |b - A x| / |b| <= tol with a recomputed residual;
<a, b> = sum conj(a) b and the real part of <r, z> is used; inner CG scalars are
per sub-lattice; blocks have even extents and keep global parity; a direction
with a single block keeps its periodic wrap inside the block.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import dwf_operator as op


# ----------------------------------------------------------------------------
# Plain CG and fixed-iteration CG
# ----------------------------------------------------------------------------
def cg(apply_A, b, tol: float, maxiter: int = 100000):
    """Plain CG on A x = b from x_0 = 0 (Algorithm 1 with M = 1).

    Stops when the recomputed residual |b - A x| / |b| <= tol. Returns
    (x, iterations, true relative residual).
    """
    bnorm = np.sqrt(op.norm2(b))
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = op.norm2(r)
    it = 0
    while it < maxiter:
        Ap = apply_A(p)
        alpha = rr / op.vdot(p, Ap).real
        x = x + alpha * p
        r = r - alpha * Ap
        rr_new = op.norm2(r)
        it += 1
        if np.sqrt(rr_new) <= tol * bnorm:
            rt = b - apply_A(x)
            res = np.sqrt(op.norm2(rt)) / bnorm
            if res <= tol:
                return x, it, res
            r = rt
            rr_new = op.norm2(r)
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
    rt = b - apply_A(x)
    return x, it, np.sqrt(op.norm2(rt)) / bnorm


def cg_fixed(apply_A, r, k: int):
    """k iterations of plain CG on A z = r from z = 0 (the paper's inner solve,
    Sec. 3: a fixed count, no precision-based stop). Returns z."""
    z = np.zeros_like(r)
    res = r.copy()
    p = res.copy()
    rr = op.norm2(res)
    for _ in range(k):
        if rr == 0.0:
            break
        Ap = apply_A(p)
        pAp = op.vdot(p, Ap).real
        alpha = rr / pAp
        z = z + alpha * p
        res = res - alpha * Ap
        rr_new = op.norm2(res)
        beta = rr_new / rr
        p = res + beta * p
        rr = rr_new
    return z


def cg_stop(apply_A, r, kmax: int, eps: float):
    """CG on A z = r from z = 0 that stops at the first iteration whose
    recursively updated residual satisfies |r_k| <= eps |r|, or after kmax
    iterations (the inner solve with a residual stop instead of a fixed k, a
    variant the paper's Sec. 4 invites). Returns (z, iterations)."""
    z = np.zeros_like(r)
    res = r.copy()
    p = res.copy()
    rr = op.norm2(res)
    stop = eps * eps * rr
    k = 0
    while k < kmax and rr > stop and rr > 0.0:
        Ap = apply_A(p)
        alpha = rr / op.vdot(p, Ap).real
        z = z + alpha * p
        res = res - alpha * Ap
        rr_new = op.norm2(res)
        p = res + (rr_new / rr) * p
        rr = rr_new
        k += 1
    return z, k


def pcg(apply_A, apply_Minv, b, tol: float, maxiter: int = 100000, x0=None):
    """Algorithm 1: preconditioned CG on A x = b, x_0 = 0 (or the given x0,
    with r_0 = b - A x_0).

    alpha_k = <r_k, z_k> / <p_k, A p_k>; x += alpha p; r -= alpha A p;
    z = M^-1 r; beta_k = <z_{k+1}, r_{k+1}> / <z_k, r_k>; p = z + beta p.
    Converged when the recomputed residual satisfies |b - A x| / |b| <= tol.
    Returns (x, outer iterations, true relative residual).
    """
    bnorm = np.sqrt(op.norm2(b))
    if x0 is None:
        x = np.zeros_like(b)
        r = b.copy()
    else:
        x = x0.copy()
        r = b - apply_A(x)
        if np.sqrt(op.norm2(r)) <= tol * bnorm:
            return x, 0, np.sqrt(op.norm2(r)) / bnorm
    z = apply_Minv(r)
    p = z.copy()
    rz = op.vdot(r, z).real
    it = 0
    while it < maxiter:
        Ap = apply_A(p)
        alpha = rz / op.vdot(p, Ap).real
        x = x + alpha * p
        r = r - alpha * Ap
        it += 1
        if np.sqrt(op.norm2(r)) <= tol * bnorm:
            rt = b - apply_A(x)
            res = np.sqrt(op.norm2(rt)) / bnorm
            if res <= tol:
                return x, it, res
            r = rt
        z = apply_Minv(r)
        rz_new = op.vdot(z, r).real
        beta = rz_new / rz
        p = z + beta * p
        rz = rz_new
    rt = b - apply_A(x)
    return x, it, np.sqrt(op.norm2(rt)) / bnorm


# ----------------------------------------------------------------------------
# Sub-lattices (the paper's per-processor blocks)
# ----------------------------------------------------------------------------
def block_origins(dims, block):
    """Origins (x, y, z, t) of the blocks of extent `block` tiling `dims`."""
    for d, bl in zip(dims, block):
        if bl <= 0 or d % bl != 0 or bl % 2 != 0:
            raise ValueError("block extents must be even and divide the lattice")
    ranges = [range(0, d, bl) for d, bl in zip(dims, block)]
    # x fastest
    return [(x, y, z, t) for t, z, y, x in itertools.product(*reversed(ranges))]


def block_mask(act: op.Action, block, origin) -> np.ndarray:
    """Boolean (T,Z,Y,X) mask of the sites of one block (the projector P_s)."""
    t, z, y, x = np.indices(act.shape4)
    m = np.ones(act.shape4, dtype=bool)
    for coord, o, bl in zip((x, y, z, t), origin, block):
        m &= (coord >= o) & (coord < o + bl)
    return m


def project(psi: np.ndarray, mask4: np.ndarray) -> np.ndarray:
    return psi * mask4[None, :, :, :, :, None, None]


def a_block(act: op.Action, U, x, mf: float, mask4, schur: str = "asym") -> np.ndarray:
    """A_s x = P_s D_PC^dag D_PC P_s x on the full lattice (snake terms kept).

    This is the definition of Sec. 2.3: Dirichlet conditions on the whole
    normal operator, so every path that leaves the block and comes back
    contributes. schur="sym": the same with the symmetric form's normal
    operator."""
    return project(op.normal_op(schur)(act, U, project(x, mask4), mf), mask4)


def a_block_truncated(act: op.Action, U, x, mf: float, mask4) -> np.ndarray:
    """The snake-truncated block operator of Sec. 2.3: Dirichlet conditions on
    each of the four hops in turn, i.e. every M^4 is replaced by P_s M^4 P_s."""

    def mpc_t(v, dag):
        t = project(op.restrict_parity(op.m4(act, U, project(v, mask4), mf, dag), 1), mask4)
        t = op.m5inv(act, t, mf, dag)
        t = project(op.restrict_parity(op.m4(act, U, t, mf, dag), 0), mask4)
        return op.m5(act, v, mf, dag) - t

    xs = project(x, mask4)
    return project(mpc_t(mpc_t(xs, False), True), mask4)


# ----------------------------------------------------------------------------
# Box form of A_s: the block plus a two-site halo cut out as a small lattice.
# ----------------------------------------------------------------------------
def box_extent(L: int, bl: int) -> int:
    """Extent of the cut-out box in one direction: the block plus two sites on
    each side, or the whole direction when that does not fit."""
    return bl + 4 if L >= bl + 4 else L


def extract_box(act: op.Action, U, origin, block):
    """Cut the box around one block out of the lattice.

    Returns (box action, box links, box -> lattice coordinate maps). The box is
    a small periodic lattice whose links are the lattice links with the
    boundary sign of the lattice folded in; the box's own wrap links are never
    reached by a path that contributes to A_s on the block, because every
    contributing path stays within two hops of the block."""
    ext, coords = [], []
    for L, o, bl in zip(act.dims, origin, block):
        e = box_extent(L, bl)
        ext.append(e)
        start = o - 2 if e == bl + 4 else 0
        coords.append((start + np.arange(e)) % L)
    bx, by, bz, bt = coords
    Ub = U[:, bt][:, :, bz][:, :, :, by][:, :, :, :, bx].copy()
    if act.antiperiodic:
        # the t link leaving t = Lt-1 carries the antiperiodic sign
        sel = bt == act.dims[3] - 1
        Ub[3, sel] *= -1.0
    box = op.Action(dims=tuple(ext), Ls=act.Ls, M5=act.M5, b=act.b, c=act.c, antiperiodic=False)
    return box, Ub, coords


def a_block_box(act: op.Action, U, x, mf: float, origin, block, schur: str = "asym") -> np.ndarray:
    """A_s x computed on the cut-out box; equal to a_block (pinned by a test).

    The box origin is chosen so that box parity equals lattice parity (all
    offsets are even because the block origin and extents are even)."""
    box, Ub, (bx, by, bz, bt) = extract_box(act, U, origin, block)
    xb = x[:, bt][:, :, bz][:, :, :, by][:, :, :, :, bx]
    inb = np.ones(box.shape4, dtype=bool)
    t, z, y, xx = np.indices(box.shape4)
    for coord, c_lat, o, bl in zip((xx, y, z, t), (bx, by, bz, bt), origin, block):
        inb &= (c_lat[coord] >= o) & (c_lat[coord] < o + bl)
    yb = project(op.normal_op(schur)(box, Ub, project(xb, inb), mf), inb)
    out = np.zeros_like(x)
    T, Z, Y, X = np.meshgrid(bt, bz, by, bx, indexing="ij")
    out[:, T[inb], Z[inb], Y[inb], X[inb]] = yb[:, inb]
    return out


# ----------------------------------------------------------------------------
# Multisplitting preconditioner and MSPCG
# ----------------------------------------------------------------------------
def ms_precondition(act: op.Action, U, r, mf: float, block, k: int,
                    snake: bool = True, form: str = "box", inner_tol: float = 0.0,
                    schur: str = "asym") -> np.ndarray:
    """z = M^-1 r with M = (+)_s A_s (Sec. 2.4): on every block, k CG iterations
    on A_s z_s = r_s from a zero guess, with block-local scalars; no coupling
    between blocks. inner_tol > 0: each block stops early once its residual
    fell by inner_tol (cg_stop, at most k iterations)."""
    z = np.zeros_like(r)
    for origin in block_origins(act.dims, block):
        mask = block_mask(act, block, origin)
        if not snake:
            A = lambda v, m=mask: a_block_truncated(act, U, v, mf, m)
        elif form == "box":
            A = lambda v, o=origin: a_block_box(act, U, v, mf, o, block, schur)
        else:
            A = lambda v, m=mask: a_block(act, U, v, mf, m, schur)
        rs = project(r, mask)
        zs = cg_stop(A, rs, k, inner_tol)[0] if inner_tol > 0 else cg_fixed(A, rs, k)
        z += project(zs, mask)
    return z


def mspcg(act: op.Action, U, b, mf: float, block, k: int, tol: float,
          maxiter: int = 100000, snake: bool = True, inner_tol: float = 0.0,
          schur: str = "asym"):
    """MSPCG: Algorithm 1 with the multisplitting preconditioner, on the normal
    equation of the paper's D_PC (schur="asym") or of the symmetric form."""
    A = lambda v: op.normal_op(schur)(act, U, v, mf)
    Minv = lambda v: ms_precondition(act, U, v, mf, block, k, snake, inner_tol=inner_tol,
                                     schur=schur)
    return pcg(A, Minv, b, tol, maxiter)
