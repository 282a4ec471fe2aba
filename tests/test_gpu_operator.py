"""GPU operator parity: the CUDA kernels (through the C ABI) against the FP64 oracle.

Tolerances (relative, max-norm over the field):
* FP64 paths: 1e-12.
* FP32 paths: 1e-5 (one FP32 operator apply; the error is a few ulps of the
  largest terms, ~1e-6 relative).
* FP16 / BF16 fields: every stored spinor is rounded to 11 / 8 significant
  bits relative to its (site, s) maximum.
* The block operator and the block preconditioner are checked element by
  element: every (site, s) against its own maximum (bounds derived at BTOL).
"""
import numpy as np
import pytest

from oracle import dwf_operator as op
from oracle import pointwise
from oracle import solvers as sv
from paper_1811_08488_gb300 import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5,
       # FP16/BF16: input and output rounded to 11 / 8 bits of their (site, s)
       # maximum, links to FP16: about 3 roundings of 2^-11 / 2^-8
       "fp16": 3e-3, "bf16": 2.5e-2}


def dwf():
    from paper_1811_08488_gb300 import dwf as d
    return d


def relerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def elem_relerr(got, want):
    """Largest, over the (s, site) elements of a canonical half field, of
    max|got - want| / max|want| with both maxima over that element's own 24
    reals: every element is held to the tolerance relative to its own size."""
    g = np.stack([got.real, got.imag], -1)
    w = np.stack([want.real, want.imag], -1)
    num = np.abs(g - w).max(axis=(-3, -2, -1))
    den = np.abs(w).max(axis=(-3, -2, -1))
    assert (den > 0).all()
    return float((num / den).max())


class Setup:
    def __init__(self, dims, Ls, b=1.5, c=0.5, M5=1.8, eps=0.4, seed=1, antiperiodic=True,
                 recon12=False):
        self.act = op.Action(dims=tuple(dims), Ls=Ls, M5=M5, b=b, c=c, antiperiodic=antiperiodic)
        self.Uc = syn.gauge_field(dims, eps, seed)
        self.U = op.gauge_to_mu_major(self.Uc)
        self.ctx = dwf().Context(dims, Ls, b=b, c=c, M5=M5, t_antiperiodic=antiperiodic,
                                 recon12=recon12)
        self.ctx.gauge_load(self.Uc)

    def to_native(self, halves, prec):
        """halves: list of canonical half fields (one per rhs) -> native device field."""
        canon = torch.from_numpy(np.ascontiguousarray(np.stack(halves))).cuda()
        nat = self.ctx.new_field(prec, len(halves))
        self.ctx.field_import(nat, prec, canon, len(halves))
        return nat

    def from_native(self, nat, prec, nrhs):
        canon = torch.zeros(self.ctx.canon_shape(nrhs), dtype=torch.complex128, device="cuda")
        self.ctx.field_export(canon, nat, prec, nrhs)
        torch.cuda.synchronize()
        return [c for c in canon.cpu().numpy()]

    def source(self, seed):
        return syn.half_field(self.act.dims, self.act.Ls, seed)


SHAPES = [
    ((4, 4, 4, 4), 4, dict()),
    ((2, 2, 2, 2), 4, dict()),                 # L = 2: x+mu and x-mu are the same site
    ((4, 6, 2, 8), 5, dict(b=1.0, c=0.0)),     # Shamir, odd Ls, ragged extents
    ((6, 4, 4, 2), 8, dict(antiperiodic=False)),
]


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16", "bf16"])
def test_import_export_roundtrip(prec):
    S = Setup((4, 2, 4, 6), 3)
    h = [S.source(5), S.source(6)]
    got = S.from_native(S.to_native(h, prec), prec, 2)
    for g, w in zip(got, h):
        if prec == "fp64":
            assert np.array_equal(g, w)
        elif prec == "fp32":
            assert relerr(g, w) < 1e-7
        else:
            # every real is stored relative to the maximum of its (site, s):
            # rounding error <= 2^-11 (FP16) or 2^-8 (BF16) of that maximum
            site_max = np.maximum(np.abs(w.real), np.abs(w.imag)).max(axis=(-2, -1))
            err = np.abs(g - w).max(axis=(-2, -1))
            bound = (2.0 ** -11 if prec == "fp16" else 2.0 ** -8) * np.sqrt(2) * 1.01
            assert (err <= bound * site_max).all()


@pytest.mark.parametrize("dims,Ls,kw", SHAPES)
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16", "bf16"])
@pytest.mark.parametrize("dagger", [0, 1])
def test_dslash_eo(dims, Ls, kw, prec, dagger):
    S = Setup(dims, Ls, **kw)
    masses = [0.03, 0.2]
    ins = [S.source(11), S.source(12)]
    for out_par in (0, 1):
        nat_in = S.to_native(ins, prec)
        nat_out = S.ctx.new_field(prec, 2)
        S.ctx.dslash_eo(nat_out, nat_in, out_par, dagger, prec, masses)
        got = S.from_native(nat_out, prec, 2)
        for r in range(2):
            full_in = op.half_to_full(ins[r], 1 - out_par)
            want = op.full_to_half(op.m4(S.act, S.U, full_in, masses[r], bool(dagger)), out_par)
            assert relerr(got[r], want) < TOL[prec], (out_par, r)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("dagger", [0, 1])
@pytest.mark.parametrize("Ls,kw", [(4, dict()), (12, dict()), (7, dict(b=1.0, c=0.0))])
def test_m5_and_m5inv(prec, dagger, Ls, kw):
    S = Setup((4, 2, 2, 4), Ls, **kw)
    masses = [0.01, 0.5]
    ins = [S.source(21), S.source(22)]
    nat_in = S.to_native(ins, prec)
    for fn, ref in ((S.ctx.m5, op.m5), (S.ctx.m5inv, op.m5inv)):
        out = S.ctx.new_field(prec, 2)
        fn(out, nat_in, dagger, prec, masses)
        got = S.from_native(out, prec, 2)
        for r in range(2):
            want = op.full_to_half(ref(S.act, op.half_to_full(ins[r], 0), masses[r], bool(dagger)), 0)
            assert relerr(got[r], want) < TOL[prec]


@pytest.mark.parametrize("dims,Ls,kw", SHAPES[:3])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_mpc_and_mdagm(dims, Ls, kw, prec):
    S = Setup(dims, Ls, **kw)
    masses = [0.05, 0.01]
    ins = [S.source(31), S.source(32)]
    nat_in = S.to_native(ins, prec)
    for dagger in (0, 1):
        out = S.ctx.new_field(prec, 2)
        S.ctx.mpc(out, nat_in, dagger, prec, masses)
        got = S.from_native(out, prec, 2)
        for r in range(2):
            want = op.full_to_half(op.mpc(S.act, S.U, op.half_to_full(ins[r], 0), masses[r],
                                          bool(dagger)), 0)
            assert relerr(got[r], want) < TOL[prec]
    out = S.ctx.new_field(prec, 2)
    S.ctx.mdagm(out, nat_in, prec, masses)
    got = S.from_native(out, prec, 2)
    for r in range(2):
        want = op.full_to_half(op.mdagm(S.act, S.U, op.half_to_full(ins[r], 0), masses[r]), 0)
        assert relerr(got[r], want) < TOL[prec]


def test_mdagm_hermitian_positive_fp64():
    """<x, A y> = <A x, y> and <x, A x> > 0 on the GPU in FP64."""
    S = Setup((4, 4, 4, 8), 6)
    x, y = S.source(41), S.source(42)
    nx, ny = S.to_native([x], "fp64"), S.to_native([y], "fp64")
    ax, ay = S.ctx.new_field("fp64"), S.ctx.new_field("fp64")
    S.ctx.mdagm(ax, nx, "fp64", 0.02)
    S.ctx.mdagm(ay, ny, "fp64", 0.02)
    Ax, Ay = S.from_native(ax, "fp64", 1)[0], S.from_native(ay, "fp64", 1)[0]
    lhs, rhs = np.vdot(x, Ay), np.vdot(Ax, y)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    assert np.vdot(x, Ax).real > 0


# ----------------------------------------------------------------------------
# block operator and preconditioner
# ----------------------------------------------------------------------------
# Element-wise bounds (each (site, s) against its own maximum). FP32 storage:
# a few hundred FP32 roundings along the four-hop chain, 1e-5. FP16 / BF16
# storage: four stored intermediates, each rounded to 2^-11 / 2^-8 of its own
# (site, s) maximum, so about 4 * 2^-11 = 2e-3 (FP16) and 1.6e-2 (BF16) of the
# terms that meet in one output element; an output element may be a few times
# smaller than those terms (partial cancellation of the M_5 and hop parts), so
# the bounds are 1e-2 and 8e-2. Any indexing or region error is O(1) and the
# FP32 case resolves errors down to 1e-5.
BTOL = {"fp32": 1e-5, "fp16": 1e-2, "bf16": 8e-2}


@pytest.mark.parametrize("dims,block", [((8, 4, 6, 4), (2, 2, 2, 4)), ((4, 8, 4, 8), (4, 2, 2, 4)),
                                        ((8, 8, 8, 8), (4, 4, 4, 4))])
@pytest.mark.parametrize("inner", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("snake", [1, 0])
def test_block_apply(dims, block, inner, snake):
    S = Setup(dims, 4)
    masses = [0.05, 0.3]
    ins = [S.source(51), S.source(52)]
    prm = dwf().default_params(block=block, inner=inner, snake=snake)
    nat_in = S.to_native(ins, "fp32")
    out = S.ctx.new_field("fp32", 2)
    S.ctx.block_apply(out, nat_in, prm, masses)
    got = S.from_native(out, "fp32", 2)
    origins = sv.block_origins(dims, block)
    for r in range(2):
        x = op.half_to_full(ins[r], 0)
        want = np.zeros_like(x)
        for o in origins:
            m = sv.block_mask(S.act, block, o)
            f = sv.a_block if snake else sv.a_block_truncated
            want += f(S.act, S.U, sv.project(x, m), masses[r], m)
        want = op.full_to_half(want, 0)
        err = elem_relerr(got[r], want)
        assert err < BTOL[inner], (r, err)


@pytest.mark.parametrize("inner", ["fp32", "fp16"])
@pytest.mark.parametrize("k", [1, 3, 6])
def test_block_precond(inner, k):
    S = Setup((8, 4, 4, 8), 4)
    block = (4, 4, 4, 4)
    masses = [0.05]
    r_in = [S.source(61)]
    prm = dwf().default_params(block=block, inner=inner, inner_iters=k)
    nat_r = S.to_native(r_in, "fp32")
    z = S.ctx.new_field("fp32", 1)
    S.ctx.block_precond(z, nat_r, prm, masses)
    got = S.from_native(z, "fp32", 1)[0]
    want = op.full_to_half(sv.ms_precondition(S.act, S.U, op.half_to_full(r_in[0], 0), masses[0],
                                              block, k, form="definition"), 0)
    err = elem_relerr(got, want)
    # k CG steps with block scalars formed from reductions over the whole
    # block: an element's error is set by the block's scale, not its own, so
    # the bound is wider than the operator's (FP32: 1e-5 per step; FP16:
    # 5e-2)
    assert err < (1e-5 * k if inner == "fp32" else 5e-2), err


@pytest.fixture(scope="module")
def production_blocks():
    """16^4 x Ls=12 lattice cut into the 8^3 x 16 blocks of the benchmark
    workload (8 blocks), so that every block's distance-1 and distance-2 rings
    and its per-block links have their production size. The oracle's box form
    of A_s (pinned against the definition on small lattices) gives A_s x on two
    of the blocks, and 2 inner CG steps on one of them."""
    S = Setup((16, 16, 16, 16), 12, eps=0.4, seed=1005)
    block, mf, k = (8, 8, 8, 16), 0.01, 2
    src = S.source(2005)
    x = op.half_to_full(src, 0)
    origins = sv.block_origins(S.act.dims, block)
    even = op.parity_mask(S.act.shape4) == 0
    want = {}
    for o in (origins[0], origins[-1]):
        m = sv.block_mask(S.act, block, o)
        want[o] = (m & even, sv.a_block_box(S.act, S.U, sv.project(x, m), mf, o, block))
    o = origins[-1]
    m = sv.block_mask(S.act, block, o)
    z = sv.cg_fixed(lambda v: sv.a_block_box(S.act, S.U, v, mf, o, block), sv.project(x, m), k)
    return S, block, mf, k, src, want, (m & even, z)


@pytest.mark.parametrize("inner", ["fp32", "fp16"])
def test_block_apply_production_shape(production_blocks, inner):
    S, block, mf, k, src, want, _ = production_blocks
    prm = dwf().default_params(block=block, inner=inner)
    out = S.ctx.new_field("fp32", 1)
    S.ctx.block_apply(out, S.to_native([src], "fp32"), prm, [mf])
    got = op.half_to_full(S.from_native(out, "fp32", 1)[0], 0)
    for o, (sel, w) in want.items():
        err = elem_relerr(got[:, sel], w[:, sel])
        assert err < BTOL[inner], (o, err)


@pytest.mark.parametrize("inner", ["fp32", "fp16"])
def test_block_precond_production_shape(production_blocks, inner):
    S, block, mf, k, src, _, (sel, zwant) = production_blocks
    prm = dwf().default_params(block=block, inner=inner, inner_iters=k)
    z = S.ctx.new_field("fp32", 1)
    S.ctx.block_precond(z, S.to_native([src], "fp32"), prm, [mf])
    got = op.half_to_full(S.from_native(z, "fp32", 1)[0], 0)
    err = elem_relerr(got[:, sel], zwant[:, sel])
    assert err < (1e-5 * k if inner == "fp32" else 5e-2), err


def test_dslash_full_size_sampled():
    """16^3x32 x Ls=12 (the measured workload): FP32 M^4 at sampled sites
    against the point-by-point oracle."""
    S = Setup((16, 16, 16, 32), 12, eps=0.4, seed=1001)
    mf = 0.01
    src = S.source(2001)
    nat_in = S.to_native([src], "fp32")
    out = S.ctx.new_field("fp32", 1)
    S.ctx.dslash_eo(out, nat_in, 0, 0, "fp32", [mf])
    got = S.from_native(out, "fp32", 1)[0]
    rng = np.random.default_rng(0)
    for _ in range(24):
        x, y, z, t = (int(rng.integers(0, L)) for L in S.act.dims)
        x = (x // 2) * 2 + ((y + z + t) % 2)  # even site
        s = int(rng.integers(0, 12))
        want = pointwise.m4_at(S.act, S.Uc, src, (x, y, z, t), s, mf)
        g = got[s, t, z, y, x // 2]
        assert np.abs(g - want).max() < 1e-5 * np.abs(want).max()


# ----------------------------------------------------------------------------
# reconstruct-12 links: FP32/FP16 link records keep two rows and the boundary
# sign; the operators must agree with the oracle at the same tolerances
# (the third row is rebuilt from rows that are SU(3) to FP64 accuracy).
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("dims,Ls,kw", [((4, 4, 4, 4), 4, dict()), ((4, 6, 2, 8), 5, dict(b=1.0, c=0.0)),
                                        ((6, 4, 4, 2), 8, dict(antiperiodic=False))])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16", "bf16"])
@pytest.mark.parametrize("dagger", [0, 1])
def test_dslash_eo_recon12(dims, Ls, kw, prec, dagger):
    S = Setup(dims, Ls, recon12=True, **kw)
    masses = [0.03, 0.2]
    ins = [S.source(13), S.source(14)]
    for out_par in (0, 1):
        nat_in = S.to_native(ins, prec)
        nat_out = S.ctx.new_field(prec, 2)
        S.ctx.dslash_eo(nat_out, nat_in, out_par, dagger, prec, masses)
        got = S.from_native(nat_out, prec, 2)
        for r in range(2):
            full_in = op.half_to_full(ins[r], 1 - out_par)
            want = op.full_to_half(op.m4(S.act, S.U, full_in, masses[r], bool(dagger)), out_par)
            assert relerr(got[r], want) < TOL[prec], (out_par, r)


def test_mdagm_and_block_apply_recon12():
    S = Setup((8, 4, 6, 4), 4, recon12=True)
    masses = [0.05, 0.3]
    ins = [S.source(53), S.source(54)]
    nat_in = S.to_native(ins, "fp32")
    out = S.ctx.new_field("fp32", 2)
    S.ctx.mdagm(out, nat_in, "fp32", masses)
    got = S.from_native(out, "fp32", 2)
    for r in range(2):
        want = op.full_to_half(op.mdagm(S.act, S.U, op.half_to_full(ins[r], 0), masses[r]), 0)
        assert relerr(got[r], want) < TOL["fp32"]
    block = (2, 2, 2, 4)
    for inner in ("fp32", "fp16"):
        prm = dwf().default_params(block=block, inner=inner)
        out = S.ctx.new_field("fp32", 2)
        S.ctx.block_apply(out, nat_in, prm, masses)
        got = S.from_native(out, "fp32", 2)
        for r in range(2):
            x = op.half_to_full(ins[r], 0)
            want = np.zeros_like(x)
            for o in sv.block_origins(S.act.dims, block):
                m = sv.block_mask(S.act, block, o)
                want += sv.a_block(S.act, S.U, sv.project(x, m), masses[r], m)
            want = op.full_to_half(want, 0)
            err = elem_relerr(got[r], want)
            assert err < BTOL[inner], (inner, r, err)


def test_mspcg_solve_recon12():
    S = Setup((4, 4, 4, 8), 6, recon12=True)
    mf = 0.05
    b = S.source(55)
    bt = torch.from_numpy(b[None].copy()).cuda()
    x = torch.zeros_like(bt)
    prm = dwf().default_params(block=(2, 2, 2, 4), inner="fp16", inner_iters=4, tol=1e-10)
    st, info = S.ctx.solve(x, bt, [mf], prm)
    assert st == 0 and info[0]["converged"]
    xf = op.half_to_full(x[0].cpu().numpy(), 0)
    bf = op.half_to_full(b, 0)
    r = bf - op.mdagm(S.act, S.U, xf, mf)
    assert np.sqrt(op.norm2(r) / op.norm2(bf)) <= 1e-10
