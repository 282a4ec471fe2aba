"""Full-size workloads on the GPU, checked by the FP64 oracle or by properties
that hold at any size.

* Shamir 8^4 x 8, plain FP64 CG: oracle residual and oracle solution.
* Moebius 16^3 x 32 x 12 (the benchmark solve, MSPCG with 8^3 x 16 blocks,
  k = 6, FP16 inner): oracle FP64 residual of the GPU solution.
* Moebius 16^3 x 32 x 12 with 16 right-hand sides of log-spaced masses in one
  call (per-rhs early exit): every rhs converges, lighter masses need more
  iterations, oracle residual of the lightest.
* Moebius 24^3 x 64 x 16 (m_f 0.003, the benchmark's headline solve, MSPCG
  with 12^3 x 16 blocks, k = 6, FP16 inner): the oracle recomputes the FP64
  residual of the GPU solution over the whole lattice, slab by slab on the
  host's cores.
* The multisplitting preconditioner at full size is block diagonal: z on a
  block depends only on r on that block.
"""
import numpy as np
import pytest

from oracle import dwf_operator as op
from oracle import solvers as sv
from paper_1811_08488_gb300 import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dwf():
    from paper_1811_08488_gb300 import dwf as d
    return d


def load(name, nrhs=None):
    w = syn.WORKLOADS[name]
    U, srcs = syn.workload_inputs(name, nrhs)
    act = op.Action(dims=w["dims"], Ls=w["Ls"], M5=w["M5"], b=w["b"], c=w["c"])
    ctx = dwf().Context(w["dims"], w["Ls"], b=w["b"], c=w["c"], M5=w["M5"])
    ctx.gauge_load(U)
    return w, act, U, srcs, ctx


def oracle_resid(act, U, x_half, b_half, mf):
    xf = op.half_to_full(x_half, 0)
    bf = op.half_to_full(b_half, 0)
    r = bf - op.mdagm(act, U, xf, mf)
    return np.sqrt(op.norm2(r) / op.norm2(bf))


def solve(ctx, srcs, masses, **kw):
    b = torch.from_numpy(np.ascontiguousarray(np.stack(srcs))).cuda()
    x = torch.zeros_like(b)
    st, info = ctx.solve(x, b, masses, dwf().default_params(**kw))
    return st, info, x.cpu().numpy()


def test_shamir_8x8x8x8_plain_cg_fp64():
    w, act, U, srcs, ctx = load("shamir_8^4x8")
    mf = w["mf"][0]
    st, info, x = solve(ctx, srcs, [mf], inner_iters=0, outer=dwf().DWF_FP64, tol=1e-10)
    assert st == 0 and info[0]["converged"]
    Um = op.gauge_to_mu_major(U)
    assert oracle_resid(act, Um, x[0], srcs[0], mf) <= 1e-10
    xo, it, _ = sv.cg(lambda v: op.mdagm(act, Um, v, mf), op.half_to_full(srcs[0], 0), 1e-11)
    rel = np.linalg.norm(x[0] - op.full_to_half(xo, 0)) / np.linalg.norm(xo)
    assert rel < 1e-8


def test_mobius_16x16x16x32_mspcg_benchmark_solve():
    w, act, U, srcs, ctx = load("mobius_16^3x32x12")
    mf = w["mf"][0]
    st, info, x = solve(ctx, srcs, [mf], inner_iters=6, block=w["block"], inner="fp16",
                        tol=1e-10)
    assert st == 0 and info[0]["converged"]
    assert oracle_resid(act, op.gauge_to_mu_major(U), x[0], srcs[0], mf) <= 1e-10


def test_mobius_24x24x24x64_mspcg_oracle_residual():
    """The benchmark's headline solve. Host memory: the inputs and the solution
    (about 4 GB) and the oracle's worker processes (about 1.5 GB each, up to 16
    of them). The oracle's FP64 |b - A x| / |b| must be <= 1e-10 and agree with
    the library's own FP64 recomputation."""
    from oracle import slabs
    w, act, U, srcs, ctx = load("mobius_24^3x64x16")
    mf = w["mf"][0]
    st, info, x = solve(ctx, srcs, [mf], inner_iters=6, block=w["block"], inner="fp16",
                        tol=1e-10)
    ctx.close()
    assert st == 0 and info[0]["converged"] and info[0]["true_resid"] <= 1e-10
    b = srcs[0]
    r = b - slabs.mdagm_half(act, U, x[0], mf, slab=4)
    res = float(np.sqrt(np.vdot(r, r).real / np.vdot(b, b).real))
    assert res <= 1e-10
    assert abs(res - info[0]["true_resid"]) <= 1e-3 * res


def test_mobius_16_rhs_log_spaced_masses_one_call():
    w, act, U, srcs, ctx = load("mobius_16^3x32x12_16rhs")
    masses = w["mf"]
    st, info, x = solve(ctx, srcs, masses, inner_iters=6, block=w["block"], inner="fp16",
                        tol=1e-10)
    assert st == 0
    assert all(i["converged"] and i["true_resid"] <= 1e-10 for i in info)
    its = [i["outer_iters"] for i in info]
    assert its[0] >= its[-1] and its[0] > its[-1] + 5, its
    assert oracle_resid(act, op.gauge_to_mu_major(U), x[0], srcs[0], masses[0]) <= 1e-10


def test_preconditioner_is_block_diagonal_at_full_size():
    w, act, U, srcs, ctx = load("mobius_16^3x32x12")
    mf = w["mf"][0]
    block = w["block"]
    prm = dwf().default_params(block=block, inner="fp16", inner_iters=6)
    full = srcs[0]
    # r restricted to block 0 (origin 0): zero elsewhere
    mask = sv.block_mask(act, block, (0, 0, 0, 0))
    r0 = op.full_to_half(sv.project(op.half_to_full(full, 0), mask), 0)
    outs = []
    for r in (full, r0):
        canon = torch.from_numpy(r[None].copy()).cuda()
        nat, z = ctx.new_field("fp32"), ctx.new_field("fp32")
        ctx.field_import(nat, "fp32", canon)
        ctx.block_precond(z, nat, prm, [mf])
        got = torch.zeros_like(canon)
        ctx.field_export(got, z, "fp32")
        torch.cuda.synchronize()
        outs.append(op.half_to_full(got.cpu().numpy()[0], 0))
    z_full, z_0 = outs
    inside = mask[None, :, :, :, :, None, None]
    # nothing leaks out of the block
    assert np.abs(np.where(inside, 0, z_0)).max() == 0.0
    # and on the block it is the same as with r everywhere
    diff = np.abs(np.where(inside, z_full - z_0, 0)).max()
    assert diff <= 1e-6 * np.abs(np.where(inside, z_full, 0)).max()


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("fp16", 3e-3)])
@pytest.mark.parametrize("dagger", [0, 1])
def test_m5inv_gemm_sixteen_rhs_full_size_sampled(prec, tol, dagger):
    """The tensor-core M_5^-1 in the launch the benchmark times (16^3x32 x 12,
    16 right-hand sides of log-spaced masses, one call) against the oracle's
    dense inverse of M_5 on sampled (site, rhs) columns."""
    name = "mobius_16^3x32x12_16rhs"
    w = syn.WORKLOADS[name]
    act = op.Action(dims=w["dims"], Ls=w["Ls"], M5=w["M5"], b=w["b"], c=w["c"])
    ctx = dwf().Context(w["dims"], w["Ls"], b=w["b"], c=w["c"], M5=w["M5"])
    _, srcs = syn.workload_inputs(name)
    masses = list(w["mf"])
    nr = len(masses)
    canon = torch.from_numpy(np.ascontiguousarray(np.stack(srcs))).cuda()
    fin, fout = ctx.new_field(prec, nr), ctx.new_field(prec, nr)
    ctx.field_import(fin, prec, canon, nr)
    ctx.m5inv_gemm(fout, fin, dagger, prec, masses)
    got = torch.zeros_like(canon)
    ctx.field_export(got, fout, prec, nr)
    stored = torch.zeros_like(canon)
    ctx.field_export(stored, fin, prec, nr)  # the input as stored (FP16 rounding included)
    torch.cuda.synchronize()
    got, stored = got.cpu().numpy(), stored.cpu().numpy()
    rng = np.random.default_rng(7)
    shape = got.shape[2:6]  # t, z, y, xh
    err = scale = 0.0
    for _ in range(32):
        r = int(rng.integers(0, nr))
        t, z, y, xh = (int(rng.integers(0, L)) for L in shape)
        minv = np.linalg.inv(op.m5_matrix(act, masses[r], bool(dagger)))
        col = stored[r, :, t, z, y, xh].reshape(w["Ls"] * 4, 3)
        want = (minv @ col).reshape(w["Ls"], 4, 3)
        err = max(err, np.abs(got[r, :, t, z, y, xh] - want).max())
        scale = max(scale, np.abs(want).max())
    assert err <= tol * scale, err / scale
