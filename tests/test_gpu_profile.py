"""Hop-kernel timer (dwf_profile_enable / dwf_profile_read).

The timer must not change any result, must count every hop launch into the
slot of its kernel, and must report the compulsory bytes of each launch."""
import numpy as np
import pytest

from paper_1811_08488_gb300 import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DIMS, LS, MF = (8, 8, 8, 16), 8, 0.05


def setup():
    from paper_1811_08488_gb300 import dwf
    ctx = dwf.Context(DIMS, LS, b=1.5, c=0.5, M5=1.8)
    ctx.gauge_load(syn.gauge_field(DIMS, 0.4, 17))
    canon = torch.from_numpy(syn.half_field(DIMS, LS, 18)[None].copy()).cuda()
    return dwf, ctx, canon


def by_name(stats):
    return {s["name"]: s for s in stats}


def test_nothing_recorded_until_enabled():
    dwf, ctx, canon = setup()
    fin, fout = ctx.new_field("fp32"), ctx.new_field("fp32")
    ctx.field_import(fin, "fp32", canon)
    ctx.dslash_eo(fout, fin, 0, 0, "fp32", [MF])
    assert ctx.profile_read() == []


def test_dslash_launches_bytes_and_identical_results():
    dwf, ctx, canon = setup()
    fin, fa, fb = ctx.new_field("fp32"), ctx.new_field("fp32"), ctx.new_field("fp32")
    ctx.field_import(fin, "fp32", canon)
    ctx.dslash_eo(fa, fin, 0, 0, "fp32", [MF])
    ctx.profile(True)
    for _ in range(3):
        ctx.dslash_eo(fb, fin, 0, 0, "fp32", [MF])
    ctx.dslash_eo(fb, fin, 1, 1, "fp32", [MF])
    st = by_name(ctx.profile_read())
    pre = st["hop2_kernel<F32,0,1,0,0>"]
    dag = st["hop2_kernel<F32,1,0,0,1>"]
    assert pre["launches"] == 3 and dag["launches"] == 1
    V4 = int(np.prod(DIMS))
    per = 2 * (V4 // 2) * LS * 96 + V4 * 4 * 72  # spinor in + out, links once
    assert pre["alg_bytes"] == 3 * per and dag["alg_bytes"] == per
    assert 0 < pre["seconds"] < 1 and 0 < dag["seconds"] < 1
    # same output with the timer on as off
    ctx.dslash_eo(fb, fin, 0, 0, "fp32", [MF])
    torch.cuda.synchronize()
    assert torch.equal(fa, fb)
    # off: counters kept, nothing added
    ctx.profile(False)
    ctx.dslash_eo(fb, fin, 0, 0, "fp32", [MF])
    assert by_name(ctx.profile_read())["hop2_kernel<F32,0,1,0,0>"]["launches"] == 4
    # on again: reset
    ctx.profile(True)
    assert ctx.profile_read() == []


def test_solve_counts_block_operator_hops_and_keeps_the_solution():
    dwf, ctx, canon = setup()
    prm = dwf.default_params(block=(4, 4, 4, 8), inner="fp16", inner_iters=4, tol=1e-10)
    x0 = torch.zeros_like(canon)
    st0, info0 = ctx.solve(x0, canon, [MF], prm)
    ctx.profile(True)
    x1 = torch.zeros_like(canon)
    st1, info1 = ctx.solve(x1, canon, [MF], prm)
    stats = by_name(ctx.profile_read())
    ctx.profile(False)
    assert st0 == 0 and st1 == 0
    assert info0[0]["outer_iters"] == info1[0]["outer_iters"]
    assert torch.equal(x0, x1)
    # block operator: hops 3 and 4 are the FP16 adjoint with its epilogue, two
    # per inner iteration; each preconditioner application runs k of them
    k = 4
    blk_dag = stats["hop2_kernel<F16,1,0,0,1> [block]"]["launches"]
    blk_pre = stats["hop2_kernel<F16,0,1,0,1> [block]"]["launches"]
    blk_mid = stats["hop2_kernel<F16,0,0,0,1> [block]"]["launches"]
    assert blk_dag == 2 * blk_pre == 2 * blk_mid
    assert blk_pre % k == 0 and blk_pre // k >= info1[0]["outer_iters"]
    # outer operator in FP32, reliable updates in FP64
    assert stats["hop2_kernel<F32,1,0,0,1>"]["launches"] >= 2 * info1[0]["outer_iters"]
    assert any(n.startswith("hop_kernel<F64") for n in stats)
    total = sum(s["seconds"] for s in stats.values())
    assert 0 < total < info1[0]["seconds"]
    # dslash_gbs: the outer operator's FP32 hops of this solve (timer on)
    outer = [s for n, s in stats.items() if n.startswith("hop2_kernel<F32") and "[block]" not in n]
    gbs = sum(s["alg_bytes"] for s in outer) / sum(s["seconds"] for s in outer) / 1e9
    assert info1[0]["dslash_gbs"] > 0
    assert abs(info1[0]["dslash_gbs"] - gbs) < 1e-6 * gbs
    assert info0[0]["dslash_gbs"] == -1.0  # timer off


def test_block_operator_with_fp32_storage_has_its_own_slots():
    """With FP32 inner storage the block operator runs the same kernel
    instantiations as the outer FP32 operator; its launches are counted apart
    (" [block]"), so dslash_gbs covers the outer operator only."""
    dwf, ctx, canon = setup()
    prm = dwf.default_params(block=(4, 4, 4, 8), inner="fp32", inner_iters=2, tol=1e-10)
    ctx.profile(True)
    st, info = ctx.solve(torch.zeros_like(canon), canon, [MF], prm)
    stats = by_name(ctx.profile_read())
    ctx.profile(False)
    assert st == 0
    assert stats["hop2_kernel<F32,1,0,0,1> [block]"]["launches"] % 2 == 0
    assert stats["hop2_kernel<F32,1,0,0,1>"]["launches"] >= 2 * info[0]["outer_iters"]
    assert info[0]["dslash_gbs"] > 0


def test_profile_read_argument_errors():
    dwf, ctx, canon = setup()
    import ctypes as C
    n = C.c_int(0)
    assert dwf.lib().dwf_profile_read(ctx._h, None, 1, C.byref(n)) == 1  # INVALID_ARG
    assert dwf.lib().dwf_profile_read(ctx._h, None, 0, None) == 1
    assert dwf.lib().dwf_profile_enable(ctx._h, 2) == 1
