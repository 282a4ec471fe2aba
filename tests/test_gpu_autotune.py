"""Block-shape autotuner (dwf_autotune_block) and mspcg_solve with block = 0."""
import numpy as np
import pytest

from oracle import dwf_operator as op
from paper_1811_08488_gb300 import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DIMS, LS, MF = (8, 8, 8, 16), 8, 0.05
# b^3 x bt, b in {4, 6, 8, ...}, b/2 <= bt <= 2b, dividing 8^3 x 16, >= 2 blocks
CANDIDATES = {(4, 4, 4, 4), (4, 4, 4, 8), (8, 8, 8, 4), (8, 8, 8, 8)}


def setup():
    from paper_1811_08488_gb300 import dwf
    act = op.Action(dims=DIMS, Ls=LS, M5=1.8, b=1.5, c=0.5)
    Uc = syn.gauge_field(DIMS, 0.4, 7)
    ctx = dwf.Context(DIMS, LS, b=1.5, c=0.5, M5=1.8)
    ctx.gauge_load(Uc)
    b = torch.from_numpy(syn.half_field(DIMS, LS, 8)[None].copy()).cuda()
    return dwf, act, Uc, ctx, b


def test_autotune_picks_a_candidate_and_solve_uses_it():
    dwf, act, Uc, ctx, b = setup()
    prm = dwf.default_params(block=(0, 0, 0, 0), inner="fp16", inner_iters=4, tol=1e-10)
    blk, pred = ctx.autotune_block(b, [MF], prm, trial=6)
    assert tuple(blk) in CANDIDATES
    assert np.isfinite(pred) and pred > 0
    # block = 0 reuses the tuned shape: the same iterations as naming it
    x0 = torch.zeros_like(b)
    st, info0 = ctx.solve(x0, b, [MF], prm)
    x1 = torch.zeros_like(b)
    st1, info1 = ctx.solve(x1, b, [MF], dwf.default_params(block=blk, inner="fp16",
                                                             inner_iters=4, tol=1e-10))
    assert st == 0 and st1 == 0
    assert info0[0]["outer_iters"] == info1[0]["outer_iters"]
    assert torch.equal(x0, x1)
    # and the solution is the oracle's to the tolerance
    U = op.gauge_to_mu_major(Uc)
    xf = op.half_to_full(x0[0].cpu().numpy(), 0)
    bf = op.half_to_full(b[0].cpu().numpy(), 0)
    r = bf - op.mdagm(act, U, xf, MF)
    assert np.sqrt(op.norm2(r) / op.norm2(bf)) <= 1e-10


def test_solve_with_block_zero_tunes_on_first_call():
    dwf, act, Uc, ctx, b = setup()
    prm = dwf.default_params(block=(0, 0, 0, 0), inner="fp16", inner_iters=3, tol=1e-9)
    x = torch.zeros_like(b)
    st, info = ctx.solve(x, b, [MF], prm)
    assert st == 0 and info[0]["converged"] and info[0]["true_resid"] <= 1e-9


def test_autotune_rejects_plain_cg():
    dwf, act, Uc, ctx, b = setup()
    prm = dwf.default_params(inner_iters=0)
    with pytest.raises(dwf.DwfError) as e:
        ctx.autotune_block(b, [MF], prm, trial=4)
    assert e.value.code == 1  # INVALID_ARG


def test_autotune_without_candidates_is_unsupported():
    """2^3 x 4 has no block of extent >= 4 in every direction: no candidate."""
    from paper_1811_08488_gb300 import dwf
    ctx = dwf.Context((2, 2, 2, 4), 4, b=1.5, c=0.5, M5=1.8)
    ctx.gauge_load(syn.gauge_field((2, 2, 2, 4), 0.4, 3))
    b = torch.from_numpy(syn.half_field((2, 2, 2, 4), 4, 4)[None].copy()).cuda()
    prm = dwf.default_params(block=(0, 0, 0, 0), inner_iters=3)
    with pytest.raises(dwf.DwfError) as e:
        ctx.autotune_block(b, [MF], prm, trial=4)
    assert e.value.code == 2  # UNSUPPORTED
    with pytest.raises(dwf.DwfError) as e:
        ctx.solve(torch.zeros_like(b), b, [MF], prm)
    assert e.value.code == 2


def test_autotune_with_host_buffers():
    """io_on_host: the tuner's trial solves read b from host memory too."""
    dwf, act, Uc, ctx, b = setup()
    bh = b.cpu().numpy().copy()
    prm = dwf.default_params(block=(0, 0, 0, 0), inner="fp16", inner_iters=4, tol=1e-10,
                             io_on_host=1)
    blk, pred = ctx.autotune_block(bh, [MF], prm, trial=4)
    assert tuple(blk) in CANDIDATES and pred > 0
    xh = np.zeros_like(bh)
    st, info = ctx.solve(xh, bh, [MF], prm)
    assert st == 0 and info[0]["converged"]
