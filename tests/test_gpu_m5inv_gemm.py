"""Tensor-core M_5^-1 (dwf_m5inv_gemm) against the FP64 oracle's dense inverse.

Tolerances (relative, max-norm over the field):
* FP32 fields: both GEMM operands are split into two FP16 parts scaled per
  (site, chirality) slab; the dropped lo*lo product and the FP32 tensor-memory
  accumulation leave about 2^-21 of the slab maximum per term, times at most
  Ls terms: 1e-5 (the bound of the FP32 operators).
* FP16 / BF16 fields: input and output rounded to 11 / 8 bits of their
  (site, s) maximum, the A operand to 11 bits: 3e-3 / 2.5e-2 as for dslash.
Sizes: 48 even sites (one full CTA of 32 sites and a ragged one of 16) and
512 sites (16 CTAs); Ls = 4, 7, 12 (one K step), 16 (the largest single
step), 20 and 32 (the largest Ls a context takes; two K steps, N = 32).
"""
import numpy as np
import pytest

from oracle import dwf_operator as op
from paper_1811_08488_gb300 import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp16": 3e-3, "bf16": 2.5e-2}


def dwf():
    from paper_1811_08488_gb300 import dwf as d
    return d


def relerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


class Setup:
    def __init__(self, dims, Ls, b=1.5, c=0.5, M5=1.8):
        self.act = op.Action(dims=tuple(dims), Ls=Ls, M5=M5, b=b, c=c)
        self.ctx = dwf().Context(dims, Ls, b=b, c=c, M5=M5)

    def to_native(self, halves, prec):
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

    def want(self, half, mf, dagger):
        return op.full_to_half(op.m5inv(self.act, op.half_to_full(half, 0), mf, bool(dagger)), 0)


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("dagger", [0, 1])
@pytest.mark.parametrize("dims,Ls,kw", [((4, 2, 2, 6), 12, dict()), ((4, 2, 2, 6), 4, dict()),
                                        ((4, 2, 2, 6), 7, dict(b=1.0, c=0.0)),
                                        ((8, 4, 4, 8), 16, dict()), ((4, 2, 2, 6), 20, dict()),
                                        ((4, 2, 2, 6), 32, dict())])
def test_m5inv_gemm_matches_oracle(prec, dagger, dims, Ls, kw):
    S = Setup(dims, Ls, **kw)
    masses = [0.01, 0.3, 0.9]
    ins = [S.source(71 + r) for r in range(3)]
    nat_in = S.to_native(ins, prec)
    out = S.ctx.new_field(prec, 3)
    S.ctx.m5inv_gemm(out, nat_in, dagger, prec, masses)
    got = S.from_native(out, prec, 3)
    for r in range(3):
        assert relerr(got[r], S.want(ins[r], masses[r], dagger)) < TOL[prec], r


def test_m5inv_gemm_agrees_with_closed_form_kernel_fp32():
    """The GEMM form and the closed-form recursion (dwf_m5inv) on the same FP32 field."""
    S = Setup((8, 4, 4, 8), 12)
    masses = [0.02, 0.2]
    nat_in = S.to_native([S.source(81), S.source(82)], "fp32")
    a, b = S.ctx.new_field("fp32", 2), S.ctx.new_field("fp32", 2)
    for dagger in (0, 1):
        S.ctx.m5inv_gemm(a, nat_in, dagger, "fp32", masses)
        S.ctx.m5inv(b, nat_in, dagger, "fp32", masses)
        ga, gb = S.from_native(a, "fp32", 2), S.from_native(b, "fp32", 2)
        for r in range(2):
            assert relerr(ga[r], gb[r]) < 2e-6


def test_m5inv_gemm_sixteen_rhs_and_site_scales():
    """All 16 right-hand sides in one launch, with per-site magnitudes spread
    over 12 decades: the per-(site, chirality) scaling keeps every site's
    relative error small, not just the largest ones."""
    S = Setup((4, 2, 2, 6), 12)
    masses = list(syn.log_spaced_masses(0.001, 0.05, 16))
    ins = [S.source(90 + r) for r in range(16)]
    # magnitudes per (t, z, y, xh) site
    rng = np.random.default_rng(5)
    mags = 10.0 ** rng.integers(-6, 7, size=ins[0].shape[1:5])
    ins = [h * mags[None, :, :, :, :, None, None] for h in ins]
    nat_in = S.to_native(ins, "fp32")
    out = S.ctx.new_field("fp32", 16)
    S.ctx.m5inv_gemm(out, nat_in, 0, "fp32", masses)
    got = S.from_native(out, "fp32", 16)
    for r in range(16):
        want = S.want(ins[r], masses[r], 0)
        err = np.abs(got[r] - want).max(axis=(0, 5, 6)) / np.abs(want).max(axis=(0, 5, 6))
        assert err.max() < 1e-5, (r, err.max())


def test_m5inv_gemm_zero_field_and_errors():
    S = Setup((4, 2, 2, 6), 12)
    z = S.to_native([np.zeros_like(S.source(1))], "fp32")
    out = S.ctx.new_field("fp32", 1)
    S.ctx.m5inv_gemm(out, z, 0, "fp32", [0.1])
    assert np.abs(S.from_native(out, "fp32", 1)[0]).max() == 0.0
    d = dwf()
    f64 = S.ctx.new_field("fp64", 1)
    o64 = S.ctx.new_field("fp64", 1)
    with pytest.raises(d.DwfError) as e:
        S.ctx.m5inv_gemm(o64, f64, 0, "fp64", [0.1])
    assert e.value.code == 2  # UNSUPPORTED


def test_m5inv_gemm_bounded_wait_expires_and_context_survives(monkeypatch):
    """Failure detection without a fault: DWF_TEST_STARVE_WAIT=1 makes every
    CTA wait, after its MMAs, on a barrier phase nothing completes. The wait
    gives up after 1 ms, the CTA frees its tensor memory and the call returns
    DWF_ERR_TIMEOUT; the next call on the same context is exact again."""
    S = Setup((4, 2, 2, 6), 12)
    d = dwf()
    src = S.source(5)
    nat_in = S.to_native([src], "fp32")
    out = S.ctx.new_field("fp32", 1)
    monkeypatch.setenv("DWF_TEST_STARVE_WAIT", "1")
    with pytest.raises(d.DwfError) as e:
        S.ctx.m5inv_gemm(out, nat_in, 0, "fp32", [0.1])
    assert e.value.code == 5  # TIMEOUT
    monkeypatch.delenv("DWF_TEST_STARVE_WAIT")
    S.ctx.m5inv_gemm(out, nat_in, 0, "fp32", [0.1])
    assert relerr(S.from_native(out, "fp32", 1)[0], S.want(src, 0.1, 0)) < TOL["fp32"]
