"""dwf_mdagm_noalloc against dwf_mdagm (through the C ABI).

The no-allocation variant serves callers that cannot call cudaMalloc: programs
whose own pool allocator owns the device memory, and host loops that must not
take cudaMalloc's implicit device synchronisation. It keeps its temporaries in
the library's fixed device scratch array instead, so it must give the same
result as the allocating entry point, also on the second call in a row (the
array then holds the first call's temporaries), and must refuse lattices whose
temporaries do not fit. This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1811_08488_gb300 import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


def relerr(a, b):
    return (a - b).abs().max().item() / max(b.abs().max().item(), 1e-300)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_matches_allocating_entry_point(prec):
    from paper_1811_08488_gb300 import dwf
    dims, Ls, masses = (4, 4, 4, 8), 6, [0.03, 0.1]
    ctx = dwf.Context(dims, Ls, b=1.5, c=0.5, M5=1.8)
    ctx.gauge_load(syn.gauge_field(dims, 0.4, 7))
    for call in range(2):  # two calls in a row share the scratch array
        srcs = np.stack([syn.half_field(dims, Ls, 100 + 10 * call + r) for r in range(2)])
        canon = torch.from_numpy(srcs).cuda()
        fin = ctx.new_field(prec, 2)
        ctx.field_import(fin, prec, canon, 2)
        want_n, got_n = ctx.new_field(prec, 2), ctx.new_field(prec, 2)
        ctx.mdagm(want_n, fin, prec, masses)
        ctx.mdagm_noalloc(got_n, fin, prec, masses)
        want, got = torch.zeros_like(canon), torch.zeros_like(canon)
        ctx.field_export(want, want_n, prec, 2)
        ctx.field_export(got, got_n, prec, 2)
        torch.cuda.synchronize()
        assert relerr(got, want) <= TOL[prec], (prec, call)
    ctx.close()


def test_noalloc_refuses_fields_beyond_its_scratch():
    from paper_1811_08488_gb300 import dwf
    dims, Ls = (16, 16, 16, 16), 8  # 3 FP32 temporaries = 72 MiB > scratch
    ctx = dwf.Context(dims, Ls)
    assert 3 * ctx.field_bytes("fp32") > dwf.NOALLOC_SCRATCH_BYTES
    f, g = ctx.new_field("fp32"), ctx.new_field("fp32")
    with pytest.raises(dwf.DwfError) as e:
        ctx.mdagm_noalloc(g, f, "fp32", [0.1])
    assert e.value.code == 1 and "DWF_NOALLOC_SCRATCH_BYTES" in str(e.value)
    ctx.close()


def test_noalloc_rejects_a_nan_mass():
    """Like dwf_mdagm, the no-allocation variant refuses a NaN quark mass."""
    from paper_1811_08488_gb300 import dwf
    dims, Ls = (4, 4, 4, 4), 4
    ctx = dwf.Context(dims, Ls)
    ctx.gauge_load(syn.gauge_field(dims, 0.4, 8))
    f, g = ctx.new_field("fp32"), ctx.new_field("fp32")
    for fn in (ctx.mdagm, ctx.mdagm_noalloc):
        with pytest.raises(dwf.DwfError) as e:
            fn(g, f, "fp32", [float("nan")])
        assert e.value.code == 1 and "NaN" in str(e.value)
    ctx.close()
