"""Low modes and deflation on the GPU against the FP64 oracle (oracle/deflation.py).

* dwf_deflate (z = V Lambda^-1 V^+ r, the kernels of the deflated start and
  of the coarse correction) element by element against the oracle's
  coarse_correction, for FP32 and FP64 fields, 1 to 4 right-hand sides (the
  tile shapes of the multi-dot kernel) and 1 to 33 vectors (ragged tiles),
  with V in FP32 and in FP16, and at the 16^3x32 x Ls=12 size;
* dwf_field_convert between FP32, FP64 and FP16;
* dwf_eig_lowmodes against numpy's eigh of the oracle's dense A on a
  4x2x2x4 x Ls=4 lattice: Ritz values, the invariant subspace and the
  orthonormality of the Ritz vectors;
* mspcg_solve_deflated: the true residual recomputed by the oracle, and fewer
  outer iterations than without deflation, for MSPCG and plain CG.

Tolerances: FP32 vectors V carry 2^-24 relative rounding, the multi-dot sums
are FP64 over compensated FP32 partials, the combination accumulates in FP32
(FP64 for FP64 fields): 1e-5 relative (max-norm) for FP32 results, 1e-6 for
FP64 results whose inputs V are FP32. Eigen-pairs: the Rayleigh-Ritz step
works on FP32 A applications (relative error about 1e-6 of lambda_max), so
Ritz values are compared to 2e-5 lambda_max and subspaces (n_ev at a spectral
gap of relative width g) to 1e-3 / g.
"""
import numpy as np
import pytest

from oracle import deflation as df
from oracle import dwf_operator as op
from oracle import solvers as sv
from paper_1811_08488_gb300 import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MOB = dict(b=1.5, c=0.5, M5=1.8)


def dwf():
    from paper_1811_08488_gb300 import dwf as d
    return d


def setup(dims, Ls, seed, eps=0.4, **kw):
    a = dict(MOB)
    a.update(kw)
    act = op.Action(dims=tuple(dims), Ls=Ls, **a)
    Uc = syn.gauge_field(dims, eps, seed)
    ctx = dwf().Context(dims, Ls, **a)
    ctx.gauge_load(Uc)
    return act, op.gauge_to_mu_major(Uc), ctx


def to_native(ctx, halves, prec):
    canon = torch.from_numpy(np.ascontiguousarray(np.stack(halves))).cuda()
    nat = ctx.new_field(prec, len(halves))
    ctx.field_import(nat, prec, canon, len(halves))
    return nat


def to_native_many(ctx, halves, prec):
    """More than 16 fields: imported 16 at a time into one buffer."""
    nat = ctx.new_field(prec, len(halves))
    rs = ctx.field_bytes(prec, 1)
    for b0 in range(0, len(halves), 16):
        part = halves[b0:b0 + 16]
        canon = torch.from_numpy(np.ascontiguousarray(np.stack(part))).cuda()
        ctx.field_import(nat[b0 * rs:(b0 + len(part)) * rs], prec, canon, len(part))
    return nat


def from_native_many(ctx, nat, prec, n):
    rs = ctx.field_bytes(prec, 1)
    out = []
    for b0 in range(0, n, 16):
        k = min(16, n - b0)
        canon = torch.zeros(ctx.canon_shape(k), dtype=torch.complex128, device="cuda")
        ctx.field_export(canon, nat[b0 * rs:(b0 + k) * rs], prec, k)
        torch.cuda.synchronize()
        out.extend(c for c in canon.cpu().numpy())
    return out


def relerr(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("fp64", 1e-6)])
@pytest.mark.parametrize("n_ev,nrhs", [(1, 1), (5, 2), (12, 3), (33, 1), (9, 4)])
@pytest.mark.parametrize("accumulate", [0, 1])
def test_deflate_matches_oracle(prec, tol, n_ev, nrhs, accumulate):
    dims, Ls = (4, 4, 2, 6), 4
    act, U, ctx = setup(dims, Ls, 301)
    V = [syn.half_field(dims, Ls, 400 + j) for j in range(n_ev)]
    lam = np.linspace(0.05, 2.0, n_ev)
    r = [syn.half_field(dims, Ls, 500 + k) for k in range(nrhs)]
    z0 = [syn.half_field(dims, Ls, 600 + k) for k in range(nrhs)]
    Vn = to_native_many(ctx, V, "fp32")
    rn = to_native(ctx, r, prec)
    zn = to_native(ctx, z0, prec)
    ctx.deflate(zn, rn, Vn, lam, prec, nrhs, accumulate=accumulate)
    got = from_native_many(ctx, zn, prec, nrhs)
    for k in range(nrhs):
        want = df.coarse_correction(V, lam, r[k]) + (z0[k] if accumulate else 0)
        assert relerr(got[k], want) < tol, (k, relerr(got[k], want))


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("n_ev,nrhs", [(1, 1), (17, 2), (24, 4)])
def test_deflate_fp16_vectors_match_oracle(prec, n_ev, nrhs):
    """V stored in FP16 with per-(site, s) scales (dwf_field_convert from FP32):
    every element of V carries a relative rounding of at most 2^-11 of its
    (site, s) maximum, so the projection and the combination are within about
    3 * 2^-11 of the FP64 result (tolerance 2e-3)."""
    dims, Ls = (4, 4, 2, 6), 4
    act, U, ctx = setup(dims, Ls, 302)
    V = [syn.half_field(dims, Ls, 410 + j) for j in range(n_ev)]
    lam = np.linspace(0.05, 2.0, n_ev)
    r = [syn.half_field(dims, Ls, 510 + k) for k in range(nrhs)]
    V32 = to_native_many(ctx, V, "fp32")
    V16 = ctx.new_field("fp16", n_ev)
    ctx.field_convert(V16, "fp16", V32, "fp32", n_ev)
    rn = to_native(ctx, r, prec)
    zn = ctx.new_field(prec, nrhs)
    ctx.deflate(zn, rn, V16, lam, prec, nrhs, vprec="fp16")
    got = from_native_many(ctx, zn, prec, nrhs)
    for k in range(nrhs):
        want = df.coarse_correction(V, lam, r[k])
        assert relerr(got[k], want) < 2e-3, (k, relerr(got[k], want))


def test_field_convert_round_trips():
    """FP32 -> FP64 -> FP32 is exact; FP32 -> FP16 keeps every element within
    2^-11 of its (site, s) maximum; FP16 -> FP32 -> FP16 is exact."""
    dims, Ls = (4, 4, 2, 6), 6
    ctx = dwf().Context(dims, Ls, **MOB)
    halves = [syn.half_field(dims, Ls, 520 + k) for k in range(3)]
    f32 = to_native(ctx, halves, "fp32")
    f64, back = ctx.new_field("fp64", 3), ctx.new_field("fp32", 3)
    ctx.field_convert(f64, "fp64", f32, "fp32", 3)
    ctx.field_convert(back, "fp32", f64, "fp64", 3)
    torch.cuda.synchronize()
    assert torch.equal(back, f32)
    f16, b32, b16 = ctx.new_field("fp16", 3), ctx.new_field("fp32", 3), ctx.new_field("fp16", 3)
    ctx.field_convert(f16, "fp16", f32, "fp32", 3)
    ctx.field_convert(b32, "fp32", f16, "fp16", 3)
    ctx.field_convert(b16, "fp16", b32, "fp32", 3)
    torch.cuda.synchronize()
    assert torch.equal(b16, f16)
    got = from_native_many(ctx, f16, "fp16", 3)
    for k in range(3):
        g = np.stack([got[k].real, got[k].imag], -1)
        w = np.stack([halves[k].real, halves[k].imag], -1)
        elem_max = np.abs(w).max(axis=(-3, -2, -1), keepdims=True)
        assert (np.abs(g - w) / elem_max).max() <= 2.0 ** -11 * 1.01


def test_deflate_full_size_16x16x16x32():
    """dwf_deflate on the 16^3x32 x Ls=12 lattice (8 vectors, 2 right-hand
    sides), every element against the oracle."""
    dims, Ls = (16, 16, 16, 32), 12
    ctx = dwf().Context(dims, Ls, **MOB)
    n_ev, nrhs = 8, 2
    V = [syn.half_field(dims, Ls, 700 + j) for j in range(n_ev)]
    lam = np.geomspace(0.01, 1.0, n_ev)
    r = [syn.half_field(dims, Ls, 800 + k) for k in range(nrhs)]
    Vn = to_native_many(ctx, V, "fp32")
    rn = to_native(ctx, r, "fp32")
    zn = ctx.new_field("fp32", nrhs)
    ctx.deflate(zn, rn, Vn, lam, "fp32", nrhs)
    got = from_native_many(ctx, zn, "fp32", nrhs)
    for k in range(nrhs):
        want = np.zeros_like(r[k])
        for v, l in zip(V, lam):
            want += v * (np.vdot(v.reshape(-1), r[k].reshape(-1)) / l)
        assert relerr(got[k], want) < 1e-5


def dense_even(act, fn):
    par = op.parity_mask(act.shape4)
    mask = np.broadcast_to(par[None, :, :, :, :, None, None], act.shape5).reshape(-1) == 0
    idx = np.flatnonzero(mask)
    cols = []
    for j in idx:
        e = np.zeros(mask.size, dtype=complex)
        e[j] = 1
        cols.append(fn(e.reshape(act.shape5)).reshape(-1)[idx])
    return np.array(cols).T, idx


def half_to_vec(act, idx, half):
    return op.half_to_full(half, 0).reshape(-1)[idx]


@pytest.mark.parametrize("schur", [0, 1])
def test_eig_lowmodes_match_dense_eigh(schur):
    dims, Ls = (4, 2, 2, 4), 4
    act, U, ctx = setup(dims, Ls, 311, eps=0.5)
    mf = 0.02
    form = "sym" if schur else "asym"
    Ad, idx = dense_even(act, lambda v: op.normal_op(form)(act, U, v, mf))
    w, Q = np.linalg.eigh(0.5 * (Ad + Ad.conj().T))
    gaps = np.diff(w[:24]) / w.max()
    n_ev = int(np.argmax(gaps[4:16])) + 5
    g = gaps[n_ev - 1]
    m = n_ev + 8
    start = [syn.half_field(dims, Ls, 900 + j) for j in range(m)]
    Vn = to_native_many(ctx, start, "fp32")
    prm = dwf().default_eig_params(n_ev=n_ev, degree=16, max_passes=80, tol=2e-6,
                                   schur=schur)
    theta, resid, info = ctx.eig_lowmodes(Vn, m, mf, prm)
    assert info["converged"] == 1 and info["passes"] < 80, info
    assert w.max() <= info["lambda_max"] <= 1.1 * w.max() * 1.001
    assert np.all(np.diff(theta) >= 0)
    assert np.abs(theta[:n_ev] - w[:n_ev]).max() < 2e-5 * w.max()
    assert resid[:n_ev].max() <= 2e-6 * info["lambda_max"]
    vecs = from_native_many(ctx, Vn, "fp32", m)
    Vm = np.stack([half_to_vec(act, idx, v) for v in vecs[:n_ev]], axis=1)
    assert np.abs(Vm.conj().T @ Vm - np.eye(n_ev)).max() < 1e-5
    Qv, _ = np.linalg.qr(Vm)
    dist = np.linalg.norm(Qv @ Qv.conj().T - Q[:, :n_ev] @ Q[:, :n_ev].conj().T, 2)
    assert dist < 1e-3 / g, (dist, g)


def test_eig_lowmodes_rejects_bad_arguments():
    dims, Ls = (4, 2, 2, 4), 4
    act, U, ctx = setup(dims, Ls, 311)
    Vn = ctx.new_field("fp32", 4)
    d = dwf()
    with pytest.raises(d.DwfError):
        ctx.eig_lowmodes(Vn, 4, 0.02, d.default_eig_params(n_ev=5))   # n_ev > m
    with pytest.raises(d.DwfError):
        ctx.eig_lowmodes(Vn, 65, 0.02, d.default_eig_params(n_ev=4))  # m > 64
    with pytest.raises(d.DwfError):
        ctx.deflate(ctx.new_field("fp32", 1), ctx.new_field("fp32", 1), Vn, [1.0, -1.0], "fp32")
    with pytest.raises(d.DwfError) as e:  # FP16 V with more than 4 right-hand sides
        ctx.deflate(ctx.new_field("fp32", 5), ctx.new_field("fp32", 5), Vn, [1.0], "fp32", 5,
                    vprec="fp16")
    assert e.value.code == 2


@pytest.mark.parametrize("k,vprec", [(0, "fp32"), (3, "fp32"), (3, "fp16")])
def test_deflated_solve_fewer_iterations(k, vprec):
    """Low modes from dwf_eig_lowmodes; the deflated solve (start and coarse
    correction) converges with the oracle's recomputed residual <= 1e-10 and
    needs fewer outer iterations than the same solve without deflation."""
    dims, Ls = (8, 8, 4, 8), 4
    act, U, ctx = setup(dims, Ls, 321, eps=0.3)
    mf = 0.005
    n_ev, m = 12, 20
    Vn = to_native_many(ctx, [syn.half_field(dims, Ls, 1000 + j) for j in range(m)], "fp32")
    theta, resid, info = ctx.eig_lowmodes(
        Vn, m, mf, dwf().default_eig_params(n_ev=n_ev, degree=24, max_passes=60, tol=1e-5))
    assert info["converged"] == 1, info
    b = syn.half_field(dims, Ls, 1100)
    bt = torch.from_numpy(b[None].copy()).cuda()
    prm = dwf().default_params(block=(4, 4, 4, 4), inner_iters=k, inner="fp16", tol=1e-10)
    x0 = torch.zeros_like(bt)
    st, info0 = ctx.solve(x0, bt, [mf], prm)
    rs = ctx.field_bytes(vprec, 1)
    if vprec == "fp16":
        V16 = ctx.new_field("fp16", n_ev)
        ctx.field_convert(V16, "fp16", Vn, "fp32", n_ev)
        Vn = V16
    for coarse in (0, 1):
        x = torch.zeros_like(bt)
        st, info1 = ctx.solve_deflated(x, bt, [mf], prm, Vn[:n_ev * rs], theta[:n_ev],
                                       coarse=coarse, vprec=vprec)
        assert st == 0 and info1[0]["converged"] == 1
        xf = op.half_to_full(x.cpu().numpy()[0], 0)
        bf = op.half_to_full(b, 0)
        res = np.sqrt(op.norm2(bf - op.mdagm(act, U, xf, mf)) / op.norm2(bf))
        assert res <= 1e-10
        assert info1[0]["outer_iters"] < info0[0]["outer_iters"], (coarse, info0, info1)


def test_deflated_solve_matches_oracle_iteration_count():
    """Exact low modes (the oracle's dense eigh, imported as FP32): the GPU's
    deflated MSPCG takes the oracle's outer iteration count to within 2 (FP32
    outer iterations against FP64)."""
    dims, Ls = (4, 2, 2, 4), 4
    act, U, ctx = setup(dims, Ls, 331, eps=0.3)
    mf = 0.01
    Ad, idx = dense_even(act, lambda v: op.mdagm(act, U, v, mf))
    w, Q = np.linalg.eigh(0.5 * (Ad + Ad.conj().T))
    n_ev = 8
    full = np.zeros(int(np.prod(act.shape5)), dtype=complex)
    V = []
    for j in range(n_ev):
        f = full.copy()
        f[idx] = Q[:, j]
        V.append(op.full_to_half(f.reshape(act.shape5), 0))
    b = syn.half_field(dims, Ls, 1200)
    block = (2, 2, 2, 2)
    _, it_o, _ = df.deflated_mspcg(act, U, op.half_to_full(b, 0), mf, block, 3, 1e-10,
                                   [op.half_to_full(v, 0) for v in V], w[:n_ev])
    Vn = to_native_many(ctx, V, "fp32")
    bt = torch.from_numpy(b[None].copy()).cuda()
    x = torch.zeros_like(bt)
    prm = dwf().default_params(block=block, inner_iters=3, inner="fp32", tol=1e-10)
    st, info = ctx.solve_deflated(x, bt, [mf], prm, Vn, w[:n_ev], coarse=1)
    assert st == 0 and info[0]["converged"] == 1
    assert abs(info[0]["outer_iters"] - it_o) <= 2, (info[0]["outer_iters"], it_o)


def test_deflated_solve_flexible_coarse_unsupported():
    dims, Ls = (4, 2, 2, 4), 4
    act, U, ctx = setup(dims, Ls, 311)
    Vn = ctx.new_field("fp32", 2)
    bt = torch.from_numpy(syn.half_field(dims, Ls, 5)[None].copy()).cuda()
    prm = dwf().default_params(block=(2, 2, 2, 2), inner_iters=2, flexible=1)
    with pytest.raises(dwf().DwfError) as e:
        ctx.solve_deflated(torch.zeros_like(bt), bt, [0.1], prm, Vn, [1.0, 2.0], coarse=1)
    assert e.value.code == 2
