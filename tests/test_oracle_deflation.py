"""Pins of oracle/deflation.py (low modes of A and deflated MSPCG) against
closed forms and dense brute force, independent of the oracle's own code:

* the Chebyshev filter against cos(d arccos x) / cosh(d arccosh x) on a
  diagonal operator (catches a wrong degree, a wrong interval map, a wrong
  recurrence sign);
* the Rayleigh-Ritz step and the subspace iteration against numpy's eigh of
  the dense A on a 2^4 x Ls=4 lattice (eigenvalues and the invariant
  subspace);
* the deflated start against the Galerkin condition V^dag (b - A x_0) = 0 and,
  with the full eigenbasis, against the dense solve x = A^-1 b;
* the coarse correction against A^-1 P_V r from a dense solve.
"""
import numpy as np
import pytest

from oracle import deflation as df
from oracle import dwf_operator as op
from oracle import solvers as sv
from paper_1811_08488_gb300 import synthetic as syn

MOB = dict(M5=1.8, b=1.5, c=0.5)


def cheb_closed(d, x):
    x = np.asarray(x, dtype=float)
    out = np.empty_like(x)
    inside = np.abs(x) <= 1
    out[inside] = np.cos(d * np.arccos(x[inside]))
    xo = x[~inside]
    out[~inside] = np.sign(xo) ** d * np.cosh(d * np.arccosh(np.abs(xo)))
    return out


@pytest.mark.parametrize("d", [1, 2, 7, 20])
def test_chebyshev_filter_closed_form(d):
    lam = np.array([0.001, 0.02, 0.3, 1.0, 2.5, 4.0, 6.0])
    a, b = 0.5, 6.0
    y = np.ones_like(lam) + 0.25j
    out = df.chebyshev_filter(lambda v: lam * v, [y], d, a, b)[0]
    want = cheb_closed(d, (2 * lam - (a + b)) / (b - a)) * y
    assert np.abs(out - want).max() <= 1e-12 * np.abs(want).max()
    # bounded by 1 on [a, b], growing below a
    inner = (lam >= a) & (lam <= b)
    assert np.all(np.abs(out[inner] / y[inner]) <= 1 + 1e-12)


def dense_even(act, fn):
    """Dense matrix of fn on the even half of the lattice (columns = unit vectors)."""
    par = op.parity_mask(act.shape4)
    mask = np.broadcast_to(par[None, :, :, :, :, None, None], act.shape5).reshape(-1) == 0
    idx = np.flatnonzero(mask)
    n = mask.size
    cols = []
    for j in idx:
        e = np.zeros(n, dtype=complex)
        e[j] = 1
        cols.append(fn(e.reshape(act.shape5)).reshape(-1)[idx])
    return np.array(cols).T, idx


@pytest.fixture(scope="module")
def brute():
    act = op.Action(dims=(2, 2, 2, 2), Ls=4, **MOB)
    U = op.gauge_to_mu_major(syn.gauge_field(act.dims, 0.5, 5))
    mf = 0.02
    A = lambda v: op.mdagm(act, U, v, mf)
    Ad, idx = dense_even(act, A)
    w, Q = np.linalg.eigh(0.5 * (Ad + Ad.conj().T))
    return act, U, mf, A, Ad, idx, w, Q


def to_field(act, idx, vec):
    f = np.zeros(int(np.prod(act.shape5)), dtype=complex)
    f[idx] = vec
    return f.reshape(act.shape5)


def from_field(idx, f):
    return f.reshape(-1)[idx]


def even_random(act, seed):
    return op.half_to_full(syn.half_field(act.dims, act.Ls, seed), 0)


def projector_distance(Va, Vb):
    """|P_a - P_b| (spectral norm) of the orthogonal projectors onto two
    subspaces of equal dimension."""
    Qa, _ = np.linalg.qr(Va)
    Qb, _ = np.linalg.qr(Vb)
    return np.linalg.norm(Qa @ Qa.conj().T - Qb @ Qb.conj().T, 2)


def test_rayleigh_ritz_exact_on_invariant_subspace(brute):
    act, U, mf, A, Ad, idx, w, Q = brute
    # a basis of span(eigenvectors 3, 10, 40) mixed by a random matrix
    rng = np.random.default_rng(1)
    sel = [3, 10, 40]
    mix = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
    W = [to_field(act, idx, Q[:, sel] @ mix[:, j]) for j in range(3)]
    theta, V = df.rayleigh_ritz(A, W)
    assert np.abs(theta - w[sel]).max() < 1e-12 * w.max()
    G = np.array([[op.vdot(a, b) for b in V] for a in V])
    assert np.abs(G - np.eye(3)).max() < 1e-12
    for t, v in zip(theta, V):
        assert np.sqrt(op.norm2(A(v) - t * v)) < 1e-10 * w.max()


def test_lambda_max_estimate_bounds_the_spectrum(brute):
    act, U, mf, A, Ad, idx, w, Q = brute
    est = df.lambda_max_estimate(A, even_random(act, 7))
    assert w.max() <= est <= 1.1 * w.max() * (1 + 1e-12)


def test_lowmodes_match_dense_eigh(brute):
    act, U, mf, A, Ad, idx, w, Q = brute
    # n_ev at a gap of the dense spectrum, so that the wanted subspace is unique
    gaps = np.diff(w[:16]) / w[:16][1:]
    n_ev = int(np.argmax(gaps[5:12])) + 6
    m = n_ev + 6
    V0 = [even_random(act, 100 + j) for j in range(m)]
    lam_max = df.lambda_max_estimate(A, V0[0])
    theta, V, res, passes = df.lowmodes(A, V0, n_ev, degree=16, passes=60, lam_max=lam_max,
                                        tol=1e-11)
    assert passes < 60
    assert np.abs(theta[:n_ev] - w[:n_ev]).max() < 1e-9 * w.max()
    assert res[:n_ev].max() <= 1e-11 * lam_max
    Vm = np.stack([from_field(idx, v) for v in V[:n_ev]], axis=1)
    assert projector_distance(Vm, Q[:, :n_ev]) < 1e-6


def test_deflated_start_galerkin_and_full_basis(brute):
    act, U, mf, A, Ad, idx, w, Q = brute
    b = even_random(act, 9)
    n_ev = 12
    V = [to_field(act, idx, Q[:, j]) for j in range(n_ev)]
    x0 = df.coarse_correction(V, w[:n_ev], b)
    r0 = b - A(x0)
    proj = np.array([op.vdot(v, r0) for v in V])
    assert np.abs(proj).max() < 1e-12 * np.sqrt(op.norm2(b))
    # the full eigenbasis gives the solution itself
    Vall = [to_field(act, idx, Q[:, j]) for j in range(len(w))]
    x = df.coarse_correction(Vall, w, b)
    want = np.linalg.solve(Ad, from_field(idx, b))
    assert np.abs(from_field(idx, x) - want).max() < 1e-9 * np.abs(want).max()


def test_coarse_correction_is_inverse_on_the_subspace(brute):
    act, U, mf, A, Ad, idx, w, Q = brute
    r = even_random(act, 10)
    n_ev = 9
    V = [to_field(act, idx, Q[:, j]) for j in range(n_ev)]
    z = df.coarse_correction(V, w[:n_ev], r)
    Qv = Q[:, :n_ev]
    Pr = Qv @ (Qv.conj().T @ from_field(idx, r))
    want = np.linalg.solve(Ad, Pr)
    assert np.abs(from_field(idx, z) - want).max() < 1e-10 * np.abs(want).max()


def test_deflated_mspcg_converges_in_fewer_iterations():
    """On a 4x2x2x4 x Ls=4 lattice with small m_f and the 8 lowest eigenpairs
    of the dense A: the deflated solve reaches the tolerance with a recomputed
    residual and needs fewer outer iterations than plain MSPCG; with k = 0 the
    same holds for CG."""
    act = op.Action(dims=(4, 2, 2, 4), Ls=4, **MOB)
    U = op.gauge_to_mu_major(syn.gauge_field(act.dims, 0.3, 21))
    mf = 0.01
    A = lambda v: op.mdagm(act, U, v, mf)
    Ad, idx = dense_even(act, A)
    w, Q = np.linalg.eigh(0.5 * (Ad + Ad.conj().T))
    b = even_random(act, 22)
    n_ev = 8
    V = [to_field(act, idx, Q[:, j]) for j in range(n_ev)]
    block = (2, 2, 2, 2)
    x, it_d, res_d = df.deflated_mspcg(act, U, b, mf, block, 3, 1e-10, V, w[:n_ev])
    _, it_ms, _ = sv.mspcg(act, U, b, mf, block, 3, 1e-10)
    assert res_d <= 1e-10
    assert np.sqrt(op.norm2(b - A(x)) / op.norm2(b)) <= 1e-10
    assert it_d < it_ms, (it_d, it_ms)
    _, it_cg_d, res_cg = df.deflated_mspcg(act, U, b, mf, block, 0, 1e-10, V, w[:n_ev])
    _, it_cg, _ = sv.cg(A, b, 1e-10)
    assert res_cg <= 1e-10 and it_cg_d < it_cg, (it_cg_d, it_cg)


def test_pcg_with_initial_guess_matches_zero_start_on_exact_guess(brute):
    """x0 = A^-1 b (dense) is returned at once; x0 = 0 reproduces the zero start."""
    act, U, mf, A, Ad, idx, w, Q = brute
    b = even_random(act, 12)
    xs = to_field(act, idx, np.linalg.solve(Ad, from_field(idx, b)))
    x, it, res = sv.pcg(A, lambda v: v, b, 1e-10, x0=xs)
    assert it == 0 and res <= 1e-10
    x1, it1, _ = sv.pcg(A, lambda v: v, b, 1e-10, x0=np.zeros_like(b))
    x2, it2, _ = sv.pcg(A, lambda v: v, b, 1e-10)
    assert it1 == it2 and np.abs(x1 - x2).max() == 0


def test_lowmodes_of_the_symmetric_form_match_dense_eigh(brute):
    """The same subspace iteration on A_sym = D_sym^dag D_sym (the symmetric
    Schur form's normal operator) against numpy's eigh of its dense matrix."""
    act, U, mf, _, _, idx, _, _ = brute
    A = lambda v: op.mdagm_sym(act, U, v, mf)
    Ad, _ = dense_even(act, A)
    w, Q = np.linalg.eigh(0.5 * (Ad + Ad.conj().T))
    gaps = np.diff(w[:16]) / w[:16][1:]
    n_ev = int(np.argmax(gaps[5:12])) + 6
    m = n_ev + 6
    V0 = [even_random(act, 300 + j) for j in range(m)]
    lam_max = df.lambda_max_estimate(A, V0[0])
    theta, V, res, passes = df.lowmodes(A, V0, n_ev, degree=16, passes=80, lam_max=lam_max,
                                        tol=1e-11)
    assert passes < 80
    assert np.abs(theta[:n_ev] - w[:n_ev]).max() < 1e-9 * w.max()
    Vm = np.stack([from_field(idx, v) for v in V[:n_ev]], axis=1)
    assert projector_distance(Vm, Q[:, :n_ev]) < 1e-6
