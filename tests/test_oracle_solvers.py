"""Pins of the oracle's solvers and of the Dirichlet block operator A_s."""
import numpy as np
import pytest

from oracle import dwf_operator as op
from oracle import solvers as sv
from paper_1811_08488_gb300 import synthetic as syn

RNG = np.random.default_rng(3)
MOB = dict(M5=1.8, b=1.5, c=0.5)


def rand_even(act):
    psi = RNG.normal(size=act.shape5) + 1j * RNG.normal(size=act.shape5)
    return op.restrict_parity(psi, 0)


def gauge(act, eps=0.4, seed=12):
    return op.gauge_to_mu_major(syn.gauge_field(act.dims, eps, seed))


def dense_on(fn, act, mask4):
    """Dense matrix of fn on the even sites of mask4 (all s, spin, colour)."""
    even = (op.parity_mask(act.shape4) == 0) & mask4
    m5 = np.broadcast_to(even[None, :, :, :, :, None, None], act.shape5).reshape(-1)
    idx = np.flatnonzero(m5)
    n = m5.size
    cols = []
    for j in idx:
        e = np.zeros(n, dtype=complex)
        e[j] = 1
        cols.append(fn(e.reshape(act.shape5)).reshape(-1)[idx])
    return np.array(cols).T, idx


# ----------------------------------------------------------------------------
# CG against dense LU
# ----------------------------------------------------------------------------
def test_cg_matches_dense_solve():
    act = op.Action(dims=(2, 2, 2, 2), Ls=4, **MOB)
    U = gauge(act, eps=0.5)
    mf = 0.1
    A, idx = dense_on(lambda v: op.mdagm(act, U, v, mf), act, np.ones(act.shape4, bool))
    b = rand_even(act)
    x, it, res = sv.cg(lambda v: op.mdagm(act, U, v, mf), b, 1e-13)
    assert res <= 1e-13
    xd = np.linalg.solve(A, b.reshape(-1)[idx])
    assert np.abs(x.reshape(-1)[idx] - xd).max() < 1e-10 * np.abs(xd).max()


# ----------------------------------------------------------------------------
# A_s: definition, box form, Hermiticity, snake terms
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("dims,block", [
    ((8, 4, 6, 4), (2, 2, 2, 4)),   # x: box 6 < L; y: L = b + 2; z: L = b + 4; t: one block
    ((4, 8, 4, 8), (4, 2, 2, 4)),   # x: one block; y: box 6 < L; t: box = L
])
def test_block_operator_box_equals_definition(dims, block):
    act = op.Action(dims=dims, Ls=3, **MOB)
    U = gauge(act)
    mf = 0.05
    origins = sv.block_origins(act.dims, block)
    for origin in [origins[0], origins[len(origins) // 2], origins[-1]]:
        mask = sv.block_mask(act, block, origin)
        x = sv.project(rand_even(act), mask)
        want = sv.a_block(act, U, x, mf, mask)
        got = sv.a_block_box(act, U, x, mf, origin, block)
        assert np.abs(got - want).max() < 1e-13 * np.abs(want).max()


def test_block_operator_hermitian_pd_and_snake_terms():
    act = op.Action(dims=(4, 4, 2, 4), Ls=4, **MOB)
    U = gauge(act)
    mf = 0.05
    block = (2, 2, 2, 2)
    origin = (2, 0, 0, 2)
    mask = sv.block_mask(act, block, origin)
    As, idx = dense_on(lambda v: sv.a_block(act, U, v, mf, mask), act, mask)
    assert np.abs(As - As.conj().T).max() < 1e-13 * np.abs(As).max()
    assert np.linalg.eigvalsh(As).min() > 0
    # the snake terms are O(1): the truncated operator differs
    At, _ = dense_on(lambda v: sv.a_block_truncated(act, U, v, mf, mask), act, mask)
    assert np.abs(As - At).max() > 0.05 * np.abs(As).max()
    assert np.abs(At - At.conj().T).max() < 1e-13 * np.abs(At).max()


def test_single_block_is_whole_operator():
    act = op.Action(dims=(4, 2, 2, 4), Ls=3, **MOB)
    U = gauge(act)
    mf = 0.05
    mask = sv.block_mask(act, act.dims, (0, 0, 0, 0))
    x = rand_even(act)
    A = op.mdagm(act, U, x, mf)
    assert np.abs(sv.a_block(act, U, x, mf, mask) - A).max() < 1e-13 * np.abs(A).max()
    assert np.abs(sv.a_block_box(act, U, x, mf, (0, 0, 0, 0), act.dims) - A).max() < 1e-13 * np.abs(A).max()


# ----------------------------------------------------------------------------
# fixed-k inner CG
# ----------------------------------------------------------------------------
@pytest.fixture(scope="module")
def small_block():
    act = op.Action(dims=(4, 4, 4, 4), Ls=4, **MOB)
    U = gauge(act, seed=5)
    mf = 0.05
    block = (2, 2, 2, 2)
    origin = (0, 2, 2, 0)
    mask = sv.block_mask(act, block, origin)
    Aop = lambda v: sv.a_block(act, U, v, mf, mask)
    As, idx = dense_on(Aop, act, mask)
    r = sv.project(rand_even(act), mask)
    return act, Aop, As, idx, r


def test_inner_cg_k1_closed_form(small_block):
    act, Aop, As, idx, r = small_block
    z = sv.cg_fixed(Aop, r, 1)
    want = op.norm2(r) / op.vdot(r, Aop(r)).real * r
    assert np.abs(z - want).max() < 1e-14 * np.abs(want).max()


@pytest.mark.parametrize("k", [2, 3, 5])
def test_inner_cg_is_krylov_optimal(small_block, k):
    """CG_k minimises the A-norm error over the Krylov space K_k(A_s, r)."""
    act, Aop, As, idx, r = small_block
    rv = r.reshape(-1)[idx]
    V = [rv]
    for _ in range(k - 1):
        V.append(As @ V[-1])
    Q, _ = np.linalg.qr(np.array(V).T)
    c = np.linalg.solve(Q.conj().T @ As @ Q, Q.conj().T @ rv)
    want = Q @ c
    z = sv.cg_fixed(Aop, r, k).reshape(-1)[idx]
    assert np.abs(z - want).max() < 1e-9 * np.abs(want).max()


@pytest.mark.parametrize("eps", [0.5, 0.1, 0.02])
def test_inner_cg_with_residual_stop(small_block, eps):
    """cg_stop takes the first k whose CG residual is <= eps |r|: its result is
    the Krylov-optimal solution in K_k (dense Galerkin), whose residual
    |r - A_s z| meets the stop, while the optimal one in K_{k-1} does not."""
    act, Aop, As, idx, r = small_block
    rv = r.reshape(-1)[idx]
    z, k = sv.cg_stop(Aop, r, 50, eps)
    assert 1 <= k < 50
    want = krylov_optimal(As, rv, k)
    assert np.abs(z.reshape(-1)[idx] - want).max() < 1e-9 * np.abs(want).max()
    assert np.linalg.norm(rv - As @ want) <= eps * np.linalg.norm(rv) * (1 + 1e-9)
    if k > 1:
        prev = krylov_optimal(As, rv, k - 1)
        assert np.linalg.norm(rv - As @ prev) > eps * np.linalg.norm(rv)
    # eps = 0 is the fixed-count solve
    z0, k0 = sv.cg_stop(Aop, r, 3, 0.0)
    assert k0 == 3 and np.abs(z0 - sv.cg_fixed(Aop, r, 3)).max() == 0.0


def test_inner_cg_many_iterations_is_exact(small_block):
    act, Aop, As, idx, r = small_block
    z = sv.cg_fixed(Aop, r, 120).reshape(-1)[idx]
    want = np.linalg.solve(As, r.reshape(-1)[idx])
    assert np.abs(z - want).max() < 1e-10 * np.abs(want).max()


# ----------------------------------------------------------------------------
# The multisplitting preconditioner M^-1 = (+)_s CG_k(A_s) (Sec. 2.4): the
# assembly over several blocks against a dense block-diagonal construction
# ----------------------------------------------------------------------------
def krylov_optimal(A, r, k):
    """The A-norm-optimal approximation of A^-1 r in K_k(A, r), computed densely
    (Galerkin projection on an orthonormal Krylov basis), which is what k CG
    steps from a zero guess produce in exact arithmetic."""
    V = [r]
    for _ in range(k - 1):
        V.append(A @ V[-1])
    Q, _ = np.linalg.qr(np.array(V).T)
    return Q @ np.linalg.solve(Q.conj().T @ A @ Q, Q.conj().T @ r)


@pytest.fixture(scope="module")
def four_blocks():
    """4x4x2x2 x Ls=2 lattice cut into 2^4 blocks: two blocks in x and two in y,
    one block (keeping its periodic wrap) in z and t. Dense A = D_PC^+ D_PC on
    all even sites, from the oracle's pinned operator."""
    act = op.Action(dims=(4, 4, 2, 2), Ls=2, **MOB)
    U = gauge(act, seed=21)
    mf = 0.07
    A, idx = dense_on(lambda v: op.mdagm(act, U, v, mf), act, np.ones(act.shape4, bool))
    block = (2, 2, 2, 2)
    sels = []
    for o in sv.block_origins(act.dims, block):
        m = sv.block_mask(act, block, o)
        m5 = np.broadcast_to(m[None, :, :, :, :, None, None], act.shape5).reshape(-1)
        sels.append((o, m, np.flatnonzero(m5[idx])))
    r = rand_even(act)
    return act, U, mf, A, idx, block, sels, r


def test_block_partition_covers_even_sites_once(four_blocks):
    act, U, mf, A, idx, block, sels, r = four_blocks
    assert len(sels) == 4
    allsel = np.concatenate([s for _, _, s in sels])
    assert np.array_equal(np.sort(allsel), np.arange(len(idx)))


def test_ms_precondition_symmetric_form_is_block_diagonal_stack(four_blocks):
    """The same stacking for the symmetric Schur form: on every block the
    Krylov-optimal solution with the dense sub-matrix of A_sym, with and
    without an inner residual stop (the stop applied per block)."""
    act, U, mf, A, idx, block, sels, r = four_blocks
    Asym, idx2 = dense_on(lambda v: op.mdagm_sym(act, U, v, mf), act, np.ones(act.shape4, bool))
    assert np.array_equal(idx, idx2)
    rv = r.reshape(-1)[idx]
    for inner_tol in (0.0, 0.3):
        z = sv.ms_precondition(act, U, r, mf, block, 4, form="definition", schur="sym",
                               inner_tol=inner_tol).reshape(-1)[idx]
        for origin, _, sel in sels:
            As = Asym[np.ix_(sel, sel)]
            k = 4
            if inner_tol:
                k = next(j for j in range(1, 5)
                         if np.linalg.norm(rv[sel] - As @ krylov_optimal(As, rv[sel], j))
                         <= inner_tol * np.linalg.norm(rv[sel]) or j == 4)
            want = krylov_optimal(As, rv[sel], k)
            assert np.abs(z[sel] - want).max() < 1e-11 * np.abs(want).max(), (origin, inner_tol)


@pytest.mark.parametrize("form", ["definition", "box"])
@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_ms_precondition_is_block_diagonal_stack(four_blocks, form, k):
    """z = M^-1 r equals, on every block s, the Krylov-optimal k-step solution
    of the dense sub-matrix A[s, s] (= P_s A P_s, Sec. 2.3) with the block's
    part of r; the blocks do not couple."""
    act, U, mf, A, idx, block, sels, r = four_blocks
    z = sv.ms_precondition(act, U, r, mf, block, k, form=form).reshape(-1)[idx]
    rv = r.reshape(-1)[idx]
    for origin, _, sel in sels:
        want = krylov_optimal(A[np.ix_(sel, sel)], rv[sel], k)
        assert np.abs(z[sel] - want).max() < 1e-12 * np.abs(want).max(), origin


def test_ms_precondition_truncated_is_block_diagonal_stack(four_blocks):
    """The same stacking with the snake-truncated block operator (snake = 0),
    whose dense form comes block by block from a_block_truncated."""
    act, U, mf, A, idx, block, sels, r = four_blocks
    k = 3
    z = sv.ms_precondition(act, U, r, mf, block, k, snake=False)
    for origin, mask, _ in sels:
        At, bidx = dense_on(lambda v, m=mask: sv.a_block_truncated(act, U, v, mf, m), act, mask)
        want = krylov_optimal(At, r.reshape(-1)[bidx], k)
        got = z.reshape(-1)[bidx]
        assert np.abs(got - want).max() < 1e-12 * np.abs(want).max(), origin


# ----------------------------------------------------------------------------
# A on large lattices, slab by slab (oracle/slabs.py)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("antiperiodic", [True, False])
def test_slab_evaluation_equals_whole_lattice(antiperiodic):
    """A x evaluated in t slabs of 2 rows, each on a small periodic lattice
    with a four-row halo and the antiperiodic sign folded into the links,
    equals op.mdagm on the whole lattice (A has range 4)."""
    from oracle import slabs
    act = op.Action(dims=(4, 2, 2, 12), Ls=3, antiperiodic=antiperiodic, **MOB)
    Uc = syn.gauge_field(act.dims, 0.5, 31)
    x = op.full_to_half(rand_even(act), 0)
    want = op.full_to_half(op.mdagm(act, op.gauge_to_mu_major(Uc), op.half_to_full(x, 0), 0.04), 0)
    got = slabs.mdagm_half(act, Uc, x, 0.04, slab=2, workers=2)
    assert np.abs(got - want).max() < 1e-13 * np.abs(want).max()


# ----------------------------------------------------------------------------
# MSPCG (Algorithm 1 with the multisplitting preconditioner)
# ----------------------------------------------------------------------------
def test_mspcg_solves_and_matches_dense():
    act = op.Action(dims=(4, 2, 2, 4), Ls=4, **MOB)
    U = gauge(act, eps=0.5, seed=8)
    mf = 0.05
    b = rand_even(act)
    x, it, res = sv.mspcg(act, U, b, mf, (2, 2, 2, 2), 4, 1e-10)
    assert res <= 1e-10
    A, idx = dense_on(lambda v: op.mdagm(act, U, v, mf), act, np.ones(act.shape4, bool))
    xd = np.linalg.solve(A, b.reshape(-1)[idx])
    cond = np.linalg.cond(A)
    assert np.abs(x.reshape(-1)[idx] - xd).max() <= 10 * cond * 1e-10 * np.abs(xd).max()
    xc, itc, _ = sv.cg(lambda v: op.mdagm(act, U, v, mf), b, 1e-10)
    assert it < itc


def test_mspcg_symmetric_form_and_inner_stop_give_the_full_system_solution():
    """MSPCG on the normal equation of the symmetric form, and with an inner
    residual stop, reaches the same even solution of D psi = phi as the paper's
    form (both normal equations have it as their unique solution)."""
    act = op.Action(dims=(4, 2, 2, 4), Ls=4, **MOB)
    U = gauge(act, eps=0.5, seed=8)
    mf = 0.05
    phi = RNG.normal(size=act.shape5) + 1j * RNG.normal(size=act.shape5)
    phi_e, phi_o = op.restrict_parity(phi, 0), op.restrict_parity(phi, 1)
    sols = []
    for schur, inner_tol in (("asym", 0.0), ("sym", 0.0), ("asym", 0.2)):
        b = op.normal_source(act, U, phi_e, phi_o, mf, schur)
        x, it, res = sv.mspcg(act, U, b, mf, (2, 2, 2, 2), 4, 1e-11, schur=schur,
                              inner_tol=inner_tol)
        assert res <= 1e-11
        sols.append(x)
    for x in sols[1:]:
        assert np.abs(x - sols[0]).max() < 1e-8 * np.abs(sols[0]).max()


def test_mspcg_one_block_large_k_converges_at_once():
    act = op.Action(dims=(2, 2, 2, 4), Ls=4, **MOB)
    U = gauge(act, eps=0.5, seed=9)
    mf = 0.1
    b = rand_even(act)
    x, it, res = sv.mspcg(act, U, b, mf, act.dims, 150, 1e-10)
    assert res <= 1e-10
    assert it <= 2


@pytest.mark.slow
def test_table1_trends_on_synthetic_field():
    """Trends of the paper's Table 1 (Sec. 3): MSPCG needs fewer outer
    iterations than plain CG, more inner iterations help with diminishing
    returns, and keeping the snake terms matters (Sec. 2.3)."""
    act = op.Action(dims=(4, 4, 4, 8), Ls=4, **MOB)
    U = gauge(act, eps=0.45, seed=13)
    mf = 0.01
    b = rand_even(act)
    block = (4, 4, 4, 4)
    tol = 1e-6
    A = lambda v: op.mdagm(act, U, v, mf)
    _, plain, _ = sv.cg(A, b, tol)
    its = {}
    for k in (2, 4, 8):
        _, its[k], res = sv.mspcg(act, U, b, mf, block, k, tol)
        assert res <= tol
    assert its[2] < plain
    assert its[2] >= its[4] >= its[8]
    _, trunc, _ = sv.mspcg(act, U, b, mf, block, 4, tol, snake=False)
    assert its[4] < trunc
