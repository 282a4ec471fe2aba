"""Pins of the FP64 oracle operator against facts it does not compute itself.

Each test checks the oracle against a closed form, an algebraic identity, a
symmetry, or a dense brute-force construction, chosen so that a dropped term,
a wrong sign or index, or a transposed operand fails at least one of them.
"""
import os

import numpy as np
import pytest

from oracle import dwf_operator as op
from oracle import pointwise
from paper_1811_08488_gb300 import synthetic as syn

RNG = np.random.default_rng(7)


def rand5(act, parity=None):
    psi = RNG.normal(size=act.shape5) + 1j * RNG.normal(size=act.shape5)
    if parity is not None:
        psi = op.restrict_parity(psi, parity)
    return psi


def gauge(act, eps=0.4, seed=11):
    return op.gauge_to_mu_major(syn.gauge_field(act.dims, eps, seed))


MOB = dict(M5=1.8, b=1.5, c=0.5)


# ----------------------------------------------------------------------------
# synthetic inputs
# ----------------------------------------------------------------------------
def test_splitmix64_published_values():
    path = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed0.txt")
    want = [int(l, 16) for l in open(path) if l.strip() and not l.startswith("#")]
    got = [int(v) for v in syn.splitmix64(0, 3)]
    assert got == want


def test_parallel_draws_equal_serial_draws():
    """Large fields are drawn in slabs by worker processes; each slab reads its
    own part of the counter-based stream, so the arrays are the same."""
    dims = (4, 4, 2, 6)
    assert np.array_equal(syn.gauge_field(dims, 0.4, 3),
                          syn.gauge_field(dims, 0.4, 3, parallel_min=1))
    assert np.array_equal(syn.half_field(dims, 5, 3), syn.half_field(dims, 5, 3, parallel_min=1))
    n = syn.normal(9, 20)
    assert np.array_equal(syn.normal(9, 8, 12), n[12:])


def test_gauge_is_su3():
    U = syn.gauge_field((4, 4, 4, 4), 0.4, 5)
    I = np.eye(3)
    err = np.abs(U @ np.conj(np.swapaxes(U, -1, -2)) - I).max()
    assert err < 1e-14
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-14
    # Re tr exp(i eps H) / 3 = 1 - eps^2 tr(H^2) / 6 + O(eps^4) and E tr(H^2) = 4
    # for H = sum_a h_a lambda_a / 2 with tr(lambda_a lambda_b) = 2 delta_ab
    U = syn.gauge_field((4, 4, 4, 4), 0.1, 5)
    tr = np.einsum("...ii", U).real.mean() / 3
    assert abs(tr - (1 - 0.01 * 4 / 6)) < 1e-3


# ----------------------------------------------------------------------------
# gamma matrices
# ----------------------------------------------------------------------------
def test_clifford_algebra_and_chiral_basis():
    for m in range(4):
        assert np.allclose(op.GAMMA[m], op.GAMMA[m].conj().T)
        for n in range(4):
            ac = op.GAMMA[m] @ op.GAMMA[n] + op.GAMMA[n] @ op.GAMMA[m]
            assert np.allclose(ac, 2 * np.eye(4) * (m == n))
    assert np.allclose(op.GAMMA5, np.diag([1, 1, -1, -1]))


def test_half_full_roundtrip():
    act = op.Action(dims=(4, 2, 4, 6), Ls=3)
    h = syn.half_field(act.dims, act.Ls, 3)
    for p in (0, 1):
        f = op.half_to_full(h, p)
        # the full array lives on parity p only
        assert np.allclose(op.restrict_parity(f, 1 - p), 0)
        assert np.array_equal(op.full_to_half(f, p), h)
    # explicit site check: x = 2*xh + ((parity + y + z + t) % 2)
    f = op.half_to_full(h, 1)
    s, t, z, y, xh = 2, 5, 3, 1, 1
    x = 2 * xh + ((1 + y + z + t) % 2)
    assert np.array_equal(f[s, t, z, y, x], h[s, t, z, y, xh])


# ----------------------------------------------------------------------------
# free field: momentum-space closed form
# ----------------------------------------------------------------------------
def dw_momentum(p, M5):
    """Free Wilson operator in momentum space:
    D_W(p) = i sum_mu g_mu sin p_mu + sum_mu (1 - cos p_mu) - M5."""
    D = (sum(1 - np.cos(pm) for pm in p) - M5) * np.eye(4, dtype=complex)
    for mu in range(4):
        D = D + 1j * np.sin(p[mu]) * op.GAMMA[mu]
    return D


def c_dense(Ls, mf):
    """C on (s, spin): (C psi)_s = P_- psi_{s+1} + P_+ psi_{s-1}, -mf on the wrap."""
    C = np.zeros((Ls * 4, Ls * 4), dtype=complex)
    for s in range(Ls):
        sp, wp = (s + 1) % Ls, (-mf if s == Ls - 1 else 1.0)
        sm, wm = (s - 1) % Ls, (-mf if s == 0 else 1.0)
        C[4 * s:4 * s + 4, 4 * sp:4 * sp + 4] += wp * op.P_MINUS
        C[4 * s:4 * s + 4, 4 * sm:4 * sm + 4] += wm * op.P_PLUS
    return C


def d_momentum(p, act, mf):
    """D(p) = D_W(p) (b + c C) + (1 - C) on (s, spin)."""
    Ls = act.Ls
    DW = np.kron(np.eye(Ls), dw_momentum(p, act.M5))
    C = c_dense(Ls, mf)
    I = np.eye(4 * Ls)
    return DW @ (act.b * I + act.c * C) + (I - C)


def momenta(dims, antiperiodic=True):
    Lx, Ly, Lz, Lt = dims
    out = []
    for nx in range(Lx):
        for ny in range(Ly):
            for nz in range(Lz):
                for nt in range(Lt):
                    pt = (2 * nt + (1 if antiperiodic else 0)) * np.pi / Lt
                    out.append((2 * np.pi * nx / Lx, 2 * np.pi * ny / Ly, 2 * np.pi * nz / Lz, pt))
    return out


def plane_wave(act, p, chi, col):
    t, z, y, x = np.indices(act.shape4)
    ph = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    # chi: (Ls, 4) ; col: (3,)
    return np.einsum("tzyx,si,a->stzyxia", ph, chi, col)


@pytest.mark.parametrize("params", [dict(M5=1.8, b=1.0, c=0.0), MOB])
def test_free_field_plane_wave(params):
    act = op.Action(dims=(4, 4, 6, 8), Ls=5, **params)
    U = op.gauge_to_mu_major(syn.unit_gauge(act.dims))
    mf = 0.07
    for p in [(0, 0, 0, np.pi / 8), (np.pi / 2, np.pi, 2 * np.pi / 3, 3 * np.pi / 8),
              (3 * np.pi / 2, np.pi / 2, 4 * np.pi / 3, 13 * np.pi / 8)]:
        chi = RNG.normal(size=(act.Ls, 4)) + 1j * RNG.normal(size=(act.Ls, 4))
        col = RNG.normal(size=3) + 1j * RNG.normal(size=3)
        psi = plane_wave(act, p, chi, col)
        got = op.dwf_full(act, U, psi, mf)
        want = plane_wave(act, p, (d_momentum(p, act, mf) @ chi.reshape(-1)).reshape(act.Ls, 4), col)
        assert np.abs(got - want).max() < 1e-12


def test_free_field_spectrum_matches_momentum_space():
    """The whole spectrum of D^dag D on a free 2^3x4 lattice equals the union over
    momenta of eig(D(p)^dag D(p)), each three times (colour)."""
    act = op.Action(dims=(2, 2, 2, 4), Ls=4, **MOB)
    mf = 0.1
    U = op.gauge_to_mu_major(syn.unit_gauge(act.dims))
    n = int(np.prod(act.shape5))
    cols = []
    for j in range(n):
        e = np.zeros(n, dtype=complex)
        e[j] = 1
        cols.append(op.dwf_full(act, U, e.reshape(act.shape5), mf).reshape(-1))
    D = np.array(cols).T
    lat = np.sort(np.linalg.eigvalsh(D.conj().T @ D))
    mom = []
    for p in momenta(act.dims):
        Dp = d_momentum(p, act, mf)
        mom.extend(list(np.linalg.eigvalsh(Dp.conj().T @ Dp)) * 3)
    mom = np.sort(np.array(mom))
    assert lat.shape == mom.shape
    assert np.abs(lat - mom).max() < 1e-10
    # the chiral mode: the lowest eigenvalue is far below the bulk
    assert lat[0] < 0.05 * lat[-1]


def test_mobius_gamma5_hermiticity_of_dminus_inverse_d():
    """For Moebius, Gamma5 = g5 R5 makes D_-^{-1} D Hermitian in momentum space,
    with D_- = c D_W - 1 (R5 reflects s). D(p) is read off the oracle."""
    act = op.Action(dims=(4, 4, 4, 8), Ls=6, **MOB)
    mf = 0.05
    U = op.gauge_to_mu_major(syn.unit_gauge(act.dims))
    R5 = np.fliplr(np.eye(act.Ls))
    G5 = np.kron(R5, op.GAMMA5)
    for p in [(np.pi / 2, 0, np.pi, np.pi / 8), (np.pi / 2, np.pi / 2, 3 * np.pi / 2, 5 * np.pi / 8)]:
        # read D(p) off the oracle column by column
        Dp = np.zeros((4 * act.Ls, 4 * act.Ls), dtype=complex)
        col = np.array([1.0, 0, 0], dtype=complex)
        site = (1, 2, 3, 1)  # (t, z, y, x) index where the phase is read
        t, z, y, x = site
        ph = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
        for j in range(4 * act.Ls):
            chi = np.zeros(4 * act.Ls, dtype=complex)
            chi[j] = 1
            out = op.dwf_full(act, U, plane_wave(act, p, chi.reshape(act.Ls, 4), col), mf)
            Dp[:, j] = out[:, t, z, y, x, :, 0].reshape(-1) / ph
        Dm = np.kron(np.eye(act.Ls), act.c * dw_momentum(p, act.M5) - np.eye(4))
        H = np.linalg.solve(Dm, Dp)
        assert np.abs(G5 @ H @ G5 - H.conj().T).max() < 1e-12


# ----------------------------------------------------------------------------
# symmetries with a random gauge field
# ----------------------------------------------------------------------------
def test_wilson_gamma5_hermiticity():
    act = op.Action(dims=(4, 4, 4, 4), Ls=2, M5=1.8)
    U = gauge(act)
    x, y = rand5(act), rand5(act)
    DW = lambda v: (4 - act.M5) * v - 0.5 * op.dhop(act, U, v)
    g5 = lambda v: op.spin(op.GAMMA5, v)
    lhs = op.vdot(x, g5(DW(g5(y))))
    rhs = op.vdot(DW(x), y)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_shamir_gamma5_r5_hermiticity():
    act = op.Action(dims=(4, 4, 4, 4), Ls=6, M5=1.8, b=1.0, c=0.0)
    U = gauge(act)
    mf = 0.03
    x, y = rand5(act), rand5(act)
    G5 = lambda v: op.spin(op.GAMMA5, v[::-1])
    lhs = op.vdot(x, G5(op.dwf_full(act, U, G5(y), mf)))
    rhs = op.vdot(op.dwf_full(act, U, x, mf), y)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_mobius_is_not_gamma5_r5_hermitian():
    """Guard against using the Shamir shortcut for the Moebius adjoint."""
    act = op.Action(dims=(4, 4, 4, 4), Ls=6, **MOB)
    U = gauge(act)
    x, y = rand5(act), rand5(act)
    G5 = lambda v: op.spin(op.GAMMA5, v[::-1])
    lhs = op.vdot(x, G5(op.dwf_full(act, U, G5(y), 0.03)))
    rhs = op.vdot(op.dwf_full(act, U, x, 0.03), y)
    assert abs(lhs - rhs) > 1e-3 * abs(lhs)


@pytest.mark.parametrize("name", ["dhop", "cmat", "m5", "mphi", "m5inv", "m4", "dwf_full", "mpc"])
def test_adjoint_identities(name):
    act = op.Action(dims=(4, 2, 2, 4), Ls=4, **MOB)
    U = gauge(act)
    mf = 0.02
    x, y = rand5(act), rand5(act)
    if name == "mpc":
        x, y = op.restrict_parity(x, 0), op.restrict_parity(y, 0)
    f = {
        "dhop": lambda v, d: op.dhop(act, U, v, d),
        "cmat": lambda v, d: op.cmat(v, mf, d),
        "m5": lambda v, d: op.m5(act, v, mf, d),
        "mphi": lambda v, d: op.mphi(act, v, mf, d),
        "m5inv": lambda v, d: op.m5inv(act, v, mf, d),
        "m4": lambda v, d: op.m4(act, U, v, mf, d),
        "dwf_full": lambda v, d: op.dwf_full(act, U, v, mf, d),
        "mpc": lambda v, d: op.mpc(act, U, v, mf, d),
    }[name]
    lhs = op.vdot(x, f(y, False))
    rhs = op.vdot(f(x, True), y)
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), 1.0)


def test_gauge_covariance():
    act = op.Action(dims=(4, 4, 2, 4), Ls=4, **MOB)
    U = gauge(act)
    mf = 0.05
    g = syn.random_su3(act.shape4, 99)  # g(x) on (T,Z,Y,X)
    gd = np.conj(np.swapaxes(g, -1, -2))
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[mu] = g @ U[mu] @ op.shift4(gd, mu, +1)
    psi = rand5(act)
    gpsi = op.colour(g, psi)
    lhs = op.dwf_full(act, Ug, gpsi, mf)
    rhs = op.colour(g, op.dwf_full(act, U, psi, mf))
    assert np.abs(lhs - rhs).max() < 1e-12
    # the paper's literal U^dag on the forward hop is not covariant
    def dhop_literal(v):
        out = np.zeros_like(v)
        for mu in range(4):
            bc = -1.0 if mu == 3 else 1.0
            out += op.spin(op.ID4 - op.GAMMA[mu], op.colour(op.dagger3(Ug[mu]), op.shift5(v, mu, 1, bc)))
            out += op.spin(op.ID4 + op.GAMMA[mu], op.colour(op.dagger3(op.shift4(Ug[mu], mu, -1)),
                                                             op.shift5(v, mu, -1, bc)))
        return out
    def dhop_literal_U(v):
        out = np.zeros_like(v)
        for mu in range(4):
            bc = -1.0 if mu == 3 else 1.0
            out += op.spin(op.ID4 - op.GAMMA[mu], op.colour(op.dagger3(U[mu]), op.shift5(v, mu, 1, bc)))
            out += op.spin(op.ID4 + op.GAMMA[mu], op.colour(op.dagger3(op.shift4(U[mu], mu, -1)),
                                                             op.shift5(v, mu, -1, bc)))
        return out
    assert np.abs(dhop_literal(gpsi) - op.colour(g, dhop_literal_U(psi))).max() > 1e-2


# ----------------------------------------------------------------------------
# M_5^-1: geometric-series closed form
# ----------------------------------------------------------------------------
def m5inv_closed_form(act, mf, dagger=False):
    """Per chirality M_5 = alpha (1 - r S) with r = -beta/alpha and S^Ls = -mf, so
    M_5^-1 = [alpha (1 + mf r^Ls)]^-1 sum_{k<Ls} r^k S^k. S moves s-1 -> s on the
    upper spins (P_+) and s+1 -> s on the lower spins (P_-); the adjoint swaps them."""
    Ls, a, bt = act.Ls, act.alpha, act.beta
    r = -bt / a
    out = np.zeros((4 * Ls, 4 * Ls))
    for chir, spins in ((+1, (0, 1)), (-1, (2, 3))):
        S = np.zeros((Ls, Ls))
        down = (chir == +1) != dagger  # S takes psi_{s-1}
        for s in range(Ls):
            if down:
                S[s, (s - 1) % Ls] = -mf if s == 0 else 1.0
            else:
                S[s, (s + 1) % Ls] = -mf if s == Ls - 1 else 1.0
        acc = np.zeros((Ls, Ls))
        Sk = np.eye(Ls)
        for k in range(Ls):
            acc += r ** k * Sk
            Sk = Sk @ S
        acc /= a * (1 + mf * r ** Ls)
        for sp in spins:
            out[sp::4, sp::4] = acc
    return out


@pytest.mark.parametrize("params,Ls", [(dict(M5=1.8, b=1.0, c=0.0), 8), (MOB, 12), (MOB, 5)])
@pytest.mark.parametrize("dagger", [False, True])
def test_m5inv_closed_form(params, Ls, dagger):
    act = op.Action(dims=(2, 2, 2, 2), Ls=Ls, **params)
    mf = 0.01
    M = op.m5_matrix(act, mf, dagger)
    Minv = m5inv_closed_form(act, mf, dagger)
    assert np.abs(Minv @ M - np.eye(4 * Ls)).max() < 1e-13
    assert np.abs(np.linalg.inv(M) - Minv).max() < 1e-13
    # and the oracle's function inverts the oracle's M_5
    psi = rand5(act)
    assert np.abs(op.m5inv(act, op.m5(act, psi, mf, dagger), mf, dagger) - psi).max() < 1e-13


# ----------------------------------------------------------------------------
# dense brute force on 2^4 x Ls=4
# ----------------------------------------------------------------------------
def dense(fn, shape, mask=None):
    n = int(np.prod(shape))
    idx = np.arange(n) if mask is None else np.flatnonzero(mask.reshape(-1))
    cols = []
    for j in idx:
        e = np.zeros(n, dtype=complex)
        e[j] = 1
        cols.append(fn(e.reshape(shape)).reshape(-1)[idx])
    return np.array(cols).T, idx


@pytest.fixture(scope="module")
def brute():
    act = op.Action(dims=(2, 2, 2, 2), Ls=4, **MOB)
    U = gauge(act, eps=0.5, seed=3)
    mf = 0.04
    D, _ = dense(lambda v: op.dwf_full(act, U, v, mf), act.shape5)
    par = op.parity_mask(act.shape4)
    full_par = np.broadcast_to(par[None, :, :, :, :, None, None], act.shape5).reshape(-1)
    e = np.flatnonzero(full_par == 0)
    o = np.flatnonzero(full_par == 1)
    return act, U, mf, D, e, o


def test_dense_even_odd_blocks(brute):
    act, U, mf, D, e, o = brute
    # diagonal blocks are M_5 (constant in space-time), off-diagonal blocks are M^4
    M5d, _ = dense(lambda v: op.m5(act, v, mf), act.shape5)
    assert np.abs(D[np.ix_(e, e)] - M5d[np.ix_(e, e)]).max() < 1e-14
    assert np.abs(D[np.ix_(o, o)] - M5d[np.ix_(o, o)]).max() < 1e-14


def test_dense_schur_complement(brute):
    act, U, mf, D, e, o = brute
    Dee, Deo, Doe, Doo = D[np.ix_(e, e)], D[np.ix_(e, o)], D[np.ix_(o, e)], D[np.ix_(o, o)]
    Dpc_dense = Dee - Deo @ np.linalg.solve(Doo, Doe)
    even = op.parity_mask(act.shape4) == 0
    mask5 = np.broadcast_to(even[None, :, :, :, :, None, None], act.shape5)
    Dpc, idx = dense(lambda v: op.mpc(act, U, v, mf), act.shape5, mask5)
    assert np.array_equal(idx, e)
    assert np.abs(Dpc - Dpc_dense).max() < 1e-12
    Dpcd, _ = dense(lambda v: op.mpc(act, U, v, mf, True), act.shape5, mask5)
    assert np.abs(Dpcd - Dpc_dense.conj().T).max() < 1e-12
    A, _ = dense(lambda v: op.mdagm(act, U, v, mf), act.shape5, mask5)
    assert np.abs(A - Dpc_dense.conj().T @ Dpc_dense).max() < 1e-12
    w = np.linalg.eigvalsh(0.5 * (A + A.conj().T))
    assert w.min() > 0


def test_schur_solution_solves_full_system(brute):
    """Solve D_PC psi_e = phi_hat_e, reconstruct psi_o, and check D psi = phi."""
    act, U, mf, D, e, o = brute
    phi = rand5(act)
    phi_e, phi_o = op.restrict_parity(phi, 0), op.restrict_parity(phi, 1)
    phat = op.source_prep(act, U, phi_e, phi_o, mf)
    even = op.parity_mask(act.shape4) == 0
    mask5 = np.broadcast_to(even[None, :, :, :, :, None, None], act.shape5)
    Dpc, idx = dense(lambda v: op.mpc(act, U, v, mf), act.shape5, mask5)
    sol = np.linalg.solve(Dpc, phat.reshape(-1)[idx])
    psi_e = np.zeros(phi.size, dtype=complex)
    psi_e[idx] = sol
    psi_e = psi_e.reshape(act.shape5)
    psi_o = op.odd_reconstruct(act, U, psi_e, phi_o, mf)
    psi = psi_e + psi_o
    assert np.abs(D @ psi.reshape(-1) - phi.reshape(-1)).max() < 1e-11


def test_symmetric_schur_form_dense(brute):
    """D_sym = 1 - M_5^-1 M^4_eo M_5^-1 M^4_oe equals D_ee^-1 (D_ee - D_eo D_oo^-1
    D_oe) built from the dense full matrix, its adjoint is the conjugate
    transpose, and A_sym = D_sym^dag D_sym is Hermitian positive definite."""
    act, U, mf, D, e, o = brute
    Dee, Deo, Doe, Doo = D[np.ix_(e, e)], D[np.ix_(e, o)], D[np.ix_(o, e)], D[np.ix_(o, o)]
    Dsym_dense = np.linalg.solve(Dee, Dee - Deo @ np.linalg.solve(Doo, Doe))
    even = op.parity_mask(act.shape4) == 0
    mask5 = np.broadcast_to(even[None, :, :, :, :, None, None], act.shape5)
    Dsym, idx = dense(lambda v: op.mpc_sym(act, U, v, mf), act.shape5, mask5)
    assert np.abs(Dsym - Dsym_dense).max() < 1e-12
    Dsymd, _ = dense(lambda v: op.mpc_sym(act, U, v, mf, True), act.shape5, mask5)
    assert np.abs(Dsymd - Dsym_dense.conj().T).max() < 1e-12
    A, _ = dense(lambda v: op.mdagm_sym(act, U, v, mf), act.shape5, mask5)
    assert np.abs(A - Dsym_dense.conj().T @ Dsym_dense).max() < 1e-12
    assert np.linalg.eigvalsh(0.5 * (A + A.conj().T)).min() > 0


@pytest.mark.parametrize("schur", ["asym", "sym"])
def test_normal_equation_solution_solves_full_system(brute, schur):
    """The normal equation of either Schur form, with its right-hand side
    normal_source, gives the even half of the solution of D psi = phi."""
    act, U, mf, D, e, o = brute
    phi = rand5(act)
    phi_e, phi_o = op.restrict_parity(phi, 0), op.restrict_parity(phi, 1)
    b = op.normal_source(act, U, phi_e, phi_o, mf, schur)
    even = op.parity_mask(act.shape4) == 0
    mask5 = np.broadcast_to(even[None, :, :, :, :, None, None], act.shape5)
    A, idx = dense(lambda v: op.normal_op(schur)(act, U, v, mf), act.shape5, mask5)
    psi_e = np.zeros(phi.size, dtype=complex)
    psi_e[idx] = np.linalg.solve(A, b.reshape(-1)[idx])
    psi_e = psi_e.reshape(act.shape5)
    psi = psi_e + op.odd_reconstruct(act, U, psi_e, phi_o, mf)
    assert np.abs(D @ psi.reshape(-1) - phi.reshape(-1)).max() < 1e-10


def test_pointwise_matches_full_array():
    act = op.Action(dims=(4, 4, 2, 6), Ls=5, **MOB)
    Uc = syn.gauge_field(act.dims, 0.4, 21)
    U = op.gauge_to_mu_major(Uc)
    mf = 0.03
    half_o = syn.half_field(act.dims, act.Ls, 77)
    full_o = op.half_to_full(half_o, 1)
    out = op.m4(act, U, full_o, mf)
    for site, s in [((0, 0, 0, 0), 0), ((3, 1, 1, 5), 4), ((1, 3, 0, 2), 2), ((2, 0, 1, 5), 0)]:
        x, y, z, t = site
        if (x + y + z + t) % 2 != 0:
            continue
        got = pointwise.m4_at(act, Uc, half_o, site, s, mf)
        assert np.abs(got - out[s, t, z, y, x]).max() < 1e-13
