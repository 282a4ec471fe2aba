"""Even-odd Moebius domain-wall operator in plain numpy (FP64).

Test infrastructure only (see oracle/__init__.py).

Paper, Sec. 2.2: the 4D even-odd form of the Moebius DWF Dirac matrix is
[[M_5, M^4_eo], [M^4_oe, M_5]], with M^4 = D^w M_phi and D^w the Wilson hop
(eq. for D^w), M_5 and M_phi constant in space-time. The paper defers the entries of
M_5 and M_phi to Brower et al. (2014); the standard Moebius (Cayley) form is
used here:

    D_W      = (4 - M5) - 1/2 Dhop
    Dhop     = sum_mu (1 - g_mu) U_mu(x) d(x+mu, y) + (1 + g_mu) U_mu(x-mu)^dag d(x-mu, y)
    (C psi)_s = P_- psi_{s+1} + P_+ psi_{s-1},  psi_{Ls} = -mf psi_0,  psi_{-1} = -mf psi_{Ls-1}
    D        = D_W (b + c C) + (1 - C)
             = [b(4-M5)+1] + [c(4-M5)-1] C  -  1/2 Dhop (b + c C)

so M_5 = alpha + beta C with alpha = b(4-M5)+1, beta = c(4-M5)-1, M_phi = b + c C,
and M^4 = -1/2 Dhop M_phi (M_phi acts first, as in the paper's M^4 = D^w M_phi).
The forward hop carries U_mu(x); the paper's dagger on it is read as a typo
(gauge covariance fixes it; see tests/test_oracle_operator.py).

Gamma matrices: chiral basis, g_k = [[0, -i s_k], [i s_k, 0]], g_4 = [[0, 1], [1, 0]],
g_5 = g_1 g_2 g_3 g_4 = diag(1, 1, -1, -1), P_+- = (1 +- g_5)/2.
Boundary conditions: periodic in x, y, z; antiperiodic in t (switchable).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# ----------------------------------------------------------------------------
# Gamma matrices
# ----------------------------------------------------------------------------
PAULI = [
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
]


def _gammas():
    g = []
    for k in range(3):
        m = np.zeros((4, 4), dtype=np.complex128)
        m[0:2, 2:4] = -1j * PAULI[k]
        m[2:4, 0:2] = 1j * PAULI[k]
        g.append(m)
    m = np.zeros((4, 4), dtype=np.complex128)
    m[0:2, 2:4] = np.eye(2)
    m[2:4, 0:2] = np.eye(2)
    g.append(m)
    return g


GAMMA = _gammas()
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
ID4 = np.eye(4, dtype=np.complex128)
P_PLUS = 0.5 * (ID4 + GAMMA5)
P_MINUS = 0.5 * (ID4 - GAMMA5)


# ----------------------------------------------------------------------------
# Parameters and lattice helpers
# ----------------------------------------------------------------------------
@dataclass
class Action:
    """Moebius DWF action. Shamir is b = 1, c = 0."""
    dims: tuple  # (Lx, Ly, Lz, Lt)
    Ls: int
    M5: float = 1.8
    b: float = 1.0
    c: float = 0.0
    antiperiodic: bool = True

    @property
    def alpha(self):
        return self.b * (4.0 - self.M5) + 1.0

    @property
    def beta(self):
        return self.c * (4.0 - self.M5) - 1.0

    @property
    def shape4(self):
        Lx, Ly, Lz, Lt = self.dims
        return (Lt, Lz, Ly, Lx)

    @property
    def shape5(self):
        return (self.Ls,) + self.shape4 + (4, 3)


def parity_mask(shape4) -> np.ndarray:
    """parity = (x + y + z + t) mod 2 on a (T, Z, Y, X) grid (paper eq. parity)."""
    t, z, y, x = np.indices(shape4)
    return (x + y + z + t) % 2


def gauge_to_mu_major(U_canon: np.ndarray) -> np.ndarray:
    """U[t][z][y][x][mu][a][b] -> U[mu][t][z][y][x][a][b]."""
    return np.ascontiguousarray(np.moveaxis(U_canon, 4, 0))


def half_to_full(half: np.ndarray, parity: int) -> np.ndarray:
    """Canonical parity half field [s][t][z][y][xh][4][3] -> full 5D array."""
    Ls, Lt, Lz, Ly, Xh = half.shape[:5]
    full = np.zeros((Ls, Lt, Lz, Ly, 2 * Xh, 4, 3), dtype=np.complex128)
    t, z, y = np.indices((Lt, Lz, Ly))
    off = (parity + y + z + t) % 2  # x = 2*xh + off
    for o in (0, 1):
        sel = off == o
        ts, zs, ys = t[sel], z[sel], y[sel]
        full[:, ts, zs, ys, o::2] = half[:, ts, zs, ys, :]
    return full


def full_to_half(full: np.ndarray, parity: int) -> np.ndarray:
    Ls, Lt, Lz, Ly, X = full.shape[:5]
    half = np.zeros((Ls, Lt, Lz, Ly, X // 2, 4, 3), dtype=np.complex128)
    t, z, y = np.indices((Lt, Lz, Ly))
    off = (parity + y + z + t) % 2
    for o in (0, 1):
        sel = off == o
        ts, zs, ys = t[sel], z[sel], y[sel]
        half[:, ts, zs, ys, :] = full[:, ts, zs, ys, o::2]
    return half


def restrict_parity(full: np.ndarray, parity: int) -> np.ndarray:
    m = parity_mask(full.shape[1:5]) == parity
    return full * m[None, :, :, :, :, None, None]


# ----------------------------------------------------------------------------
# Building blocks
# ----------------------------------------------------------------------------
def spin(P: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """Apply a 4x4 spin matrix: out[..., i, a] = sum_j P[i, j] psi[..., j, a]."""
    return np.einsum("ij,...ja->...ia", P, psi)


def colour(U: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """out[s, x, i, a] = sum_b U[x, a, b] psi[s, x, i, b]; U is (T,Z,Y,X,3,3)."""
    return psi @ np.swapaxes(U, -1, -2)


def dagger3(U: np.ndarray) -> np.ndarray:
    return np.conj(np.swapaxes(U, -1, -2))


def shift5(psi: np.ndarray, mu: int, step: int, bc: float) -> np.ndarray:
    """out(x) = psi(x + step*mu_hat) on a 5D field, with the factor bc applied
    where the shift wraps around the lattice (bc = -1: antiperiodic)."""
    axis = 4 - mu  # axes: s, t, z, y, x
    out = np.roll(psi, -step, axis=axis)
    if bc != 1.0:
        L = psi.shape[axis]
        idx = [slice(None)] * psi.ndim
        idx[axis] = L - 1 if step == 1 else 0
        out[tuple(idx)] *= bc
    return out


def shift4(U: np.ndarray, mu: int, step: int) -> np.ndarray:
    """out(x) = U(x + step*mu_hat) on a (T,Z,Y,X,...) array (no sign)."""
    return np.roll(U, -step, axis=3 - mu)


def dhop(act: Action, U: np.ndarray, psi: np.ndarray, dagger: bool = False) -> np.ndarray:
    """Wilson hop (paper eq. for D^w, with U on the forward term).

    Dhop psi(x) = sum_mu (1 - g_mu) U_mu(x) psi(x+mu) + (1 + g_mu) U_mu(x-mu)^dag psi(x-mu).
    Its adjoint has the projector signs exchanged:
    Dhop^dag psi(x) = sum_mu (1 + g_mu) U_mu(x) psi(x+mu) + (1 - g_mu) U_mu(x-mu)^dag psi(x-mu).
    U is mu-major: U[mu][t][z][y][x][a][b].
    """
    sgn = 1.0 if dagger else -1.0
    out = np.zeros_like(psi)
    for mu in range(4):
        bc = -1.0 if (act.antiperiodic and mu == 3) else 1.0
        fwd = shift5(psi, mu, +1, bc)
        out += spin(ID4 + sgn * GAMMA[mu], colour(U[mu], fwd))
        Ub = shift4(U[mu], mu, -1)
        bwd = shift5(psi, mu, -1, bc)
        out += spin(ID4 - sgn * GAMMA[mu], colour(dagger3(Ub), bwd))
    return out


def s_shift(psi: np.ndarray, step: int, mf: float) -> np.ndarray:
    """out_s = psi_{s+step}, with psi_{Ls} = -mf psi_0 and psi_{-1} = -mf psi_{Ls-1}."""
    out = np.roll(psi, -step, axis=0)
    Ls = psi.shape[0]
    if step == 1:
        out[Ls - 1] *= -mf
    else:
        out[0] *= -mf
    return out


def cmat(psi: np.ndarray, mf: float, dagger: bool = False) -> np.ndarray:
    """(C psi)_s = P_- psi_{s+1} + P_+ psi_{s-1};  (C^dag psi)_s = P_+ psi_{s+1} + P_- psi_{s-1}."""
    if not dagger:
        return spin(P_MINUS, s_shift(psi, +1, mf)) + spin(P_PLUS, s_shift(psi, -1, mf))
    return spin(P_PLUS, s_shift(psi, +1, mf)) + spin(P_MINUS, s_shift(psi, -1, mf))


def m5(act: Action, psi: np.ndarray, mf: float, dagger: bool = False) -> np.ndarray:
    """M_5 = alpha + beta C (paper eq. (dirac_equation) diagonal blocks)."""
    return act.alpha * psi + act.beta * cmat(psi, mf, dagger)


def mphi(act: Action, psi: np.ndarray, mf: float, dagger: bool = False) -> np.ndarray:
    """M_phi = b + c C."""
    return act.b * psi + act.c * cmat(psi, mf, dagger)


def m5_matrix(act: Action, mf: float, dagger: bool = False) -> np.ndarray:
    """M_5 as a dense (Ls*4) x (Ls*4) matrix on the (s, spin) index."""
    Ls = act.Ls
    n = Ls * 4
    M = np.zeros((n, n), dtype=np.complex128)
    for j in range(n):
        e = np.zeros((Ls, 1, 1, 1, 1, 4, 1), dtype=np.complex128)
        e[j // 4, 0, 0, 0, 0, j % 4, 0] = 1
        M[:, j] = m5(act, e, mf, dagger).reshape(Ls, 4).reshape(n)
    return M


def apply_ls_spin_matrix(M: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """Apply a dense matrix on the (s, spin) index, identical on sites and colour."""
    Ls = psi.shape[0]
    Mr = M.reshape(Ls, 4, Ls, 4)
    return np.einsum("sitj,t...ja->s...ia", Mr, psi)


def m5inv(act: Action, psi: np.ndarray, mf: float, dagger: bool = False) -> np.ndarray:
    """M_5^{-1} by dense inversion of M_5 on (s, spin) (its plain definition)."""
    return apply_ls_spin_matrix(np.linalg.inv(m5_matrix(act, mf, dagger)), psi)


def m4(act: Action, U, psi, mf: float, dagger: bool = False) -> np.ndarray:
    """M^4 = -1/2 Dhop M_phi; its adjoint is -1/2 M_phi^dag Dhop^dag.

    On a full lattice M^4 maps each parity to the other, so M^4_eo and M^4_oe
    (paper Sec. 2.2) are M^4 restricted to odd inputs / even inputs.
    """
    if not dagger:
        return -0.5 * dhop(act, U, mphi(act, psi, mf), dagger=False)
    return -0.5 * mphi(act, dhop(act, U, psi, dagger=True), mf, dagger=True)


def dwf_full(act: Action, U, psi, mf: float, dagger: bool = False) -> np.ndarray:
    """The unpreconditioned 5D operator D = M_5 + M^4 on the full lattice."""
    return m5(act, psi, mf, dagger) + m4(act, U, psi, mf, dagger)


def mpc(act: Action, U, psi_e, mf: float, dagger: bool = False) -> np.ndarray:
    """D_PC = M_5 - M^4_eo M_5^-1 M^4_oe (paper eq. (dirac_equation)); input and
    output are even-parity full arrays. The adjoint is M_5^dag - (M^4_oe)^dag
    M_5^-dag (M^4_eo)^dag."""
    t = restrict_parity(m4(act, U, psi_e, mf, dagger), 1)
    t = m5inv(act, t, mf, dagger)
    t = restrict_parity(m4(act, U, t, mf, dagger), 0)
    return m5(act, psi_e, mf, dagger) - t


def mdagm(act: Action, U, psi_e, mf: float) -> np.ndarray:
    """A = D_PC^dag D_PC (paper eq. (normal_equation) and eq. (DdagD))."""
    return mpc(act, U, mpc(act, U, psi_e, mf, False), mf, True)


def mpc_sym(act: Action, U, psi_e, mf: float, dagger: bool = False) -> np.ndarray:
    """The symmetric Schur form D_sym = 1 - M_5^-1 M^4_eo M_5^-1 M^4_oe on even
    fields, the even-odd reduction with the diagonal block divided out (a
    variant of the paper's D_PC of eq. (dirac_equation); D_PC psi_e = phi_hat_e
    and D_sym psi_e = M_5^-1 phi_hat_e have the same solution). The adjoint is
    1 - (M^4_oe)^dag M_5^-dag (M^4_eo)^dag M_5^-dag."""
    if not dagger:
        t = restrict_parity(m4(act, U, psi_e, mf), 1)
        t = m5inv(act, t, mf)
        t = restrict_parity(m4(act, U, t, mf), 0)
        return psi_e - m5inv(act, t, mf)
    t = m5inv(act, psi_e, mf, True)
    t = restrict_parity(m4(act, U, t, mf, True), 1)
    t = m5inv(act, t, mf, True)
    t = restrict_parity(m4(act, U, t, mf, True), 0)
    return psi_e - t


def mdagm_sym(act: Action, U, psi_e, mf: float) -> np.ndarray:
    """A_sym = D_sym^dag D_sym, the normal operator of the symmetric form."""
    return mpc_sym(act, U, mpc_sym(act, U, psi_e, mf, False), mf, True)


def normal_op(schur: str):
    """The normal operator of a Schur form: "asym" (the paper's D_PC) or "sym"."""
    return {"asym": mdagm, "sym": mdagm_sym}[schur]


def source_prep(act: Action, U, phi_e, phi_o, mf: float) -> np.ndarray:
    """phi_hat_e = phi_e - M^4_eo M_5^-1 phi_o (paper eq. (dirac_equation))."""
    t = m5inv(act, phi_o, mf)
    return phi_e - restrict_parity(m4(act, U, t, mf), 0)


def normal_source(act: Action, U, phi_e, phi_o, mf: float, schur: str = "asym") -> np.ndarray:
    """Right-hand side of the normal equation of a Schur form for D psi = phi:
    D_PC^dag phi_hat_e, or D_sym^dag M_5^-1 phi_hat_e for the symmetric form."""
    ph = source_prep(act, U, phi_e, phi_o, mf)
    if schur == "asym":
        return mpc(act, U, ph, mf, True)
    return mpc_sym(act, U, m5inv(act, ph, mf), mf, True)


def odd_reconstruct(act: Action, U, psi_e, phi_o, mf: float) -> np.ndarray:
    """psi_o = M_5^-1 (phi_o - M^4_oe psi_e), the second row of the even-odd system."""
    return m5inv(act, phi_o - restrict_parity(m4(act, U, psi_e, mf), 1), mf)


def vdot(a: np.ndarray, b: np.ndarray) -> complex:
    """<a, b> = sum conj(a) b."""
    return np.vdot(a.reshape(-1), b.reshape(-1))


def norm2(a: np.ndarray) -> float:
    return float(np.vdot(a.reshape(-1), a.reshape(-1)).real)
