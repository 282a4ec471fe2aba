"""Low modes of A = D_PC^dag D_PC and deflated MSPCG, in plain numpy (FP64).

Test infrastructure only (see oracle/__init__.py).

Paper reference: Sec. 1. For the measurement phase, where many right-hand
sides are solved with one Dirac matrix, eigen-space methods (EigCG; the
implicitly restarted Lanczos algorithm with a Chebyshev polynomial) compute
low-lying eigenvectors once, which lowers the effective condition number of
every later solve. The paper names these methods but gives no algorithm, and
does not combine them with MSPCG. Readings used here (listed in the design
notes as well):

* The low modes come from Chebyshev-filtered subspace iteration with a
  Rayleigh-Ritz step: the subspace V (m vectors) is replaced by
  W = T_d(L(A)) V, where T_d is the Chebyshev polynomial of degree d and L
  maps the unwanted interval [a, b] onto [-1, 1] (a = the largest Ritz value
  of the current subspace, b >= the largest eigenvalue of A); then the Ritz
  pairs of A on span(W) replace V. T_d stays bounded by 1 on [a, b] and grows
  below a, so the low end of the spectrum is amplified.
* The modes enter MSPCG twice. The start x_0 = V Lambda^-1 V^dag b (Galerkin:
  V^dag (b - A x_0) = 0 for exact eigenpairs) and an additive coarse
  correction of the preconditioner, z = M_ms^-1 r + V Lambda^-1 V^dag r (for
  exact eigenpairs V Lambda^-1 V^dag = A^-1 P_V with P_V the projector onto
  span(V)). With positive Ritz values the correction is Hermitian positive
  semi-definite, so the preconditioner stays positive definite for any V, and
  Algorithm 1 applies unchanged.

Fields are the oracle's full-lattice even half fields (see dwf_operator).
"""
from __future__ import annotations

import numpy as np

from . import dwf_operator as op
from . import solvers as sv


def chebyshev_filter(apply_A, Y, degree: int, a: float, b: float):
    """T_degree(L(A)) y for every y in Y, L(t) = (2 t - (a + b)) / (b - a).

    Three-term recurrence T_0 = 1, T_1(x) = x, T_{j+1}(x) = 2 x T_j(x) -
    T_{j-1}(x), with x = L(A) applied as (A y - c y) / e, c = (a + b) / 2,
    e = (b - a) / 2.
    """
    if degree < 1:
        raise ValueError("degree must be at least 1")
    c = 0.5 * (a + b)
    e = 0.5 * (b - a)
    out = []
    for y in Y:
        t_prev = y
        t_cur = (apply_A(y) - c * y) / e
        for _ in range(2, degree + 1):
            t_next = 2.0 * (apply_A(t_cur) - c * t_cur) / e - t_prev
            t_prev, t_cur = t_cur, t_next
        out.append(t_cur)
    return out


def rayleigh_ritz(apply_A, W):
    """Ritz pairs of A on span(W): an orthonormal basis Q of span(W) (numpy QR),
    H = Q^dag A Q, H = S diag(theta) S^dag (numpy eigh, ascending), V = Q S.
    Returns (theta, V as a list of fields shaped like W[0])."""
    shape = W[0].shape
    Wm = np.stack([w.reshape(-1) for w in W], axis=1)
    Q, _ = np.linalg.qr(Wm)
    AQ = np.stack([apply_A(Q[:, j].reshape(shape)).reshape(-1) for j in range(Q.shape[1])], axis=1)
    H = Q.conj().T @ AQ
    H = 0.5 * (H + H.conj().T)
    theta, S = np.linalg.eigh(H)
    V = Q @ S
    return theta, [V[:, j].reshape(shape) for j in range(V.shape[1])]


def ritz_residuals(apply_A, theta, V):
    """|A v_j - theta_j v_j| for every Ritz pair."""
    return np.array([np.sqrt(op.norm2(apply_A(v) - t * v)) for t, v in zip(theta, V)])


def lambda_max_estimate(apply_A, v0, steps: int = 30, margin: float = 1.1) -> float:
    """Upper estimate of A's largest eigenvalue: `steps` power iterations from
    v0, the last Rayleigh quotient times `margin`."""
    v = v0 / np.sqrt(op.norm2(v0))
    q = 0.0
    for _ in range(steps):
        w = apply_A(v)
        q = op.vdot(v, w).real
        v = w / np.sqrt(op.norm2(w))
    return margin * q


def lowmodes(apply_A, V0, n_ev: int, degree: int, passes: int, lam_max: float,
             tol: float = 0.0):
    """Chebyshev-filtered subspace iteration from the start vectors V0 (m >= n_ev).

    A Rayleigh-Ritz step on V0 first; then every pass filters the current Ritz
    vectors with T_degree on [a, lam_max], a = the largest current Ritz value
    (at most lam_max / 2), and takes the Ritz pairs of the filtered subspace.
    Stops after `passes` passes, or earlier once the n_ev lowest Ritz pairs
    have |A v - theta v| <= tol * lam_max (tol > 0).
    Returns (theta, V, residuals, passes done), all m pairs in ascending order.
    """
    theta, V = rayleigh_ritz(apply_A, V0)
    done = 0
    res = ritz_residuals(apply_A, theta, V)
    for _ in range(passes):
        if tol > 0 and res[:n_ev].max() <= tol * lam_max:
            break
        a = min(float(theta[-1]), 0.5 * lam_max)
        W = chebyshev_filter(apply_A, V, degree, a, lam_max)
        theta, V = rayleigh_ritz(apply_A, W)
        res = ritz_residuals(apply_A, theta, V)
        done += 1
    return theta, V, res, done


def coarse_correction(V, lam, r):
    """V Lambda^-1 V^dag r = sum_j v_j <v_j, r> / lambda_j."""
    z = np.zeros_like(r)
    for v, l in zip(V, lam):
        z = z + v * (op.vdot(v, r) / l)
    return z


def deflated_mspcg(act: op.Action, U, b, mf: float, block, k: int, tol: float, V, lam,
                   maxiter: int = 100000, snake: bool = True, inner_tol: float = 0.0,
                   schur: str = "asym"):
    """Algorithm 1 from x_0 = V Lambda^-1 V^dag b with the preconditioner
    z = M_ms^-1 r + V Lambda^-1 V^dag r (M_ms the multisplitting preconditioner
    of Sec. 2.4; plain CG's z = r when k = 0)."""
    A = lambda v: op.normal_op(schur)(act, U, v, mf)
    if k > 0:
        ms = lambda v: sv.ms_precondition(act, U, v, mf, block, k, snake, inner_tol=inner_tol,
                                          schur=schur)
    else:
        ms = lambda v: v
    Minv = lambda v: ms(v) + coarse_correction(V, lam, v)
    x0 = coarse_correction(V, lam, b)
    return sv.pcg(A, Minv, b, tol, maxiter, x0=x0)
