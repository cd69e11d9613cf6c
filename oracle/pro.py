"""Orthogonality estimates of partial reorthogonalisation (the omega
recurrence) for Golub-Kahan-Lanczos after a thick restart -- TEST
INFRASTRUCTURE ONLY (loaded by tests/; shares no code with the CUDA library).

Section 3 (choice of reorthogonalisation strategy) reorthogonalises only when
an estimate of the loss of orthogonality exceeds a threshold, as in the
partial reorthogonalisation of PROPACK that the paper compares against.  The
paper gives no formulas; the estimates here follow from the two GKL relations
alone, written for the upper-triangular projected matrix B that a thick
restart leaves (kept values on the diagonal, a spike column after them):

    A v_j = sum_{i<=j} B_ij u_i   (u_j enters with B_jj = alpha_j),
    A^T u_j = sum_{l<=j+1} B_jl v_l  (v_{j+1} enters with B_j,j+1 = beta_j).

With mu_jk ~ u_j^T u_k and nu_jk ~ v_j^T v_k, taking inner products of the
first relation with u_k (k < j) and of the second with v_k (k <= j) gives

    alpha_j mu_jk      = sum_{l<=j} B_kl nu_lj - sum_{i<j} B_ij mu_ik,
    beta_j  nu_{j+1,k} = sum_{i<=k} B_ik mu_ij - sum_{l<=j} B_jl nu_lk,

and each step adds rounding of about eps (alpha_j + beta) with the sign of
the sum, so that the estimates grow like the true loss does.  The sums here run
over the whole dense B, with no use of its sparsity: a reader can check them
against the relations above term by term.

cycle_after_restart() runs one cycle after a thick restart with NO
reorthogonalisation at all, so that the true inner products U^T U and V^T V
show the loss of orthogonality that the estimates have to track.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class ProTrace:
    mu_est: np.ndarray    # (l, l) estimates of u_j^T u_k, filled for the cycle's new j
    nu_est: np.ndarray    # (l+1, l+1) estimates of v_j^T v_k
    mu_true: np.ndarray   # the computed inner products U^T U
    nu_true: np.ndarray   # V^T V
    B: np.ndarray         # (l, l+1) projected matrix of the cycle (kept block, spike, new bidiagonal part)
    kk: int               # vectors kept by the restart
    ell: int


def mu_row(B, mu, nu, j, alpha):
    """mu_jk for k < j from the first relation (no rounding term):
    (sum_{l<=j} B_kl nu_lj - sum_{i<j} B_ij mu_ik) / alpha_j."""
    return np.array([B[k, :j + 1] @ nu[:j + 1, j] - B[:j, j] @ mu[:j, k] for k in range(j)]) / alpha


def nu_row(B, mu, nu, j, beta):
    """nu_{j+1,k} for k <= j from the second relation (no rounding term):
    (sum_{i<=k} B_ik mu_ij - sum_{l<=j} B_jl nu_lk) / beta_j."""
    return np.array([B[:k + 1, k] @ mu[:k + 1, j] - B[j, :j + 1] @ nu[:j + 1, k] for k in range(j + 1)]) / beta


def _orth(x, W):
    if W.shape[1]:
        x = x - W @ (W.T @ x)
        x = x - W @ (W.T @ x)
    return x


def cycle_after_restart(A: np.ndarray, k_keep: int, ell: int, v0, eps: float = 2.0 ** -53) -> ProTrace:
    """One fully reorthogonalised cycle of l steps, a thick restart keeping
    k_keep Ritz vectors and the last v (section 3), then the steps k_keep..l-1
    of the next cycle without reorthogonalisation, tracking the estimates."""
    n, m = A.shape
    U = np.zeros((n, ell))
    V = np.zeros((m, ell + 1))
    B = np.zeros((ell, ell + 1))
    V[:, 0] = v0 / np.linalg.norm(v0)
    # first cycle: full reorthogonalisation (the bases start orthonormal)
    for j in range(ell):
        w = _orth(A @ V[:, j], U[:, :j])
        B[j, j] = np.linalg.norm(w)
        U[:, j] = w / B[j, j]
        z = _orth(A.T @ U[:, j], V[:, :j + 1])
        B[j, j + 1] = np.linalg.norm(z)
        V[:, j + 1] = z / B[j, j + 1]
    # thick restart: U <- U P_kk, V <- [V_l Q_kk, v_l], B <- diag(s_kk) with the spike in column kk
    P, s, Qt = np.linalg.svd(B[:, :ell])
    beta = B[ell - 1, ell]
    kk = k_keep
    U[:, :kk] = U @ P[:, :kk]
    V[:, :kk], V[:, kk] = V[:, :ell] @ Qt.T[:, :kk], V[:, ell].copy()
    U[:, kk:] = 0.0
    V[:, kk + 1:] = 0.0
    B[:] = 0.0
    B[np.arange(kk), np.arange(kk)] = s[:kk]
    B[:kk, kk] = beta * P[ell - 1, :kk]
    # estimates start at eps between distinct kept vectors (orthonormal to rounding)
    mu = np.full((ell, ell), eps)
    nu = np.full((ell + 1, ell + 1), eps)
    np.fill_diagonal(mu, 1.0)
    np.fill_diagonal(nu, 1.0)
    # second cycle, steps kk..l-1, no reorthogonalisation
    for j in range(kk, ell):
        w = A @ V[:, j] - U[:, :j] @ B[:j, j]
        alpha = np.linalg.norm(w)
        U[:, j] = w / alpha
        B[j, j] = alpha
        bprev = B[j - 1, j] if j > kk else 0.0
        t = mu_row(B, mu, nu, j, alpha)
        mu[j, :j] = mu[:j, j] = t + np.copysign(eps * (alpha + bprev) / alpha, t)
        z = A.T @ U[:, j] - V[:, :j + 1] @ B[j, :j + 1]
        beta = np.linalg.norm(z)
        V[:, j + 1] = z / beta
        B[j, j + 1] = beta
        t = nu_row(B, mu, nu, j, beta)
        nu[j + 1, :j + 1] = nu[:j + 1, j + 1] = t + np.copysign(eps * (alpha + beta) / beta, t)
    return ProTrace(mu, nu, U.T @ U, V.T @ V, B, kk, ell)
