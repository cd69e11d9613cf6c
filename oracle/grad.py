"""Gradients of top-k singular values and PC scores with respect to per-SNP
and per-sample weights -- TEST INFRASTRUCTURE ONLY (dense, FP64, small sizes).

The paper (arXiv:1808.03374) has no differentiation; the formulas below are the
standard first-order perturbation theory of the SVD, written out here.

Weighted matrix A = diag(s) A0 diag(w), A0 the standardised genotype matrix.
For a simple singular value sigma_i with vectors (u_i, v_i):
    d sigma_i = u_i^T dA v_i.
PC scores S = A V_k (n x k).  With M = A^T A, the right vector moves by
    d v_i = (sigma_i^2 I - M)^+ dM v_i,   dM = dA^T A + A^T dA,
so for an adjoint S_bar with columns s_i, b_i = A^T s_i and
    x_i = sum_{l != i} v_l (v_l^T b_i) / (sigma_i^2 - sigma_l^2)
(the sum over every eigenvector of M, including its null space, eigenvalue 0):
    A_bar = sum_i [ sigma_bar_i u_i v_i^T + s_i v_i^T + sigma_i u_i x_i^T + (A x_i) v_i^T ].
Then dL/dw_j = sum_r A_bar_rj A_rj / w_j and dL/ds_r = sum_j A_bar_rj A_rj / s_r.

The sign of each (u_i, v_i) pair follows the library's rule (largest-magnitude
entry of v_i positive), which makes S a function of A away from ties.
"""
from __future__ import annotations

import numpy as np

import oracle


def weighted_dense(packed, n, s, w):
    M = oracle.Matrix.from_packed(packed, n)
    A0 = M.dense()
    return A0 * s[:, None] * w[None, :], A0


def svd_signed(A):
    U, sg, Vt = np.linalg.svd(A, full_matrices=True)
    r = min(A.shape)
    V = Vt.T
    for i in range(r):
        j = int(np.argmax(np.abs(V[:, i])))
        if V[j, i] < 0:
            V[:, i] = -V[:, i]
            U[:, i] = -U[:, i]
    return U, sg, V


def loss(A, k, c, r):
    """L = sum_i c_i sigma_i^2 + || S r ||^2 with S = A V_k (PC scores)."""
    U, sg, V = svd_signed(A)
    S = A @ V[:, :k]
    return float(np.sum(c * sg[:k] ** 2) + np.sum((S @ r) ** 2))


def loss_grad(A, A0, s, w, k, c, r):
    """(L, dL/ds, dL/dw) from the adjoint formula with the full SVD."""
    n, m = A.shape
    U, sg, V = svd_signed(A)
    rank = min(n, m)
    sig = sg[:k]
    S = A @ V[:, :k]
    L = float(np.sum(c * sig ** 2) + np.sum((S @ r) ** 2))
    sbar_sig = 2 * c * sig
    Sbar = 2 * np.outer(S @ r, r)  # n x k
    ev = np.zeros(m)
    ev[:rank] = sg[:rank] ** 2     # eigenvalues of A^T A (null space: 0)
    Abar = np.zeros_like(A)
    for i in range(k):
        si = Sbar[:, i]
        b = A.T @ si
        coef = V.T @ b
        den = ev[i] - ev
        den[i] = np.inf
        x = V @ (coef / den)
        Abar += np.outer(sbar_sig[i] * U[:, i] + si + A @ x, V[:, i]) + sig[i] * np.outer(U[:, i], x)
    gw = (Abar * A).sum(0) / w
    gs = (Abar * A).sum(1) / s
    return L, gs, gw


def sigma_grad_closed_form(A, s, w, k, c):
    """For L = sum_i c_i sigma_i^2 only: dL/dw_j = sum_i 2 c_i sigma_i^2 v_ij^2 / w_j,
    dL/ds_r = sum_i 2 c_i sigma_i^2 u_ri^2 / s_r."""
    U, sg, V = svd_signed(A)
    gw = (2 * c * sg[:k] ** 2 * V[:, :k] ** 2).sum(1) / w
    gs = (2 * c * sg[:k] ** 2 * U[:, :k] ** 2).sum(1) / s
    return gs, gw


def loss_grad_cg(M, k, c, r, ell, v0, tol_cg=1e-12, maxit=2000):
    """(L, dL/ds, dL/dw) without forming A: the oracle's own FP64 GKL triplets,
    the known part of x_i from the computed vectors, and the complement part
    y_i from conjugate gradients on P (sigma_i^2 I - A^T A) P y = P b_i
    (P = I - V_k V_k^T), every product through the oracle's A.v / A^T.u.
    M is an oracle.Matrix carrying the weights s and w."""
    res = oracle.gkl(M, k=k + 1, ell=ell, tol=1e-13, v0=v0, maxit=5000)
    assert res.converged
    sig, U, V = res.sigma[:k], res.U[:, :k], res.V[:, :k]
    S = U * sig
    L = float(np.sum(c * sig ** 2) + np.sum((S @ r) ** 2))
    sbar_sig = 2 * c * sig
    Sbar = 2 * np.outer(S @ r, r)
    n, m = M.n, M.m
    X = np.zeros((m, k))
    for i in range(k):
        if not np.any(Sbar[:, i]):
            continue
        b = M.rmatvec(Sbar[:, i])
        coef = V.T @ b
        den = sig[i] ** 2 - sig ** 2
        den[i] = np.inf
        x = V @ (coef / den)
        proj = lambda z: z - V @ (V.T @ z)
        rr_vec = proj(proj(b))
        y = np.zeros(m)
        p = rr_vec.copy()
        rr = rr_vec @ rr_vec
        r0 = np.sqrt(rr)
        for _ in range(maxit):
            if np.sqrt(rr) <= tol_cg * r0 or r0 == 0:
                break
            q = proj(proj(sig[i] ** 2 * p - M.rmatvec(M.matvec(p))))
            alpha = rr / (p @ q)
            y += alpha * p
            rr_vec -= alpha * q
            rn = rr_vec @ rr_vec
            p = rr_vec + (rn / rr) * p
            rr = rn
        X[:, i] = x + y
    gw = np.zeros(m)
    gs = np.zeros(n)
    wt = M.w if M.w is not None else np.ones(m)
    st = M.s if M.s is not None else np.ones(n)
    for i in range(k):
        pi = sbar_sig[i] * U[:, i]
        if np.any(Sbar[:, i]):
            pi = pi + Sbar[:, i] + M.matvec(X[:, i])
            gw += X[:, i] * M.rmatvec(sig[i] * U[:, i])
            gs += sig[i] * U[:, i] * M.matvec(X[:, i])
        gw += V[:, i] * M.rmatvec(pi)
        gs += pi * M.matvec(V[:, i])
    return L, gs / st, gw / wt, res


def finite_difference(A0, s, w, k, c, r, coords_w, coords_s, h=1e-6):
    """Central differences of the loss in chosen weight coordinates."""
    def L(s_, w_):
        return loss(A0 * s_[:, None] * w_[None, :], k, c, r)
    gw, gs = [], []
    for j in coords_w:
        wp, wm = w.copy(), w.copy()
        wp[j] += h
        wm[j] -= h
        gw.append((L(s, wp) - L(s, wm)) / (2 * h))
    for i in coords_s:
        sp, sm = s.copy(), s.copy()
        sp[i] += h
        sm[i] -= h
        gs.append((L(sp, w) - L(sm, w)) / (2 * h))
    return np.array(gs), np.array(gw)
