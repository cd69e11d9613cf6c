"""The paper's two thick-restart options, restated to compare their cost --
TEST INFRASTRUCTURE ONLY (loaded by tests/; shares no code with the CUDA
library).

Section 3 (thick restarting) offers restarts with ordinary Ritz values or
with harmonic Ritz values, and states that ordinary Ritz values suffice for
the top principal components.  Both restarts are written here over one
Golub-Kahan-Lanczos expansion with full reorthogonalisation (classical
Gram-Schmidt twice), so that they differ only in the small problem that
chooses the kept vectors.

After a cycle, U (n x l) and V (m x (l+1)) are orthonormal, with
    A V_l = U B,   A^T U = V B^ (exactly, up to rounding),
where B = U^T A V_l is l x l and B^ = [B, beta e_l] = U^T A V is l x (l+1).
The projected matrix U^T A V is assembled from the Gram-Schmidt coefficients
of the expansion: projecting A v_j on U gives column j (and the new vector's
norm its next entry), projecting A^T u_i on V gives row i -- no products
beyond the expansion's own.

* Ordinary Ritz: B = P S Q^T.  Kept: U P_k', V_l Q_k' and the last v; the
  triplet (U p_i, s_i, V_l q_i) has A V_l q_i = s_i U p_i and
  ||A^T U p_i - s_i V_l q_i|| = beta |P[l-1, i]|.
* Harmonic Ritz (of A^T A with respect to span(V_l), target 0): the harmonic
  Ritz values solve (A^T A V y)^T (A^T A V y - theta^2 V y) = 0; with
  A^T A V_l = V B^^T B this gives B^ B^^T (B y) = theta^2 (B y), so they are the
  singular values of B^ = P^ S^ Q^^T, with harmonic Ritz vectors
  V_l B^-1 p^_i.  Kept (the augmented restart, as in Baglama and Reichel's
  restarted bidiagonalisation methods): U p^_i and V q^_i, which
  satisfy A^T U p^_i = s^_i V q^_i exactly, and the next left vector u_l:
  A V q^_i = s^_i U p^_i + alpha_l Q^[last, i] u_l, so the residual is
  alpha_l |Q^[last, i]|; the expansion then continues from A^T u_l.  After
  such a restart the bases lead with a left vector, and the cycle's
  augmented matrix is U^T A V with as many columns as rows.

The operator is a dense array or any object with n, m, matvec and rmatvec
(the C oracle's packed Matrix), so that the comparison can run at sizes where
a dense copy does not fit; only the products of the expansion are counted (in
pairs: one A v and one A^T u).

`python -m oracle.restarts [workload:n:m ...]` prints both restarts' pair and
restart counts on scaled-down copies of the benchmark workloads (compare()).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class RestartResult:
    sigma: np.ndarray
    U: np.ndarray
    V: np.ndarray
    resid: np.ndarray
    pairs: float
    restarts: int
    converged: bool


def _project(x, W):
    """Classical Gram-Schmidt twice: x minus its projection on the orthonormal
    columns of W, and the projection's coefficients (the sum of both passes)."""
    c = np.zeros(W.shape[1])
    if W.shape[1]:
        for _ in range(2):
            d = W.T @ x
            x = x - W @ d
            c += d
    return x, c


def gkl_restarted(A, k: int, ell: int, tol: float, v0, variant: str = "ritz", k_keep: int = 0,
                  maxit: int = 500) -> RestartResult:
    """Top-k singular triplets of A (n x m: a dense array, or an operator with
    n, m, matvec and rmatvec) by GKL with full reorthogonalisation and thick
    restarts of the given variant ("ritz" or "harmonic"); converged when
    max_{i<k} r_i <= tol sigma_1."""
    if variant not in ("ritz", "harmonic"):
        raise ValueError(variant)
    if isinstance(A, np.ndarray):
        n, m = A.shape
        mv, rmv = (lambda x: A @ x), (lambda y: A.T @ y)
    else:
        n, m = A.n, A.m
        mv, rmv = A.matvec, A.rmatvec
    kk = k_keep or k + (ell - k) // 2
    U = np.zeros((n, ell + 1))
    V = np.zeros((m, ell + 2))
    Bh = np.zeros((ell + 2, ell + 2))  # U^T A V over the nu x nv columns in use
    v0 = np.asarray(v0, dtype=np.float64)
    V[:, 0] = v0 / np.linalg.norm(v0)
    nu, nv = 0, 1
    last_v = True  # the last vector added is a v: the next product is A v
    products = 0
    restarts = 0
    for _ in range(maxit):
        # expand until V has l + 1 columns (l after a harmonic restart, whose bases
        # lead with a left vector), the last one a v: both restarts then add the
        # same number of products per cycle, 2 (l - k')
        target = ell + 1 if variant == "ritz" or restarts == 0 else ell
        while not (nv >= target and last_v):
            if last_v:
                w, c = _project(mv(V[:, nv - 1]), U[:, :nu])
                alpha = np.linalg.norm(w)
                Bh[nu, :] = 0.0  # the new u is orthogonal to A v_i for every earlier v_i
                Bh[:nu, nv - 1] = c
                Bh[nu, nv - 1] = alpha
                U[:, nu] = w / alpha
                nu += 1
            else:
                z, d = _project(rmv(U[:, nu - 1]), V[:, :nv])
                beta = np.linalg.norm(z)
                Bh[:, nv] = 0.0  # the new v is orthogonal to A^T u_i for every earlier u_i
                Bh[nu - 1, :nv] = d
                Bh[nu - 1, nv] = beta
                V[:, nv] = z / beta
                nv += 1
            products += 1
            last_v = not last_v
        if variant == "ritz":
            beta = Bh[ell - 1, ell]
            P, s, Qt = np.linalg.svd(Bh[:ell, :ell])
            Q = Qt.T
            resid = np.abs(beta * P[ell - 1, :])
            if np.max(resid[:k]) <= tol * s[0]:
                return RestartResult(s[:k], U[:, :ell] @ P[:, :k], V[:, :ell] @ Q[:, :k], resid[:k], products / 2,
                                     restarts, True)
            spike = P[:, :kk].T @ Bh[:ell, ell]
            U[:, :kk] = U[:, :ell] @ P[:, :kk]
            V[:, :kk], V[:, kk] = V[:, :ell] @ Q[:, :kk], V[:, ell]
            Bh[:] = 0.0
            Bh[:kk, :kk] = np.diag(s[:kk])
            Bh[:kk, kk] = spike
            nu, nv, last_v = kk, kk + 1, True
        else:
            # the next left vector u_l (one more product), then the augmented problem
            w, c = _project(mv(V[:, nv - 1]), U[:, :nu])
            alpha = np.linalg.norm(w)
            u_next = w / alpha
            products += 1
            Bh[:nu, nv - 1] = c
            # l x (l + 1) in the first cycle, l x l after
            P, s, Qt = np.linalg.svd(Bh[:nu, :nv], full_matrices=False)
            Q = Qt.T
            resid = np.abs(alpha * Q[-1, :])
            if np.max(resid[:k]) <= tol * s[0]:
                return RestartResult(s[:k], U[:, :nu] @ P[:, :k], V[:, :nv] @ Q[:, :k], resid[:k], products / 2,
                                     restarts, True)
            U[:, :kk], U[:, kk] = U[:, :nu] @ P[:, :kk], u_next
            V[:, :kk] = V[:, :nv] @ Q[:, :kk]
            Bh[:] = 0.0
            Bh[:kk, :kk] = np.diag(s[:kk])
            Bh[kk, :kk] = alpha * Q[-1, :kk]
            nu, nv, last_v = kk + 1, kk, False
        restarts += 1
    return RestartResult(s[:k], U[:, :k], V[:, :k], resid[:k], products / 2, restarts, False)


DENSE_LIMIT = 2 * 10**8  # entries: above this the products are the C oracle's packed ones


def compare(cases=None, k: int = 20, ell: int = 50, tol: float = 1e-6):
    """Pairs and restarts of both restarts on scaled-down copies of the
    benchmark's workloads (the same population structure, allele-frequency law
    and missingness at a smaller n x m); yields one row per case and variant.
    Small cases run on a dense copy with LAPACK's singular values beside them;
    larger ones run matrix-free on the packed matrix, and the two variants'
    values are compared with each other."""
    from dataclasses import replace

    import synth
    from oracle import Matrix

    cases = cases or [("large_200k_x_1m", 2000, 20_000), ("large_200k_x_1m", 4000, 40_000),
                      ("fp32_pro_10k_x_100k", 2000, 20_000), ("block_50k_x_500k", 3000, 30_000)]
    for name, n, m in cases:
        spec = replace(synth.CONFIGS[name].geno, n=n, m=m)
        M = Matrix.from_packed(synth.genotypes(spec).packed, n)
        v0 = synth.normal_vec(4, 0, m)
        if n * m <= DENSE_LIMIT:
            op = M.dense()
            sv = np.linalg.svd(op, compute_uv=False)
        else:
            op, sv = M, None
        results = {}
        for variant in ("ritz", "harmonic"):
            r = gkl_restarted(op, k=k, ell=ell, tol=tol, v0=v0, variant=variant, maxit=2000)
            results[variant] = r
            row = dict(workload=name, n=n, m=m, variant=variant, converged=r.converged, pairs=r.pairs,
                       restarts=r.restarts)
            if sv is not None:
                row["sigma_rel_err"] = float(np.max(np.abs(r.sigma - sv[:k]) / sv[:k]))
                row["gap_k"] = float((sv[k - 1] - sv[k]) / sv[0])
            else:
                ref = results["ritz"].sigma
                row["sigma_rel_diff_vs_ritz"] = float(np.max(np.abs(r.sigma - ref) / ref))
                row["min_gap_top_k"] = float(np.min(-np.diff(r.sigma)) / r.sigma[0])
            yield row


if __name__ == "__main__":
    import sys

    # optional cases as workload:n:m arguments, e.g. large_200k_x_1m:20000:200000
    args = [a.split(":") for a in sys.argv[1:]]
    for row in compare([(a[0], int(a[1]), int(a[2])) for a in args] or None):
        print(" ".join(f"{k}={v:.3g}" if isinstance(v, float) else f"{k}={v}" for k, v in row.items()), flush=True)
