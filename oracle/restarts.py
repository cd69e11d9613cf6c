"""The paper's two thick-restart options, restated to compare their cost --
TEST INFRASTRUCTURE ONLY (loaded by tests/; shares no code with the CUDA
library).

Section 3 (thick restarting) offers restarts with ordinary Ritz values or
with harmonic Ritz values, and states that ordinary Ritz values suffice for
the top principal components.  Both restarts are written here over one
explicit, fully reorthogonalised Golub-Kahan-Lanczos expansion, so that they
differ only in the small problem that chooses the kept vectors.

After a cycle, U (n x l) and V (m x (l+1)) are orthonormal, with
    A V_l = U B,   A^T U = V B^ (exactly, up to rounding),
where B = U^T A V_l is l x l and B^ = [B, beta e_l] = U^T A V is l x (l+1).

* Ordinary Ritz: B = P S Q^T.  Kept: U P_k', V_l Q_k' and the last v; the
  triplet (U p_i, s_i, V_l q_i) has A V_l q_i = s_i U p_i and
  ||A^T U p_i - s_i V_l q_i|| = beta |P[l-1, i]|.
* Harmonic Ritz (of A^T A with respect to span(V_l), target 0): the harmonic
  Ritz values solve (A^T A V y)^T (A^T A V y - theta^2 V y) = 0; with
  A^T A V_l = V B^^T B this gives B^ B^^T (B y) = theta^2 (B y), so they are the
  singular values of B^ = P^ S^ Q^^T, with harmonic Ritz vectors
  V_l B^-1 p^_i.  Kept (the augmented restart): U p^_i and V q^_i, which
  satisfy A^T U p^_i = s^_i V q^_i exactly, and the next left vector u_l:
  A V q^_i = s^_i U p^_i + alpha_l Q^[last, i] u_l, so the residual is
  alpha_l |Q^[last, i]|; the expansion then continues from A^T u_l.  After
  such a restart the bases lead with a left vector, and the cycle's
  augmented matrix is U^T A V with as many columns as rows.

The products are dense numpy products of the oracle's operator (small sizes
only), and the projected matrices are formed as U^T A V from the bases, so
that both restarts rest on the same arithmetic; only the products of the
expansion are counted (in pairs: one A v and one A^T u).

`python -m oracle.restarts` prints both restarts' pair and restart counts on
scaled-down copies of the benchmark workloads (compare()).
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


def _orth(x, W):
    """x minus its projection on the orthonormal columns of W, twice (CGS2)."""
    if W.shape[1]:
        x = x - W @ (W.T @ x)
        x = x - W @ (W.T @ x)
    return x


def gkl_restarted(A: np.ndarray, k: int, ell: int, tol: float, v0, variant: str = "ritz", k_keep: int = 0,
                  maxit: int = 500) -> RestartResult:
    """Top-k singular triplets of the dense matrix A (n x m) by GKL with full
    reorthogonalisation and thick restarts of the given variant ("ritz" or
    "harmonic"); converged when max_{i<k} r_i <= tol sigma_1."""
    if variant not in ("ritz", "harmonic"):
        raise ValueError(variant)
    n, m = A.shape
    kk = k_keep or k + (ell - k) // 2
    V = (np.asarray(v0, dtype=np.float64) / np.linalg.norm(v0))[:, None]
    U = np.zeros((n, 0))
    last_v = True  # the last vector added is a v: the next product is A v
    products = 0
    restarts = 0
    for _ in range(maxit):
        # expand until V has l + 1 columns (l after a harmonic restart, whose bases
        # lead with a left vector), the last one a v: both restarts then add the
        # same number of products per cycle, 2 (l - k')
        target = ell + 1 if variant == "ritz" or restarts == 0 else ell
        while not (V.shape[1] >= target and last_v):
            if last_v:
                w = _orth(A @ V[:, -1], U)
                U = np.column_stack([U, w / np.linalg.norm(w)])
            else:
                z = _orth(A.T @ U[:, -1], V)
                V = np.column_stack([V, z / np.linalg.norm(z)])
            products += 1
            last_v = not last_v
        if variant == "ritz":
            Bh = U.T @ (A @ V)  # l x (l + 1): [B, beta e_l]
            beta = float(Bh[ell - 1, ell])
            P, s, Qt = np.linalg.svd(Bh[:, :ell])
            Q = Qt.T
            resid = np.abs(beta * P[ell - 1, :])
            if np.max(resid[:k]) <= tol * s[0]:
                return RestartResult(s[:k], U @ P[:, :k], V[:, :ell] @ Q[:, :k], resid[:k], products / 2,
                                     restarts, True)
            U = U @ P[:, :kk]
            V = np.column_stack([V[:, :ell] @ Q[:, :kk], V[:, ell]])
            last_v = True
        else:
            # the next left vector u_l (one more product), then the augmented problem
            w = _orth(A @ V[:, -1], U)
            alpha = np.linalg.norm(w)
            u_next = w / alpha
            products += 1
            Bh = U.T @ (A @ V)  # l x (l + 1) in the first cycle, l x l after
            P, s, Qt = np.linalg.svd(Bh, full_matrices=False)
            Q = Qt.T
            resid = np.abs(alpha * Q[-1, :])
            if np.max(resid[:k]) <= tol * s[0]:
                return RestartResult(s[:k], U @ P[:, :k], V @ Q[:, :k], resid[:k], products / 2, restarts, True)
            U = np.column_stack([U @ P[:, :kk], u_next])
            V = V @ Q[:, :kk]
            last_v = False
        restarts += 1
    return RestartResult(s[:k], U[:, :k], V[:, :k], resid[:k], products / 2, restarts, False)


def compare(cases=None, k: int = 20, ell: int = 50, tol: float = 1e-6):
    """Pairs and restarts of both restarts on scaled-down copies of the
    benchmark's workloads (the same population structure, allele-frequency law
    and missingness at n x m small enough for dense products); yields one row
    per case and variant."""
    from dataclasses import replace

    import synth
    from oracle import Matrix

    cases = cases or [("large_200k_x_1m", 2000, 20_000), ("large_200k_x_1m", 4000, 40_000),
                      ("fp32_pro_10k_x_100k", 2000, 20_000), ("block_50k_x_500k", 3000, 30_000)]
    for name, n, m in cases:
        spec = replace(synth.CONFIGS[name].geno, n=n, m=m)
        A = Matrix.from_packed(synth.genotypes(spec).packed, n).dense()
        v0 = synth.normal_vec(4, 0, m)
        sv = np.linalg.svd(A, compute_uv=False)
        for variant in ("ritz", "harmonic"):
            r = gkl_restarted(A, k=k, ell=ell, tol=tol, v0=v0, variant=variant, maxit=2000)
            yield dict(workload=name, n=n, m=m, variant=variant, converged=r.converged, pairs=r.pairs,
                       restarts=r.restarts, sigma_rel_err=float(np.max(np.abs(r.sigma - sv[:k]) / sv[:k])),
                       gap_k=float((sv[k - 1] - sv[k]) / sv[0]))


if __name__ == "__main__":
    for row in compare():
        print(" ".join(f"{k}={v:.3g}" if isinstance(v, float) else f"{k}={v}" for k, v in row.items()), flush=True)
