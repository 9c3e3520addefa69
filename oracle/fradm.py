"""Plain FP64 CPU oracle for FR-ADM / FixedRankOptStep / FR-Nys.

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously-correct
reference that the CUDA path is checked against.  Only the test suite, the
package smoke check and the benchmark's CPU-baseline leg may import it; the
product path never calls it and shares no code with it.

Everything here is float64 numpy, written in the order and notation of the
paper (Ros et al., "Fast and Robust Fixed-Rank Matrix Recovery"):

  * Sym, P_ST, P_O, P_SPD ............ Sec. 2 (notation) and Sec. 4.1, Eq. (9)/(10)
  * fixed_rank_opt_step .............. Algorithm 3 (FixedRankOptStep)
  * fixed_rank_opt_full .............. Algorithm 4 (FixedRankOptFull, Appendix)
  * fr_adm ........................... Algorithm 1 (FR-ADM), Eq. (4)
  * fr_nys ........................... Algorithm 2 (FR-Nys)

Library primitives used as single steps: matrix products, numpy.linalg.eigh
(for (A^T A)^{-1/2}) and numpy.linalg.svd (for the thin-SVD form of P_O and
for the pseudo-inverse in FR-Nys).  No blocking, fusion or algebraic
reordering: every m x n intermediate of the algorithms is formed densely.

Readings of points the paper leaves open (all shared with the CUDA path only
through the arguments, never through code):
  * rho: the paper only requires rho > 1; it is an argument here.
  * "while not converged": stop when ||M - L - S||_F / ||M||_F <= tol, or
    after max_iter iterations.
  * V_0 = I_{n x r} (the printed "I_{r x n}" is the transpose); U_0 is never
    read by Algorithm 3, B_0 = I_r.
  * The S- and Y-steps use mu_k (the value before the continuation update).
  * P_O requires rank(A) = r; a Gram matrix whose smallest eigenvalue is not
    positive raises RankDeficient instead of returning garbage.
  * FR-Nys pseudo-inverse: dense SVD pseudo-inverse of the l x l block,
    truncated to its r largest singular values (rank(L_L) = r).
"""
from __future__ import annotations

import dataclasses

import numpy as np


class RankDeficient(ArithmeticError):
    """P_O was given an m x r matrix whose rank is below r (Eq. 9 assumes full rank)."""


# --------------------------------------------------------------------------
# Operators of Sec. 2 / Sec. 4.1
# --------------------------------------------------------------------------

def sym(A: np.ndarray) -> np.ndarray:
    """Sym(A) = (A + A^T) / 2, the symmetric part (Sec. 2)."""
    A = np.asarray(A, dtype=np.float64)
    return 0.5 * (A + A.T)


def soft_threshold(X: np.ndarray, delta: float) -> np.ndarray:
    """P_ST[X] = max(0, X - delta) + min(0, X + delta), entrywise (Sec. 2)."""
    X = np.asarray(X, dtype=np.float64)
    return np.maximum(0.0, X - delta) + np.minimum(0.0, X + delta)


def inv_sqrt_spd(G: np.ndarray) -> np.ndarray:
    """G^{-1/2} of a symmetric positive definite r x r matrix via eigh."""
    w, E = np.linalg.eigh(sym(G))
    if not (w[0] > 0.0) or w[0] <= 1e-14 * w[-1]:
        raise RankDeficient(f"Gram matrix not positive definite: eigenvalues {w[0]:.3e} .. {w[-1]:.3e}")
    return (E * (1.0 / np.sqrt(w))) @ E.T


def stiefel_projector(A: np.ndarray) -> np.ndarray:
    """P_O[A] = A (A^T A)^{-1/2} for full-rank A (Sec. 4.1.1, Eq. 9)."""
    A = np.asarray(A, dtype=np.float64)
    return A @ inv_sqrt_spd(A.T @ A)


def stiefel_projector_svd(A: np.ndarray) -> np.ndarray:
    """P_O[A] = Q S^T from the thin SVD A = Q Sigma S^T (Sec. 4.1.1, first form of Eq. 9)."""
    Q, _, St = np.linalg.svd(np.asarray(A, dtype=np.float64), full_matrices=False)
    return Q @ St


def spd_projector(A: np.ndarray) -> np.ndarray:
    """P_SPD[A] = Sym(A) (Sec. 4.1.2, Eq. 10); valid because U, V are orthonormal."""
    return sym(A)


# --------------------------------------------------------------------------
# Algorithm 3 / Algorithm 4
# --------------------------------------------------------------------------

def fixed_rank_opt_step(X, U0, B0, V0):
    """One ADM step on St x SPD x St (Algorithm 3, FixedRankOptStep).

    U_bar = P_O[X V0 B0];  V_bar = P_O[X^T U_bar B0];  B_bar = Sym(U_bar^T X V_bar).
    U0 is accepted for symmetry with the paper's signature but not read.
    """
    del U0
    X = np.asarray(X, dtype=np.float64)
    U_bar = stiefel_projector(X @ V0 @ B0)
    V_bar = stiefel_projector(X.T @ U_bar @ B0)
    B_bar = spd_projector(U_bar.T @ X @ V_bar)
    return U_bar, B_bar, V_bar


def fixed_rank_opt_full(M, U0, B0, V0, n_iter: int):
    """Algorithm 4 (FixedRankOptFull): iterate Algorithm 3 on a fixed M.

    Returns the list of (U_i, B_i, V_i) for i = 1..n_iter so that tests can
    inspect every iterate (convergence to the TSVD, Theorem 2).
    """
    out = []
    U, B, V = U0, B0, V0
    for _ in range(n_iter):
        U, B, V = fixed_rank_opt_step(M, U, B, V)
        out.append((U, B, V))
    return out


# --------------------------------------------------------------------------
# Algorithm 1: FR-ADM
# --------------------------------------------------------------------------

@dataclasses.dataclass
class FRADMResult:
    U: np.ndarray            # m x r, Stiefel
    B: np.ndarray            # r x r, symmetric
    V: np.ndarray            # n x r, Stiefel
    L: np.ndarray            # m x n, L = U B V^T
    S: np.ndarray            # m x n
    Y: np.ndarray            # m x n, final multiplier
    Y_prev: np.ndarray       # m x n, multiplier entering the last iteration
    mu: float                # mu after the last continuation update
    mu_last: float           # mu used by the last S/Y step
    iters: int
    residuals: list          # ||M - L - S||_F / ||M||_F after each iteration
    converged: bool


def fr_adm(M, r: int, *, rho: float = 1.5, mu0: float = 1.0, mu_max: float = 1e9,
           tol: float = 1e-9, max_iter: int = 500, fixed_iters: int | None = None) -> FRADMResult:
    """Algorithm 1 (FR-ADM) in float64, with every m x n matrix dense.

    Per iteration k (Algorithm 1, Eq. 4):
        L_{k+1} = FixedRankOptStep(M - S_k + Y_k / mu_k, U_k, B_k, V_k)
        S_{k+1} = P_ST_{1/mu_k}(M - L_{k+1} + Y_k / mu_k)
        Y_{k+1} = Y_k + mu_k (M - L_{k+1} - S_{k+1})
        mu_{k+1} = min(mu_bar, rho mu_k)
    Initial values: S = L = Y = 0, mu = mu0 (= 1 in the paper), B_0 = I_r,
    V_0 = I_{n x r}.  With fixed_iters set, exactly that many iterations run
    and the tolerance is ignored.
    """
    M = np.asarray(M, dtype=np.float64)
    m, n = M.shape
    if not (1 <= r <= min(m, n)):
        raise ValueError("need 1 <= r <= min(m, n)")
    if rho <= 1.0:
        raise ValueError("rho must exceed 1")
    S = np.zeros((m, n))
    Y = np.zeros((m, n))
    mu = float(mu0)
    U = np.eye(m, r)
    B = np.eye(r)
    V = np.eye(n, r)
    normM = np.linalg.norm(M)
    residuals = []
    converged = False
    Y_prev = Y
    mu_last = mu
    k = 0
    n_max = fixed_iters if fixed_iters is not None else max_iter
    while k < n_max:
        X = M - S + Y / mu
        U, B, V = fixed_rank_opt_step(X, U, B, V)
        L = U @ B @ V.T
        S = soft_threshold(M - L + Y / mu, 1.0 / mu)
        Y_prev = Y
        Y = Y + mu * (M - L - S)
        mu_last = mu
        mu = min(mu_max, rho * mu)
        k += 1
        res = np.linalg.norm(M - L - S) / normM
        residuals.append(res)
        if fixed_iters is None and res <= tol:
            converged = True
            break
    L = U @ B @ V.T
    return FRADMResult(U=U, B=B, V=V, L=L, S=S, Y=Y, Y_prev=Y_prev, mu=mu, mu_last=mu_last,
                       iters=k, residuals=residuals, converged=converged)


# --------------------------------------------------------------------------
# Algorithm 2: FR-Nys
# --------------------------------------------------------------------------

@dataclasses.dataclass
class FRNysResult:
    L: np.ndarray            # m x n, in the row order of the input M (sampled: L at the samples)
    S: np.ndarray            # m x n, in the row order of the input M (sampled: S at the samples)
    left: FRADMResult        # FR-ADM on the m x l column block of the shuffled M
    top: FRADMResult         # FR-ADM on the l x n row block of the shuffled M
    perm: np.ndarray         # row permutation: shuffled row i is input row perm[i]


def truncated_pinv(A: np.ndarray, r: int) -> np.ndarray:
    """Pseudo-inverse of A keeping its r largest singular values (dense SVD)."""
    Q, s, Wt = np.linalg.svd(np.asarray(A, dtype=np.float64), full_matrices=False)
    return (Wt[:r].T / s[:r]) @ Q[:, :r].T


def fr_nys(M, r: int, l: int, perm, *, sample=None, **adm_kwargs) -> FRNysResult:
    """Algorithm 2 (FR-Nys).

    M_tilde = rows of M shuffled by `perm` (M_tilde[i] = M[perm[i]]);
    (L_L, S_L) = FR-ADM(M_tilde[:, :l], r); (L_T, S_T) = FR-ADM(M_tilde[:l, :], r);
    L = L_L (L_L[:l, :l])^+ L_T;  S = M_tilde - L.  Both are returned in the
    row order of the input M (the shuffle is undone at the end).

    sample = (ii, jj): instead of the dense m x n L and S, return their entries at the input-order
    positions (ii[k], jj[k]) only, each from the same formula (row inv[ii[k]] of L_L (L_L[:l, :l])^+
    times column jj[k] of L_T, inv the inverse shuffle), so that large inputs need no m x n
    intermediate beyond M itself.
    """
    M = np.asarray(M)
    m, n = M.shape
    perm = np.asarray(perm, dtype=np.int64)
    if not np.array_equal(np.sort(perm), np.arange(m)):
        raise ValueError("perm must be a permutation of range(m)")
    if not (r <= l <= min(m, n)):
        raise ValueError("need r <= l <= min(m, n)")
    # the two blocks of M_tilde: M_tilde[:, :l] = M[perm, :l] and M_tilde[:l, :] = M[perm[:l], :]
    left = fr_adm(np.asarray(M[perm, :l], dtype=np.float64), r, **adm_kwargs)
    top = fr_adm(np.asarray(M[perm[:l], :], dtype=np.float64), r, **adm_kwargs)
    L_L, L_T = left.L, top.L
    P = L_L @ truncated_pinv(L_L[:l, :l], r)          # m x l: L_L (L_L[:l, :l])^+
    if sample is not None:
        ii, jj = (np.asarray(x, dtype=np.int64) for x in sample)
        inv = np.empty(m, dtype=np.int64)
        inv[perm] = np.arange(m)
        Ls = np.einsum("kl,lk->k", P[inv[ii]], L_T[:, jj])
        Ss = np.asarray(M[ii, jj], dtype=np.float64) - Ls
        return FRNysResult(L=Ls, S=Ss, left=left, top=top, perm=perm)
    Mt = np.asarray(M, dtype=np.float64)[perm]
    Lt = P @ L_T
    St = Mt - Lt
    L = np.empty_like(Lt)
    S = np.empty_like(St)
    L[perm] = Lt
    S[perm] = St
    return FRNysResult(L=L, S=S, left=left, top=top, perm=perm)
