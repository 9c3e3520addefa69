"""The rewrites the GPU path is built on, checked in float64 against the definitions they replace.

The kernels never form S_k, X_k or the thin products the way Algorithms 1 and 3 write them: the
fused sweep keeps only the multiplier Y and the difference Delta = X_{k+1} - L_{k+1}; the W pass
reads Delta (tensor-core path: Delta^T P); the projector is r x r work and a row transform; B
comes from r x r products; FR-Nys keeps an r x r core.  Each test below builds the quantity both
ways on random data (the definitions through the oracle's own step functions) and requires
agreement to rounding, so a wrong sign, a dropped term or a swapped mu in a rewrite fails here
before any kernel runs.
"""
import numpy as np

from oracle import fradm as O

RNG = np.random.default_rng(2024)
m, n, r = 120, 90, 8


def _stiefel(rows, cols):
    Q, _ = np.linalg.qr(RNG.standard_normal((rows, cols)))
    return Q


def _state():
    U = _stiefel(m, r)
    V = _stiefel(n, r)
    A = RNG.standard_normal((r, r))
    B = A @ A.T + r * np.eye(r)                       # SPD
    M = U @ B @ V.T + np.where(RNG.random((m, n)) < 0.05, RNG.uniform(-5, 5, (m, n)), 0.0)
    Y = np.clip(RNG.standard_normal((m, n)), -1.0, 1.0)
    return U, B, V, M, Y


def _close(a, b, tol=1e-11):
    a, b = np.asarray(a), np.asarray(b)
    assert np.linalg.norm(a - b) <= tol * max(1.0, np.linalg.norm(b)), np.linalg.norm(a - b)


def test_multiplier_step_is_a_clip_and_the_residual_a_difference_of_multipliers():
    # Algorithm 1: S_{k+1} = P_ST(M - L + Y_k / mu, 1 / mu), Y_{k+1} = Y_k + mu (M - L - S_{k+1})
    U, B, V, M, Y = _state()
    L = U @ B @ V.T
    mu = 0.7
    z = M - L + Y / mu
    S1 = O.soft_threshold(z, 1.0 / mu)
    Y1 = Y + mu * (M - L - S1)
    _close(Y1, np.clip(mu * z, -1.0, 1.0))            # what the sweep stores
    _close(M - L - S1, (Y1 - Y) / mu)                 # what the residual sums
    _close(S1, O.soft_threshold(z, 1.0 / mu))         # the output pass rebuilds S from z


def test_next_fixed_rank_input_is_L_plus_delta():
    # X_{k+1} = M - S_{k+1} + Y_{k+1} / mu_{k+1} = L_{k+1} + Delta,
    # Delta = Y_{k+1} (1 / mu_k + 1 / mu_{k+1}) - Y_k / mu_k
    U, B, V, M, Y = _state()
    L = U @ B @ V.T
    mu, mu_next = 0.7, 0.7 * 1.5
    z = M - L + Y / mu
    S1 = O.soft_threshold(z, 1.0 / mu)
    Y1 = Y + mu * (M - L - S1)
    X1 = M - S1 + Y1 / mu_next
    Delta = Y1 * (1.0 / mu + 1.0 / mu_next) - Y / mu
    _close(X1, L + Delta)


def test_thin_products_from_delta():
    # P = X V_bar = U_bar B_bar + Delta V_bar (V_bar^T V_bar = I);
    # W = X^T U_new = C (U^T U_new) + Delta^T U_new = (Delta^T P) T_U + C H, C = V B, H = U^T U_new
    U, B, V, M, Y = _state()
    L = U @ B @ V.T
    Delta = RNG.standard_normal((m, n))
    X = L + Delta
    P = X @ V
    _close(P, U @ B + Delta @ V)
    G = P.T @ P
    T_U = B @ O.inv_sqrt_spd(B @ G @ B)
    U_new = P @ T_U
    C = V @ B
    H = U.T @ U_new
    W = X.T @ U_new
    _close(W, C @ H + Delta.T @ U_new)
    _close(W, (Delta.T @ P) @ T_U + C @ H)


def test_projector_is_an_r_by_r_transform_and_B_needs_no_extra_pass():
    # P_O[P B] = P T, T = B (B G B)^{-1/2}, G = P^T P (Eq. 9, full-rank form), and the result
    # is the step of Algorithm 3; B_bar = Sym(U_bar^T X V_bar) = Sym(G_W T_V) (Eq. 10)
    U, B, V, M, Y = _state()
    X = M - O.soft_threshold(M, 0.5)
    P = X @ V
    T_U = B @ O.inv_sqrt_spd(B @ (P.T @ P) @ B)
    U_bar = P @ T_U
    _close(U_bar, O.stiefel_projector(P @ B))
    _close(U_bar, O.stiefel_projector_svd(P @ B))
    W = X.T @ U_bar
    G_W = W.T @ W
    T_V = B @ O.inv_sqrt_spd(B @ G_W @ B)
    V_bar = W @ T_V
    _close(V_bar, O.stiefel_projector(W @ B))
    B_bar = O.sym(G_W @ T_V)
    _close(B_bar, O.spd_projector(U_bar.T @ X @ V_bar))
    U_ref, B_ref, V_ref = O.fixed_rank_opt_step(X, U, B, V)
    _close(U_bar, U_ref)
    _close(V_bar, V_ref)
    _close(B_bar, B_ref)
    # the sweep rebuilds L from C = V_bar B_bar: L = U_bar C^T
    _close(U_bar @ (V_bar @ B_bar).T, U_bar @ B_bar @ V_bar.T)


def test_nystrom_core_equals_the_dense_pseudo_inverse_route():
    # L = L_L (L_L[:l, :l])^+ L_T (Algorithm 2) with L_L = U_L B_L V_L^T and L_T = U_T B_T V_T^T:
    # with A = U_L[:l] B_L, (L_L[:l, :l])^+ = V_L (A^T A)^{-1} A^T, so
    # L = U_L [B_L (A^T A)^{-1} A^T U_T B_T] V_T^T, an r x r core
    mm, nn, l = 150, 110, 30
    U_L, V_L = _stiefel(mm, r), _stiefel(l, r)
    U_T, V_T = _stiefel(l, r), _stiefel(nn, r)
    B_L = np.diag(RNG.uniform(1.0, 3.0, r))
    B_T = np.diag(RNG.uniform(1.0, 3.0, r))
    L_L = U_L @ B_L @ V_L.T
    L_T = U_T @ B_T @ V_T.T
    dense = L_L @ O.truncated_pinv(L_L[:l, :l], r) @ L_T
    A = U_L[:l] @ B_L
    core = B_L @ np.linalg.solve(A.T @ A, A.T @ U_T @ B_T)
    _close(U_L @ core @ V_T.T, dense, tol=1e-10)
    # polar form of the result: Core = Ua diag(sigma) Vc^T -> U = U_L Ua, B = diag(sigma), V = V_T Vc
    Ua, sig, Vct = np.linalg.svd(core)
    _close((U_L @ Ua) @ np.diag(sig) @ (V_T @ Vct.T).T, dense, tol=1e-10)
