"""Pins for the FP64 CPU oracle: each checks it against something other than itself.

The sources are closed forms and optimality statements of the paper (Sec. 2,
Sec. 4.1, Eq. 9, Eq. 10, Lemma 1, Theorem 2, Eq. 11), textbook routines that
reach the same result by another route (SVD, QR orthogonal iteration,
least squares, grid search), and the numbers the paper prints for its
synthetic recipe (Table 1).
"""
import os

import numpy as np
import pytest
import scipy.linalg

from oracle import fradm as O
from paper_1503_03004_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand(seed, *shape):
    return synth.rng(seed).standard_normal(shape)


def _stiefel(seed, m, r):
    Q, _ = np.linalg.qr(_rand(seed, m, r))
    return Q


# ---------------------------------------------------------------- Sec. 2 operators

def test_soft_threshold_is_prox_of_l1_by_grid_search():
    # P_ST_delta(x) = argmin_s 0.5 (s - x)^2 + delta |s|   (Sec. 2 definition)
    grid = np.linspace(-6, 6, 240001)
    for delta in (0.0, 0.3, 1.0, 2.5):
        for x in (-5.0, -2.6, -1.0, -0.2, 0.0, 0.1, 0.99, 1.0, 1.7, 4.2):
            f = 0.5 * (grid - x) ** 2 + delta * np.abs(grid)
            s_star = grid[np.argmin(f)]
            assert abs(O.soft_threshold(np.array([x]), delta)[0] - s_star) <= 1e-4


def test_soft_threshold_special_values():
    x = np.array([-3.0, -1.0, -0.5, 0.0, 0.5, 1.0, 3.0])
    np.testing.assert_array_equal(O.soft_threshold(x, 1.0), [-2.0, 0.0, 0.0, 0.0, 0.0, 0.0, 2.0])
    np.testing.assert_array_equal(O.soft_threshold(x, 0.0), x)


def test_sym_is_orthogonal_projection_onto_symmetric_matrices():
    A = _rand(1, 7, 7)
    S = O.sym(A)
    np.testing.assert_array_equal(S, S.T)
    np.testing.assert_allclose(O.sym(S), S, rtol=0, atol=0)
    # A - Sym(A) is antisymmetric, hence Frobenius-orthogonal to every symmetric matrix
    Z = O.sym(_rand(2, 7, 7))
    assert abs(np.sum((A - S) * Z)) < 1e-12


# ---------------------------------------------------------------- Eq. 9: P_O

def test_stiefel_projector_two_forms_agree():
    # Eq. 9 gives P_O[A] = Q S^T (thin SVD) and, for full rank, A (A^T A)^{-1/2}
    for seed, (m, r) in enumerate([(9, 1), (12, 3), (40, 7), (200, 25)]):
        A = _rand(10 + seed, m, r)
        np.testing.assert_allclose(O.stiefel_projector(A), O.stiefel_projector_svd(A), atol=1e-12)


def test_stiefel_projector_rank_one_is_normalisation():
    a = _rand(3, 11, 1)
    np.testing.assert_allclose(O.stiefel_projector(a), a / np.linalg.norm(a), atol=1e-15)


def test_stiefel_projector_properties():
    A = _rand(4, 50, 6) @ np.diag([1, 2, 3, 5, 8, 13.0])
    U = O.stiefel_projector(A)
    np.testing.assert_allclose(U.T @ U, np.eye(6), atol=1e-13)          # on St_{m,r}
    np.testing.assert_allclose(O.stiefel_projector(U), U, atol=1e-13)  # idempotent
    H = U.T @ A                                                       # polar factor: SPD
    np.testing.assert_allclose(H, H.T, atol=1e-12)
    assert np.linalg.eigvalsh(O.sym(H))[0] > 0


def test_inverse_square_root_matches_scipy_sqrtm():
    A = _rand(5, 30, 8)
    G = A.T @ A
    np.testing.assert_allclose(O.inv_sqrt_spd(G), np.linalg.inv(scipy.linalg.sqrtm(G).real), atol=1e-12)


def test_stiefel_projector_rejects_rank_deficient():
    A = _rand(6, 20, 3)
    A[:, 2] = A[:, 0] + A[:, 1]
    with pytest.raises(O.RankDeficient):
        O.stiefel_projector(A)


def test_procrustes_optimality_against_random_stiefel_points():
    # Eq. 9: U = P_O[M V B] minimises ||M - U B V^T||_F over St_{m,r}
    m, n, r = 30, 20, 4
    M, V = _rand(7, m, n), _stiefel(8, n, r)
    B = O.sym(_rand(9, r, r)) + 4 * np.eye(r)
    U = O.stiefel_projector(M @ V @ B)
    f = np.linalg.norm(M - U @ B @ V.T)
    for s in range(200):
        Up = O.stiefel_projector(U + 0.05 * _rand(100 + s, m, r))
        assert f <= np.linalg.norm(M - Up @ B @ V.T) + 1e-12
        Ur = _stiefel(400 + s, m, r)
        assert f <= np.linalg.norm(M - Ur @ B @ V.T) + 1e-12


# ---------------------------------------------------------------- Eq. 10: P_SPD

def test_spd_projector_is_least_squares_over_symmetric_matrices():
    # Eq. 10: for orthonormal U, V the minimiser of ||M - U B V^T|| over symmetric B is Sym(U^T M V).
    # Brute force: solve the least-squares problem in the r(r+1)/2 free parameters.
    m, n, r = 25, 18, 4
    M, U, V = _rand(11, m, n), _stiefel(12, m, r), _stiefel(13, n, r)
    cols, idx = [], []
    for i in range(r):
        for j in range(i, r):
            E = np.zeros((r, r))
            E[i, j] = E[j, i] = 1.0
            cols.append((U @ E @ V.T).ravel())
            idx.append((i, j))
    theta, *_ = np.linalg.lstsq(np.stack(cols, 1), M.ravel(), rcond=None)
    B_ls = np.zeros((r, r))
    for t, (i, j) in zip(theta, idx):
        B_ls[i, j] = B_ls[j, i] = t
    np.testing.assert_allclose(O.spd_projector(U.T @ M @ V), B_ls, atol=1e-12)


def test_lemma1_first_products_are_spd():
    # Lemma 1: with U = P_O[M V0 B0], V = P_O[M^T U B0] and B0 merely invertible,
    # U^T M V0 B0 and B0 U^T M V are symmetric positive definite.  The lemma's
    # proof gives V^T M^T U B0 in SPD, i.e. B0^T U^T M V; the printed B0 U^T M V
    # is the same matrix when B0 is symmetric.  Both readings are checked.
    m, n, r = 40, 30, 5
    M, V0 = _rand(21, m, n), _stiefel(22, n, r)
    B_sym_indef = O.sym(_rand(23, r, r)) @ np.diag([1, -1, 1, -1, 1.0]) @ O.sym(_rand(23, r, r))
    B_sym_indef = O.sym(B_sym_indef)
    B_general = _rand(24, r, r) + 3 * np.eye(r)
    for B0 in (B_sym_indef, B_general):
        U, _, V = O.fixed_rank_opt_step(M, None, B0, V0)
        for K in (U.T @ M @ V0 @ B0, B0.T @ U.T @ M @ V):
            np.testing.assert_allclose(K, K.T, atol=1e-10 * np.abs(K).max())
            assert np.linalg.eigvalsh(O.sym(K))[0] > 0
    # With B0 = I the SPD step needs no symmetrisation: B1 = U1^T M V1 exactly (Appendix).
    U1, B1, V1 = O.fixed_rank_opt_step(M, None, np.eye(r), V0)
    np.testing.assert_allclose(B1, U1.T @ M @ V1, atol=1e-11)
    assert np.linalg.eigvalsh(B1)[0] > 0


# ---------------------------------------------------------------- Theorem 2 / Eq. 5

def _tiny_low_rank_plus_noise(seed, m, n, r, gap=0.05):
    U, V = _stiefel(seed, m, r), _stiefel(seed + 1, n, r)
    s = np.linspace(10, 5, r)
    return U @ np.diag(s) @ V.T + gap * _rand(seed + 2, m, n)


def test_fixed_rank_opt_full_converges_to_tsvd():
    # Theorem 2 / Eq. 5: Algorithm 4 converges to the rank-r truncated SVD of M.
    m, n, r = 30, 24, 3
    M = _tiny_low_rank_plus_noise(31, m, n, r)
    it = O.fixed_rank_opt_full(M, None, np.eye(r), np.eye(n, r), 60)
    U, B, V = it[-1]
    Q, s, Wt = np.linalg.svd(M)
    T = Q[:, :r] @ np.diag(s[:r]) @ Wt[:r]
    assert np.linalg.norm(U @ B @ V.T - T) / np.linalg.norm(T) < 1e-12
    np.testing.assert_allclose(np.linalg.eigvalsh(B)[::-1], s[:r], rtol=1e-12)


def test_fixed_rank_step_is_orthogonal_iteration():
    # Theorem 2 proof: span(U_{i+1}) = span(M M^T U_i), the textbook orthogonal iteration
    m, n, r = 26, 20, 3
    M = _tiny_low_rank_plus_noise(41, m, n, r, gap=0.5)
    it = O.fixed_rank_opt_full(M, None, np.eye(r), np.eye(n, r), 6)
    for (Ui, _, _), (Uj, _, _) in zip(it[:-1], it[1:]):
        Q, _ = np.linalg.qr(M @ M.T @ Ui)
        np.testing.assert_allclose(Uj @ Uj.T, Q @ Q.T, atol=1e-12)
    # and the projector error contracts like (sigma_{r+1}/sigma_r)^2 per step
    Qs, s, _ = np.linalg.svd(M)
    P_star = Qs[:, :r] @ Qs[:, :r].T
    errs = [np.linalg.norm(U @ U.T - P_star, 2) for (U, _, _) in it]
    ratio = (s[r] / s[r - 1]) ** 2
    for a, b in zip(errs[1:-1], errs[2:]):
        assert b <= 1.5 * ratio * a + 1e-14


# ---------------------------------------------------------------- Algorithm 1

def test_s_step_minimises_augmented_lagrangian_entrywise():
    # Alg. 1 S-step: argmin_S mu/2 ||M-L-S||^2 + ||S||_1 + <Y, M-L-S>, separable per entry
    g = synth.rng(51)
    M, L, Y = g.standard_normal((4, 5)), g.standard_normal((4, 5)), g.uniform(-1, 1, (4, 5))
    mu = 1.7
    S = O.soft_threshold(M - L + Y / mu, 1.0 / mu)
    grid = np.linspace(-5, 5, 100001)
    for i in range(4):
        for j in range(5):
            f = mu / 2 * (M[i, j] - L[i, j] - grid) ** 2 + np.abs(grid) + Y[i, j] * (M[i, j] - L[i, j] - grid)
            assert abs(S[i, j] - grid[np.argmin(f)]) <= 2e-4


def test_first_iteration_closed_form():
    # First pass of Alg. 1: S = Y = 0, mu = 1, B0 = I, V0 = I_{n x r} so X = M and
    # U_1 = P_O[M[:, :r]] (thin-SVD form), V_1 = P_O[M^T U_1], B_1 = U_1^T M V_1.
    prob = synth.planted(40, 30, 4, p=0.1, amp=1.0, seed=61)
    M = prob.values_f64()
    res = O.fr_adm(M, 4, fixed_iters=1)
    U1 = O.stiefel_projector_svd(M[:, :4])
    V1 = O.stiefel_projector_svd(M.T @ U1)
    B1 = U1.T @ M @ V1
    np.testing.assert_allclose(res.U, U1, atol=1e-12)
    np.testing.assert_allclose(res.V, V1, atol=1e-12)
    np.testing.assert_allclose(res.B, B1, atol=1e-10)
    L1 = U1 @ B1 @ V1.T
    S1 = np.sign(M - L1) * np.maximum(np.abs(M - L1) - 1.0, 0.0)
    np.testing.assert_allclose(res.S, S1, atol=1e-11)
    np.testing.assert_allclose(res.Y, (M - L1) - S1, atol=1e-11)


def _read_table1_golden():
    rows = {}
    with open(os.path.join(GOLDEN, "paper_table1_fradm.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            m, r, err_l, err_s, iters, time_s = line.split()
            rows[int(m)] = dict(r=int(r), err_l=float(err_l), err_s=float(err_s), iters=int(iters))
    return rows


def test_paper_table1_recipe_500():
    # Table 1, m = n = 500, r = 10, 10% outliers of magnitude in [-1, 1]: the paper
    # prints Err.L 2.21e-10 after 28 iterations.  rho is unstated; rho = 1.5 is the
    # reading (it reproduces the printed iteration count).
    row = _read_table1_golden()[500]
    prob = synth.paper_table1(500, row["r"])
    M = prob.values_f64()
    L0 = prob.U0 @ prob.V0.T
    res = O.fr_adm(M, row["r"], rho=1.5, tol=1e-9)
    err_l = np.linalg.norm(res.L - L0) / np.linalg.norm(L0)
    assert res.converged
    assert err_l < 100 * row["err_l"]
    assert abs(res.iters - row["iters"]) <= 5
    np.testing.assert_array_equal(res.S != 0, prob.S0_mask)


@pytest.fixture(scope="module")
def solved_small():
    prob = synth.planted(120, 90, 5, p=0.08, amp=1.0, seed=71)
    M = prob.values_f64()
    return prob, M, O.fr_adm(M, 5, rho=1.5, tol=1e-10)


def test_fradm_invariants_at_convergence(solved_small):
    prob, M, res = solved_small
    r = 5
    assert res.converged and res.residuals[-1] <= 1e-10
    np.testing.assert_allclose(res.U.T @ res.U, np.eye(r), atol=1e-12)
    np.testing.assert_allclose(res.V.T @ res.V, np.eye(r), atol=1e-12)
    np.testing.assert_allclose(res.B, res.B.T, atol=0)
    assert np.linalg.eigvalsh(res.B)[0] > 0
    assert np.linalg.norm(M - res.L - res.S) / np.linalg.norm(M) <= 1e-10
    # Y stays in the l1 subdifferential: |Y| <= 1 and Y = sign(S) on supp(S)
    assert np.max(np.abs(res.Y)) <= 1 + 1e-12
    on = res.S != 0
    np.testing.assert_allclose(res.Y[on], np.sign(res.S[on]), atol=1e-6)


def test_fradm_planted_recovery_large_outliers():
    # 500 x 500, r = 25, 10% outliers in [-50, 50]; mu0 scaled to the data (0.05)
    prob = synth.square_fp64_500()
    M = prob.values_f64()
    L0 = prob.U0 @ prob.V0.T
    res = O.fr_adm(M, 25, rho=1.5, mu0=0.05, tol=1e-9)
    assert res.converged
    assert np.linalg.norm(res.L - L0) / np.linalg.norm(L0) < 1e-7
    np.testing.assert_array_equal(res.S != 0, prob.S0_mask)


def test_fradm_argument_checks():
    with pytest.raises(ValueError):
        O.fr_adm(np.zeros((4, 4)), 5)
    with pytest.raises(ValueError):
        O.fr_adm(np.ones((4, 4)), 1, rho=1.0)


# ---------------------------------------------------------------- Algorithm 2

def test_frnys_exact_on_rank_r_matrix_without_outliers():
    # Nystrom identity: for rank(M) = r, C W^+ R = M, so FR-Nys returns L = M, S = 0
    m, n, r, l = 80, 70, 3, 12
    M = _rand(81, m, r) @ _rand(82, r, n)
    out = O.fr_nys(M, r, l, synth.row_permutation(m, 83), rho=1.5, tol=1e-12)
    np.testing.assert_allclose(out.L, M, atol=1e-8 * np.abs(M).max())
    assert np.abs(out.S).max() < 1e-8 * np.abs(M).max()


def test_frnys_recovers_planted_low_rank():
    prob = synth.planted(300, 240, 4, p=0.05, amp=1.0, seed=91)
    M = prob.values_f64()
    L0 = prob.U0 @ prob.V0.T
    # inner FR-ADM solves use mu0 = 0.1: with mu0 = 1 the m x l block solve stalls at ~1e-2
    out = O.fr_nys(M, 4, 40, synth.row_permutation(300, 92), rho=1.5, mu0=0.1, tol=1e-10)
    assert np.linalg.norm(out.L - L0) / np.linalg.norm(L0) < 1e-8


def test_truncated_pinv_matches_numpy_pinv_on_full_rank():
    A = _rand(93, 6, 6)
    np.testing.assert_allclose(O.truncated_pinv(A, 6), np.linalg.pinv(A), atol=1e-12)


def test_frnys_sampled_output_equals_dense_output():
    # the sampled form (used at sizes where the dense m x n L cannot be formed) takes the same
    # entries of the same L_L (L_L[:l, :l])^+ L_T and M - L as the dense form
    m, n, r, l = 260, 230, 4, 40
    prob = synth.planted(m, n, r, p=0.05, amp=1.0, seed=44, dtype="f64")
    M = prob.values_f64()
    perm = synth.row_permutation(m, 45)
    dense = O.fr_nys(M, r, l, perm, rho=1.5, mu0=0.1, tol=1e-10)
    g = synth.rng(46)
    ii, jj = g.integers(0, m, 500), g.integers(0, n, 500)
    samp = O.fr_nys(M, r, l, perm, sample=(ii, jj), rho=1.5, mu0=0.1, tol=1e-10)
    np.testing.assert_allclose(samp.L, dense.L[ii, jj], rtol=0, atol=1e-12 * np.abs(dense.L).max())
    np.testing.assert_allclose(samp.S, dense.S[ii, jj], rtol=0, atol=1e-12 * np.abs(dense.L).max())
