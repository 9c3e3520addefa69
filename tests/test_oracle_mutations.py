"""Plant plausible mistakes in the oracle (on the CPU) and check that the pins catch them.

Each case monkeypatches one oracle function with a wrong variant (a sign
flip, a dropped term, a transposed operand, a wrong projector) and asserts
that at least one pin of tests/test_oracle_pins.py then fails.
"""
import numpy as np
import pytest

from oracle import fradm as O
from tests import test_oracle_pins as pins


def _fails(fn, *args):
    try:
        fn(*args)
    except (AssertionError, O.RankDeficient, np.linalg.LinAlgError):
        return True
    return False


def test_soft_threshold_sign_flip_is_caught(monkeypatch):
    monkeypatch.setattr(O, "soft_threshold",
                        lambda X, d: np.maximum(0.0, np.asarray(X) + d) + np.minimum(0.0, np.asarray(X) - d))
    assert _fails(pins.test_soft_threshold_is_prox_of_l1_by_grid_search)


def test_sym_dropped_transpose_is_caught(monkeypatch):
    monkeypatch.setattr(O, "spd_projector", lambda A: np.asarray(A, dtype=np.float64))
    assert _fails(pins.test_spd_projector_is_least_squares_over_symmetric_matrices)


def test_qr_instead_of_polar_is_caught(monkeypatch):
    monkeypatch.setattr(O, "stiefel_projector", lambda A: np.linalg.qr(np.asarray(A, dtype=np.float64))[0])
    assert _fails(pins.test_stiefel_projector_two_forms_agree)
    assert _fails(pins.test_procrustes_optimality_against_random_stiefel_points)


def test_wrong_inverse_square_root_is_caught(monkeypatch):
    real = O.inv_sqrt_spd
    monkeypatch.setattr(O, "inv_sqrt_spd", lambda G: real(G) @ real(G) @ np.asarray(G))  # G^{-1/2}... times G^{-1/2} G
    assert _fails(pins.test_inverse_square_root_matches_scipy_sqrtm)


def test_step_with_transposed_b0_is_caught(monkeypatch):
    def bad_step(X, U0, B0, V0):
        X = np.asarray(X, dtype=np.float64)
        U = O.stiefel_projector(X @ V0 @ B0.T)
        V = O.stiefel_projector(X.T @ U @ B0.T)
        return U, O.spd_projector(U.T @ X @ V), V
    monkeypatch.setattr(O, "fixed_rank_opt_step", bad_step)
    assert _fails(pins.test_lemma1_first_products_are_spd)


def test_multiplier_sign_flip_is_caught(monkeypatch):
    real = O.fr_adm

    def bad_fr_adm(M, r, **kw):
        # Y-step with the wrong sign: Y_{k+1} = Y_k - mu (M - L - S)
        M = np.asarray(M, dtype=np.float64)
        m, n = M.shape
        S = np.zeros((m, n)); Y = np.zeros((m, n)); mu = kw.get("mu0", 1.0)
        U, B, V = np.eye(m, r), np.eye(r), np.eye(n, r)
        res = []
        for _ in range(kw.get("max_iter", 60)):
            U, B, V = O.fixed_rank_opt_step(M - S + Y / mu, U, B, V)
            L = U @ B @ V.T
            S = O.soft_threshold(M - L + Y / mu, 1.0 / mu)
            Y = Y - mu * (M - L - S)
            mu = min(1e9, kw.get("rho", 1.5) * mu)
            res.append(np.linalg.norm(M - L - S) / np.linalg.norm(M))
            if res[-1] <= kw.get("tol", 1e-9):
                break
        return O.FRADMResult(U=U, B=B, V=V, L=U @ B @ V.T, S=S, Y=Y, Y_prev=Y, mu=mu, mu_last=mu,
                             iters=len(res), residuals=res, converged=res[-1] <= kw.get("tol", 1e-9))
    monkeypatch.setattr(O, "fr_adm", bad_fr_adm)
    assert _fails(pins.test_paper_table1_recipe_500)
    monkeypatch.setattr(O, "fr_adm", real)


def test_threshold_with_updated_mu_is_caught(monkeypatch):
    # S-step thresholding at 1/mu_{k+1} instead of 1/mu_k (order of Alg. 1 lines swapped)
    def bad_fr_adm(M, r, **kw):
        M = np.asarray(M, dtype=np.float64)
        m, n = M.shape
        S = np.zeros((m, n)); Y = np.zeros((m, n)); mu = kw.get("mu0", 1.0); rho = kw.get("rho", 1.5)
        U, B, V = np.eye(m, r), np.eye(r), np.eye(n, r)
        fixed = kw.get("fixed_iters")
        for _ in range(fixed or 60):
            U, B, V = O.fixed_rank_opt_step(M - S + Y / mu, U, B, V)
            L = U @ B @ V.T
            mu_next = min(1e9, rho * mu)
            S = O.soft_threshold(M - L + Y / mu, 1.0 / mu_next)
            Y = Y + mu * (M - L - S)
            mu = mu_next
        return O.FRADMResult(U=U, B=B, V=V, L=U @ B @ V.T, S=S, Y=Y, Y_prev=Y, mu=mu, mu_last=mu,
                             iters=fixed or 60, residuals=[0.0], converged=True)
    monkeypatch.setattr(O, "fr_adm", bad_fr_adm)
    assert _fails(pins.test_first_iteration_closed_form)
