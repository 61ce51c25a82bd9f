"""Pins for the oracle's t-SVD pieces against closed forms and Proposition 1."""

import numpy as np
import scipy.sparse as sp

from oracle.tsvd import brute_force_update, embedding_from_tsvd, randomized_tsvd, t_svd
from tests.helpers import dense_from_pairs, load_closed_form_spectra


def test_tsvd_matches_closed_form_spectra():
    for name, pairs, sv in load_closed_form_spectra():
        A = dense_from_pairs(pairs)
        U, s, V = t_svd(A, len(sv))
        np.testing.assert_allclose(s, sv, atol=1e-12, err_msg=name)
        # Eq. "ne": X Y^T reproduces the rank-d truncation; at full rank it is A itself
        X, Y = embedding_from_tsvd(U, s, V)
        np.testing.assert_allclose(X @ Y.T, A, atol=1e-12, err_msg=name)


def test_disjoint_cliques_spectrum():
    # c disjoint K_k: sigma = k-1 (c times), then 1 (c(k-1) times)
    k, c = 5, 4
    pairs = []
    for b in range(c):
        o = b * k
        pairs += [(o + i, o + j) for i in range(k) for j in range(i + 1, k)]
    A = dense_from_pairs(pairs)
    _, s, _ = t_svd(A, c * k)
    np.testing.assert_allclose(s[:c], k - 1, atol=1e-12)
    np.testing.assert_allclose(s[c:], 1.0, atol=1e-12)


def test_randomized_tsvd_exact_on_gapped_spectrum():
    # star K_{1,25} plus a disjoint K_6: sigma = 5, 5, 5, 1, ... ; rank-3 RSVD is exact
    pairs = [(0, i) for i in range(1, 26)]
    pairs += [(26 + i, 26 + j) for i in range(6) for j in range(i + 1, 6)]
    A = dense_from_pairs(pairs)
    rng = np.random.default_rng(1)
    Om = rng.standard_normal((A.shape[0], 8))
    U, s, V = randomized_tsvd(sp.csr_matrix(A), Om, 3, power_iters=4)
    np.testing.assert_allclose(s, [5.0, 5.0, 5.0], atol=1e-10)
    np.testing.assert_allclose(U.T @ U, np.eye(3), atol=1e-12)
    # the rank-3 product equals the exact rank-3 truncation (unique: gap 5 -> 1)
    Ue, se, Ve = t_svd(A, 3)
    np.testing.assert_allclose((U * s) @ V.T, (Ue * se) @ Ve.T, atol=1e-9)


def test_brute_force_update_single_edge_from_zero():
    # two isolated nodes, add the edge (0, 1): the t-SVD of e_0 e_1^T has sigma_1 = 1
    X1 = np.zeros((2, 1))
    Y1 = np.zeros((2, 1))
    dA = np.zeros((2, 2))
    dA[0, 1] = 1.0
    X2, Y2, s = brute_force_update(X1, Y1, dA, 1)
    assert abs(s[0] - 1.0) < 1e-15
    np.testing.assert_allclose(X2 @ Y2.T, dA, atol=1e-15)


def test_proposition_1_residual_norm():
    # |(I - U U^T) x| = sqrt(|x|^2 - |U^T x|^2) for orthonormal U (Prop. 1)
    rng = np.random.default_rng(3)
    for n, d in [(50, 5), (200, 40)]:
        U, _ = np.linalg.qr(rng.standard_normal((n, d)))
        for _ in range(5):
            x = rng.standard_normal(n)
            lhs = np.linalg.norm(x - U @ (U.T @ x))
            rhs = np.sqrt(x @ x - np.sum((U.T @ x) ** 2))
            assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(x)
