"""Pins of the oracle's sparse adjacency (adaptive lasso + BIC, the reading
for pruned output) against closed forms, limits, a library routine and
recovery of a known graph."""
import numpy as np
import pytest

import gen
import oracle


def test_orthogonal_design_is_a_soft_threshold():
    # predecessors uncorrelated with each other: every coordinate decouples,
    # b_j(lam) = S(C_jk, lam w_j) / C_jj exactly
    C = np.diag([2.0, 0.5, 1.5, 3.0])
    C[3, :3] = C[:3, 3] = [0.8, -0.3, 0.05]
    n = 1000
    path = oracle.adaptive_lasso_path(C, 3, [0, 1, 2], n, eps=1e-3, n_lambda=15)
    cjj = np.array([2.0, 0.5, 1.5])
    cpk = np.array([0.8, -0.3, 0.05])
    w = 1.0 / np.abs(cpk / cjj)
    for lam, b, bic in path:
        ref = np.sign(cpk) * np.maximum(np.abs(cpk) - lam * w, 0.0) / cjj
        assert np.max(np.abs(b - ref)) < 1e-15
        rss = C[3, 3] - 2 * b @ cpk + b @ (cjj * b)
        assert abs(bic - (n * np.log(rss) + np.count_nonzero(b) * np.log(n))) < 1e-9


def test_vanishing_penalty_gives_least_squares():
    ds = gen.cfg1(n=3000)
    X = ds.X.astype(np.float64)
    Xc = X - X.mean(axis=0)
    C = Xc.T @ Xc / X.shape[0]
    k = int(ds.order[-1])
    pred = ds.order[:-1]
    path = oracle.adaptive_lasso_path(C, k, pred, X.shape[0], eps=1e-13, n_lambda=30)
    ols, *_ = np.linalg.lstsq(Xc[:, pred], Xc[:, k], rcond=None)
    assert np.max(np.abs(path[-1][1] - ols)) < 1e-8


def test_path_point_matches_sklearn_lasso():
    lm = pytest.importorskip("sklearn.linear_model")
    st = gen.Stream(5)
    n, q = 2000, 6
    Z = st.laplace(1.0, n * q).reshape(n, q)
    Z[:, 1] += 0.5 * Z[:, 0]
    y = Z @ np.array([0.9, 0.0, -0.4, 0.05, 0.0, 0.7]) + st.laplace(1.0, n)
    X = np.column_stack([Z, y])
    Xc = X - X.mean(axis=0)
    C = Xc.T @ Xc / n
    path = oracle.adaptive_lasso_path(C, q, np.arange(q), n, n_lambda=12, eps=1e-2)
    b_ols = np.linalg.solve(C[:q, :q], C[:q, q])
    w = 1.0 / np.abs(b_ols)
    for lam, b, _ in path[3::3]:
        # the weighted problem is a plain lasso on the columns divided by w
        m = lm.Lasso(alpha=lam, fit_intercept=False, tol=1e-14, max_iter=100000)
        m.fit(Xc[:, :q] / w, Xc[:, q])
        assert np.max(np.abs(b - m.coef_ / w)) < 1e-7


def test_rss_from_covariance_equals_residual_of_the_data():
    ds = gen.cfg2(n=4000, d=12)
    X = ds.X.astype(np.float64)
    Xc = X - X.mean(axis=0)
    n = X.shape[0]
    C = Xc.T @ Xc / n
    k, pred = int(ds.order[8]), ds.order[:8]
    for lam, b, bic in oracle.adaptive_lasso_path(C, k, pred, n, n_lambda=8):
        rss = np.sum((Xc[:, k] - Xc[:, pred] @ b) ** 2) / n
        assert abs(bic - (n * np.log(rss) + np.count_nonzero(b) * np.log(n))) < 1e-6


def test_recovers_the_true_support_at_large_n():
    # adaptive lasso + BIC is consistent for the support: at n = 40000 the
    # pruned graph of the true order is the true graph (a stray tiny
    # coefficient in at most two of ten random graphs), values close
    exact = 0
    for seed in range(70, 80):
        ds = gen.cfg1(seed=seed, n=40000)
        B = oracle.prune_adjacency(ds.X, ds.order)
        exact += np.array_equal(B != 0, ds.B != 0)
        assert np.all((B != 0) | (ds.B == 0))          # no true edge is lost
        assert np.max(np.abs(B - ds.B)) < 0.05
    assert exact >= 8


def test_every_path_point_satisfies_the_lasso_optimality_conditions():
    # KKT of the weighted lasso at each grid lam: C_Pk - C_PP b = lam w sign(b)
    # on the support, |C_jk - (C_PP b)_j| <= lam w_j off it
    ds = gen.cfg2(seed=1002, n=5000, d=40)
    X = ds.X.astype(np.float64)
    Xc = X - X.mean(axis=0)
    n = X.shape[0]
    C = Xc.T @ Xc / n
    worst = 0.0
    for pos in range(1, ds.d):
        k, pred = int(ds.order[pos]), ds.order[:pos]
        cpp, cpk = C[np.ix_(pred, pred)], C[pred, k]
        w = 1.0 / np.abs(np.linalg.solve(cpp, cpk))
        for lam, b, _ in oracle.adaptive_lasso_path(C, k, pred, n):
            g = cpk - cpp @ b
            on = b != 0
            worst = max(worst,
                        np.max(np.abs(g[on] - lam * w[on] * np.sign(b[on])), initial=0.0) / lam,
                        np.max(np.abs(g[~on]) - lam * w[~on], initial=0.0) / lam)
    assert worst < 1e-6
