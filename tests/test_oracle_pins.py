"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, a Gaussian quadrature, an exact invariant, a special case that reduces
to a textbook or library routine, brute force on a tiny input, or the
identifiability property the paper relies on (Sec. 2.2, Sec. 3.1).
"""
import math

import numpy as np
import pytest
from scipy import integrate

import gen
import oracle

SQ2PI = math.sqrt(2.0 * math.pi)


def _quad(f, lo=-40.0, hi=40.0):
    return integrate.quad(f, lo, hi, epsabs=1e-15, epsrel=1e-13, limit=400)[0]


def _phi(z):
    return math.exp(-0.5 * z * z) / SQ2PI


def _lc(z):
    return math.log(math.cosh(z))


def _g2(z):
    return z * math.exp(-0.5 * z * z)


# ------------------------------------------------------ entropy constants ----

def _oracle_quadratic_in_m1():
    """H(m1, 0) is an exact concave quadratic; recover its vertex and curvature."""
    xs = [0.30, 0.40, 0.50]
    hs = [oracle.entropy_from_moments(x, 0.0) for x in xs]
    A = np.vander(xs, 3)
    a, b, c = np.linalg.solve(A, hs)
    return -b / (2 * a), -a, c


def test_gamma_is_gaussian_mean_of_logcosh():
    gamma, _, _ = _oracle_quadratic_in_m1()
    gq = _quad(lambda z: _lc(z) * _phi(z))
    assert abs(gq - 0.3745672074914) < 1e-12
    assert abs(gamma - gq) < 5e-6


def test_k1_matches_gaussian_orthonormalisation_of_logcosh():
    # Max-entropy approximation: for an even G, k = 1 / (2 Var_nu(G~)) with G~
    # = G orthogonalised against 1 and nu^2 under the standard Gaussian.
    _, k1, _ = _oracle_quadratic_in_m1()
    EG = _quad(lambda z: _lc(z) * _phi(z))
    EG2 = _quad(lambda z: _lc(z) ** 2 * _phi(z))
    EGz2 = _quad(lambda z: _lc(z) * z * z * _phi(z))
    beta = (EGz2 - EG) / 2.0
    k1_quad = 1.0 / (2.0 * (EG2 - EG * EG - 2.0 * beta * beta))
    assert abs(k1 / k1_quad - 1.0) < 1e-3        # literature 79.047 vs 79.0156


def test_k2_closed_form_and_quadrature():
    h0 = oracle.entropy_from_moments(0.37457, 0.0)
    h1 = oracle.entropy_from_moments(0.37457, 0.1)
    k2 = (h0 - h1) / 0.01
    closed = 36.0 / (8.0 * math.sqrt(3.0) - 9.0)
    delta = _quad(lambda z: _g2(z) * z * _phi(z))
    e2 = _quad(lambda z: _g2(z) ** 2 * _phi(z))
    assert abs(closed - 1.0 / (2.0 * (e2 - delta * delta))) < 1e-10
    assert abs(k2 / closed - 1.0) < 2e-5


def test_gaussian_entropy_at_the_vertex():
    h = oracle.entropy_from_moments(0.37457, 0.0)
    assert abs(h - 0.5 * (1.0 + math.log(2.0 * math.pi))) < 1e-14


# ------------------------------------------------------------- moments -------

def test_moments_two_point_closed_form():
    v = np.array([2.5, -7.0] * 500)
    m1, m2 = oracle.moments(v)
    assert abs(m1 - math.log(math.cosh(1.0))) < 1e-14
    assert abs(m2) < 1e-15


def test_moments_three_point_hand_worked():
    # v = (0, 0, 3): mean 1, population variance 2, u = (-1/sqrt2, -1/sqrt2, sqrt2)
    m1, m2 = oracle.moments([0.0, 0.0, 3.0])
    r = 1.0 / math.sqrt(2.0)
    assert abs(m1 - (2 * math.log(math.cosh(r)) + math.log(math.cosh(2 * r))) / 3) < 1e-15
    assert abs(m2 - (2 * (-r) * math.exp(-0.25) + 2 * r * math.exp(-1.0)) / 3) < 1e-15


def test_moments_affine_invariance_and_sign():
    st = gen.Stream(7)
    v = st.exponential(4001)
    m1, m2 = oracle.moments(v)
    a1, a2 = oracle.moments(3.7 * v + 11.0)
    b1, b2 = oracle.moments(-v)
    assert abs(a1 - m1) < 1e-13 and abs(a2 - m2) < 1e-13
    assert abs(b1 - m1) < 1e-13 and abs(b2 + m2) < 1e-13
    assert abs(m2) > 1e-3                       # skewed: G2 moment is non-zero


@pytest.mark.parametrize("kind", ["uniform", "laplace", "exp", "student5", "normal"])
def test_moments_match_quadrature_of_known_densities(kind):
    n = 1_000_000
    st = gen.Stream(12345)
    s3 = math.sqrt(3.0)
    if kind == "uniform":
        v = st.uniform(-s3, s3, n)
        pdf, lo, hi = (lambda x: 1.0 / (2 * s3)), -s3, s3
    elif kind == "laplace":
        b = 1.0 / math.sqrt(2.0)
        v = st.laplace(b, n)
        pdf, lo, hi = (lambda x: math.exp(-abs(x) / b) / (2 * b)), -40.0, 40.0
    elif kind == "exp":
        v = st.exponential(n) - 1.0
        pdf, lo, hi = (lambda x: math.exp(-(x + 1.0))), -1.0, 60.0
    elif kind == "student5":
        sc = math.sqrt(3.0 / 5.0)
        v = st.student_t(5, n) * sc
        c5 = math.gamma(3.0) / (math.sqrt(5 * math.pi) * math.gamma(2.5))
        pdf, lo, hi = (lambda x: c5 * (1 + (x / sc) ** 2 / 5) ** -3 / sc), -400.0, 400.0
    else:
        v = st.normal(n)
        pdf, lo, hi = _phi, -40.0, 40.0
    m1, m2 = oracle.moments(v)
    t1 = integrate.quad(lambda x: _lc(x) * pdf(x), lo, hi, limit=800, epsabs=1e-13)[0]
    t2 = integrate.quad(lambda x: _g2(x) * pdf(x), lo, hi, limit=800, epsabs=1e-13)[0]
    u = (v - v.mean()) / v.std()
    se1 = np.std(np.log(np.cosh(u))) / math.sqrt(n)
    se2 = np.std(u * np.exp(-0.5 * u * u)) / math.sqrt(n)
    assert abs(m1 - t1) < 6 * se1 + 1e-4 * se1
    assert abs(m2 - t2) < 6 * se2
    if kind == "normal":
        assert abs(oracle.entropy(v) - 0.5 * (1 + math.log(2 * math.pi))) < 1e-3
    else:
        assert oracle.entropy(v) < 0.5 * (1 + math.log(2 * math.pi))


# ------------------------------------------------------------ residual -------

def test_residual_orthogonal_to_regressor():
    st = gen.Stream(3)
    b = st.laplace(1.0, 5000) + 3.0
    a = 0.7 * b + st.uniform(-1, 1, 5000) - 2.0
    r = oracle.residual(a, b)
    assert abs(np.mean(r * (b - b.mean()))) < 1e-12 * a.std() * b.std()


def test_residual_equals_lstsq_with_intercept():
    st = gen.Stream(4)
    b = st.exponential(777)
    a = -1.3 * b + st.normal(777)
    r = oracle.residual(a, b)
    Z = np.column_stack([np.ones_like(b), b])
    coef, *_ = np.linalg.lstsq(Z, a, rcond=None)
    r_ls = a - Z @ coef
    assert np.max(np.abs((r - r.mean()) - r_ls)) < 1e-12
    slope = (a - r)[1] / b[1]
    assert abs(slope - coef[1]) < 1e-12


# ---------------------------------------------------------- Algorithm 1 -------

def _numpy_algorithm1(X):
    """Independent numpy transcription of Algorithm 1 (cross-check, tiny sizes)."""
    n, d = X.shape

    def H(v):
        u = (v - v.mean()) / v.std()
        m1 = np.mean(np.log(np.cosh(u)))
        m2 = np.mean(u * np.exp(-u * u / 2))
        return (1 + np.log(2 * np.pi)) / 2 - 79.047 * (m1 - 0.37457) ** 2 - 7.4129 * m2 ** 2

    def res(a, b):
        return a - (np.mean((a - a.mean()) * (b - b.mean())) / np.var(b)) * b

    k = np.zeros(d)
    for i in range(d):
        for j in range(d):
            if i == j:
                continue
            xi = (X[:, i] - X[:, i].mean()) / X[:, i].std()
            xj = (X[:, j] - X[:, j].mean()) / X[:, j].std()
            mi = (H(xj) + H(res(xi, xj))) - (H(xi) + H(res(xj, xi)))
            k[i] += min(0.0, mi) ** 2
    return -k


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_literal_and_memoised_modes_are_bitwise_identical(seed):
    st = gen.Stream(seed)
    d, n = 7, 257
    X = st.laplace(1.0, n * d).reshape(n, d) @ st.uniform(-1, 1, (d, d))
    a = oracle.search_step(X, literal=True, threads=3)
    b = oracle.search_step(X, literal=False, threads=2)
    assert np.array_equal(a["k_list"], b["k_list"])
    assert np.array_equal(a["I"], b["I"])
    assert np.array_equal(a["Hz"], b["Hz"])
    o1, s1 = oracle.causal_order(X, literal=True, scores=True, threads=1)
    o2, s2 = oracle.causal_order(X, literal=False, scores=True, threads=4)
    assert np.array_equal(o1, o2)
    assert np.array_equal(np.nan_to_num(s1, nan=9.0), np.nan_to_num(s2, nan=9.0))


def test_step_antisymmetry_is_exact_and_matches_brute_force():
    st = gen.Stream(11)
    d, n = 6, 300
    X = st.exponential(n * d).reshape(n, d) @ st.uniform(-1, 1, (d, d))
    r = oracle.search_step(X, literal=True)
    assert np.array_equal(r["I"], -r["I"].T)
    ref = _numpy_algorithm1(X)
    assert np.max(np.abs(r["k_list"] - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))
    assert r["m_pos"] == int(np.argmax(ref))


def test_argmax_takes_first_maximum():
    assert oracle.argmax_first([-3.0, -1.0, -1.0, -2.0]) == 1
    assert oracle.argmax_first([-0.0, 0.0]) == 0


@pytest.mark.parametrize("noise", ["uniform", "laplace", "exp"])
def test_two_variable_lingam_pair_orders_cause_first(noise):
    st = gen.Stream(99)
    n = 20000
    draw = {"uniform": lambda: st.uniform(-1, 1, n), "laplace": lambda: st.laplace(1.0, n),
            "exp": lambda: st.exponential(n)}[noise]
    x0 = draw()
    x1 = 0.8 * x0 + draw()
    X = np.column_stack([x0, x1])
    r = oracle.search_step(X)
    assert r["I"][0, 1] > 0                    # positive I(i, j) supports i -> j
    assert list(oracle.causal_order(X)) == [0, 1]
    assert list(oracle.causal_order(X[:, ::-1])) == [1, 0]


def test_single_variable():
    X = np.arange(10.0).reshape(10, 1)
    assert list(oracle.causal_order(X)) == [0]


def test_degenerate_inputs_are_errors():
    st = gen.Stream(5)
    a = st.uniform(-1, 1, 100)
    b = st.uniform(-1, 1, 100)
    with pytest.raises(oracle.OracleError) as e:
        oracle.causal_order(np.column_stack([a, 2.0 * a, b]))
    assert e.value.code == oracle.ERR_DEGENERATE
    with pytest.raises(oracle.OracleError) as e:
        oracle.causal_order(np.column_stack([a, np.full(100, 3.0)]))
    assert e.value.code == oracle.ERR_DEGENERATE
    with pytest.raises(oracle.OracleError) as e:
        oracle.causal_order(np.column_stack([a, a + b, b]))      # collinear after 2 steps
    assert e.value.code == oracle.ERR_DEGENERATE
    bad = np.column_stack([a, b])
    bad[3, 1] = np.nan
    with pytest.raises(oracle.OracleError) as e:
        oracle.causal_order(bad)
    assert e.value.code == oracle.ERR_NONFINITE


# ------------------------------------------------- recovery (identifiability) -

def test_cfg1_order_is_topological(datasets):
    ds = datasets("cfg1")
    order = oracle.causal_order(ds.X)
    assert gen.is_topological(order, ds.B)


def test_cfg2_order_is_topological(datasets):
    ds = datasets("cfg2")
    order = oracle.causal_order(ds.X)
    assert gen.is_topological(order, ds.B)


def test_paper_two_level_simulation_recovers_true_order():
    """Sec. 3.1: 50 seeds, n = 10000, d = 10, theta ~ N(0,1), noise U(0,1)."""
    bad = []
    for seed in range(50):
        ds = gen.two_level(seed)
        order = oracle.causal_order(ds.X)
        if not gen.is_topological(order, ds.B, min_abs=0.05):
            bad.append(seed)
    assert bad == []


# ------------------------------------------------------------- adjacency ------

def _orthogonal_noise(n, d, seed):
    st = gen.Stream(seed)
    E = st.laplace(1.0, n * d).reshape(n, d)
    E = E - E.mean(axis=0)
    Q, _ = np.linalg.qr(E)
    return Q * np.sqrt(n) * st.uniform(0.5, 2.0, d)


def test_adjacency_exact_when_noise_is_exactly_orthogonal():
    d, n = 8, 400
    ds = gen.cfg1(seed=77, n=n, d=d)
    E = _orthogonal_noise(n, d, 78)
    X = gen.sem_sample(ds.B, ds.order, E)
    B = oracle.fit_adjacency(X, ds.order)
    assert np.max(np.abs(B - ds.B)) < 1e-10


def test_adjacency_zero_above_order_and_ldl_identity():
    st = gen.Stream(21)
    d, n = 9, 500
    X = st.laplace(1.0, n * d).reshape(n, d) @ st.uniform(-1, 1, (d, d))
    order = st.permutation(d)
    B = oracle.fit_adjacency(X, order)
    pos = np.empty(d, dtype=int)
    pos[order] = np.arange(d)
    for k in range(d):
        for j in range(d):
            if pos[j] >= pos[k]:
                assert B[k, j] == 0.0
    Xc = X - X.mean(axis=0)
    C = (Xc.T @ Xc) / n
    Cp = C[np.ix_(order, order)]
    G = np.linalg.cholesky(Cp)
    L = G / np.diag(G)
    Bp = np.eye(d) - np.linalg.inv(L)
    assert np.max(np.abs(B[np.ix_(order, order)] - Bp)) < 1e-10


# ------------------------------------------------------------- VarLiNGAM ------

def test_varlingam_recovers_hand_built_var1():
    st = gen.Stream(31)
    d, T = 3, 40000
    B0 = np.array([[0.0, 0.0, 0.0], [0.8, 0.0, 0.0], [0.0, -0.6, 0.0]])
    M1 = np.array([[0.4, 0.0, 0.1], [0.0, 0.3, 0.0], [-0.2, 0.0, 0.25]])
    A = np.linalg.inv(np.eye(d) - B0)
    E = st.laplace(1.0 / math.sqrt(2.0), T * d).reshape(T, d)
    X = np.zeros((T, d))
    for t in range(1, T):
        X[t] = M1 @ X[t - 1] + A @ E[t]
    order, B0h, Bt, M, _ = oracle.varlingam(X, lags=1)
    assert list(order) == [0, 1, 2]
    assert np.max(np.abs(M[0] - M1)) < 0.03
    assert np.max(np.abs(B0h - B0)) < 0.03
    assert np.max(np.abs(Bt[0] - (np.eye(d) - B0) @ M1)) < 0.04


# ------------------------------------------------ residuals along an order ----

def test_residuals_along_order_equal_lstsq_on_removed_variables():
    """After t steps, each remaining column is x_i minus its least-squares fit
    (with intercept) on the t removed variables: Sec. 2.2's sequential
    regressions span the same space as one regression on all of them."""
    ds = gen.cfg2(seed=71, n=1500, d=9)
    order = oracle.causal_order(ds.X)
    res = oracle.Residuals(ds.X, order)
    X = ds.X.astype(np.float64)
    for t in (1, 3, 6, 8):
        res.advance(t)
        removed = order[:t]
        assert sorted(res.U) == sorted(set(range(9)) - set(int(v) for v in removed))
        Z = np.column_stack([np.ones(X.shape[0]), X[:, removed]])
        for i in res.U:
            coef, *_ = np.linalg.lstsq(Z, X[:, i], rcond=None)
            r_ls = X[:, i] - Z @ coef
            r = res.data[:, i]
            assert np.max(np.abs((r - r.mean()) - r_ls)) < 1e-10 * X[:, i].std()


def test_residuals_reproduce_the_oracle_loop_scores_at_later_steps():
    """Scoring rows on the residual state of step t gives the k_list the
    oracle's own loop recorded at step t (bitwise: same helpers, same order)."""
    ds = gen.cfg2(seed=72, n=900, d=8)
    order, sc = oracle.causal_order(ds.X, scores=True)
    res = oracle.Residuals(ds.X, order)
    for t in (0, 2, 5):
        res.advance(t)
        U = res.U
        rows = np.arange(U.size, dtype=np.int32)
        k = oracle.row_scores(res.data, rows, U=U)
        assert np.array_equal(k, sc[t, U])
        assert int(U[np.argmax(k)]) == int(order[t])
