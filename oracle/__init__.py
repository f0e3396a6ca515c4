"""FP64 CPU oracle for the DirectLiNGAM causal-ordering path -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline
leg and ``--impl reference`` arm) may import this package.  It shares no code
with the CUDA path (``paper_2403_03772_gb300``) and neither imports the other.

Pieces and the passage each follows (AcceleratedLiNGAM, arXiv 2403.03772):

* ``causal_order`` / ``search_step`` -- Algorithm 1 and the DirectLiNGAM loop
  of Sec. 2.2, in plain C (``lingam_oracle.c``, FP64, OpenMP over pairs only).
* ``fit_adjacency`` -- Sec. 1: each variable is regressed by least squares on
  the variables earlier in the causal order; the coefficients form the
  weighted adjacency matrix B[effect, cause] (Sec. 4.1 calls it the "weighted
  adjacency matrix").  ``numpy.linalg.lstsq`` per row on the centred data.
* ``varlingam`` -- Sec. 3.2: least-squares VAR fit (intercept included, as in
  the statsmodels estimator named in Sec. 4.2), DirectLiNGAM on the
  innovations, then B_tau = (I - B0) M_tau.

Parity pins live in ``tests/test_oracle_*.py``.  Everything here is pinned
except the three literature constants K1, GAMMA and K2 of the entropy
approximation beyond what quadrature and the closed form of K2 fix.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lingam_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIBPATH = os.path.join(_LIBDIR, "liblingam_oracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_NONFINITE, ERR_DEGENERATE, ERR_NOMEM = 0, 1, 2, 3, 5


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what} failed with status {code}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (no fast-math, no FMA contraction)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if (not force and os.path.exists(_LIBPATH)
            and os.path.getmtime(_LIBPATH) >= os.path.getmtime(_SRC)):
        return _LIBPATH
    tmp = _LIBPATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIBPATH)
    return _LIBPATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIBPATH)
        D, I64, I32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int
        PD, PI32 = ctypes.POINTER(D), ctypes.POINTER(ctypes.c_int32)
        lib.oracle_search_step.argtypes = [PD, I64, I64, PI32, I64, PD, I32, I32, PD, PD, PD,
                                           ctypes.POINTER(I32)]
        lib.oracle_row_scores.argtypes = [PD, I64, I64, PI32, I64, PI32, I64, I32, PD]
        lib.oracle_causal_order.argtypes = [PD, I64, I64, I32, I32, PI32, PD, I64]
        lib.oracle_causal_order_prior.argtypes = [PD, I64, I64, I32, I32,
                                                  ctypes.POINTER(ctypes.c_int8), PI32, PD, I64]
        lib.oracle_regress_along.argtypes = [PD, I64, I64, PI32, ctypes.POINTER(I64), PI32,
                                             I64, I64]
        lib.oracle_moments.argtypes = [PD, I64, PD, PD, PD, PD]
        lib.oracle_entropy.argtypes = [PD, I64, PD, PD]
        lib.oracle_entropy_from_moments.argtypes = [D, D]
        lib.oracle_entropy_from_moments.restype = D
        lib.oracle_residual.argtypes = [PD, PD, I64, PD, PD]
        lib.oracle_standardize.argtypes = [PD, I64, PD, PD]
        lib.oracle_diff_mutual_info.argtypes = [PD, PD, PD, PD, I64, PD, PD]
        lib.oracle_argmax_first.argtypes = [PD, I64]
        lib.oracle_mean.argtypes = [PD, I64]
        lib.oracle_mean.restype = D
        lib.oracle_max_threads.restype = I32
        _lib = lib
        return lib


def _pd(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def _check(code: int, what: str):
    if code != OK:
        raise OracleError(code, what)


# ------------------------------------------------------------- primitives ----

def standardize(x) -> np.ndarray:
    x = _f64(x)
    out = np.empty_like(x)
    tmp = np.empty_like(x)
    _check(_load().oracle_standardize(_pd(x), x.size, _pd(out), _pd(tmp)), "standardize")
    return out


def residual(a, b) -> np.ndarray:
    """_residual(a, b) = a - (cov(a, b)/var(b)) b, cov and var normalised by 1/n."""
    a, b = _f64(a), _f64(b)
    out = np.empty_like(a)
    tmp = np.empty_like(a)
    _check(_load().oracle_residual(_pd(a), _pd(b), a.size, _pd(out), _pd(tmp)), "residual")
    return out


def moments(v) -> tuple[float, float]:
    """(E[log cosh u], E[u exp(-u^2/2)]) of v standardised by its own mean/std."""
    v = _f64(v)
    m1, m2, var = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    tmp = np.empty_like(v)
    _check(_load().oracle_moments(_pd(v), v.size, ctypes.byref(m1), ctypes.byref(m2),
                                  ctypes.byref(var), _pd(tmp)), "moments")
    return m1.value, m2.value


def entropy(v) -> float:
    v = _f64(v)
    h = ctypes.c_double()
    tmp = np.empty_like(v)
    _check(_load().oracle_entropy(_pd(v), v.size, ctypes.byref(h), _pd(tmp)), "entropy")
    return h.value


def entropy_from_moments(m1: float, m2: float) -> float:
    return _load().oracle_entropy_from_moments(float(m1), float(m2))


def diff_mutual_info(xi_std, xj_std, ri_j, rj_i) -> float:
    arrs = [_f64(a) for a in (xi_std, xj_std, ri_j, rj_i)]
    out = ctypes.c_double()
    tmp = np.empty_like(arrs[0])
    _check(_load().oracle_diff_mutual_info(*[_pd(a) for a in arrs], arrs[0].size,
                                           ctypes.byref(out), _pd(tmp)), "diff_mutual_info")
    return out.value


def argmax_first(v) -> int:
    v = _f64(v)
    return int(_load().oracle_argmax_first(_pd(v), v.size))


# ----------------------------------------------------------- one step -------

def search_step(R, U=None, literal: bool = False, threads: int | None = None,
                ref_var=None) -> dict:
    """Algorithm 1 on data R ([n, d] samples x variables) over variables U.

    Returns k_list [p], I [p, p] (I[a, b] = I(U[a], U[b])), Hz [p] and m (the
    chosen original index) and m_pos."""
    R = np.asarray(R, dtype=np.float64)
    n, d = R.shape
    Rc = np.ascontiguousarray(R.T)                   # column-major by variable
    U = np.arange(d, dtype=np.int32) if U is None else np.ascontiguousarray(U, dtype=np.int32)
    p = U.size
    kl = np.empty(p)
    I = np.empty((p, p))
    Hz = np.empty(p)
    mpos = ctypes.c_int()
    ref = None if ref_var is None else _f64(ref_var)
    code = _load().oracle_search_step(
        _pd(Rc), n, n, U.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), p,
        _pd(ref) if ref is not None else None, int(bool(literal)),
        int(threads or default_threads()), _pd(kl), _pd(I), _pd(Hz), ctypes.byref(mpos))
    _check(code, "search_step")
    return {"k_list": kl, "I": I, "Hz": Hz, "m_pos": mpos.value, "m": int(U[mpos.value])}


def row_scores(R, rows, U=None, threads: int | None = None) -> np.ndarray:
    """Algorithm 1's k for the positions ``rows`` of U only (literal loop)."""
    R = np.asarray(R, dtype=np.float64)
    n, d = R.shape
    Rc = np.ascontiguousarray(R.T)
    U = np.arange(d, dtype=np.int32) if U is None else np.ascontiguousarray(U, dtype=np.int32)
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    out = np.empty(rows.size)
    P32 = ctypes.POINTER(ctypes.c_int32)
    code = _load().oracle_row_scores(_pd(Rc), n, n, U.ctypes.data_as(P32), U.size,
                                     rows.ctypes.data_as(P32), rows.size,
                                     int(threads or default_threads()), _pd(out))
    _check(code, "row_scores")
    return out


def causal_order(X, literal: bool = False, threads: int | None = None,
                 scores: bool = False, max_steps: int = 0, prior=None):
    """DirectLiNGAM causal order of X ([n, d]); optionally the per-step scores
    (row t = k_list of step t at the original indices, NaN once removed).

    prior: optional [d, d] ancestry knowledge, prior[i, j] = 1 if x_j is known
    to be an ancestor of x_i, 0 if known not to be, -1 unknown (a reading:
    the paper has none).  A variable is chosen only when no remaining
    variable is a known ancestor of it, and only among the known-exogenous
    remaining variables when there are any; the scores are unchanged."""
    X = _f64(X)
    n, d = X.shape
    order = np.empty(d, dtype=np.int32)
    sc = np.empty((d, d)) if scores else None
    P32 = ctypes.POINTER(ctypes.c_int32)
    if prior is None:
        code = _load().oracle_causal_order(
            _pd(X), n, d, int(bool(literal)), int(threads or default_threads()),
            order.ctypes.data_as(P32), _pd(sc) if sc is not None else None, int(max_steps))
    else:
        pk = np.ascontiguousarray(prior, dtype=np.int8)
        if pk.shape != (d, d) or not np.isin(pk, (-1, 0, 1)).all():
            raise OracleError(1, "causal_order: prior must be [d, d] with entries -1, 0, 1")
        code = _load().oracle_causal_order_prior(
            _pd(X), n, d, int(bool(literal)), int(threads or default_threads()),
            pk.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)), order.ctypes.data_as(P32),
            _pd(sc) if sc is not None else None, int(max_steps))
    _check(code, "causal_order")
    return (order, sc) if scores else order


class Residuals:
    """Sec. 2.2's residual data along a given order, step by step.

    ``advance(t)`` regresses order[t_now .. t) out of the remaining variables
    (the oracle's own helper, in its own sequence); ``data`` is then the [n, d]
    residual matrix (removed variables keep their last values) and ``U`` the
    remaining variables ascending, i.e. the state at which step t of the
    oracle's loop scores when ``order`` is the oracle's order."""

    def __init__(self, X, order):
        X = _f64(X)
        self.n, self.d = X.shape
        self._R = np.ascontiguousarray(X.T)
        self._U = np.arange(self.d, dtype=np.int32)
        self._p = ctypes.c_int64(self.d)
        self._order = np.ascontiguousarray(order, dtype=np.int32)
        self.t = 0

    def advance(self, t: int):
        if t < self.t or t > self.d:
            raise OracleError(1, "Residuals.advance: steps only move forward")
        P32 = ctypes.POINTER(ctypes.c_int32)
        code = _load().oracle_regress_along(
            _pd(self._R), self.n, self.d, self._U.ctypes.data_as(P32), ctypes.byref(self._p),
            self._order.ctypes.data_as(P32), self.t, t)
        _check(code, "regress_along")
        self.t = t
        return self

    @property
    def U(self) -> np.ndarray:
        return self._U[: self._p.value].copy()

    @property
    def data(self) -> np.ndarray:
        return self._R.T


# ------------------------------------------------------------ adjacency -----

def adjacency_rows(X, order, rows=None) -> np.ndarray:
    """Rows of the weighted adjacency B for the variables ``rows`` (original
    indices; default all): B[k, pred(k)] = least-squares coefficients of x_k
    on every variable before it in ``order`` (centred data, so the intercept
    drops out).  Returns a [len(rows), d] array."""
    X = np.asarray(X, dtype=np.float64)
    Xc = X - X.mean(axis=0)
    d = X.shape[1]
    order = np.asarray(order, dtype=np.int64)
    pos = np.empty(d, dtype=np.int64)
    pos[order] = np.arange(d)
    rows = order if rows is None else np.asarray(rows, dtype=np.int64)
    out = np.zeros((len(rows), d))
    for r, k in enumerate(rows):
        pred = order[:pos[k]]
        if pred.size == 0:
            continue
        coef, *_ = np.linalg.lstsq(Xc[:, pred], Xc[:, k], rcond=None)
        out[r, pred] = coef
    return out


def fit_adjacency(X, order) -> np.ndarray:
    d = np.asarray(X).shape[1]
    rows = np.arange(d)
    return adjacency_rows(X, order, rows)


# ------------------------------------------------------------- VarLiNGAM ----

def var_fit(Xt, lags: int = 1):
    """Least-squares VAR(lags) with intercept.  Returns (M [lags, d, d], E)
    where x(t) = c + sum_tau M[tau-1] x(t-tau) + E(t), E the residuals."""
    Xt = np.asarray(Xt, dtype=np.float64)
    T, d = Xt.shape
    Y = Xt[lags:]
    Z = np.hstack([np.ones((T - lags, 1))] + [Xt[lags - tau:T - tau] for tau in range(1, lags + 1)])
    coef, *_ = np.linalg.lstsq(Z, Y, rcond=None)       # [(1 + lags d), d]
    E = Y - Z @ coef
    M = np.stack([coef[1 + (tau - 1) * d:1 + tau * d].T for tau in range(1, lags + 1)])
    return M, E


def varlingam(Xt, lags: int = 1, threads: int | None = None, order=None):
    """VarLiNGAM (Sec. 3.2): returns order, B0 [d, d], Btau [lags, d, d], M, E.

    ``order`` may be passed to skip the ordering (for sampled checks)."""
    M, E = var_fit(Xt, lags)
    if order is None:
        order = causal_order(E, threads=threads)
    B0 = fit_adjacency(E, order)
    d = B0.shape[0]
    Btau = np.stack([(np.eye(d) - B0) @ M[tau] for tau in range(lags)])
    return np.asarray(order), B0, Btau, M, E


# ------------------------------------------------ downstream of the graph ---

def total_effects(B) -> np.ndarray:
    """Total causal effects of a linear acyclic model x = B x + e (Sec. 4.2
    ranks nodes "by measuring the total causal effects"): x = (I - B)^-1 e,
    so T[i, j] = d x_i / d e_j, the sum over every directed path j -> i of the
    product of its edge weights (T[i, i] = 1).  ``numpy.linalg.solve``."""
    B = _f64(B)
    d = B.shape[0]
    return np.linalg.solve(np.eye(d) - B, np.eye(d))


def var_window_graph(B0, Btau) -> np.ndarray:
    """Adjacency of the time-unrolled VarLiNGAM graph over the nodes
    [x(t - lags), ..., x(t - 1), x(t)] (Sec. 3.2): B0 acts within every time
    slice and B_tau from slice s - tau to slice s.  Block (s, s') of the
    (lags+1) d square matrix is B_{s - s'} (B0 on the diagonal)."""
    B0 = _f64(B0)
    Bt = _f64(Btau)
    lags, d = Bt.shape[0], B0.shape[0]
    q = (lags + 1) * d
    A = np.zeros((q, q))
    for s in range(lags + 1):
        A[s * d:(s + 1) * d, s * d:(s + 1) * d] = B0
        for tau in range(1, s + 1):
            A[s * d:(s + 1) * d, (s - tau) * d:(s - tau + 1) * d] = Bt[tau - 1]
    return A


def influence(T) -> tuple[np.ndarray, np.ndarray]:
    """Exerted and received influence of every node from the total effects T
    (Sec. 4.2, Table 2): exert[j] = sum_{i != j} |T[i, j]|,
    receive[i] = sum_{j != i} |T[i, j]|."""
    A = np.abs(_f64(T))
    np.fill_diagonal(A, 0.0)
    return A.sum(axis=0), A.sum(axis=1)


def top_k(score, k: int) -> np.ndarray:
    """Indices of the k largest scores, larger first, equal scores to the
    smaller index (a stable sort of -score)."""
    score = _f64(score)
    return np.argsort(-score, kind="stable")[:k].astype(np.int32)


def bootstrap_edge_stats(Bs, threshold: float = 0.0) -> tuple[np.ndarray, np.ndarray]:
    """Edge statistics over bootstrap resamples: the fraction of resamples in
    which |B[i, j]| > threshold, and the mean of B[i, j]."""
    Bs = _f64(Bs)
    return (np.abs(Bs) > threshold).mean(axis=0), Bs.mean(axis=0)


# ------------------------------------------------------- sparse adjacency ---

def adaptive_lasso_path(C, k, pred, n: int, gamma: float = 1.0, n_lambda: int = 60,
                        eps: float = 1e-6, max_events: int | None = None):
    """Sparse regression of variable k on its predecessors ``pred`` (the paper
    only says "regressing"; this is the reading for pruned output): the
    adaptive lasso of Zou (2006) in covariance form,

        min_b  1/2 b' C_PP b - b' C_Pk + lam sum_j w_j |b_j|,
        w_j = |b_ols_j|^-gamma,  b_ols = C_PP^-1 C_Pk,

    on C = Xc'Xc / n, at lam_i = lam_max eps^(i / (L - 1)), i = 0 .. L-1,
    lam_max = (1 + 1e-9) max_j |C_jk| / w_j.  With beta_j = w_j b_j it is a
    plain lasso on Ct = D C_PP D, ct = D C_Pk, D = diag(1 / w), whose
    minimiser (unique: C_PP is positive definite) is piecewise linear in lam.
    The path is followed exactly by the homotopy of Osborne, Presnell and
    Turlach (2000) / the lasso form of LARS (Efron et al. 2004): with the
    active set A and signs s_A, beta_A = Ct_AA^-1 (ct_A - lam s_A) and the
    correlations rho = ct - Ct beta satisfy rho_A = lam s_A, |rho_j| <= lam
    off A; lam decreases to the next of: an inactive |rho_j| reaching lam
    (j joins with the sign of rho_j), an active beta_j reaching 0 (j leaves),
    or the next grid value (a path point).  A variable is not dropped in the
    event right after it joined nor re-joined right after it left (rounding
    puts it a hair off the boundary).  Variables with b_ols_j = 0 stay 0.
    Each path point carries BIC = n log(RSS/n) + df log n with
    RSS/n = C_kk - 2 b'C_Pk + b'C_PP b and df the nonzeros.
    Returns [(lam, b, bic)] over the grid (empty when lam_max is 0)."""
    C = _f64(C)
    pred = np.asarray(pred, dtype=np.int64)
    q = pred.size
    if q == 0:
        return []
    Cpp = C[np.ix_(pred, pred)]
    cpk = C[pred, k]
    ckk = C[k, k]
    b_ols = np.linalg.solve(Cpp, cpk)
    use = b_ols != 0.0
    D = np.where(use, np.abs(np.where(use, b_ols, 1.0)) ** gamma, 0.0)   # 1 / w
    Ct = Cpp * np.outer(D, D)
    ct = cpk * D
    lam_top = float(np.max(np.abs(ct)))
    lam_max = lam_top * (1.0 + 1e-9)
    if not lam_max > 0.0:
        return []
    grid = lam_max * eps ** (np.arange(n_lambda) / (n_lambda - 1))
    path = []

    def record(lam, beta):
        b = beta * D
        rss = ckk - 2.0 * (b @ cpk) + b @ Cpp @ b
        bic = n * np.log(max(rss, 1e-300)) + np.count_nonzero(b) * np.log(n)
        path.append((lam, b, bic))

    beta = np.zeros(q)
    gi = 0
    while gi < n_lambda and grid[gi] >= lam_top:      # above the first join: b = 0
        record(grid[gi], beta)
        gi += 1
    first = int(np.argmax(np.abs(ct)))
    A, sign = [first], {first: 1.0 if ct[first] > 0.0 else -1.0}
    lam, left, fresh = lam_top, -1, first
    for _ in range(max_events or 20 * q + 100):
        if gi >= n_lambda:
            break
        Ai = np.array(A)
        sA = np.array([sign[j] for j in A])
        G = Ct[np.ix_(Ai, Ai)]
        bA = np.linalg.solve(G, ct[Ai] - lam * sA)
        dA = np.linalg.solve(G, sA)            # d beta_A / d(-lam)
        rho = ct - Ct[:, Ai] @ bA
        a = Ct[:, Ai] @ dA                     # d rho / d lam
        active = np.zeros(q, dtype=bool)
        active[Ai] = True
        step, kind, who = lam - grid[gi], "grid", -1
        for j in range(q):
            if active[j] or not use[j] or j == left:
                continue
            if abs(rho[j]) >= lam:             # on or past the boundary: joins now
                step, kind, who = 0.0, "join", j
                break
            for num, den in ((lam - rho[j], 1.0 - a[j]), (lam + rho[j], 1.0 + a[j])):
                if den > 0.0 and num / den < step:
                    step, kind, who = num / den, "join", j
        for t, j in enumerate(A):
            if j != fresh and dA[t] != 0.0:
                dl = -bA[t] / dA[t]
                if 1e-12 * lam < dl < step:
                    step, kind, who = dl, "drop", j
        left = fresh = -1
        if kind == "grid":
            lam = grid[gi]
            beta[:] = 0.0
            beta[Ai] = np.linalg.solve(G, ct[Ai] - lam * sA)
            record(lam, beta)
            gi += 1
        elif kind == "join":
            lam -= step
            sign[who] = 1.0 if rho[who] - step * a[who] > 0.0 else -1.0
            A.append(who)
            fresh = who
        else:
            lam -= step
            A.remove(who)
            left = who
    return path


def adaptive_lasso_row(C, k, pred, n: int, gamma: float = 1.0, n_lambda: int = 60,
                       eps: float = 1e-6) -> np.ndarray:
    """The path point of ``adaptive_lasso_path`` with the smallest BIC (the
    first one on ties); zeros when the path is empty."""
    path = adaptive_lasso_path(C, k, pred, n, gamma, n_lambda, eps)
    if not path:
        return np.zeros(np.asarray(pred).size)
    best = min(range(len(path)), key=lambda i: (path[i][2], i))
    return path[best][1]


def prune_adjacency(X, order, gamma: float = 1.0, n_lambda: int = 60,
                    eps: float = 1e-6) -> np.ndarray:
    """Sparse weighted adjacency: ``adaptive_lasso_row`` for every variable on
    the variables before it in ``order``; B[k, pred(k)] = its coefficients."""
    X = _f64(X)
    n, d = X.shape
    Xc = X - X.mean(axis=0)
    C = Xc.T @ Xc / n
    order = np.asarray(order, dtype=np.int64)
    B = np.zeros((d, d))
    for pos_k, k in enumerate(order):
        pred = order[:pos_k]
        B[k, pred] = adaptive_lasso_row(C, k, pred, n, gamma, n_lambda, eps)
    return B
