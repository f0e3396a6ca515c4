"""Seeded synthetic inputs shaped like the paper's workloads.

This module is shared by the FP64 oracle tests and the GPU path.  It holds none
of the method's arithmetic: it only draws structural equation models and
samples from them.

Every random number starts as a PCG64 uniform double (``Generator.random``,
whose stream numpy keeps stable across versions).  Every transform uses only
IEEE-754 ``+ - * /``, ``sqrt``, ``frexp`` and comparisons, one numpy ufunc at a
time, plus a series logarithm written here.  numpy's own vectorised ``log`` /
``cos`` are avoided on purpose: their last-bit results differ between x86-64
and aarch64 builds, and the data must be byte-identical on x86 and Arm.

Workloads (n = samples, d = variables; the paper writes X as [m, dim]):

* ``cfg1``  d=10,  n=1000   random DAG, edge prob 0.3, weights +-U[0.5,2],
  noise U(-sqrt3, sqrt3).
* ``cfg2``  d=100, n=5000   Erdos-Renyi DAG, mean in-degree 2, weights
  +-U[0.5,2], per-variable noise Laplace(0,1/sqrt2) | Exp(1)-1 | U(-sqrt3,sqrt3).
* ``cfg3``  d=1000, n=10000 scale-free DAG (preferential attachment, 2 parents
  per node), weights +-U[0.3,1], noise Student-t(5)*sqrt(3/5).  Stands in for
  the Perturb-CITE-seq shape of Sec. 4.1 (n ~ 5e4-7.5e4, d ~ 961-964).
* ``cfg4``  VAR(1), d=487, T=2500 (+500 burn-in), sparse lag matrix scaled to
  spectral radius 0.5, instantaneous DAG with mean in-degree 1.5, Laplace
  innovations.  Stands in for the S&P 500 shape of Sec. 4.2 (d=487, lag 1).
* ``cfg5``  128 bootstrap resamples of one d=200, n=4000 cfg2-style dataset,
  plus 64 cfg2-style instances with d ~ U{50..400}, n ~ U{1000..8000}.
* ``two_level``  the validation generator of Sec. 3.1: a two-level DAG,
  theta ~ N(0,1), noise Uniform(0,1).
"""
from __future__ import annotations

import hashlib
from dataclasses import dataclass, field

import numpy as np

LN2 = 0.6931471805599453
SQRT3 = 1.7320508075688772
SQRT_HALF = 0.7071067811865476

SEEDS = {1: 1001, 2: 1002, 3: 1003, 4: 1004, 5: 1005, 6: 1006}


def series_log(x: np.ndarray) -> np.ndarray:
    """Natural log of positive float64 values using only IEEE basic operations.

    x = m * 2**e with m in [sqrt(1/2), sqrt(2)); log m = 2*atanh(s) with
    s = (m-1)/(m+1), |s| <= 0.1716, summed to 13 odd terms (< 1e-17 relative).
    """
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)
    low = m < SQRT_HALF
    m = np.where(low, m * 2.0, m)
    e = np.where(low, e - 1, e).astype(np.float64)
    s = (m - 1.0) / (m + 1.0)
    s2 = s * s
    term = s.copy()
    acc = s.copy()
    for k in range(1, 14):
        term = term * s2
        acc = acc + term / float(2 * k + 1)
    return 2.0 * acc + e * LN2


class Stream:
    """Distributions built on PCG64 uniform doubles only (see module doc)."""

    def __init__(self, seed):
        if isinstance(seed, np.random.SeedSequence):
            self.rng = np.random.Generator(np.random.PCG64(seed))
        else:
            self.rng = np.random.Generator(np.random.PCG64(int(seed)))

    def random(self, size) -> np.ndarray:
        return self.rng.random(size)

    def uniform(self, lo: float, hi: float, size) -> np.ndarray:
        return lo + (hi - lo) * self.rng.random(size)

    def open01(self, size) -> np.ndarray:
        u = self.rng.random(size)
        return np.where(u == 0.0, 0.5, u)

    def normal(self, size: int) -> np.ndarray:
        """Marsaglia polar method (no trigonometry)."""
        size = int(size)
        out = np.empty(size, dtype=np.float64)
        filled = 0
        while filled < size:
            k = size - filled
            m = k // 2 + k // 4 + 16
            u = 2.0 * self.rng.random(m) - 1.0
            v = 2.0 * self.rng.random(m) - 1.0
            s = u * u + v * v
            ok = (s > 0.0) & (s < 1.0)
            u, v, s = u[ok], v[ok], s[ok]
            f = np.sqrt((-2.0 * series_log(s)) / s)
            z = np.empty(2 * s.size, dtype=np.float64)
            z[0::2] = u * f
            z[1::2] = v * f
            take = min(z.size, k)
            out[filled:filled + take] = z[:take]
            filled += take
        return out

    def laplace(self, b: float, size: int) -> np.ndarray:
        """Laplace(0, b) by inverse CDF."""
        u = self.open01(size) - 0.5
        a = np.abs(u)
        w = 1.0 - 2.0 * a
        w = np.where(w <= 0.0, 2.0 ** -53, w)
        mag = -b * series_log(w)
        return np.where(u < 0.0, -mag, mag)

    def exponential(self, size: int) -> np.ndarray:
        """Exp(1) by inverse CDF."""
        return -series_log(1.0 - self.rng.random(size))

    def student_t(self, nu: int, size: int) -> np.ndarray:
        """Student-t with integer nu: Z / sqrt(chi2_nu / nu)."""
        z0 = self.normal(size)
        chi = np.zeros(size, dtype=np.float64)
        for _ in range(nu):
            zk = self.normal(size)
            chi = chi + zk * zk
        return z0 / np.sqrt(chi / float(nu))

    def permutation(self, n: int) -> np.ndarray:
        return np.argsort(self.rng.random(n), kind="stable").astype(np.int64)

    def integers(self, lo: int, hi_inclusive: int, size) -> np.ndarray:
        span = hi_inclusive - lo + 1
        v = np.floor(self.rng.random(size) * span).astype(np.int64) + lo
        return np.minimum(v, hi_inclusive)

    def signed_uniform(self, lo: float, hi: float, size) -> np.ndarray:
        mag = self.uniform(lo, hi, size)
        sign = self.rng.random(size) < 0.5
        return np.where(sign, -mag, mag)


@dataclass
class Dataset:
    """X: float32 [n, d] row-major samples x variables (the paper's layout)."""
    X: np.ndarray
    B: np.ndarray                  # true weighted adjacency, B[child, parent]
    order: np.ndarray              # one true causal order (topological)
    name: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.X.shape[0])

    @property
    def d(self) -> int:
        return int(self.X.shape[1])

    def digest(self) -> str:
        return hashlib.sha256(np.ascontiguousarray(self.X).tobytes()).hexdigest()[:16]


def sem_sample(B: np.ndarray, order: np.ndarray, E: np.ndarray) -> np.ndarray:
    """x_k = sum_j B[k, j] x_j + e_k, evaluated in causal order, parents in
    ascending index, one elementwise multiply-add at a time (fixed rounding)."""
    n, d = E.shape
    X = np.zeros((n, d), dtype=np.float64)
    for k in order:
        col = E[:, k].copy()
        for j in np.nonzero(B[k])[0]:
            col = col + B[k, j] * X[:, j]
        X[:, k] = col
    return X


def _random_dag(st: Stream, d: int, p_edge: float, wlo: float, whi: float):
    perm = st.permutation(d)
    mask = st.random((d, d)) < p_edge
    w = st.signed_uniform(wlo, whi, (d, d))
    B = np.zeros((d, d), dtype=np.float64)
    for a in range(d):
        for b in range(a + 1, d):
            if mask[a, b]:
                B[perm[b], perm[a]] = w[a, b]
    return B, perm


def _noise_mix(st: Stream, n: int, d: int) -> np.ndarray:
    """Per-variable noise: Laplace(0,1/sqrt2), Exp(1)-1 or U(-sqrt3,sqrt3), prob 1/3 each."""
    kind = st.integers(0, 2, d)
    E = np.empty((n, d), dtype=np.float64)
    for k in range(d):
        if kind[k] == 0:
            E[:, k] = st.laplace(SQRT_HALF, n)
        elif kind[k] == 1:
            E[:, k] = st.exponential(n) - 1.0
        else:
            E[:, k] = st.uniform(-SQRT3, SQRT3, n)
    return E


def cfg1(seed=SEEDS[1], n: int = 1000, d: int = 10) -> Dataset:
    st = Stream(seed)
    B, perm = _random_dag(st, d, 0.3, 0.5, 2.0)
    E = st.uniform(-SQRT3, SQRT3, (n, d))
    X = sem_sample(B, perm, E)
    return Dataset(X.astype(np.float32), B, perm, f"cfg1_d{d}_n{n}")


def cfg2(seed=SEEDS[2], n: int = 5000, d: int = 100) -> Dataset:
    st = Stream(seed)
    B, perm = _random_dag(st, d, 4.0 / (d - 1), 0.5, 2.0)
    E = _noise_mix(st, n, d)
    X = sem_sample(B, perm, E)
    return Dataset(X.astype(np.float32), B, perm, f"cfg2_d{d}_n{n}")


def long_n(seed=SEEDS[6], n: int = 1_000_000, d: int = 100) -> Dataset:
    """The paper's long-sample case (Sec. 2.3 and its CPU benchmark figure:
    1e6 observations of 100 variables, 7 hours for a sequential CPU run),
    drawn with the cfg2 generator (ER DAG, mean in-degree 2, mixed noise)."""
    ds = cfg2(seed=seed, n=n, d=d)
    ds.name = f"long_n_d{d}_n{n}"
    return ds


def cfg3(seed=SEEDS[3], n: int = 10000, d: int = 1000) -> Dataset:
    st = Stream(seed)
    # Preferential attachment over nodes 0..d-1 in insertion order.
    deg = np.zeros(d, dtype=np.int64)
    parents = [[] for _ in range(d)]
    if d > 1:
        parents[1] = [0]
        deg[0] += 1
        deg[1] += 1
    for k in range(2, d):
        u = st.random(2)
        wts = deg[:k] + 1
        cum = np.cumsum(wts)
        first = int(np.searchsorted(cum, u[0] * float(cum[-1]), side="right"))
        first = min(first, k - 1)
        wts2 = wts.copy()
        wts2[first] = 0
        cum2 = np.cumsum(wts2)
        second = int(np.searchsorted(cum2, u[1] * float(cum2[-1]), side="right"))
        second = min(second, k - 1)
        if second == first:  # only reachable through float edge cases
            second = (first + 1) % k
        parents[k] = sorted([first, second])
        deg[first] += 1
        deg[second] += 1
        deg[k] += 2
    relabel = st.permutation(d)          # node k -> variable relabel[k]
    w = st.signed_uniform(0.3, 1.0, (d, 2))
    B = np.zeros((d, d), dtype=np.float64)
    for k in range(d):
        for q, par in enumerate(parents[k]):
            B[relabel[k], relabel[par]] = w[k, q]
    order = relabel.copy()               # insertion order is topological
    E = st.student_t(5, n * d).reshape(n, d) * np.sqrt(3.0 / 5.0)
    X = sem_sample(B, order, E)
    return Dataset(X.astype(np.float32), B, order, f"cfg3_d{d}_n{n}")


def _round_sig(x: float, digits: int = 9) -> float:
    return float(f"{x:.{digits}e}")


@dataclass
class VarDataset:
    """Xt: float32 [T, d] time series; M1 reduced-form lag matrix; B0 instantaneous DAG."""
    Xt: np.ndarray
    M1: np.ndarray
    B0: np.ndarray
    order: np.ndarray
    name: str = ""

    def digest(self) -> str:
        return hashlib.sha256(np.ascontiguousarray(self.Xt).tobytes()).hexdigest()[:16]


def cfg4(seed=SEEDS[4], T: int = 2500, d: int = 487, burn: int = 500,
         m_density: float = 0.02, b0_indeg: float = 1.5) -> VarDataset:
    st = Stream(seed)
    mmask = st.random((d, d)) < m_density
    mval = st.signed_uniform(0.05, 0.2, (d, d))
    M1 = np.where(mmask, mval, 0.0)
    rad = float(np.max(np.abs(np.linalg.eigvals(M1)))) if mmask.any() else 0.0
    if rad > 0:
        M1 = M1 * _round_sig(0.5 / rad)
    B0, perm = _random_dag(st, d, (2.0 * b0_indeg) / (d - 1), 0.2, 0.8)
    Ttot = T + burn
    E = st.laplace(SQRT_HALF, Ttot * d).reshape(Ttot, d)
    V = sem_sample(B0, perm, E)          # V = (I - B0)^-1 e, row per time step
    # padded sparse rows of M1 for a fixed-order matvec
    nz = [np.nonzero(M1[k])[0] for k in range(d)]
    width = max(1, max(len(z) for z in nz))
    cols = np.zeros((d, width), dtype=np.int64)
    vals = np.zeros((d, width), dtype=np.float64)
    for k in range(d):
        cols[k, :len(nz[k])] = nz[k]
        vals[k, :len(nz[k])] = M1[k, nz[k]]
    X = np.zeros((Ttot, d), dtype=np.float64)
    prev = np.zeros(d, dtype=np.float64)
    for t in range(Ttot):
        acc = V[t].copy()
        for q in range(width):
            acc = acc + vals[:, q] * prev[cols[:, q]]
        X[t] = acc
        prev = acc
    return VarDataset(X[burn:].astype(np.float32), M1, B0, perm, f"cfg4_d{d}_T{T}")


@dataclass
class BatchInstance:
    X: np.ndarray                   # float32 [n_src, d] source data
    rows: np.ndarray | None         # int32 [n] resample rows, or None
    name: str = ""

    def data(self) -> np.ndarray:
        return self.X if self.rows is None else self.X[self.rows]


def cfg5(seed=SEEDS[5], n_resamples: int = 128, base_d: int = 200, base_n: int = 4000,
         n_uneven: int = 64, d_range=(50, 400), n_range=(1000, 8000)) -> list[BatchInstance]:
    ss = np.random.SeedSequence(int(seed))
    base_ss, rows_ss, sizes_ss, inst_ss = ss.spawn(4)
    base = cfg2(base_ss, n=base_n, d=base_d)
    out = []
    rst = Stream(rows_ss)
    for r in range(n_resamples):
        rows = rst.integers(0, base_n - 1, base_n).astype(np.int32)
        out.append(BatchInstance(base.X, rows, f"boot{r}"))
    sst = Stream(sizes_ss)
    ds = sst.integers(d_range[0], d_range[1], n_uneven)
    ns = sst.integers(n_range[0], n_range[1], n_uneven)
    for k, child in enumerate(inst_ss.spawn(n_uneven)):
        ds_k = cfg2(child, n=int(ns[k]), d=int(ds[k]))
        out.append(BatchInstance(ds_k.X, None, f"inst{k}_d{ds[k]}_n{ns[k]}"))
    return out


def two_level(seed: int, n: int = 10000, d: int = 10, p_edge: float = 0.5) -> Dataset:
    """Sec. 3.1 validation data: level-0 nodes feed level-1 nodes only,
    theta ~ N(0,1), noise Uniform(0,1)."""
    st = Stream(seed)
    level = (st.random(d) < 0.5).astype(np.int64)
    if level.min() == level.max():
        level[0] = 1 - level[0]
    mask = st.random((d, d)) < p_edge
    theta = st.normal(d * d).reshape(d, d)
    B = np.zeros((d, d), dtype=np.float64)
    for i in range(d):
        for j in range(d):
            if level[i] == 1 and level[j] == 0 and mask[i, j]:
                B[i, j] = theta[i, j]
    order = np.concatenate([np.nonzero(level == 0)[0], np.nonzero(level == 1)[0]])
    E = st.uniform(0.0, 1.0, (n, d))
    X = sem_sample(B, order, E)
    return Dataset(X.astype(np.float32), B, order, f"two_level_s{seed}")


def residual_samples(d: int, n: int) -> int:
    """Unit of work: one ordered pair (i, j) at one sample, summed over the
    ordering steps p = d..2:  n * sum p(p-1) = n (d+1) d (d-1) / 3."""
    return n * (d + 1) * d * (d - 1) // 3


def is_topological(order, B: np.ndarray, min_abs: float = 0.0) -> bool:
    """True when no edge with |weight| > min_abs points backwards in ``order``."""
    pos = np.empty(len(order), dtype=np.int64)
    pos[np.asarray(order)] = np.arange(len(order))
    child, parent = np.nonzero(np.abs(B) > min_abs)
    return bool(np.all(pos[parent] < pos[child]))


def ancestors(B: np.ndarray) -> np.ndarray:
    """anc[i, j] = True when x_j is an ancestor of x_i in the DAG of B
    (B[child, parent] != 0), by repeated composition of the parent relation."""
    par = np.asarray(B) != 0
    anc = par.copy()
    while True:
        nxt = anc | ((anc.astype(np.int64) @ par.astype(np.int64)) > 0)
        if (nxt == anc).all():
            return anc
        anc = nxt


def prior_from_dag(st: Stream, B: np.ndarray, reveal: float = 0.3) -> np.ndarray:
    """Ancestry knowledge consistent with the DAG of B: each ordered pair
    (i, j), i != j, is revealed with probability ``reveal`` as 1 (x_j is an
    ancestor of x_i) or 0 (it is not); the rest are -1 (unknown)."""
    d = B.shape[0]
    anc = ancestors(B)
    pk = np.where(anc, 1, 0).astype(np.int8)
    hide = st.random((d, d)) >= reveal
    pk[hide] = -1
    np.fill_diagonal(pk, -1)
    return pk
