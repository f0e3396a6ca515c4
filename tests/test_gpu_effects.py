"""GPU parity of the graph read-outs (Sec. 4.2): total causal effects, the
time-unrolled VarLiNGAM graph, influence rankings and bootstrap edge
statistics, against the FP64 oracle on the same inputs."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2403_03772_gb300 as pkg
    c = pkg.Context(0, "mixed")
    yield c
    c.close()


def _dag(seed, d, density):
    st = gen.Stream(seed)
    perm = st.permutation(d)
    keep = st.uniform(0.0, 1.0, d * d).reshape(d, d) < density
    w = st.signed_uniform(0.2, 0.9, d * d).reshape(d, d)
    B = np.zeros((d, d))
    for a in range(d):
        for b in range(a):
            if keep[a, b]:
                B[perm[a], perm[b]] = w[a, b]
    return B, perm.astype(np.int32)


@pytest.mark.parametrize("d,density,seed", [(1, 0.0, 1), (6, 0.6, 2), (57, 0.1, 3), (300, 0.01, 4)])
def test_total_effects_match_oracle(ctx, d, density, seed):
    B, perm = _dag(seed, d, density)
    T = ctx.total_effects(B, perm)
    ref = oracle.total_effects(B)
    assert np.max(np.abs(T - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_edge_against_the_order_is_refused(ctx):
    import paper_2403_03772_gb300 as pkg
    B, perm = _dag(5, 8, 0.5)
    B[perm[0], perm[7]] = 0.3          # an edge from a later to an earlier variable
    with pytest.raises(pkg.LingamError):
        ctx.total_effects(B, perm)
    with pytest.raises(pkg.LingamError):
        ctx.total_effects(B, np.zeros(8, dtype=np.int32))   # not a permutation


def test_effects_of_the_estimated_graph(ctx, datasets):
    ds = datasets("cfg2")
    order = ctx.causal_order(ds.X)
    B = ctx.fit_adjacency(ds.X, order)
    T = ctx.total_effects(B, order)
    ref = oracle.total_effects(B)
    assert np.max(np.abs(T - ref)) <= 1e-10 * max(1.0, np.max(np.abs(ref)))
    ex, rc, rex, rrc = ctx.influence(T)
    oex, orc = oracle.influence(ref)
    assert np.max(np.abs(ex - oex)) <= 1e-9 * np.max(oex)
    assert np.max(np.abs(rc - orc)) <= 1e-9 * np.max(orc)
    # ranks are integers decided on the GPU's own scores: compare them with the
    # oracle's ranking of those same scores, and the top 5 with the oracle's
    assert list(rex) == list(oracle.top_k(ex, len(ex)))
    assert list(rrc) == list(oracle.top_k(rc, len(rc)))
    assert set(rex[:5]) == set(oracle.top_k(oex, 5))


def test_varlingam_window_effects(ctx, datasets):
    ds = datasets("cfg4")
    order, B0, Bt = ctx.varlingam_fit(ds.Xt, lags=1)
    T = ctx.varlingam_total_effects(B0, Bt, order)
    ref = oracle.total_effects(oracle.var_window_graph(B0, Bt))
    assert T.shape == (2 * ds.Xt.shape[1],) * 2
    assert np.max(np.abs(T - ref)) <= 1e-10 * max(1.0, np.max(np.abs(ref)))
    ex, rc, rex, rrc = ctx.influence(T)
    oex, orc = oracle.influence(ref)
    assert np.max(np.abs(ex - oex)) <= 1e-9 * np.max(oex)
    assert list(rex) == list(oracle.top_k(ex, len(ex)))


def test_bootstrap_edge_stats(ctx):
    st = gen.Stream(77)
    n, d = 2000, 30
    X = st.laplace(1.0, n * d).reshape(n, d)
    X[:, 1:] += 0.6 * X[:, :-1]
    X = X.astype(np.float32)
    insts = [(X, gen.Stream(100 + k).integers(0, n - 1, n).astype(np.int32)) for k in range(12)]
    _, Bs = ctx.causal_order_batch(insts, adjacency=True)
    for thr in [0.0, 0.05, 0.3]:
        prob, mean = ctx.bootstrap_edge_stats(Bs, thr)
        oprob, omean = oracle.bootstrap_edge_stats(np.stack(Bs), thr)
        assert np.array_equal(prob, oprob)
        assert np.max(np.abs(mean - omean)) <= 1e-15


def _assert_rows_on_oracle_path(X, order, B):
    """Every row of the GPU's pruned B is a point of the oracle's adaptive
    lasso path whose BIC is the minimum up to 1e-3 (two path points whose
    BIC differ by less than that are a tie of the model selection, and a
    1e-10 change in the adaptive weights can swap them)."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    Xc = X - X.mean(axis=0)
    C = Xc.T @ Xc / n
    for pos, k in enumerate(order):
        pred = order[:pos]
        if pos == 0:
            assert np.all(B[k] == 0)
            continue
        path = oracle.adaptive_lasso_path(C, k, pred, n)
        row = B[k, pred]
        if not path:
            assert np.all(row == 0)
            continue
        best = min(b for _, _, b in path)
        near = [b for _, b, bic in path if bic <= best + 1e-3]
        assert any(np.array_equal(row != 0, b != 0) and np.max(np.abs(row - b)) < 1e-6
                   for b in near), (int(k), row, near)
        others = np.delete(np.arange(B.shape[0]), pred)
        assert np.all(B[k, others] == 0)


@pytest.mark.parametrize("seed,n,d", [(71, 40000, 10), (1002, 5000, 40)])
def test_pruned_adjacency_matches_oracle(ctx, seed, n, d):
    ds = gen.cfg1(seed=seed, n=n, d=d) if d <= 10 else gen.cfg2(seed=seed, n=n, d=d)
    B = ctx.prune_adjacency(ds.X, ds.order)
    _assert_rows_on_oracle_path(ds.X, ds.order, B)


def test_pruned_adjacency_of_the_estimated_order(ctx, datasets):
    ds = datasets("cfg1")
    order = ctx.causal_order(ds.X)
    B = ctx.prune_adjacency(ds.X, order)
    _assert_rows_on_oracle_path(ds.X, order, B)
    # a pruned row never has more edges than its least-squares row
    assert np.count_nonzero(B) <= np.count_nonzero(ctx.fit_adjacency(ds.X, order))
