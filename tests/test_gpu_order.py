"""GPU parity: the CUDA causal-ordering path through the C ABI against the FP64
oracle (element by element on the same seeded inputs).

Orders must be identical integer permutations; per-step scores M(i) within
1e-4 of the step's max |M| (+1e-12); first-step I(i, j) within a bound
derived from FP32 moment errors (1e-11 for the double-float form, 1e-10 for
FP64); adjacency within 1e-5 absolute.
"""
import numpy as np
import pytest

import gen
import oracle
from gpu_util import B_ABS, read_golden_order, scores_close

pytestmark = pytest.mark.gpu

PRECS = ["fp32", "mixed", "fp64", "df"]


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


@pytest.fixture(scope="module")
def ctx(torch_cuda):
    import paper_2403_03772_gb300 as pkg
    c = {p: pkg.Context(0, p) for p in PRECS}
    yield c
    for v in c.values():
        v.close()


def _dev(torch, X, prec):
    dt = torch.float64 if prec == "fp64" else torch.float32
    return torch.as_tensor(np.asarray(X), dtype=dt).to("cuda:0")


def _random_sem(seed, n, d, noise="mix"):
    st = gen.Stream(seed)
    B, perm = gen._random_dag(st, d, min(1.0, 3.0 / max(1, d - 1)), 0.3, 1.2)
    E = gen._noise_mix(st, n, d)
    return gen.sem_sample(B, perm, E).astype(np.float32), B


# ---------------------------------------------------------------- step 0 ----

@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape", [(1000, 10, 1), (1300, 37, 2), (513, 24, 3), (260, 3, 4)])
def test_first_step_measures_match_oracle(ctx, torch_cuda, prec, shape):
    n, d, seed = shape
    X, _ = _random_sem(seed, n, d)
    I, M = ctx[prec].step_measures(_dev(torch_cuda, X, prec))
    ref = oracle.search_step(X.astype(np.float64))
    # I: FP32 moments carry ~1e-7 relative error; h = -K1 (m1-g)^2 - K2 m2^2
    # amplifies it by 2 K1 |m1 - g| <= ~20 -> a few e-6 absolute on I.
    # double-float: terms carry <= ~3e-14 absolute error, so I stays far
    # below the 1e-10 bound the re-score tier assumes for it
    tolI = {"fp64": 1e-10, "df": 1e-11}.get(prec, 5e-5)
    assert np.max(np.abs(I - ref["I"])) < tolI
    scale = np.max(np.abs(ref["k_list"]))
    assert np.max(np.abs(M - ref["k_list"])) <= 1e-4 * scale + 1e-12


# ------------------------------------------------------------- full order ---

@pytest.mark.parametrize("prec", PRECS)
def test_cfg1_order_and_scores(ctx, torch_cuda, datasets, prec):
    ds = datasets("cfg1")
    gold, dig = read_golden_order("cfg1")
    assert dig == ds.digest()
    order, scores = ctx[prec].causal_order(_dev(torch_cuda, ds.X, prec), scores=True)
    assert list(order) == list(gold)
    assert gen.is_topological(order, ds.B)
    _, ref_scores = oracle.causal_order(ds.X, scores=True)
    assert scores_close(scores, ref_scores) <= 0


@pytest.mark.parametrize("prec", ["fp32", "mixed", "df"])
def test_cfg2_order_and_scores(ctx, torch_cuda, datasets, prec):
    ds = datasets("cfg2")
    gold, dig = read_golden_order("cfg2")
    assert dig == ds.digest()
    order, scores = ctx[prec].causal_order(_dev(torch_cuda, ds.X, prec), scores=True)
    assert list(order) == list(gold)
    _, ref_scores = oracle.causal_order(ds.X, scores=True)
    assert scores_close(scores, ref_scores) <= 0


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape", [(300, 2, 11), (777, 17, 12), (2049, 40, 13), (1500, 67, 14)])
def test_random_ragged_orders_match_oracle(ctx, torch_cuda, prec, shape):
    n, d, seed = shape
    X, _ = _random_sem(seed, n, d)
    order, scores = ctx[prec].causal_order(_dev(torch_cuda, X, prec), scores=True)
    ref, ref_scores = oracle.causal_order(X, scores=True)
    assert list(order) == list(ref)
    assert scores_close(scores, ref_scores) <= 0


def test_single_variable(ctx, torch_cuda):
    X = np.arange(20, dtype=np.float32).reshape(20, 1)
    assert list(ctx["fp32"].causal_order(_dev(torch_cuda, X, "fp32"))) == [0]


def test_host_device_and_layouts_agree(ctx, torch_cuda):
    X, _ = _random_sem(21, 900, 23)
    c = ctx["fp32"]
    a = c.causal_order(_dev(torch_cuda, X, "fp32"))
    b = c.causal_order(X)                                  # host numpy, row-major
    f = c.causal_order(np.asfortranarray(X))               # host, column-major
    t = c.causal_order(_dev(torch_cuda, X.T, "fp32").t())  # device, column-major
    assert list(a) == list(b) == list(f) == list(t)
    assert list(a) == list(oracle.causal_order(X))


def test_repeated_calls_and_shape_changes(ctx, torch_cuda):
    c = ctx["mixed"]
    for seed, (n, d) in enumerate([(700, 12), (1400, 30), (700, 12), (350, 5)]):
        X, _ = _random_sem(100 + seed, n, d)
        assert list(c.causal_order(_dev(torch_cuda, X, "mixed"))) == list(oracle.causal_order(X))


# ------------------------------------------------------------- errors -------

def test_error_codes(ctx, torch_cuda):
    import paper_2403_03772_gb300 as pkg
    c = ctx["fp32"]
    st = gen.Stream(3)
    a = st.uniform(-1, 1, 400)
    b = st.laplace(1.0, 400)
    X = np.column_stack([a, 2.0 * a, b]).astype(np.float32)
    with pytest.raises(pkg.LingamError) as e:
        c.causal_order(_dev(torch_cuda, X, "fp32"))
    assert e.value.code == pkg.ERR_DEGENERATE
    X = np.column_stack([a, b]).astype(np.float32)
    X[7, 1] = np.nan
    with pytest.raises(pkg.LingamError) as e:
        c.causal_order(_dev(torch_cuda, X, "fp32"))
    assert e.value.code == pkg.ERR_NONFINITE
    X = st.uniform(-1, 1, (3, 5)).astype(np.float32)
    with pytest.raises(pkg.LingamError) as e:
        c.causal_order(_dev(torch_cuda, X, "fp32"))
    assert e.value.code == pkg.ERR_DEGENERATE
    # the context keeps working after errors
    X, _ = _random_sem(5, 500, 6)
    assert list(c.causal_order(_dev(torch_cuda, X, "fp32"))) == list(oracle.causal_order(X))


# ------------------------------------------------------------- adjacency ----

def test_adjacency_matches_oracle(ctx, torch_cuda, datasets):
    ds = datasets("cfg2")
    gold, _ = read_golden_order("cfg2")
    B = ctx["fp32"].fit_adjacency(_dev(torch_cuda, ds.X, "fp32"), gold)
    ref = oracle.fit_adjacency(ds.X, gold)
    assert np.max(np.abs(B - ref)) < B_ABS
    Bd = torch_cuda.empty((ds.d, ds.d), dtype=torch_cuda.float64, device="cuda:0")
    ctx["fp32"].fit_adjacency(_dev(torch_cuda, ds.X, "fp32"), gold, out=Bd)
    assert np.array_equal(Bd.cpu().numpy(), B)


def test_adjacency_true_order_cfg1(ctx, torch_cuda, datasets):
    ds = datasets("cfg1")
    B = ctx["fp32"].fit_adjacency(ds.X, ds.order)
    assert np.max(np.abs(B - oracle.fit_adjacency(ds.X, ds.order))) < B_ABS


def test_stats_report_the_run(ctx, torch_cuda, datasets):
    ds = datasets("cfg2")
    c = ctx["fp32"]
    c.causal_order(_dev(torch_cuda, ds.X, "fp32"))
    st = c.stats()
    assert st["total_ms"] > 0 and st["graph_nodes"] >= 7 * (ds.d - 1)
    assert st["cond_bodies"] == 0 and st["cond_nodes"] == 0   # plain graph by default


@pytest.mark.parametrize("prec", ["mixed", "fp32"])
def test_conditional_rescore_blocks_keep_the_order(torch_cuda, datasets, prec):
    """With conditional_rescore each step's re-score launches sit under a
    conditional graph node set by the select kernel; the order and the score
    history must be those of the plain graph (and the oracle's)."""
    import paper_2403_03772_gb300 as pkg
    ds = datasets("cfg2")
    gold, _ = read_golden_order("cfg2")
    X = _dev(torch_cuda, ds.X, prec)
    with pkg.Context(0, prec, conditional_rescore=True) as c:
        order, scores = c.causal_order(X, scores=True)
        st = c.stats()
        again = c.causal_order(X)
    assert list(order) == list(again) == list(gold)
    assert st["cond_bodies"] == ds.d - 1
    assert 6 * (ds.d - 1) <= st["cond_nodes"] < st["graph_nodes"]
    with pkg.Context(0, prec) as c:
        _, plain = c.causal_order(X, scores=True)
    np.testing.assert_array_equal(np.nan_to_num(scores), np.nan_to_num(plain))


@pytest.mark.parametrize("tie", [300.0, 1e7])
def test_rescore_tiers_keep_the_order(torch_cuda, datasets, tie):
    """Widened error bounds push many steps through the double-float tier
    (and, at 1e7, the double-float near-ties on to FP64); the order and the
    scores must still be the oracle's."""
    import paper_2403_03772_gb300 as pkg
    ds = datasets("cfg2")
    gold, _ = read_golden_order("cfg2")
    with pkg.Context(0, "mixed", tie_scale=tie) as c:
        order, scores = c.causal_order(_dev(torch_cuda, ds.X, "mixed"), scores=True)
        st = c.stats()
    assert list(order) == list(gold)
    assert st["df_candidates"] > 0
    if tie > 1e4:
        assert st["fp64_candidates"] > 0
    _, ref_scores = oracle.causal_order(ds.X, scores=True)
    assert scores_close(scores, ref_scores) <= 0


@pytest.mark.parametrize("prec,tie", [("mixed", 300.0), ("fp32", 100.0), ("df", 1.0)])
def test_split_sample_ranges_keep_the_order(torch_cuda, prec, tie):
    """n = 40000 cuts every high-precision work item into several sample
    ranges (partial sums added in range order); widened bounds send many
    candidates through those passes.  Order and scores stay the oracle's."""
    import paper_2403_03772_gb300 as pkg
    X, _ = _random_sem(21, 40000, 60)
    with pkg.Context(0, prec, tie_scale=tie) as c:
        order, scores = c.causal_order(_dev(torch_cuda, X, prec), scores=True)
        st = c.stats()
    ref, ref_scores = oracle.causal_order(X, scores=True)
    assert list(order) == list(ref)
    assert scores_close(scores, ref_scores) <= 0
    if prec != "df":
        assert st["df_candidates"] > 0
