"""GPU parity at the full d=1000, n=10000 gene-expression-shaped workload, in
the launch configuration bench.py times.

The FP64 oracle cannot order this size within a test (~1e5 core-seconds), so
the checks are (a) the stored oracle order written by
tests/golden/make_golden.py, when present; (b) first-step scores M(i) of
sampled variables, which the oracle computes one by one (literal Algorithm 1
rows); (c) properties that hold at any size; (d) adjacency rows along the true
causal order against the oracle's least squares; (e) scores of sampled
variables at later steps, on the oracle's residual data replayed along the
GPU's order (Sec. 2.2), one literal Algorithm 1 row at a time.
"""
import numpy as np
import pytest

import gen
import oracle
from gpu_util import B_ABS, M_ABS, M_REL, read_golden_order

pytestmark = pytest.mark.gpu

SAMPLED = [0, 1, 137, 500, 998, 999]


@pytest.fixture(scope="module")
def cfg3(datasets):
    return datasets("cfg3")


@pytest.fixture(scope="module")
def runs(cfg3):
    import torch
    import paper_2403_03772_gb300 as pkg
    X = torch.from_numpy(cfg3.X).to("cuda:0")
    out = {}
    for prec in ["fp32", "mixed"]:
        with pkg.Context(0, prec) as c:
            order, scores = c.causal_order(X, scores=True)
            out[prec] = (order, scores, c.stats())
    return out


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_order_is_a_permutation_and_first_step_rows_match(cfg3, runs, prec):
    order, scores, _ = runs[prec]
    assert sorted(order) == list(range(cfg3.d))
    ref_rows = oracle.row_scores(cfg3.X, SAMPLED)
    row0 = scores[0]
    scale = np.max(np.abs(row0))
    assert np.all(np.abs(row0[SAMPLED] - ref_rows) <= M_REL * scale + M_ABS)
    # the chosen first variable scores at least as high as every sampled one
    m0 = order[0]
    ref_m0 = oracle.row_scores(cfg3.X, [m0])[0]
    assert ref_m0 >= np.max(ref_rows) - (M_REL * scale + M_ABS)
    # the step-0 argmax is the GPU's first variable
    assert np.argmax(row0) == m0


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_order_matches_stored_oracle_order(cfg3, runs, prec):
    gold, dig = read_golden_order("cfg3")
    if gold is None:
        pytest.skip("the d=1000 oracle order has not been stored yet")
    assert dig == cfg3.digest()
    order = runs[prec][0]
    assert list(order) == list(gold)


def test_adjacency_rows_along_true_order(cfg3):
    import torch
    import paper_2403_03772_gb300 as pkg
    X = torch.from_numpy(cfg3.X).to("cuda:0")
    with pkg.Context(0, "fp32") as c:
        B = c.fit_adjacency(X, cfg3.order)
    rows = [int(cfg3.order[k]) for k in (1, 10, 400, 999)]
    ref = oracle.adjacency_rows(cfg3.X, cfg3.order, rows)
    assert np.max(np.abs(B[rows] - ref)) < B_ABS


LATER_STEPS = (1, 200, 500)


@pytest.fixture(scope="module")
def later_rows(cfg3, runs):
    """Oracle rows at LATER_STEPS on the residual data along the mixed form's
    order (which the stored-order test pins to the oracle's)."""
    order = runs["mixed"][0]
    res = oracle.Residuals(cfg3.X, order)
    out = {}
    for t in LATER_STEPS:
        res.advance(t)
        U = res.U
        pos = sorted({0, U.size // 3, U.size // 2, U.size - 1,
                      int(np.searchsorted(U, order[t]))})
        out[t] = (U, U[pos], oracle.row_scores(res.data, pos, U=U))
    return out


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_later_step_rows_match_oracle(runs, later_rows, prec):
    order, scores, _ = runs[prec]
    assert list(order[:max(LATER_STEPS) + 1]) == list(runs["mixed"][0][:max(LATER_STEPS) + 1])
    for t, (U, vars_, ref) in later_rows.items():
        row = scores[t]
        assert np.all(np.isfinite(row[U])) and np.all(np.isnan(np.delete(row, U)))
        scale = np.max(np.abs(row[U]))
        assert np.all(np.abs(row[vars_] - ref) <= M_REL * scale + M_ABS), t
        assert int(np.nanargmax(row)) == int(order[t])
