"""GPU: the pair-kernel autotuner.  Every tile configuration and split
schedule it can choose must give the oracle's order; its tables round-trip
through the C ABI and the JSON cache; bad tables are refused."""
import numpy as np
import pytest

import oracle
from gpu_util import read_golden_order, scores_close

pytestmark = pytest.mark.gpu

import os as _os
import re as _re

N_CFG = int(_re.search(r"#define LINGAM_PAIR_TILES (\d+)", open(_os.path.join(
    _os.path.dirname(_os.path.dirname(_os.path.abspath(__file__))), "include", "lingam.h")).read()).group(1))


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_autotune_table_is_valid(torch_cuda, prec):
    import paper_2403_03772_gb300 as pkg
    with pkg.Context(0, prec) as c:
        t = c.autotune(5000, 300)
        assert 1 <= t["count"] <= 8 and t["precision"] == pkg.PREC[prec]
        assert t["p_max"][-1] >= 300
        assert all(0 <= x < N_CFG for x in t["tile"])
        assert all(x >= 1 for x in t["ctas_per_sm"])
        assert all(ms > 0 for ms in t["ms"])
        assert c.tuning() == t


@pytest.fixture(scope="module")
def cfg2_ref(datasets):
    ds = datasets("cfg2")
    return ds, oracle.causal_order(ds.X, scores=True)[1]


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
@pytest.mark.parametrize("tile", range(N_CFG))
@pytest.mark.parametrize("ctas", [1, 6])
def test_every_tile_gives_the_oracle_order(torch_cuda, cfg2_ref, prec, tile, ctas):
    import paper_2403_03772_gb300 as pkg
    ds, ref_scores = cfg2_ref
    gold, _ = read_golden_order("cfg2")
    with pkg.Context(0, prec) as c:
        c.set_tuning({"count": 1, "precision": pkg.PREC[prec], "p_max": [2 ** 31 - 1],
                      "tile": [tile], "ctas_per_sm": [ctas]})
        order, scores = c.causal_order(torch_cuda.as_tensor(ds.X).cuda(), scores=True)
    assert list(order) == list(gold)
    assert scores_close(scores, ref_scores) <= 0


def test_tuned_batch_matches_oracle(torch_cuda):
    import gen
    import paper_2403_03772_gb300 as pkg
    st = gen.Stream(4242)
    insts = []
    for n, d in [(900, 40), (1500, 70), (700, 33)]:
        X = st.laplace(1.0, n * d).reshape(n, d).astype(np.float32)
        X[:, 1:] += 0.5 * X[:, :-1]
        insts.append((X, None))
    with pkg.Context(0, "mixed") as c:
        c.autotune(1500, 70, instances=3)
        orders = c.causal_order_batch(insts)
    for (X, _), o in zip(insts, orders):
        assert list(o) == list(oracle.causal_order(X))


def test_cache_round_trip(torch_cuda, tmp_path):
    import paper_2403_03772_gb300 as pkg
    path = str(tmp_path / "tune.json")
    with pkg.Context(0, "mixed") as c:
        t1 = c.autotune(3000, 150, cache=path)
    with pkg.Context(0, "mixed") as c:
        t2 = c.autotune(3000, 150, cache=path)
        assert t2 == t1
        assert c.tuning() == t1


def test_bad_tables_are_refused(torch_cuda):
    import paper_2403_03772_gb300 as pkg
    with pkg.Context(0, "mixed") as c:
        good = c.tuning()
        for bad in [{"tile": [N_CFG]}, {"ctas_per_sm": [0]}, {"count": 0},
                    {"count": 2, "p_max": [100, 50], "tile": [0, 0], "ctas_per_sm": [4, 4]}]:
            t = dict(good, **bad)
            with pytest.raises(pkg.LingamError):
                c.set_tuning(t)
        assert c.tuning() == good
    with pkg.Context(0, "df") as c:
        with pytest.raises(pkg.LingamError):
            c.autotune(1000, 50)
