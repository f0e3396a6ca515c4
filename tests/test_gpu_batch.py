"""GPU parity of the batched form (bootstrap resamples + uneven instances in
one graph) against the FP64 oracle, per instance."""
import numpy as np
import pytest

import gen
import oracle
from gpu_util import B_ABS, read_cfg5_golden

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2403_03772_gb300 as pkg
    c = {p: pkg.Context(0, p) for p in ["fp32", "mixed", "df"]}
    yield c
    for v in c.values():
        v.close()


def _small_batch():
    base = gen.cfg2(seed=501, n=1500, d=24)
    st = gen.Stream(502)
    insts = []
    for r in range(5):
        insts.append((base.X, st.integers(0, base.n - 1, base.n).astype(np.int32)))
    for k, (n, d) in enumerate([(700, 9), (2100, 33), (1200, 17), (3000, 40), (900, 2)]):
        insts.append((gen.cfg2(seed=600 + k, n=n, d=d).X, None))
    insts.append((gen.Stream(610).laplace(1.0, 500).reshape(500, 1).astype(np.float32), None))
    return insts


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_small_batch_matches_oracle(ctx, prec):
    insts = _small_batch()
    orders = ctx[prec].causal_order_batch(insts)
    for (X, rows), o in zip(insts, orders):
        data = X if rows is None else X[rows]
        assert list(o) == list(oracle.causal_order(data))


def test_batch_equals_single_calls(ctx):
    insts = _small_batch()
    c = ctx["mixed"]
    orders = c.causal_order_batch(insts)
    for (X, rows), o in zip(insts, orders):
        data = X if rows is None else X[rows]
        assert list(o) == list(c.causal_order(np.ascontiguousarray(data)))


def test_batch_adjacency(ctx):
    insts = _small_batch()[:8]
    orders, Bs = ctx["fp32"].causal_order_batch(insts, adjacency=True)
    for (X, rows), o, B in zip(insts, orders, Bs):
        data = X if rows is None else X[rows]
        assert np.max(np.abs(B - oracle.fit_adjacency(data, o))) < B_ABS


def test_batch_reports_the_failing_instance(ctx):
    import paper_2403_03772_gb300 as pkg
    insts = _small_batch()[:6]
    bad = insts[5][0].copy()
    bad[3, 2] = np.inf
    insts[5] = (bad, None)
    with pytest.raises(pkg.LingamError) as e:
        ctx["fp32"].causal_order_batch(insts)
    assert e.value.code == pkg.ERR_NONFINITE and "instance 5" in str(e.value)


@pytest.mark.parametrize("prec", ["mixed"])
def test_cfg5_bootstrap_batch(ctx, prec):
    insts = gen.cfg5()
    gold = read_cfg5_golden()
    batch = [(inst.X, inst.rows) for inst in insts]
    orders = ctx[prec].causal_order_batch(batch)
    assert len(orders) == 192
    for inst, o in zip(insts, orders):
        assert sorted(o) == list(range(inst.X.shape[1]))
    if not gold:
        pytest.skip("stored cfg5 oracle orders are not present")
    import hashlib
    for k, (name, dig, order) in gold.items():
        data = insts[k].data()
        assert hashlib.sha256(np.ascontiguousarray(data).tobytes()).hexdigest()[:16] == dig
        assert list(orders[k]) == list(order), name
