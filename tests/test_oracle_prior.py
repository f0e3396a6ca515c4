"""Pins of the oracle's ordering under prior ancestry knowledge (a reading:
the paper has none).  The rule -- a variable may come next only if no
remaining variable is a known ancestor of it, and only the known-exogenous
remaining variables may come next when there are any -- is checked through
what it forces: complete knowledge fixes the order, ancestry knowledge makes
any data's order topological for that DAG, unknown entries change nothing,
and contradictory knowledge is refused."""
import numpy as np
import pytest

import gen
import oracle


def _independent(seed, n, d):
    st = gen.Stream(seed)
    return st.laplace(1.0, n * d).reshape(n, d)


def test_unknown_everywhere_is_no_knowledge():
    ds = gen.cfg1(n=800, d=8)
    pk = -np.ones((8, 8), dtype=np.int8)
    o1, s1 = oracle.causal_order(ds.X, scores=True)
    o2, s2 = oracle.causal_order(ds.X, scores=True, prior=pk)
    assert list(o1) == list(o2)
    assert np.array_equal(np.isnan(s1), np.isnan(s2))
    assert np.array_equal(s1[~np.isnan(s1)], s2[~np.isnan(s2)])


def test_complete_knowledge_fixes_the_order():
    d = 7
    X = _independent(11, 600, d)
    pi = np.array([4, 0, 6, 2, 5, 1, 3])
    pk = np.zeros((d, d), dtype=np.int8)
    for a in range(d):
        for b in range(a + 1, d):
            pk[pi[b], pi[a]] = 1      # pi[a] is an ancestor of pi[b]
    np.fill_diagonal(pk, -1)
    assert list(oracle.causal_order(X, prior=pk)) == list(pi)


def test_ancestry_knowledge_makes_any_order_topological():
    # data without causal structure, knowledge of a random DAG's ancestry:
    # every ancestor must come before its descendants
    d = 9
    st = gen.Stream(5)
    B, _ = gen._random_dag(st, d, 0.35, 0.5, 2.0)
    anc = gen.ancestors(B)
    pk = np.where(anc, 1, -1).astype(np.int8)
    X = _independent(6, 700, d)
    order = oracle.causal_order(X, prior=pk)
    assert gen.is_topological(order, anc.astype(np.float64))
    assert not gen.is_topological(oracle.causal_order(X), anc.astype(np.float64))


def test_known_exogenous_variable_comes_first():
    ds = gen.cfg1(n=800, d=8)
    free = oracle.causal_order(ds.X)
    k = int(free[-1])                 # the variable the data puts last
    pk = -np.ones((8, 8), dtype=np.int8)
    pk[k, :] = 0                      # nothing is an ancestor of x_k
    pk[k, k] = -1
    order = oracle.causal_order(ds.X, prior=pk)
    assert order[0] == k
    assert sorted(order) == list(range(8))


def test_contradictory_knowledge_is_refused():
    X = _independent(3, 500, 3)
    pk = -np.ones((3, 3), dtype=np.int8)
    pk[0, 1] = pk[1, 0] = 1           # x1 before x0 and x0 before x1
    pk[0, 2] = pk[1, 2] = 0
    pk[2, 0] = pk[2, 1] = 1           # ... and x2 after both: no variable may start
    with pytest.raises(oracle.OracleError):
        oracle.causal_order(X, prior=pk)
    with pytest.raises(oracle.OracleError):
        oracle.causal_order(X, prior=np.full((3, 3), 2, dtype=np.int8))


def test_known_parents_true_dag_recovers_true_order_class():
    ds = gen.cfg1(n=2000, d=10)
    pk = gen.prior_from_dag(gen.Stream(9), ds.B, reveal=0.4)
    order = oracle.causal_order(ds.X, prior=pk)
    assert gen.is_topological(order, ds.B)
