"""Pins of the oracle's downstream pieces (total causal effects, the
time-unrolled VarLiNGAM graph, influence ranking, bootstrap edge statistics)
against definitions computed another way: path enumeration, impulse
propagation, hand-worked cases and counting."""
import itertools

import numpy as np
import pytest

import gen
import oracle


def _random_dag(seed, d, density=0.6):
    st = gen.Stream(seed)
    perm = st.permutation(d)
    keep = st.uniform(0.0, 1.0, d * d).reshape(d, d) < density
    w = st.signed_uniform(0.3, 1.5, d * d).reshape(d, d)
    B = np.zeros((d, d))
    for a in range(d):
        for b in range(a):
            if keep[a, b]:
                B[perm[a], perm[b]] = w[a, b]
    return B, perm


def _path_sum(B, i, j):
    """Sum over every directed path j -> ... -> i of the product of weights."""
    d = B.shape[0]
    if i == j:
        return 1.0
    total = 0.0
    # depth-first over simple paths (a DAG has no others)
    stack = [(j, 1.0)]
    while stack:
        node, w = stack.pop()
        for nxt in range(d):
            if B[nxt, node] != 0.0:
                wn = w * B[nxt, node]
                if nxt == i:
                    total += wn
                else:
                    stack.append((nxt, wn))
    return total


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_total_effects_equal_path_sums(seed):
    B, _ = _random_dag(seed, 6)
    T = oracle.total_effects(B)
    for i, j in itertools.product(range(6), range(6)):
        assert abs(T[i, j] - _path_sum(B, i, j)) < 1e-12


def test_total_effects_chain_closed_form():
    a, b, c = 0.7, -1.3, 0.4
    B = np.zeros((3, 3))
    B[1, 0], B[2, 1], B[2, 0] = a, b, c
    T = oracle.total_effects(B)
    assert abs(T[2, 0] - (c + a * b)) < 1e-15 and abs(T[1, 0] - a) < 1e-15
    assert np.allclose(np.diag(T), 1.0) and np.all(np.triu(T, 1) == 0)


def test_var_window_graph_matches_impulse_propagation():
    d = 4
    B0, _ = _random_dag(11, d)
    st = gen.Stream(12)
    B1 = st.signed_uniform(0.05, 0.4, d * d).reshape(d, d)
    A = oracle.var_window_graph(B0, B1[None])
    T = oracle.total_effects(A)
    inv0 = np.linalg.inv(np.eye(d) - B0)
    for j in range(d):
        e = np.zeros(d)
        e[j] = 1.0
        x_prev = inv0 @ e                 # shock at t-1 propagates within slice t-1 ...
        x_now = inv0 @ (B1 @ x_prev)      # ... then through B1 and within slice t
        assert np.allclose(T[:d, j], x_prev, atol=1e-13)
        assert np.allclose(T[d:, j], x_now, atol=1e-13)
        assert np.allclose(T[:d, d + j], 0.0)   # the future does not act on the past


def test_influence_and_top_k_hand_case():
    T = np.array([[1.0, 0.0, 0.0],
                  [-2.0, 1.0, 0.0],
                  [0.5, 3.0, 1.0]])
    ex, rc = oracle.influence(T)
    assert list(ex) == [2.5, 3.0, 0.0] and list(rc) == [0.0, 2.0, 3.5]
    assert list(oracle.top_k(ex, 2)) == [1, 0]
    assert list(oracle.top_k(np.array([1.0, 2.0, 2.0, 0.5]), 3)) == [1, 2, 0]


def test_bootstrap_edge_stats_counts():
    Bs = np.zeros((4, 2, 2))
    Bs[0, 1, 0] = 0.5
    Bs[1, 1, 0] = -0.05
    Bs[2, 1, 0] = 0.2
    Bs[3, 0, 1] = 1.0
    prob, mean = oracle.bootstrap_edge_stats(Bs, threshold=0.1)
    assert prob[1, 0] == 0.5 and prob[0, 1] == 0.25 and prob[0, 0] == 0.0
    assert abs(mean[1, 0] - 0.1625) < 1e-15 and mean[0, 1] == 0.25
