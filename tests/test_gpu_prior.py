"""GPU parity of the ordering under prior ancestry knowledge: the CUDA path
(selection restricted on the device) against the FP64 oracle on the same
inputs and knowledge, in every precision form and in a batch; forced orders,
contradictions and shape mismatches."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

PRECS = ["fp32", "mixed", "df", "fp64"]


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def _dev(torch, X, prec):
    dt = torch.float64 if prec == "fp64" else torch.float32
    return torch.as_tensor(np.asarray(X), dtype=dt).to("cuda:0")


@pytest.fixture(scope="module")
def case():
    ds = gen.cfg2(seed=4711, n=3000, d=40)
    pk = gen.prior_from_dag(gen.Stream(4712), ds.B, reveal=0.3)
    ref = oracle.causal_order(ds.X, prior=pk)
    return ds, pk, ref


@pytest.mark.parametrize("prec", PRECS)
def test_partial_knowledge_matches_oracle(torch_cuda, case, prec):
    import paper_2403_03772_gb300 as pkg
    ds, pk, ref = case
    assert list(ref) != list(oracle.causal_order(ds.X))   # the knowledge matters here
    with pkg.Context(0, prec) as c:
        c.set_prior_knowledge(pk)
        order = c.causal_order(_dev(torch_cuda, ds.X, prec))
        assert list(order) == list(ref)
        c.set_prior_knowledge(None)
        assert list(c.causal_order(_dev(torch_cuda, ds.X, prec))) == list(oracle.causal_order(ds.X))


def test_complete_knowledge_forces_the_order(torch_cuda):
    import paper_2403_03772_gb300 as pkg
    d = 36
    st = gen.Stream(77)
    X = st.laplace(1.0, 2000 * d).reshape(2000, d).astype(np.float32)
    pi = st.permutation(d)
    pk = np.zeros((d, d), dtype=np.int8)
    for a in range(d):
        pk[pi[a + 1:], pi[a]] = 1
    np.fill_diagonal(pk, -1)
    with pkg.Context(0, "mixed") as c:
        c.set_prior_knowledge(pk)
        assert list(c.causal_order(_dev(torch_cuda, X, "mixed"))) == list(pi)


def test_batch_with_knowledge_matches_oracle(torch_cuda, case):
    import paper_2403_03772_gb300 as pkg
    ds, pk, _ = case
    st = gen.Stream(4713)
    insts = [(ds.X, None)] + [(ds.X, st.integers(0, ds.n - 1, ds.n).astype(np.int32))
                              for _ in range(2)]
    with pkg.Context(0, "mixed") as c:
        c.set_prior_knowledge(pk)
        orders = c.causal_order_batch([(torch_cuda.as_tensor(X).cuda(), r) for X, r in insts])
    for (X, r), o in zip(insts, orders):
        Xr = X if r is None else X[r]
        assert list(o) == list(oracle.causal_order(Xr, prior=pk))


def test_contradiction_and_mismatch_are_refused(torch_cuda, case):
    import paper_2403_03772_gb300 as pkg
    ds, pk, _ = case
    with pkg.Context(0, "mixed") as c:
        c.set_prior_knowledge(pk[:10, :10])
        with pytest.raises(pkg.LingamError):
            c.causal_order(_dev(torch_cuda, ds.X, "mixed"))        # d = 40 against 10
        bad = -np.ones((40, 40), dtype=np.int8)
        bad[:, :] = 1                                              # everyone has an ancestor
        np.fill_diagonal(bad, -1)
        c.set_prior_knowledge(bad)
        with pytest.raises(pkg.LingamError):
            c.causal_order(_dev(torch_cuda, ds.X, "mixed"))
        with pytest.raises(pkg.LingamError):
            c.set_prior_knowledge(np.full((40, 40), 3, dtype=np.int8))
        c.set_prior_knowledge(None)
        assert list(c.causal_order(_dev(torch_cuda, ds.X, "mixed"))) == list(oracle.causal_order(ds.X))
