"""GPU parity of VarLiNGAM (Sec. 3.2) against the FP64 oracle: VAR least
squares with intercept, DirectLiNGAM on the innovations, B0 by least squares
along the order, B_tau = (I - B0) M_tau."""
import numpy as np
import pytest

import gen
import oracle
from gpu_util import B_ABS, read_golden_order

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2403_03772_gb300 as pkg
    c = {p: pkg.Context(0, p) for p in ["fp32", "mixed"]}
    yield c
    for v in c.values():
        v.close()


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
@pytest.mark.parametrize("shape", [(3000, 6, 1, 1), (2500, 13, 1, 2), (4000, 9, 2, 3)])
def test_small_var_matches_oracle(ctx, prec, shape):
    T, d, lags, seed = shape
    vd = gen.cfg4(seed=seed, T=T, d=d, burn=200, m_density=0.3, b0_indeg=1.0)
    Xt = vd.Xt
    order, B0, Bt = ctx[prec].varlingam_fit(Xt, lags=lags)
    ro, rB0, rBt, rM, _ = oracle.varlingam(Xt, lags=lags)
    assert list(order) == list(ro)
    assert np.max(np.abs(B0 - rB0)) < B_ABS
    assert np.max(np.abs(Bt - rBt)) < B_ABS


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_cfg4_stock_shape(ctx, prec):
    vd = gen.cfg4()
    gold, dig = read_golden_order("cfg4")
    assert dig == vd.digest()
    order, B0, Bt = ctx[prec].varlingam_fit(vd.Xt, lags=1)
    assert list(order) == list(gold)
    # sampled rows of B0 and B1 against the oracle's least squares along the
    # stored oracle order
    M, E = oracle.var_fit(vd.Xt, 1)
    rows = [int(gold[k]) for k in (1, 50, 250, 486)]
    rB0 = oracle.adjacency_rows(E, gold, rows)
    assert np.max(np.abs(B0[rows] - rB0)) < B_ABS
    rB1 = M[0][rows] - rB0 @ M[0]          # rows of (I - B0) M_1
    assert np.max(np.abs(Bt[0][rows] - rB1)) < B_ABS
