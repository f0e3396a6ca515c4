"""GPU: the per-entry error bounds that drive the re-score tiers hold with
margin.  I(i, j) of every first-step pair from each form is compared with the
FP64 form on the same device input; the bounds are the ones the library uses
(FP32 plain 5e-6, fast 1.5e-6, double-float 1e-12), and each must stay at
least 2x (double-float: 10x) above the largest error seen.  The FP64 form
itself is pinned to the oracle in test_gpu_order.py."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

BOUND = {"fp32": 5.0e-6, "mixed": 1.5e-6, "df": 1.0e-12}
MARGIN = {"fp32": 2.0, "mixed": 2.0, "df": 10.0}


@pytest.mark.parametrize("name", ["cfg3", "cfg2", "long_n"])
def test_error_bounds_hold_with_margin(datasets, name):
    import torch
    import paper_2403_03772_gb300 as pkg
    ds = datasets(name)
    X32 = torch.from_numpy(ds.X).to("cuda:0")
    with pkg.Context(0, "fp64") as c:
        I64, _ = c.step_measures(X32.double())
    worst = {}
    for prec in ["fp32", "mixed", "df"]:
        with pkg.Context(0, prec) as c:
            I, _ = c.step_measures(X32)
        worst[prec] = float(np.max(np.abs(I - I64)))
    for prec, err in worst.items():
        assert err * MARGIN[prec] <= BOUND[prec], (prec, err, worst)
