"""The seeded generators: stable bytes, valid structure, platform-free arithmetic."""
import math

import numpy as np

import gen


def test_series_log_matches_libm():
    x = np.concatenate([np.linspace(1e-300, 1.0, 1001)[1:], [1e-308, 0.5, 1.0, 2.0, 1e300, 3.7]])
    assert np.max(np.abs(gen.series_log(x) - np.log(x)) / np.maximum(1.0, np.abs(np.log(x)))) < 4e-16


def test_streams_are_deterministic():
    a = gen.Stream(5).normal(1000)
    b = gen.Stream(5).normal(1000)
    assert np.array_equal(a, b)
    z = gen.Stream(6).normal(400000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01 and abs((z ** 4).mean() - 3) < 0.05


def test_workload_shapes_and_true_orders(datasets):
    for name, (n, d) in {"cfg1": (1000, 10), "cfg2": (5000, 100)}.items():
        ds = datasets(name)
        assert ds.X.shape == (n, d) and ds.X.dtype == np.float32
        assert gen.is_topological(ds.order, ds.B)
        assert sorted(ds.order) == list(range(d))
    assert gen.cfg1().digest() == datasets("cfg1").digest()


def test_cfg3_scale_free_structure():
    ds = gen.cfg3(n=50, d=300)
    indeg = (ds.B != 0).sum(axis=1)
    assert sorted(np.bincount(indeg)) and indeg.max() == 2 and (indeg == 0).sum() == 1
    assert gen.is_topological(ds.order, ds.B)
    outdeg = (ds.B != 0).sum(axis=0)
    assert outdeg.max() > 10            # preferential attachment grows hubs


def test_cfg4_var_is_stable_and_sparse():
    vd = gen.cfg4(T=400, d=60, burn=100)
    rad = np.max(np.abs(np.linalg.eigvals(vd.M1)))
    assert abs(rad - 0.5) < 1e-6
    assert np.isfinite(vd.Xt).all() and vd.Xt.shape == (400, 60)
    assert gen.is_topological(vd.order, vd.B0)


def test_cfg5_instances():
    insts = gen.cfg5(n_resamples=3, n_uneven=4)
    assert len(insts) == 7
    assert insts[0].rows.shape == (4000,) and insts[0].rows.max() < 4000
    for inst in insts[3:]:
        n, d = inst.X.shape
        assert 50 <= d <= 400 and 1000 <= n <= 8000


def test_residual_sample_count():
    for d, n in [(2, 3), (10, 1000), (37, 11)]:
        assert gen.residual_samples(d, n) == n * sum(p * (p - 1) for p in range(2, d + 1))
    assert gen.residual_samples(1000, 10000) == 3_333_330_000_000
