"""bench.py's host-side contract pieces that need no GPU: the recorded DRAM
traffic of the pair kernel is reported only for the sources and tile it was
measured on, the work count matches its closed form, and the count of
launched kernels leaves out the conditional re-score blocks that do not run."""
import copy

import bench
import gen


def _sources_hash(rec):
    import hashlib
    import os
    root = os.path.dirname(os.path.abspath(bench.__file__))
    blob = b"".join(open(os.path.join(root, f), "rb").read() for f in rec["sources"])
    return hashlib.sha256(blob).hexdigest()


def test_traffic_is_reported_only_for_the_measured_sources_and_tile():
    rec = bench.PAIR_TRAFFIC
    saved = copy.deepcopy(rec)
    try:
        if _sources_hash(rec) != rec["sha256"]:
            # the kernel changed since the capture: nothing is reported
            assert bench.pair_traffic([rec["tile"]]) is None
            rec["sha256"] = _sources_hash(rec)   # check the gating on a current record
        assert bench.pair_traffic([13, 13, 13, 15, rec["tile"]]) == rec["bytes_per_launch"]
        other = (rec["tile"] + 1) % 16
        assert bench.pair_traffic([rec["tile"], other]) is None
        assert bench.pair_traffic([]) is None
        rec["sha256"] = "0" * 64            # the kernel source changed since the capture
        assert bench.pair_traffic([rec["tile"]]) is None
        rec["sources"] = rec["sources"] + ["no/such/file.cu"]
        assert bench.pair_traffic([rec["tile"]]) is None
    finally:
        bench.PAIR_TRAFFIC.clear()
        bench.PAIR_TRAFFIC.update(saved)


def test_work_count_is_the_sum_over_steps():
    for d, n in [(10, 1000), (100, 5000), (1000, 10000)]:
        assert gen.residual_samples(d, n) == n * sum(p * (p - 1) for p in range(2, d + 1))


def test_oracle_errors_read_the_stored_values():
    """The bench states each GPU form's error against stored oracle values
    (it never runs the oracle there): equal values give zero error, a moved
    score or coefficient shows up, and data with another digest is not
    compared."""
    import numpy as np
    order, digest = bench.golden_order("cfg2")
    rows = bench.golden_rows("cfg2", digest)
    assert order is not None and rows is not None
    d = len(order)
    M0 = np.zeros(d)
    M0[rows["step0_vars"]] = rows["step0_M"]
    B = np.zeros((d, d))
    B[rows["B_vars"]] = rows["B_rows"]
    e = bench.oracle_errors("cfg2", digest, order, M0, B)
    assert e == {"order_equals_oracle": True, "max_rel_dM_step0": 0.0, "max_abs_dB": 0.0}
    M1 = M0.copy()
    M1[rows["step0_vars"][3]] += 1e-3 * np.max(np.abs(M0))
    B1 = B.copy()
    B1[rows["B_vars"][0], 0] += 2e-5
    swapped = list(order)
    swapped[0], swapped[1] = swapped[1], swapped[0]
    e = bench.oracle_errors("cfg2", digest, swapped, M1, B1)
    assert e["order_equals_oracle"] is False
    assert abs(e["max_rel_dM_step0"] - 1e-3) < 1e-9
    assert abs(e["max_abs_dB"] - 2e-5) < 1e-12
    assert bench.golden_rows("cfg2", "0" * 16) is None
    assert bench.oracle_errors("cfg2", "0" * 16, order)["order_equals_oracle"] is None


def test_launched_kernels_count_conditional_blocks_only_where_they_run():
    # plain graph: every kernel node runs
    assert bench.launched_nodes({"graph_nodes": 13, "cond_nodes": 0, "cond_bodies": 0,
                                 "refined_steps": 5}) == 13
    # 10 steps with a conditional block of 7 kernel nodes each; 4 steps left
    # candidates, so only their blocks run
    st = {"graph_nodes": 10 * 14, "cond_nodes": 10 * 7, "cond_bodies": 10, "refined_steps": 4}
    assert bench.launched_nodes(st) == 10 * 7 + 4 * 7
