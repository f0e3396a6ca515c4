"""A bounded device wait that runs out, through the C ABI.

lingam_set_input_gate makes the single-instance calls wait on the device
until a flag is set before they read their input.  Here the flag is never
set, so the wait must end by its limit: the kernel records a timeout and
returns, the call fails with ERR_TIMEOUT, and the same context then orders
the data correctly once the flag is released and again without a gate.  No
GPU fault is involved: the wait is on an ordinary flag in device (or mapped
host) memory that nothing writes.
"""
import time

import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["mixed", "fp32"])
def test_unreleased_gate_times_out_and_the_context_recovers(prec):
    import torch
    import paper_2403_03772_gb300 as pkg
    ds = gen.cfg2(seed=931, n=3000, d=48)
    ref = oracle.causal_order(ds.X)
    X = torch.from_numpy(ds.X).to("cuda:0")
    flag = torch.zeros(1, dtype=torch.int32, device="cuda:0")
    with pkg.Context(0, prec) as c:
        assert list(c.causal_order(X)) == list(ref)          # plan and graph exist
        c.set_input_gate(flag, 0.05)
        t0 = time.perf_counter()
        with pytest.raises(pkg.LingamError) as e:
            c.causal_order(X)
        dt = time.perf_counter() - t0
        assert e.value.code == pkg.ERR_TIMEOUT
        assert 0.05 <= dt < 10.0
        # the same context works again: once the flag is released ...
        flag.fill_(1)
        torch.cuda.synchronize()
        assert list(c.causal_order(X)) == list(ref)
        # ... and with the gate removed
        flag.zero_()
        c.set_input_gate(None)
        assert list(c.causal_order(X)) == list(ref)


def test_gate_on_mapped_host_memory_and_bad_gates():
    import torch
    import paper_2403_03772_gb300 as pkg
    ds = gen.cfg2(seed=932, n=2000, d=20)
    ref = oracle.causal_order(ds.X)
    X = torch.from_numpy(ds.X).to("cuda:0")
    host = torch.zeros(4, dtype=torch.int32).pin_memory()   # pinned: mapped under UVA
    with pkg.Context(0, "mixed") as c:
        c.set_input_gate(host.data_ptr(), 0.05)
        with pytest.raises(pkg.LingamError) as e:
            c.causal_order(X)
        assert e.value.code == pkg.ERR_TIMEOUT
        host[0] = 7                                         # the host releases the input
        assert list(c.causal_order(X)) == list(ref)
        _, M = c.step_measures(X)
        assert np.argmax(M) == ref[0]
        c.set_input_gate(None)
        dev = torch.zeros(2, dtype=torch.int32, device="cuda:0")
        for bad in [(dev.data_ptr() + 2, 1.0), (dev.data_ptr(), 0.0), (dev.data_ptr(), 61.0)]:
            with pytest.raises(pkg.LingamError) as e:
                c.set_input_gate(*bad)
            assert e.value.code == pkg.ERR_ARG
        plain = np.zeros(4, dtype=np.uint32)                  # pageable host memory
        with pytest.raises(pkg.LingamError) as e:
            c.set_input_gate(plain.ctypes.data, 1.0)
        assert e.value.code == pkg.ERR_ARG
        assert list(c.causal_order(X)) == list(ref)
