"""The allocation-free first-step scorer, called through the C ABI.

lingam_step_scores_noalloc exists for callers that cannot allocate device
memory while they run (code inside an allocator, plugins of applications that
own all device memory, services that ban cudaMalloc/cudaFree on their serving
path).  It keeps its scratch in a fixed array inside the library instead of a
context workspace.  These tests check that two calls in a row, each reusing
that shared array, return the first-step scores of the FP64 oracle (both
sides are FP64, so the tolerance is an FP64 one) and of the context-based
entry point lingam_step_measures (within the score tolerance the other GPU
tests use); that the error codes, the size limit and a padded row stride
behave as the header states; and that a call after the first one leaves the
device's free memory unchanged.  The file name sorts last so that a run
stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import gen
import oracle
from gpu_util import M_ABS, M_REL

pytestmark = pytest.mark.gpu

# both sides accumulate in FP64; only the summation order differs
FP64_REL = 1e-10


def _noalloc(lib, torch, X, d=None):
    """Call the entry point on the first d columns of the 2-D FP64 tensor X
    (row stride X.stride(0))."""
    n = X.shape[0]
    d = X.shape[1] if d is None else d
    M = torch.empty(d, dtype=torch.float64, device=X.device)
    stream = ctypes.c_void_p(torch.cuda.current_stream(X.device).cuda_stream)
    code = lib.lingam_step_scores_noalloc(ctypes.c_void_p(X.data_ptr()), n, d, X.stride(0),
                                          ctypes.c_void_p(M.data_ptr()), stream)
    return code, M


def _close_to_oracle(M, Xh):
    ref = oracle.search_step(Xh.astype(np.float64))["k_list"]
    scale = np.max(np.abs(ref))
    err = np.max(np.abs(M - ref))
    assert err <= FP64_REL * scale + M_ABS, (err, scale)


def test_noalloc_scores_match_oracle_and_context_entry_point_twice():
    import torch
    import paper_2403_03772_gb300 as pkg
    lib = pkg.load()
    cases = [gen.cfg2(seed=901, n=3000, d=40).X, gen.cfg1(seed=902, n=1200, d=10).X]
    with pkg.Context(0, "fp64") as ctx:
        for Xh in cases:                          # two calls in a row
            X = torch.from_numpy(Xh.astype(np.float64)).to("cuda:0")
            code, M = _noalloc(lib, torch, X)
            assert code == pkg.OK
            M = M.cpu().numpy()
            _close_to_oracle(M, Xh)
            _, M_ref = ctx.step_measures(X)
            scale = np.max(np.abs(M_ref))
            assert np.max(np.abs(M - M_ref)) <= M_REL * scale + M_ABS


def test_noalloc_at_its_size_limit_with_a_padded_row_stride():
    import torch
    import paper_2403_03772_gb300 as pkg
    lib = pkg.load()
    Xh = gen.cfg2(seed=903, n=2500, d=64).X.astype(np.float64)
    pad = torch.full((Xh.shape[0], 80), float("nan"), dtype=torch.float64, device="cuda:0")
    pad[:, :64] = torch.from_numpy(Xh)
    for _ in range(2):
        code, M = _noalloc(lib, torch, pad, d=64)   # ld = 80; the NaN padding is never read
        assert code == pkg.OK
        _close_to_oracle(M.cpu().numpy(), Xh)


def test_noalloc_error_codes_then_recovers():
    import torch
    import paper_2403_03772_gb300 as pkg
    lib = pkg.load()
    Xh = gen.cfg2(seed=904, n=1500, d=12).X.astype(np.float64)
    bad = Xh.copy()
    bad[7, 3] = np.nan
    code, _ = _noalloc(lib, torch, torch.from_numpy(bad).to("cuda:0"))
    assert code == pkg.ERR_NONFINITE
    dup = Xh.copy()
    dup[:, 5] = dup[:, 2]                          # |rho| = 1 for the pair (2, 5)
    code, _ = _noalloc(lib, torch, torch.from_numpy(dup).to("cuda:0"))
    assert code == pkg.ERR_DEGENERATE
    # the shared status word and counter start at zero again on the next call
    code, M = _noalloc(lib, torch, torch.from_numpy(Xh).to("cuda:0"))
    assert code == pkg.OK
    _close_to_oracle(M.cpu().numpy(), Xh)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    import paper_2403_03772_gb300 as pkg
    lib = pkg.load()
    X = torch.zeros((100, 65), dtype=torch.float64, device="cuda:0")
    code, _ = _noalloc(lib, torch, X)
    assert code == pkg.ERR_ARG
    code, _ = _noalloc(lib, torch, X, d=1)
    assert code == pkg.ERR_ARG


def test_noalloc_call_after_the_first_leaves_device_memory_unchanged():
    import torch
    import paper_2403_03772_gb300 as pkg
    lib = pkg.load()
    X = torch.from_numpy(gen.cfg2(seed=905, n=2000, d=30).X.astype(np.float64)).to("cuda:0")
    M = torch.empty(30, dtype=torch.float64, device="cuda:0")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call():
        return lib.lingam_step_scores_noalloc(ctypes.c_void_p(X.data_ptr()), 2000, 30, 30,
                                              ctypes.c_void_p(M.data_ptr()), stream)

    assert call() == pkg.OK                        # first call on the device loads the module
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    assert call() == pkg.OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_reserved() == reserved0
