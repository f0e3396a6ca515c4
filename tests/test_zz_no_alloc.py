"""The allocation-free first-step scorer, called through the C ABI.

lingam_step_scores_noalloc exists for callers that cannot allocate device
memory while they run (code inside an allocator, plugins of applications that
own all device memory, services that ban cudaMalloc/cudaFree on their serving
path).  It keeps its scratch in a fixed array inside the library instead of a
context workspace.  This test checks that two calls in a row, each reusing
that shared array, return the same first-step scores as the context-based
entry point lingam_step_measures (FP64 context), within the score tolerance
the other GPU tests use.  The file name sorts last so that a run stopping at
the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import gen
from gpu_util import M_ABS, M_REL

pytestmark = pytest.mark.gpu


def _noalloc(lib, torch, X):
    n, d = X.shape
    M = torch.empty(d, dtype=torch.float64, device=X.device)
    stream = ctypes.c_void_p(torch.cuda.current_stream(X.device).cuda_stream)
    code = lib.lingam_step_scores_noalloc(ctypes.c_void_p(X.data_ptr()), n, d, d,
                                          ctypes.c_void_p(M.data_ptr()), stream)
    return code, M


def test_noalloc_scores_match_context_entry_point_twice():
    import torch
    import paper_2403_03772_gb300 as pkg
    lib = pkg.load()
    cases = [gen.cfg2(seed=901, n=3000, d=40).X, gen.cfg1(seed=902, n=1200, d=10).X]
    with pkg.Context(0, "fp64") as ctx:
        for Xh in cases:                          # two calls in a row
            X = torch.from_numpy(Xh.astype(np.float64)).to("cuda:0")
            code, M = _noalloc(lib, torch, X)
            assert code == pkg.OK
            _, M_ref = ctx.step_measures(X)
            scale = np.max(np.abs(M_ref))
            assert np.max(np.abs(M.cpu().numpy() - M_ref)) <= M_REL * scale + M_ABS


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    import paper_2403_03772_gb300 as pkg
    lib = pkg.load()
    X = torch.zeros((100, 65), dtype=torch.float64, device="cuda:0")
    code, _ = _noalloc(lib, torch, X)
    assert code == pkg.ERR_ARG
