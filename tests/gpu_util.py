"""Helpers shared by the GPU parity tests (tolerances stated in one place)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

# Per-step scores M(i): |dM(i)| <= 1e-4 max_k |M(k)| + 1e-12 (relative to the
# step's scale, because the exogenous variable's M is ~0).
M_REL = 1e-4
M_ABS = 1e-12
# Adjacency: absolute.
B_ABS = 1e-5


def read_golden_order(name):
    """(order, digest) from tests/golden/<name>_order.txt, or (None, None)."""
    path = os.path.join(GOLDEN, f"{name}_order.txt")
    if not os.path.exists(path):
        return None, None
    digest = None
    order = None
    for line in open(path):
        if line.startswith("# data-sha256-16:"):
            digest = line.split(":")[1].strip()
        elif not line.startswith("#") and line.strip():
            order = np.array([int(v) for v in line.split()], dtype=np.int32)
    return order, digest


def read_cfg5_golden():
    path = os.path.join(GOLDEN, "cfg5_orders.txt")
    out = {}
    if not os.path.exists(path):
        return out
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        head, tail = line.split(":")
        k, name, dig = head.split()
        out[int(k)] = (name, dig, np.array([int(v) for v in tail.split()], dtype=np.int32))
    return out


class ScoreCheck(float):
    """Max violation of the per-step score tolerance (<= 0 means pass); the
    repr names the worst step."""

    def __new__(cls, value, info):
        obj = float.__new__(cls, value)
        obj.info = info
        return obj

    def __repr__(self):
        return f"{float(self):.3e} ({self.info})"


def scores_close(gpu, ref):
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(gpu))
    scale = np.nanmax(np.abs(np.where(fin, ref, np.nan)), axis=1, keepdims=True)
    scale = np.where(np.isfinite(scale), scale, 0.0)
    err = np.abs(np.where(fin, gpu - ref, 0.0))
    viol = err - (M_REL * scale + M_ABS)
    t, i = np.unravel_index(np.argmax(viol), viol.shape)
    p = int(fin[t].sum())
    info = (f"step {t} (p={p}) var {i}: gpu {gpu[t, i]:.9e} ref {ref[t, i]:.9e} "
            f"max|M| {scale[t, 0]:.3e}")
    return ScoreCheck(float(viol[t, i]), info)
