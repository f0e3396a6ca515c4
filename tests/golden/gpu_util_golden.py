"""Reader of the stored order files (shared by the golden writer and bench.py;
reads text only)."""
import numpy as np


def read_order(path):
    """(order, data digest) of a stored order file, or (None, None)."""
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None, None
    digest = order = None
    for line in lines:
        if line.startswith("# data-sha256-16:"):
            digest = line.split(":")[1].strip()
        elif not line.startswith("#") and line.strip():
            order = np.array([int(v) for v in line.split()], dtype=np.int32)
    return order, digest
