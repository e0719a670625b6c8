"""Reader for the small text fixtures under tests/golden/ ("key: v v | v v" lines)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, val = line.split(":", 1)
            rows = [r.split() for r in val.split("|")]
            out[key.strip()] = rows
    return out


def arr(rows, dtype=np.float64):
    if len(rows) == 1:
        return np.array([float(v) for v in rows[0]], dtype=dtype)
    return np.array([[float(v) for v in r] for r in rows], dtype=dtype)
