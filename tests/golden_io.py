"""Reader for the small text fixtures under tests/golden/."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_lp(name):
    """Parse lines `A ...`, `b ...`, `c ...`, `z v`, `x ...`, `y ...`, `cycle k`."""
    rows, out = [], {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            v = [float(t) for t in vals]
            if key == "A":
                rows.append(v)
            else:
                out[key] = np.array(v) if len(v) > 1 or key in "bcxy" else v[0]
    out["A"] = np.array(rows)
    return out


def read_table(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [[float(t) for t in line.split()] for line in f
                if line.strip() and not line.startswith("#")]
