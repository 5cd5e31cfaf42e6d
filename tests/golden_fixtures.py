"""Reader for the hand-worked fixtures under tests/golden/: '#' lines are
comments; 'key: numbers' is a vector; 'key:' followed by rows of numbers is a
matrix."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name: str) -> dict:
    out, key, rows = {}, None, []

    def flush():
        if key is not None and rows:
            out[key] = np.array(rows, dtype=np.float64)

    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            if ":" in line:
                flush()
                key, rest = (s.strip() for s in line.split(":", 1))
                rows = []
                if rest:
                    out[key] = np.array([float(x) for x in rest.split()], dtype=np.float64)
                    key = None
            else:
                rows.append([float(x) for x in line.split()])
    flush()
    return out
