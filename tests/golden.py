"""Readers for the small text fixtures under tests/golden/ (each file cites its source)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def philox_kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            ctr, key, out = (part.split() for part in line.split("|"))
            rows.append(tuple(np.array([int(v, 16) for v in part], dtype=np.uint32)
                              for part in (ctr, key, out)))
    return rows
