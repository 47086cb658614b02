"""Readers for the text fixtures under tests/golden/."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def paper_bounds():
    out = {}
    with open(os.path.join(GOLDEN, "paper_bounds.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            out[parts[0]] = float(parts[1])
    return out


def element_matrices():
    out = {}
    with open(os.path.join(GOLDEN, "element_matrices_1d.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, scale, rest = line.split(None, 2)
            if name.endswith("bounds"):
                out[name] = tuple(float(v) for v in rest.split())
            else:
                out[name] = (scale, np.array([[float(v) for v in row.split()] for row in rest.split(";")]))
    return out
