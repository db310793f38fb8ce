"""Test helpers: load oracle-written golden tables and paper constants."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def gram_golden(n_match, n_cont):
    return np.loadtxt(os.path.join(GOLDEN, f"fc_gram_d{n_match}_c{n_cont}.txt"))


def paper_constants():
    out = {}
    with open(os.path.join(GOLDEN, "paper_constants.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            parts = line.split()
            vals = []
            for p in parts[1:]:
                try:
                    vals.append(float(p))
                except ValueError:
                    break
            out[parts[0]] = np.array(vals)
    return out
