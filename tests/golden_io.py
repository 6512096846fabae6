"""Readers for the hand-transcribed paper fixtures under tests/golden/."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def paper_matrices():
    mats, name, rows = {}, None, []
    with open(os.path.join(GOLDEN, "paper_factors.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            if line.startswith("["):
                if name:
                    mats[name] = np.array(rows, np.int64)
                name, rows = line.strip("[]"), []
            else:
                rows.append([int(v) for v in line.split()])
    mats[name] = np.array(rows, np.int64)
    return mats


def paper_numbers():
    out = {}
    with open(os.path.join(GOLDEN, "paper_numbers.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, *vals = line.split()
            out.setdefault(key, []).append([float(v) for v in vals])
    return out
