"""Reader for the hand-worked examples under tests/golden/."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    out = {"L": [], "U": []}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, *vals = line.split()
            if key in ("L", "U"):
                out[key].append((int(vals[0]), int(vals[1]), float(vals[2])))
            elif key in ("n", "rejected"):
                out[key] = int(vals[0])
            elif key == "eps":
                out[key] = float(vals[0])
            elif key == "prefer" and vals == ["none"]:
                out[key] = None
            elif key in ("Ap", "Ai", "Q", "prefer", "piv", "etree_parent", "restart_set"):
                out[key] = np.array([int(v) for v in vals], dtype=np.int32)
            else:
                out[key] = np.array([float(v) for v in vals])
    return out


def dense_lu(g):
    n = g["n"]
    L = np.eye(n)
    U = np.zeros((n, n))
    for r, c, v in g["L"]:
        L[r, c] = v
    for r, c, v in g["U"]:
        U[r, c] = v
    return L, U
