"""Weight vectors with the dynamic range and signs of the paper's fitted weights
(Table 2, Sec. 5: 3.91e-13 s per exponentiation next to a 1.29e-4 s constant, two
negative weights), for tests of the FP64-accurate paths."""
import os

import numpy as np

GOLD = os.path.join(os.path.dirname(__file__), "golden", "table2_fury_weights.txt")


def table2_rows():
    rows = []
    for line in open(GOLD):
        if line.strip() and not line.startswith("#"):
            name, w, col = line.split()
            rows.append((name, float(w), int(col)))
    return rows


def table2_weights(n_models: int = 1, seed: int = 0) -> np.ndarray:
    """[n_models][32]: model 0 puts each Table 2 weight on its column (the stride-3
    100% row fills column 18 after the stride-2 row, so the later value stands) and
    the columns Table 2 does not name get weights log-uniform over its positive range;
    further models scale each weight by a seeded factor in [0.5, 2], signs kept."""
    rng = np.random.default_rng(seed)
    w = np.exp(rng.uniform(np.log(3.91e-13), np.log(3.55e-10), size=32))
    for _, x, c in table2_rows():
        w[c] = x
    W = np.tile(w, (n_models, 1))
    if n_models > 1:
        W[1:] *= rng.uniform(0.5, 2.0, size=(n_models - 1, 32))
    return W


def small_weight_counts(R: int, seed: int, k: int = 32) -> np.ndarray:
    """int64 [R][k] feature rows whose time sits on the columns with the smallest
    Table 2 weights: up to 1e13 exponentiations, multiplications and stride-2 loads,
    next to small counts elsewhere and the constant 1."""
    rng = np.random.default_rng(seed)
    F = rng.integers(0, 1000, size=(R, k), dtype=np.int64)
    F[:, 0] = 1
    for c in (6, 4, 18):
        F[:, c] = np.exp(rng.uniform(np.log(1e9), np.log(1e13), size=R)).astype(np.int64)
    F[::7, 6] = 10 ** 13                           # a prediction almost all exponentiation
    return F
