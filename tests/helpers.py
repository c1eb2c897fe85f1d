"""Shared test utilities: tiny-graph generators and brute-force references (no decoder arithmetic)."""
from __future__ import annotations

import itertools
import os

import numpy as np

from paper_2508_07879_gb300 import workloads as w

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_matrix(name: str) -> np.ndarray:
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([int(x) for x in line.split()])
    return np.array(rows, dtype=np.uint8)


def random_tree_pcm(rng: np.random.Generator, n_checks: int, max_deg: int = 4) -> np.ndarray:
    """A parity-check matrix whose Tanner graph is a tree (every check has degree >= 2).

    Grown from one variable: each new check attaches to one existing variable and brings
    1..max_deg-1 fresh variables, so the graph stays connected and acyclic.
    """
    n_vars = 1
    edges = []
    for c in range(n_checks):
        anchor = int(rng.integers(0, n_vars))
        fresh = int(rng.integers(1, max_deg))
        members = [anchor] + list(range(n_vars, n_vars + fresh))
        n_vars += fresh
        edges.extend((c, v) for v in members)
    h = np.zeros((n_checks, n_vars), dtype=np.uint8)
    for c, v in edges:
        h[c, v] = 1
    perm = rng.permutation(n_vars)          # scramble variable labels
    return h[:, perm]


def all_errors(n: int) -> np.ndarray:
    """All 2^n binary vectors, shape (2^n, n)."""
    return np.array(list(itertools.product((0, 1), repeat=n)), dtype=np.uint8)


def syndrome_dense(h: np.ndarray, e: np.ndarray) -> np.ndarray:
    return (np.asarray(e, dtype=np.int64) @ np.asarray(h, dtype=np.int64).T) % 2


def brute_force_min_marginals(h: np.ndarray, s: np.ndarray, gamma: np.ndarray):
    """Exact max-product LLRs by enumeration.

    cost(e) = sum_n gamma_n e_n over all e with H e^T = s;
    L_n = min_{e_n=1} cost - min_{e_n=0} cost (+inf / -inf if one side is infeasible).
    Returns (L, min cost, number of minimisers, one minimiser).
    """
    es = all_errors(h.shape[1])
    feasible = es[(syndrome_dense(h, es) == s[None, :]).all(axis=1)]
    cost = feasible.astype(np.float64) @ gamma.astype(np.float64)
    L = np.empty(h.shape[1])
    for n in range(h.shape[1]):
        c1 = cost[feasible[:, n] == 1]
        c0 = cost[feasible[:, n] == 0]
        L[n] = (c1.min() if c1.size else np.inf) - (c0.min() if c0.size else np.inf)
    best = cost.min()
    winners = np.nonzero(np.isclose(cost, best, rtol=0, atol=1e-12))[0]
    return L, best, len(winners), feasible[winners[0]]


def csr(h: np.ndarray) -> w.CSR:
    return w.csr_from_dense(h)
