"""Oracle for the Hamiltonian partitioning of Section IV-C (test infrastructure only).

TEST INFRASTRUCTURE ONLY: imported by the tests, never by the product.  Plain,
slow, obviously correct Python loops; graphs here have at most 30 nodes.

* interaction_graph -- Eq. 9: w_ij = sum of |c_k| over the terms whose Pauli
  letters on qubits i and j are both non-identity (i != j; no self-loops).
* modularity -- Eq. 10 with a resolution gamma (Section VI-C's Louvain
  resolution; gamma = 1 is Eq. 10 as printed):
  Q = 1/(2m) sum_ij [w_ij - gamma k_i k_j / (2m)] delta(c_i, c_j).
* louvain -- the Louvain method (Blondel et al.) that Section IV-C names: local
  moving of nodes between neighbouring communities while the modularity gain is
  positive, then aggregation of communities into super-nodes, repeated until a
  level moves nothing.  Readings where the paper is silent (its Louvain is a
  library call): nodes are visited in ascending order; a node moves only when
  the best gain beats staying by more than a relative 1e-12; near-equal gains go
  to the lowest community label; communities are relabelled by their lowest
  member.
* merge_small -- blocks below S_min are merged with a neighbour (Section IV-C):
  the smallest block (lowest label on ties) joins the block it shares the most
  weight with (lowest label on ties), or, with no shared weight, the smallest
  other block; repeated until every block has at least S_min qubits or one
  block is left.
* block_masks -- theta_{B_i} of Section IV-D: every layer's angle of every
  qubit of B_i (p = r n + q).
"""
from __future__ import annotations

from typing import List, Sequence

import numpy as np

REL_TIE = 1e-12


def interaction_graph(n: int, strings: Sequence[str], coeffs) -> np.ndarray:
    w = np.zeros((n, n))
    for s, c in zip(strings, coeffs):
        support = [q for q in range(n) if s[q] != "I"]
        for i in support:
            for j in support:
                if i != j:
                    w[i, j] += abs(float(c))
    return w


def modularity(w: np.ndarray, labels: Sequence[int], gamma: float = 1.0) -> float:
    n = w.shape[0]
    two_m = float(sum(w[i, j] for i in range(n) for j in range(n)))
    if two_m == 0.0:
        return 0.0
    k = [float(sum(w[i, j] for j in range(n))) for i in range(n)]
    q = 0.0
    for i in range(n):
        for j in range(n):
            if labels[i] == labels[j]:
                q += w[i, j] - gamma * k[i] * k[j] / two_m
    return q / two_m


def _canonical(labels: Sequence[int]) -> List[int]:
    """Relabel so that labels appear in order of their lowest member."""
    seen = {}
    out = []
    for c in labels:
        if c not in seen:
            seen[c] = len(seen)
        out.append(seen[c])
    return out


def _local_moving(a: np.ndarray, gamma: float, two_m: float) -> List[int]:
    """One level: communities start as singletons; sweep the nodes in ascending
    order, moving each to the neighbouring community of largest gain
    k_{i,in}(C) - gamma tot(C) k_i / (2m), until a sweep moves nothing."""
    n = a.shape[0]
    k = [float(sum(a[i, j] for j in range(n))) for i in range(n)]
    comm = list(range(n))
    tot = list(k)
    moved = True
    while moved:
        moved = False
        for i in range(n):
            old = comm[i]
            tot[old] -= k[i]
            # weight from i to each community (self-loop excluded)
            k_in = {}
            for j in range(n):
                if j != i and a[i, j] != 0.0:
                    k_in[comm[j]] = k_in.get(comm[j], 0.0) + a[i, j]
            def gain(c):
                return k_in.get(c, 0.0) - gamma * tot[c] * k[i] / two_m
            g_old = gain(old)
            tol = REL_TIE * max(abs(g_old), k[i], 1e-300)
            g_max = max([g_old] + [gain(c) for c in k_in])
            if g_max > g_old + tol:
                comm[i] = min(c for c in k_in if gain(c) >= g_max - tol)
                moved = True
            else:
                comm[i] = old
            tot[comm[i]] += k[i]
    return comm


def louvain(w: np.ndarray, gamma: float = 1.0) -> List[int]:
    n = w.shape[0]
    two_m = float(sum(w[i, j] for i in range(n) for j in range(n)))
    labels = list(range(n))
    if two_m == 0.0:
        return labels
    a = np.array(w, dtype=np.float64)
    while True:
        comm = _canonical(_local_moving(a, gamma, two_m))
        nc = max(comm) + 1
        if nc == a.shape[0]:
            break  # nothing moved at this level
        labels = [comm[c] for c in labels]
        agg = np.zeros((nc, nc))
        for i in range(a.shape[0]):
            for j in range(a.shape[0]):
                agg[comm[i], comm[j]] += a[i, j]
        a = agg
    return _canonical(labels)


def merge_small(w: np.ndarray, labels: Sequence[int], s_min: int) -> List[int]:
    labels = _canonical(labels)
    while True:
        nb = max(labels) + 1
        sizes = [labels.count(b) for b in range(nb)]
        if nb <= 1 or min(sizes) >= s_min:
            return labels
        small = min(range(nb), key=lambda b: (sizes[b], b))
        shared = [0.0] * nb
        for i in range(len(labels)):
            for j in range(len(labels)):
                if labels[i] == small and labels[j] != small:
                    shared[labels[j]] += w[i, j]
        others = [b for b in range(nb) if b != small]
        if max(shared[b] for b in others) > 0.0:
            target = min(others, key=lambda b: (-shared[b], b))
        else:
            target = min(others, key=lambda b: (sizes[b], b))
        labels = _canonical([target if c == small else c for c in labels])


def partition(w: np.ndarray, gamma: float = 1.0, s_min: int = 1) -> List[int]:
    return merge_small(w, louvain(w, gamma), s_min)


def block_masks(labels: Sequence[int], reps: int) -> np.ndarray:
    """masks[b, p] = 1 when parameter p = r n + q belongs to a qubit q of block b."""
    n = len(labels)
    nb = max(labels) + 1
    m = np.zeros((nb, n * (reps + 1)), dtype=np.uint8)
    for r in range(reps + 1):
        for q in range(n):
            m[labels[q], r * n + q] = 1
    return m
