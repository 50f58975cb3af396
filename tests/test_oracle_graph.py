"""Pins of the partitioning oracle (oracle/graph.py, Section IV-C) against facts
fixed by the mathematics: a hand-worked interaction graph (Eq. 9) and its
pair-count invariant, hand modularity values (Eq. 10) and networkx's modularity
routine, planted community structure recovered exactly and with the brute-force
maximum modularity, gamma = 0 giving the connected components, and the S_min
merge on hand-made cases; plus mutants of the oracle that the checks catch."""
import itertools
import math
import types

import numpy as np
import pytest

from oracle import graph
from paper_2607_02749_gb300 import workloads as wl


def test_interaction_graph_hand_example():
    strings = ["ZZII", "IXYI", "ZIIZ", "IIII", "ZIII", "XIXI"]
    coeffs = [2.0, -3.0, 0.5, 7.0, 1.0, -0.25]
    w = graph.interaction_graph(4, strings, coeffs)
    want = np.zeros((4, 4))
    for i, j, v in ((0, 1, 2.0), (1, 2, 3.0), (0, 3, 0.5), (0, 2, 0.25)):
        want[i, j] = want[j, i] = v
    assert np.array_equal(w, want)


def test_interaction_graph_pair_count_invariant():
    ham = wl.pauli_hamiltonian(9, 200, seed=3)
    w = graph.interaction_graph(9, ham.strings, ham.coeffs)
    assert np.allclose(w, w.T) and np.all(np.diag(w) == 0)
    expect = sum(abs(c) * math.comb(sum(ch != "I" for ch in s), 2) for s, c in zip(ham.strings, ham.coeffs))
    assert np.triu(w, 1).sum() == pytest.approx(expect, rel=1e-12)


def _two_edges():
    w = np.zeros((4, 4))
    w[0, 1] = w[1, 0] = 1.0
    w[2, 3] = w[3, 2] = 1.0
    return w


def test_modularity_hand_values():
    w = _two_edges()
    assert graph.modularity(w, [0, 0, 1, 1]) == pytest.approx(0.5)  # 2 x (1/2 - 1/4)
    assert graph.modularity(w, [0, 0, 0, 0]) == pytest.approx(0.0)
    assert graph.modularity(w, [0, 1, 2, 3]) == pytest.approx(-0.25)  # -sum (k_i / 2m)^2
    assert graph.modularity(w, [0, 0, 1, 1], gamma=2.0) == pytest.approx(0.0)
    assert graph.modularity(np.zeros((3, 3)), [0, 1, 2]) == 0.0


def test_modularity_matches_networkx():
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(0)
    for trial in range(6):
        n = 9
        w = np.triu(rng.uniform(0, 1, (n, n)) * (rng.uniform(size=(n, n)) < 0.5), 1)
        w = w + w.T
        labels = list(rng.integers(0, 3, n))
        g = nx.Graph()
        g.add_nodes_from(range(n))
        for i in range(n):
            for j in range(i + 1, n):
                if w[i, j] > 0:
                    g.add_edge(i, j, weight=w[i, j])
        comms = [{i for i in range(n) if labels[i] == c} for c in set(labels)]
        for gamma in (0.5, 1.0, 1.7):
            want = nx.algorithms.community.modularity(g, comms, weight="weight", resolution=gamma)
            assert graph.modularity(w, labels, gamma) == pytest.approx(want, abs=1e-12)


def _planted(sizes, p_in, w_out, seed):
    rng = np.random.default_rng(seed)
    n = sum(sizes)
    lab = np.repeat(np.arange(len(sizes)), sizes)
    w = np.zeros((n, n))
    for i in range(n):
        for j in range(i + 1, n):
            if lab[i] == lab[j]:
                v = rng.uniform(1.0, 2.0) if rng.uniform() < p_in else 0.0
            else:
                v = rng.uniform(0.0, w_out) if rng.uniform() < 0.3 else 0.0
            w[i, j] = w[j, i] = v
    return w, list(lab)


def _brute_force_max(w, gamma=1.0):
    n = w.shape[0]
    best = -1.0
    # restricted growth strings enumerate every partition once
    def rgs(prefix, mx):
        nonlocal best
        if len(prefix) == n:
            best = max(best, graph.modularity(w, prefix, gamma))
            return
        for c in range(mx + 2):
            yield_ = prefix + [c]
            rgs(yield_, max(mx, c))
    rgs([0], 0)
    return best


def test_louvain_recovers_planted_blocks_with_the_maximum_modularity():
    for sizes, seed in (((3, 3), 1), ((4, 3), 2), ((2, 3, 3), 3), ((3, 2, 3), 4)):
        w, lab = _planted(sizes, 1.0, 0.2, seed)
        got = graph.louvain(w)
        assert got == lab, (sizes, got)
        assert graph.modularity(w, got) == pytest.approx(_brute_force_max(w), abs=1e-12)


def test_louvain_two_cliques_and_ring_of_triangles():
    w = np.zeros((8, 8))
    for blk in (range(0, 4), range(4, 8)):
        for i, j in itertools.combinations(blk, 2):
            w[i, j] = w[j, i] = 1.0
    w[3, 4] = w[4, 3] = 0.1
    assert graph.louvain(w) == [0, 0, 0, 0, 1, 1, 1, 1]
    # six triangles in a ring joined by single edges: each triangle is a community
    t = 6
    w = np.zeros((3 * t, 3 * t))
    for b in range(t):
        for i, j in itertools.combinations(range(3 * b, 3 * b + 3), 2):
            w[i, j] = w[j, i] = 1.0
        a, c = 3 * b + 2, (3 * b + 3) % (3 * t)
        w[a, c] = w[c, a] = 1.0
    assert graph.louvain(w) == [b for b in range(t) for _ in range(3)]


def test_gamma_zero_gives_connected_components():
    w = np.zeros((7, 7))
    for i, j in ((0, 1), (1, 2), (3, 4), (5, 6)):
        w[i, j] = w[j, i] = 0.5 + i
    assert graph.louvain(w, gamma=0.0) == [0, 0, 0, 1, 1, 2, 2]


def test_merge_small_hand_cases():
    w = np.zeros((5, 5))
    for i, j, v in ((0, 1, 1.0), (1, 2, 1.0), (2, 3, 0.3), (3, 4, 0.9), (4, 0, 0.2)):
        w[i, j] = w[j, i] = v
    # block {3} (size 1) shares 0.3 with block 0 and 0.9 with block {4}
    assert graph.merge_small(w, [0, 0, 0, 1, 2], 2) == [0, 0, 0, 1, 1]
    # an isolated singleton joins the smallest other block
    w2 = np.zeros((6, 6))
    w2[0, 1] = w2[1, 0] = w2[1, 2] = w2[2, 1] = w2[3, 4] = w2[4, 3] = 1.0
    assert graph.merge_small(w2, [0, 0, 0, 1, 1, 2], 2) == [0, 0, 0, 1, 1, 1]
    assert graph.merge_small(w, [0, 0, 0, 1, 2], 10) == [0, 0, 0, 0, 0]
    assert graph.merge_small(w, [0, 1, 2, 3, 4], 1) == [0, 1, 2, 3, 4]


def test_block_masks_cover_every_parameter_once():
    labels = [0, 1, 0, 2, 1]
    m = graph.block_masks(labels, 2)
    assert m.shape == (3, 15)
    assert np.array_equal(m.sum(axis=0), np.ones(15))
    assert list(np.nonzero(m[1])[0]) == [1, 4, 6, 9, 11, 14]


# ------------------------------------------------------------------ mutants --
GRAPH_MUTANTS = {
    "eq9_signed_coefficients": ("w[i, j] += abs(float(c))", "w[i, j] += float(c)"),
    "modularity_no_resolution": ("q += w[i, j] - gamma * k[i] * k[j] / two_m", "q += w[i, j] - k[i] * k[j] / two_m"),
    "modularity_half_null": ("q += w[i, j] - gamma * k[i] * k[j] / two_m",
                             "q += w[i, j] - gamma * k[i] * k[j] / (2 * two_m)"),
    "gain_without_resolution": ("return k_in.get(c, 0.0) - gamma * tot[c] * k[i] / two_m",
                                "return k_in.get(c, 0.0) - tot[c] * k[i] / two_m"),
    "gain_keeps_own_degree": ("tot[old] -= k[i]", "pass"),
    "no_aggregation": ("labels = [comm[c] for c in labels]", "labels = [comm[c] for c in labels]; break"),
    "merge_weakest_neighbour": ("target = min(others, key=lambda b: (-shared[b], b))",
                                "target = min(others, key=lambda b: (shared[b], b))"),
}


def _graph_checks(mod) -> bool:
    try:
        w = graph.interaction_graph(4, ["ZZII", "IXYI"], [2.0, -3.0])
        if not np.array_equal(mod.interaction_graph(4, ["ZZII", "IXYI"], [2.0, -3.0]), w):
            return False
        e2 = _two_edges()
        if abs(mod.modularity(e2, [0, 0, 1, 1]) - 0.5) > 1e-12:
            return False
        if abs(mod.modularity(e2, [0, 0, 1, 1], gamma=2.0)) > 1e-12:
            return False
        for sizes, seed in (((3, 3), 1), ((2, 3, 3), 3)):
            pw, lab = _planted(sizes, 1.0, 0.2, seed)
            if mod.louvain(pw) != lab:
                return False
        t = 6
        ring = np.zeros((3 * t, 3 * t))
        for b in range(t):
            for i, j in itertools.combinations(range(3 * b, 3 * b + 3), 2):
                ring[i, j] = ring[j, i] = 1.0
            a, c = 3 * b + 2, (3 * b + 3) % (3 * t)
            ring[a, c] = ring[c, a] = 1.0
        if mod.louvain(ring) != [b for b in range(t) for _ in range(3)]:
            return False
        if mod.louvain(ring, gamma=0.1) != [0] * (3 * t):  # halves joined by 2 edges: 2 > 12 gamma
            return False
        cw = np.zeros((7, 7))
        for i, j in ((0, 1), (1, 2), (3, 4), (5, 6)):
            cw[i, j] = cw[j, i] = 0.5 + i
        if mod.louvain(cw, gamma=0.0) != [0, 0, 0, 1, 1, 2, 2]:
            return False
        mw = np.zeros((5, 5))
        for i, j, v in ((0, 1, 1.0), (1, 2, 1.0), (2, 3, 0.3), (3, 4, 0.9), (4, 0, 0.2)):
            mw[i, j] = mw[j, i] = v
        if mod.merge_small(mw, [0, 0, 0, 1, 2], 2) != [0, 0, 0, 1, 1]:
            return False
        return True
    except Exception:
        return False


def test_graph_checks_pass_on_the_oracle():
    assert _graph_checks(graph)


@pytest.mark.parametrize("name", sorted(GRAPH_MUTANTS))
def test_graph_mutant_is_caught(name):
    src = open(graph.__file__).read()
    old, new = GRAPH_MUTANTS[name]
    assert old in src, name
    mod = types.ModuleType("graph_mutant")
    exec(compile(src.replace(old, new), "graph_mutant", "exec"), mod.__dict__)
    assert not _graph_checks(mod)
