"""Parity of the library's host-side partitioning (gvqe_interaction_graph,
gvqe_partition; Section IV-C) with the partitioning oracle, through the C ABI.
No GPU: both are host code.  Graphs agree to the last bit up to summation
order; partitions are compared label for label and modularity to 1e-12."""
import numpy as np
import pytest

from oracle import graph
from paper_2607_02749_gb300 import _lib
from paper_2607_02749_gb300 import workloads as wl


def _hams():
    for n in (2, 5, 9, 14, 20, 30):
        yield n, wl.z_hamiltonian(n, 10 * n, seed=n)
        yield n, wl.pauli_hamiltonian(n, 8 * n, seed=100 + n)


def test_interaction_graph_matches_the_oracle():
    for n, ham in _hams():
        w = _lib.gvqe_interaction_graph(n, ham.strings, ham.coeffs)
        want = graph.interaction_graph(n, ham.strings, ham.coeffs)
        assert np.allclose(w, want, rtol=1e-14, atol=0), n


@pytest.mark.parametrize("gamma", [0.0, 0.5, 1.0, 1.5])
@pytest.mark.parametrize("s_min", [1, 2, 4])
def test_partition_matches_the_oracle(gamma, s_min):
    for n, ham in _hams():
        w = graph.interaction_graph(n, ham.strings, ham.coeffs)
        lab, nb, q = _lib.gvqe_partition(w, gamma, s_min)
        want = graph.partition(w, gamma, s_min)
        assert lab == want, (n, gamma, s_min)
        assert nb == max(want) + 1
        assert q == pytest.approx(graph.modularity(w, want, gamma), abs=1e-12)


def test_partition_on_planted_and_random_graphs():
    rng = np.random.default_rng(4)
    for trial in range(40):
        n = int(rng.integers(2, 31))
        w = np.triu(rng.uniform(0, 1, (n, n)) * (rng.uniform(size=(n, n)) < rng.uniform(0.1, 0.9)), 1)
        w = w + w.T
        for gamma in (0.7, 1.0, 1.3):
            lab, nb, q = _lib.gvqe_partition(w, gamma, 1)
            assert lab == graph.partition(w, gamma, 1), (trial, gamma)


def test_partition_edge_cases():
    # one qubit, no edges, all isolated
    assert _lib.gvqe_partition(np.zeros((1, 1)))[:2] == ([0], 1)
    lab, nb, q = _lib.gvqe_partition(np.zeros((4, 4)), 1.0, 1)
    assert lab == [0, 1, 2, 3] and q == 0.0
    lab, nb, q = _lib.gvqe_partition(np.zeros((4, 4)), 1.0, 2)
    assert lab == graph.partition(np.zeros((4, 4)), 1.0, 2) and nb == 2


def test_partition_rejects_bad_graphs():
    w = np.ones((3, 3)) - np.eye(3)
    bad = [w + np.eye(3), np.where(np.arange(9).reshape(3, 3) == 1, 2.0, w), -w, w * np.nan]
    for b in bad:
        with pytest.raises(_lib.GvqeError) as e:
            _lib.gvqe_partition(b)
        assert e.value.code == _lib.GVQE_EINVAL
    for args in ((w, -1.0, 1), (w, 1.0, 0)):
        with pytest.raises(_lib.GvqeError):
            _lib.gvqe_partition(*args)
    with pytest.raises(_lib.GvqeError):
        _lib.gvqe_interaction_graph(2, ["ZQ"], [1.0])
