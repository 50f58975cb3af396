"""Seeded synthetic inputs for the Graph-VQE energy/gradient path.

This module only draws random numbers and Pauli strings: it holds none of the
method's arithmetic, so both the CPU oracle and the CUDA path can consume its
output without sharing any computation.

The shapes follow the paper's workload (Section IV-A, Eq. 1-3, Eq. 6 and
Section V-A): a protein-folding Hamiltonian is a real linear combination of
Pauli strings whose coefficients are negative Miyazawa-Jernigan contact
energies plus penalty terms with weight lambda = 10.  The real MJ Hamiltonians
are not available, so the coefficient *structure* is reproduced:

* contact terms:  c ~ U(-7.5, -0.1)
* penalty terms:  c = +10  (lambda_chiral = lambda_back = lambda_overlap = 10)
* string weight:  w ~ U{1..4}, w distinct qubits drawn uniformly
* parameters:     theta ~ U(-pi, pi)  (the rotation-angle range after Eq. 7)
* seeds:          numpy PCG64, seed 0 as in Section V-A; batched instance i
                  uses seed 1000 + i.

String convention: character i of a Pauli string acts on qubit i, and qubit i
is bit i of the computational-basis index (little-endian).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

PAULI_LETTERS = "IXYZ"


@dataclasses.dataclass
class Hamiltonian:
    """A Pauli-sum H = sum_k c_k P_k (Eq. 6): strings of length n plus real coefficients."""

    n_qubits: int
    strings: List[str]
    coeffs: np.ndarray  # float64 [M]

    @property
    def n_terms(self) -> int:
        return len(self.strings)

    def abs_sum(self) -> float:
        """sum_k |c_k|, the scale the error tolerances are stated against."""
        return float(np.abs(self.coeffs).sum())

    def pauli_bytes(self) -> bytes:
        """All strings concatenated (M*n ASCII bytes), the flat form the C calls take."""
        return "".join(self.strings).encode("ascii")


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _support(rng: np.random.Generator, n: int, max_weight: int) -> np.ndarray:
    w = int(rng.integers(1, min(max_weight, n) + 1))
    return rng.choice(n, size=w, replace=False)


def z_hamiltonian(n: int, n_terms: int, seed: int = 0, contact_fraction: float = 0.75,
                  max_weight: int = 4) -> Hamiltonian:
    """Diagonal (Z-only) Hamiltonian shaped like the paper's folding Hamiltonian.

    The first round(contact_fraction * n_terms) strings carry contact energies
    c ~ U(-7.5, -0.1); the rest are penalty terms with c = +10.
    """
    rng = _rng(seed)
    n_contact = int(round(contact_fraction * n_terms))
    strings: List[str] = []
    coeffs = np.empty(n_terms, dtype=np.float64)
    for k in range(n_terms):
        letters = ["I"] * n
        for q in _support(rng, n, max_weight):
            letters[int(q)] = "Z"
        strings.append("".join(letters))
        coeffs[k] = rng.uniform(-7.5, -0.1) if k < n_contact else 10.0
    return Hamiltonian(n, strings, coeffs)


def chain_z_hamiltonian(n: int, n_terms: int, seed: int = 0, reach: int = 4, contact_fraction: float = 0.75,
                        max_weight: int = 4) -> Hamiltonian:
    """Z-only Hamiltonian with the sequence locality of Section IV-C: qubits
    2i, 2i+1 encode turn i, and most strings act on a few nearby turns.  Each
    string's support is drawn inside a window of `reach` consecutive qubits
    starting at a uniform position; coefficients as in z_hamiltonian."""
    rng = _rng(seed)
    n_contact = int(round(contact_fraction * n_terms))
    reach = max(1, min(reach, n))
    strings: List[str] = []
    coeffs = np.empty(n_terms, dtype=np.float64)
    for k in range(n_terms):
        start = int(rng.integers(0, n - reach + 1))
        letters = ["I"] * n
        for q in _support(rng, reach, max_weight):
            letters[start + int(q)] = "Z"
        strings.append("".join(letters))
        coeffs[k] = rng.uniform(-7.5, -0.1) if k < n_contact else 10.0
    return Hamiltonian(n, strings, coeffs)


def pauli_hamiltonian(n: int, n_terms: int, seed: int = 0, xy_fraction: float = 0.4,
                      max_weight: int = 4) -> Hamiltonian:
    """General Pauli-sum Hamiltonian with X/Y letters on about xy_fraction of the strings.

    Each string has weight w ~ U{1..4} on distinct uniform qubits.  With
    probability xy_fraction its letters are uniform over {X, Y, Z}, resampled
    until at least one X or Y appears; otherwise all letters are Z.
    Coefficients c ~ N(0, 1).
    """
    rng = _rng(seed)
    strings: List[str] = []
    coeffs = np.empty(n_terms, dtype=np.float64)
    for k in range(n_terms):
        support = _support(rng, n, max_weight)
        letters = ["I"] * n
        if rng.random() < xy_fraction:
            while True:
                picks = rng.integers(0, 3, size=len(support))
                if np.any(picks < 2):
                    break
            for q, p in zip(support, picks):
                letters[int(q)] = "XYZ"[int(p)]
        else:
            for q in support:
                letters[int(q)] = "Z"
        strings.append("".join(letters))
        coeffs[k] = rng.standard_normal()
    return Hamiltonian(n, strings, coeffs)


def n_params(n: int, reps: int) -> int:
    """P = n (D + 1): one RY angle per qubit per rotation layer (RY+CX reading of Eq. 8)."""
    return n * (reps + 1)


def thetas(n: int, reps: int, batch: int, seed: int = 0) -> np.ndarray:
    """theta ~ U(-pi, pi), float64 [batch][P], flattened layer-major (p = r*n + q)."""
    rng = _rng(seed)
    return rng.uniform(-math.pi, math.pi, size=(batch, n_params(n, reps)))


def active_mask(n_par: int, batch: int, seed: int = 0, lo: float = 0.3,
                hi: float = 0.6) -> np.ndarray:
    """Random active-parameter masks (Eq. 11): a fraction f ~ U(lo, hi) of entries set to 1."""
    rng = _rng(seed)
    mask = np.zeros((batch, n_par), dtype=np.uint8)
    for b in range(batch):
        k = max(1, int(round(rng.uniform(lo, hi) * n_par)))
        mask[b, rng.choice(n_par, size=k, replace=False)] = 1
    return mask


@dataclasses.dataclass
class Instance:
    """One restricted-update subproblem of the batched cluster workload."""

    n_qubits: int
    reps: int
    ham: Hamiltonian
    theta: np.ndarray  # [1][P]
    mask: np.ndarray   # [1][P] uint8


def cluster_batch(n_instances: int = 256, qubit_range: Sequence[int] = (14, 20),
                  reps_range: Sequence[int] = (2, 4), terms_per_qubit: int = 100,
                  base_seed: int = 1000) -> List[Instance]:
    """Heterogeneous batch of independent subproblems (Section IV-D block updates).

    Instance i draws everything from seed base_seed + i: n ~ U{qubit_range},
    D ~ U{reps_range}, a Z-string Hamiltonian with terms_per_qubit*n terms,
    one theta vector and one active-parameter mask with 30-60% active entries.
    """
    out: List[Instance] = []
    for i in range(n_instances):
        rng = _rng(base_seed + i)
        n = int(rng.integers(qubit_range[0], qubit_range[1] + 1))
        d = int(rng.integers(reps_range[0], reps_range[1] + 1))
        sub_seed = int(rng.integers(0, 2**31 - 1))
        ham = z_hamiltonian(n, terms_per_qubit * n, seed=sub_seed)
        th = thetas(n, d, 1, seed=sub_seed + 1)
        mk = active_mask(n_params(n, d), 1, seed=sub_seed + 2)
        out.append(Instance(n, d, ham, th, mk))
    return out


# Named workloads with the sizes used by the tests and the benchmark.
WORKLOADS = {
    # n=12, reps=2, FP64: 200 Z-strings (150 contact, 50 penalty), 64 thetas.
    "n12_reps2_z200": dict(n=12, reps=2, terms=200, batch=64, kind="z"),
    # n=24, reps=4, FP32: 2,000 Z-strings, 16 thetas.
    "n24_reps4_z2000": dict(n=24, reps=4, terms=2000, batch=16, kind="z"),
    # n=30, reps=6, FP32 (and FP64 mode): 20,000 Z-strings, 4 thetas.
    "n30_reps6_z20000": dict(n=30, reps=6, terms=20000, batch=4, kind="z"),
    # n=27, reps=2, FP32: 2,000 Z-strings, 1 theta: a profiling-size case (512 MiB state,
    # larger than L2, a few GiB on the device in total).
    "n27_reps2_z2000": dict(n=27, reps=2, terms=2000, batch=1, kind="z"),
    # n=27, reps=6, FP32: the same, with the benchmark's depth (closed-form layers 1..4
    # and two tile-pass layers): the profiling-size case of the closed-form kernels.
    "n27_reps6_z2000": dict(n=27, reps=6, terms=2000, batch=1, kind="z"),
    # n=28, reps=5, FP32: 5,000 strings over {I,X,Y,Z}, 8 thetas.
    "n28_reps5_pauli5000": dict(n=28, reps=5, terms=5000, batch=8, kind="pauli"),
    # n=26, reps=2, FP32: the same term mix, 1 theta: a profiling-size case of the
    # non-diagonal path (256 MiB state, a few GiB on the device in total).
    "n26_reps2_pauli5000": dict(n=26, reps=2, terms=5000, batch=1, kind="pauli"),
}


def make_workload(name: str, seed: int = 0, batch: Optional[int] = None):
    """Return (Hamiltonian, theta[batch][P]) for a named workload."""
    w = WORKLOADS[name]
    if w["kind"] == "z":
        ham = z_hamiltonian(w["n"], w["terms"], seed=seed)
    else:
        ham = pauli_hamiltonian(w["n"], w["terms"], seed=seed)
    th = thetas(w["n"], w["reps"], batch if batch is not None else w["batch"], seed=seed + 1)
    return ham, th
