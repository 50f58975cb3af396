"""Dense-matrix brute force for tiny registers (n <= 10), used only to pin the oracle.

Every operator is an explicit 2^n x 2^n matrix assembled from Kronecker
products of 2x2 matrices, with no bit manipulation at all, so it shares no
method with the gate-by-gate oracle:

* RY(theta) from Eq. 7, CNOT as |0><0|_c (x) I + |1><1|_c (x) X_t;
* Pauli strings as the Kronecker product of their letters (Eq. 6);
* U(theta) = product of every gate matrix in circuit order (Section IV-B);
* E = psi^dagger H psi (Eq. 4); the gradient by the parameter-shift rule
  (Eq. 13) on this dense model.

Qubit q is bit q of the basis index, so the Kronecker product runs from
qubit n-1 (leftmost factor) down to qubit 0.
"""
from __future__ import annotations

import math
from functools import reduce
from typing import Dict, Sequence

import numpy as np

I2 = np.eye(2, dtype=np.complex128)
X2 = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y2 = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
Z2 = np.array([[1, 0], [0, -1]], dtype=np.complex128)
P0 = np.array([[1, 0], [0, 0]], dtype=np.complex128)
P1 = np.array([[0, 0], [0, 1]], dtype=np.complex128)
LETTER: Dict[str, np.ndarray] = {"I": I2, "X": X2, "Y": Y2, "Z": Z2}

MAX_QUBITS = 10


def ry(theta: float) -> np.ndarray:
    """Eq. 7."""
    c, s = math.cos(theta / 2), math.sin(theta / 2)
    return np.array([[c, -s], [s, c]], dtype=np.complex128)


def rz(theta: float) -> np.ndarray:
    """The RZ of the EfficientSU2 layer (Eq. 8): exp(-i theta Z / 2)."""
    return np.array([[np.exp(-0.5j * theta), 0], [0, np.exp(0.5j * theta)]], dtype=np.complex128)


def embed(ops: Dict[int, np.ndarray], n: int) -> np.ndarray:
    """Kronecker product with ops[q] on qubit q and identity elsewhere."""
    factors = [ops.get(q, I2) for q in reversed(range(n))]
    return reduce(np.kron, factors)


def cnot(ctl: int, tgt: int, n: int) -> np.ndarray:
    return embed({ctl: P0}, n) + embed({ctl: P1, tgt: X2}, n)


def pauli(string: str) -> np.ndarray:
    n = len(string)
    return embed({q: LETTER[string[q]] for q in range(n)}, n)


def hamiltonian(strings: Sequence[str], coeffs) -> np.ndarray:
    n = len(strings[0])
    h = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    for s, c in zip(strings, coeffs):
        h += float(c) * pauli(s)
    return h


def entangler_pairs(n: int, ent: int = 0, layer: int = 1):
    """(control, target) list of the entangler of layer `layer` (1 .. reps):
    0 linear CX(0,1)..CX(n-2,n-1); 1 circular: CX(n-1,0) first, then linear;
    2 full: CX(i,j), i < j, lexicographic; 3 reverse linear: CX(n-2,n-1) down to
    CX(0,1); 4 pairwise: CX(i,i+1) for even i, then for odd i; 5 SCA: with offset
    o = layer - 1, the wrap-around chain of n gates CX(s+k, s+k+1) (indices mod n)
    starting at s = n-1-o, each gate reversed to CX(s+k+1, s+k) when o is odd."""
    if ent == 2:
        return [(i, j) for i in range(n) for j in range(i + 1, n)]
    if ent == 3:
        return [(q, q + 1) for q in reversed(range(n - 1))]
    if ent == 4:
        return [(q, q + 1) for q in range(0, n - 1, 2)] + [(q, q + 1) for q in range(1, n - 1, 2)]
    if ent == 5:
        if n < 2:
            return []
        o = (layer - 1) % n
        s = (n - 1 - o) % n
        chain = [((s + k) % n, (s + k + 1) % n) for k in range(n)]
        return [(t, c) for c, t in chain] if (layer - 1) % 2 else chain
    pairs = [(q, q + 1) for q in range(n - 1)]
    if ent == 1 and n > 1:
        pairs = [(n - 1, 0)] + pairs
    return pairs


def circuit(n: int, reps: int, theta, ent: int = 0, gates: int = 1) -> np.ndarray:
    """U(theta): rotation layer, then reps x [entangler; rotation layer] as explicit
    matrices.  A rotation layer is RY on every qubit, then (gates = 2) RZ on every
    qubit; layer r's angles start at r * gates * n."""
    assert n <= MAX_QUBITS
    th = np.asarray(theta, dtype=np.float64).reshape(-1)
    assert th.size == gates * n * (reps + 1)
    u = np.eye(1 << n, dtype=np.complex128)
    for r in range(reps + 1):
        if r > 0:
            for c, t in entangler_pairs(n, ent, r):
                u = cnot(c, t, n) @ u
        base = r * gates * n
        for q in range(n):
            u = embed({q: ry(th[base + q])}, n) @ u
        if gates == 2:
            for q in range(n):
                u = embed({q: rz(th[base + n + q])}, n) @ u
    return u


def state(n: int, reps: int, theta, ent: int = 0, gates: int = 1) -> np.ndarray:
    return circuit(n, reps, theta, ent, gates)[:, 0]


def energy(n: int, reps: int, theta, strings, coeffs, ent: int = 0, gates: int = 1) -> float:
    psi = state(n, reps, theta, ent, gates)
    return float(np.real(np.vdot(psi, hamiltonian(strings, coeffs) @ psi)))


def param_shift_grad(n: int, reps: int, theta, strings, coeffs, ent: int = 0, gates: int = 1) -> np.ndarray:
    th = np.asarray(theta, dtype=np.float64).reshape(-1)
    h = hamiltonian(strings, coeffs)
    g = np.zeros_like(th)
    for p in range(th.size):
        vals = []
        for sh in (+math.pi / 2, -math.pi / 2):
            t = th.copy()
            t[p] += sh
            psi = circuit(n, reps, t, ent, gates)[:, 0]
            vals.append(float(np.real(np.vdot(psi, h @ psi))))
        g[p] = 0.5 * (vals[0] - vals[1])
    return g
