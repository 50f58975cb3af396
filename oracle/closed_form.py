"""Closed forms that pin the oracle (and, at sizes the oracle cannot reach, the GPU path).

Every function here is derived from the mathematics of the ansatz (Section
IV-B, Eq. 7) and of Pauli sums (Eq. 6) without simulating a state vector:

* product_state_*:  reps = 0.  The state is a product of single-qubit states
  cos(t/2)|0> + sin(t/2)|1>, so <P> factorises: I -> 1, Z -> cos t, X -> sin t,
  Y -> 0.  Cost O(M n).  su2_product_state_energy: the same with RZ(p) after
  each RY(t): X -> sin t cos p, Y -> sin t sin p.
* heisenberg_reps1_energy: reps = 1 with Z-only strings.  RY(t)^dagger Z RY(t)
  = cos t Z - sin t X; conjugating X^a Z^c by the CNOT-chain permutation
  |x> -> |A x> (A = prefix XOR) gives X^(A^-1 a) Z^(A^T c) with no phase; the
  result is evaluated on the layer-0 product state (per qubit I -> 1,
  Z -> cos, X -> sin, XZ -> 0).  Exact at any n, including n = 30.
* basis_state_energy: every angle in {0, pi}.  RY(pi) maps |0> -> |1> and
  |1> -> -|0>, so the state stays a signed basis state |y> and E = E(y).
* zero_angle_energy: theta = 0 gives |0...0>, so E = sum of the coefficients of
  the strings without X or Y letters.
* Each energy is a trigonometric polynomial of degree one in every angle
  (each angle enters one RY gate), so the parameter-shift rule of Eq. 13 is
  exact; shift_grad applies it to any of these closed forms.
"""
from __future__ import annotations

import math
from typing import Callable, Sequence

import numpy as np


def _letters(s: str):
    return [(q, ch) for q, ch in enumerate(s) if ch != "I"]


def product_state_energy(theta0: Sequence[float], strings, coeffs) -> float:
    """reps = 0: E = sum_k c_k prod_q f(sigma_q, theta_q)."""
    th = np.asarray(theta0, dtype=np.float64)
    tot = 0.0
    for s, c in zip(strings, coeffs):
        v = float(c)
        for q, ch in _letters(s):
            if ch == "Z":
                v *= math.cos(th[q])
            elif ch == "X":
                v *= math.sin(th[q])
            else:  # Y
                v = 0.0
        tot += v
    return tot


def su2_product_state_energy(theta_y: Sequence[float], theta_z: Sequence[float], strings, coeffs) -> float:
    """reps = 0 with the full EfficientSU2 layer (RY then RZ): each qubit's Bloch
    vector (sin t cos p, sin t sin p, cos t) for t = theta_y, p = theta_z, so
    I -> 1, X -> sin t cos p, Y -> sin t sin p, Z -> cos t."""
    ty = np.asarray(theta_y, dtype=np.float64)
    tz = np.asarray(theta_z, dtype=np.float64)
    tot = 0.0
    for s, c in zip(strings, coeffs):
        v = float(c)
        for q, ch in _letters(s):
            if ch == "Z":
                v *= math.cos(ty[q])
            elif ch == "X":
                v *= math.sin(ty[q]) * math.cos(tz[q])
            else:
                v *= math.sin(ty[q]) * math.sin(tz[q])
        tot += v
    return tot


def product_state_grad(theta0: Sequence[float], strings, coeffs) -> np.ndarray:
    """reps = 0: the derivative of the product form, factor by factor."""
    th = np.asarray(theta0, dtype=np.float64)
    g = np.zeros(th.size)
    val = {"Z": math.cos, "X": math.sin}
    der = {"Z": lambda t: -math.sin(t), "X": math.cos}
    for s, c in zip(strings, coeffs):
        lets = _letters(s)
        if any(ch == "Y" for _, ch in lets):
            continue
        for j, (qj, chj) in enumerate(lets):
            v = float(c) * der[chj](th[qj])
            for i, (qi, chi) in enumerate(lets):
                if i != j:
                    v *= val[chi](th[qi])
            g[qj] += v
    return g


def _prefix_xor_inverse(a: int, n: int) -> int:
    """A^-1 a for A = prefix XOR: x = y xor (y << 1), masked to n bits."""
    return (a ^ (a << 1)) & ((1 << n) - 1)


def _suffix_xor(c: int, n: int) -> int:
    """A^T c: bit i is the XOR of bits j >= i of c."""
    out = 0
    acc = 0
    for i in reversed(range(n)):
        acc ^= (c >> i) & 1
        out |= acc << i
    return out


def heisenberg_reps1_energy(n: int, theta: Sequence[float], strings, coeffs) -> float:
    """reps = 1, Z-only strings: exact E at any n (cost O(M 2^w n))."""
    th = np.asarray(theta, dtype=np.float64)
    t0, t1 = th[:n], th[n:2 * n]
    cos0, sin0 = np.cos(t0), np.sin(t0)
    tot = 0.0
    for s, c in zip(strings, coeffs):
        lets = _letters(s)
        if any(ch != "Z" for _, ch in lets):
            raise ValueError("heisenberg_reps1_energy takes Z-only strings")
        qs = [q for q, _ in lets]
        w = len(qs)
        for sub in range(1 << w):
            coef = float(c)
            amask = 0
            cmask = 0
            for j, q in enumerate(qs):
                if (sub >> j) & 1:
                    coef *= -math.sin(t1[q])
                    amask |= 1 << q
                else:
                    coef *= math.cos(t1[q])
                    cmask |= 1 << q
            a2 = _prefix_xor_inverse(amask, n)
            c2 = _suffix_xor(cmask, n)
            v = coef
            for q in range(n):
                xa = (a2 >> q) & 1
                zc = (c2 >> q) & 1
                if xa and zc:
                    v = 0.0
                    break
                if xa:
                    v *= sin0[q]
                elif zc:
                    v *= cos0[q]
            tot += v
    return tot


def basis_state_energy(n: int, reps: int, flips, strings, coeffs) -> float:
    """Every angle in {0, pi} (flips[p] = 1 means theta_p = pi): E = E(y) of the final basis state."""
    f = np.asarray(flips, dtype=np.int64).reshape(-1)
    x = 0
    for r in range(reps + 1):
        if r > 0:
            y = 0
            acc = 0
            for q in range(n):
                acc ^= (x >> q) & 1
                y |= acc << q
            x = y
        for q in range(n):
            if f[r * n + q]:
                x ^= 1 << q
    tot = 0.0
    for s, c in zip(strings, coeffs):
        lets = _letters(s)
        if any(ch in "XY" for _, ch in lets):
            continue
        par = 0
        for q, _ in lets:
            par ^= (x >> q) & 1
        tot += -float(c) if par else float(c)
    return tot


def _prefix_xor(x: int, n: int) -> int:
    """Bit j of the result is x_0 ^ ... ^ x_j."""
    y = acc = 0
    for q in range(n):
        acc ^= (x >> q) & 1
        y |= acc << q
    return y


def entangler_map(x: int, n: int, ent: int = 0, layer: int = 1) -> int:
    """Basis index after the entangler of layer `layer` as a closed-form GF(2) map
    (no gate list):
    linear: y_j = x_0 ^ ... ^ x_j (each CX(q, q+1) adds the updated bit q to bit q+1);
    circular: the same after x_0 ^= x_{n-1} (the wrap-around CX(n-1, 0) acts first);
    full: y_j = x_j ^ x_{j-1}, since bit j collects x_i and, through CX(i, j) after
    bit i was updated, the running sums of the lower bits, which cancel pairwise;
    reverse linear: y_j = x_j ^ x_{j-1} as well (in descending order every CX(q, q+1)
    still sees the original bit q);
    pairwise: odd j: y_j = x_j ^ x_{j-1}; even j >= 2: y_j = x_j ^ x_{j-1} ^ x_{j-2}
    (the second half adds the updated odd bit j-1);
    SCA, offset o = layer - 1, s = n-1-o mod n, in the frame z_k = x_{s+k mod n}
    (the direction follows the parity of o itself, not of o mod n):
    even o: w_k = z_0 ^ ... ^ z_k, then w_0 ^= w_{n-1} (the last gate closes the ring);
    odd o: w_k = z_k ^ z_{k+1} for k < n-1, w_{n-1} = z_{n-1} ^ w_0; y_{s+k mod n} = w_k."""
    mask = (1 << n) - 1
    if ent in (2, 3):
        return (x ^ (x << 1)) & mask
    if ent == 4:
        y = 0
        for j in range(n):
            b = (x >> j) & 1
            if j >= 1:
                b ^= (x >> (j - 1)) & 1
            if j >= 2 and j % 2 == 0:
                b ^= (x >> (j - 2)) & 1
            y |= b << j
        return y
    if ent == 5:
        if n < 2:
            return x
        o = (layer - 1) % n
        s = (n - 1 - o) % n
        z = [(x >> ((s + k) % n)) & 1 for k in range(n)]
        if (layer - 1) % 2 == 0:
            w = [0] * n
            acc = 0
            for k in range(n):
                acc ^= z[k]
                w[k] = acc
            w[0] ^= w[n - 1]
        else:
            w = [z[k] ^ z[k + 1] for k in range(n - 1)] + [0]
            w[n - 1] = z[n - 1] ^ w[0]
        return sum(w[k] << ((s + k) % n) for k in range(n))
    if ent == 1 and n > 1:
        x ^= (x >> (n - 1)) & 1
    return _prefix_xor(x, n)


def basis_state_index(n: int, reps: int, flips, ent: int = 0) -> int:
    """Every angle in {0, pi}: the index y of the final signed basis state |y>."""
    f = np.asarray(flips, dtype=np.int64).reshape(-1)
    x = 0
    for r in range(reps + 1):
        if r > 0:
            x = entangler_map(x, n, ent, r)
        for q in range(n):
            if f[r * n + q]:
                x ^= 1 << q
    return x


def zero_angle_energy(strings, coeffs) -> float:
    """theta = 0: sum of coefficients of strings with only I/Z letters."""
    return float(sum(float(c) for s, c in zip(strings, coeffs) if all(ch in "IZ" for ch in s)))


def shift_grad(energy_fn: Callable[[np.ndarray], float], theta) -> np.ndarray:
    """Exact gradient of a degree-one trigonometric polynomial by Eq. 13."""
    th = np.asarray(theta, dtype=np.float64).reshape(-1)
    g = np.zeros(th.size)
    for p in range(th.size):
        tp = th.copy()
        tp[p] += math.pi / 2
        tm = th.copy()
        tm[p] -= math.pi / 2
        g[p] = 0.5 * (energy_fn(tp) - energy_fn(tm))
    return g
