"""Readout of a prepared state, written out plainly (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import this module.

Section IV-F: the final state |psi(theta*)> is sampled over the computational
basis states and the bitstring of highest probability is taken.  Section V-A:
8192 shots, seed 0.  Section III (with Section V-A's alpha = 0.2): CVaR-alpha,
the average energy of the lowest-alpha fraction of measurement outcomes.

The definitions used here:
  p(x)        = |psi(x)|^2, total T = sum_x p(x)
  argmax      = the smallest x of largest p(x)
  shot(u)     = the smallest x with sum_{x' <= x} p(x') > u T (inverse CDF in
                increasing x; u in [0, 1) is the caller's random number)
  E(x)        = <x|H|x> = sum over the I/Z strings k of c_k (-1)^{popcount(x & z_k)}
  CVaR_alpha  = (1 / (alpha T)) * [ sum_{E(x) < tau} p(x) E(x) + (alpha T - P(E < tau)) tau ]
                with tau the smallest energy v such that P(E <= v) >= alpha T:
                (1/alpha) * integral_0^alpha F^-1(u) du for the distribution F of E.
No binning, no chunking: cumulative sums in increasing x, one sort by energy.
"""
from __future__ import annotations

from typing import Sequence, Tuple

import numpy as np


def probabilities(psi) -> np.ndarray:
    """p(x) = |psi(x)|^2 in float64."""
    v = np.asarray(psi)
    return (v.real.astype(np.float64) ** 2 + v.imag.astype(np.float64) ** 2) if np.iscomplexobj(v) \
        else v.astype(np.float64) ** 2


def most_probable(p) -> Tuple[int, float]:
    """(smallest x of largest p(x), p(x))."""
    p = np.asarray(p, dtype=np.float64)
    x = int(np.argmax(p))  # numpy returns the first maximum
    return x, float(p[x])


def sample(p, uniforms) -> np.ndarray:
    """Shot k = smallest x whose cumulative probability exceeds uniforms[k] * T."""
    p = np.asarray(p, dtype=np.float64)
    cdf = np.cumsum(p)
    total = cdf[-1]
    t = np.asarray(uniforms, dtype=np.float64) * total
    x = np.searchsorted(cdf, t, side="right")
    nz = np.nonzero(p > 0)[0]
    last = int(nz[-1]) if nz.size else 0
    return np.minimum(x, last).astype(np.int64)


def diagonal_energies(n: int, strings: Sequence[str], coeffs) -> np.ndarray:
    """E(x) = <x|H|x> term by term (X/Y strings have zero diagonal)."""
    x = np.arange(1 << n, dtype=np.int64)
    e = np.zeros(1 << n, dtype=np.float64)
    for s, c in zip(strings, np.asarray(coeffs, dtype=np.float64)):
        if any(ch in "XY" for ch in s):
            continue
        z = 0
        for q, ch in enumerate(s):
            if ch == "Z":
                z |= 1 << q
        par = np.zeros(x.shape, dtype=np.int64)
        m = x & z
        while np.any(m):
            par ^= m & 1
            m >>= 1
        e += np.where(par == 1, -c, c)
    return e


def cvar(p, energies, alpha: float) -> float:
    """CVaR_alpha of the outcome energy under p (alpha in (0, 1])."""
    p = np.asarray(p, dtype=np.float64)
    e = np.asarray(energies, dtype=np.float64)
    order = np.argsort(e, kind="stable")
    ps, es = p[order], e[order]
    target = alpha * p.sum()
    cum = np.cumsum(ps)
    k = int(np.searchsorted(cum, target, side="left"))
    k = min(k, len(es) - 1)
    tau = es[k]
    below = es < tau
    s = float(np.sum(ps[below] * es[below]))
    pb = float(np.sum(ps[below]))
    pa = float(np.sum(ps[es == tau]))
    rest = min(max(target - pb, 0.0), pa)
    return (s + rest * tau) / target
