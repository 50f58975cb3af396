"""Pins of the readout oracle (oracle/readout.py) against facts fixed by the
mathematics: closed forms of product states, a one-qubit inverse CDF, hand
values of a two-outcome CVaR, alpha = 1 equal to the diagonal energy computed
term by term by the C oracle, alpha -> 0 equal to the lowest populated energy,
and the dense-matrix diagonal of H."""
import math

import numpy as np
import pytest

import oracle
from oracle import dense, readout
from paper_2607_02749_gb300 import workloads as wl


def _product_probs(theta0):
    n = len(theta0)
    x = np.arange(1 << n)
    p = np.ones(1 << n)
    for q, t in enumerate(theta0):
        b = (x >> q) & 1
        p *= np.where(b == 1, math.sin(t / 2) ** 2, math.cos(t / 2) ** 2)
    return p


def test_product_state_probabilities_and_argmax_closed_form():
    rng = np.random.default_rng(5)
    for n in (1, 3, 7):
        th = rng.uniform(-math.pi, math.pi, n)
        p = readout.probabilities(oracle.state(n, 0, th))
        assert np.allclose(p, _product_probs(th), atol=1e-15)
        x, pm = readout.most_probable(p)
        want = sum(1 << q for q, t in enumerate(th) if math.sin(t / 2) ** 2 > math.cos(t / 2) ** 2)
        assert x == want
        assert pm == pytest.approx(np.prod([max(math.sin(t / 2) ** 2, math.cos(t / 2) ** 2) for t in th]))


def test_argmax_takes_the_smallest_index_on_ties():
    p = np.array([0.1, 0.3, 0.2, 0.3, 0.1])
    assert readout.most_probable(p) == (1, 0.3)


def test_one_qubit_inverse_cdf():
    for t in (0.3, 1.1, 2.5):
        c2 = math.cos(t / 2) ** 2
        p = readout.probabilities(oracle.state(1, 0, [t]))
        u = np.array([0.0, c2 * 0.5, c2 - 1e-9, c2 + 1e-9, 0.999999])
        assert readout.sample(p, u).tolist() == [0, 0, 0, 1, 1]


def test_inverse_cdf_boundary_goes_up():
    # exactly representable: the cumulative probability at x = 0 equals u * T
    p = np.array([0.25, 0.75])
    assert readout.sample(p, [0.25]).tolist() == [1]
    p = np.array([0.25, 0.0, 0.75])
    assert readout.sample(p, [0.25, 0.9999]).tolist() == [2, 2]


def test_stratified_shots_match_the_probabilities():
    p = readout.probabilities(oracle.state(6, 2, wl.thetas(6, 2, 1, seed=2)[0]))
    K = 8192
    u = (np.arange(K) + 0.5) / K
    counts = np.bincount(readout.sample(p, u), minlength=p.size)
    assert np.all(np.abs(counts - K * p / p.sum()) <= 1.0 + 1e-9)


def test_zero_probability_outcomes_are_never_drawn():
    p = np.zeros(16)
    p[[3, 9]] = [0.5, 0.5]
    s = readout.sample(p, np.linspace(0, 0.999999, 101))
    assert set(s.tolist()) == {3, 9}


def test_cvar_two_outcome_hand_values():
    p = np.array([0.3, 0.7])
    e = np.array([1.0, -2.0])
    assert readout.cvar(p, e, 0.5) == pytest.approx(-2.0)
    assert readout.cvar(p, e, 0.7) == pytest.approx(-2.0)
    assert readout.cvar(p, e, 0.8) == pytest.approx((0.7 * -2.0 + 0.1 * 1.0) / 0.8)
    assert readout.cvar(p, e, 1.0) == pytest.approx(0.3 * 1.0 - 0.7 * 2.0)


def test_cvar_ties_count_fractionally():
    p = np.array([0.25, 0.25, 0.25, 0.25])
    e = np.array([0.0, -1.0, -1.0, 3.0])
    assert readout.cvar(p, e, 0.25) == pytest.approx(-1.0)
    assert readout.cvar(p, e, 0.6) == pytest.approx((0.5 * -1.0 + 0.1 * 0.0) / 0.6)


def test_diagonal_energies_match_the_dense_diagonal():
    ham = wl.pauli_hamiltonian(5, 40, seed=4)
    e = readout.diagonal_energies(5, ham.strings, ham.coeffs)
    assert np.allclose(e, np.real(np.diag(dense.hamiltonian(ham.strings, ham.coeffs))), atol=1e-12)


def test_cvar_alpha_one_is_the_diagonal_energy():
    n, reps = 6, 2
    ham = wl.z_hamiltonian(n, 60, seed=3)
    th = wl.thetas(n, reps, 1, seed=9)[0]
    p = readout.probabilities(oracle.state(n, reps, th))
    e = readout.diagonal_energies(n, ham.strings, ham.coeffs)
    want = oracle.energy(n, reps, th, ham.strings, ham.coeffs)  # the C oracle, term by term
    assert readout.cvar(p, e, 1.0) == pytest.approx(want, abs=1e-12 * ham.abs_sum())


def test_cvar_small_alpha_is_the_lowest_populated_energy_and_monotone():
    n, reps = 6, 1
    ham = wl.z_hamiltonian(n, 40, seed=8)
    th = wl.thetas(n, reps, 1, seed=1)[0]
    p = readout.probabilities(oracle.state(n, reps, th))
    e = readout.diagonal_energies(n, ham.strings, ham.coeffs)
    lowest = float(np.min(e[p > 0]))
    assert readout.cvar(p, e, 1e-12) == pytest.approx(lowest, abs=1e-9)
    vals = [readout.cvar(p, e, a) for a in np.linspace(0.01, 1.0, 40)]
    assert all(b >= a - 1e-12 for a, b in zip(vals, vals[1:]))
    assert vals[-1] <= np.sum(p * e) / p.sum() + 1e-12


# ------------------------------------------------------------------ mutants --
# Plausible mistakes planted in a copy of the readout oracle's source (CPU only)
# must each fail at least one of the checks below.  (Choosing the quantile on the
# other side of an exact cumulative-mass boundary is not among them: the CVaR is
# continuous there and both choices give the same value.)
READOUT_MUTANTS = {
    "cdf_boundary": ('x = np.searchsorted(cdf, t, side="right")', 'x = np.searchsorted(cdf, t, side="left")'),
    "argmax_last": ("x = int(np.argmax(p))", "x = int(len(p) - 1 - np.argmax(p[::-1]))"),
    "cvar_no_partial": ("return (s + rest * tau) / target", "return s / max(pb, 1e-300)"),
    "cvar_unnormalised": ("target = alpha * p.sum()", "target = alpha"),
    "z_sign": ("e += np.where(par == 1, -c, c)", "e += np.where(par == 1, c, -c)"),
    "shots_unnormalised": ("t = np.asarray(uniforms, dtype=np.float64) * total",
                           "t = np.asarray(uniforms, dtype=np.float64)"),
}


def _readout_checks(mod) -> bool:
    try:
        if mod.sample(np.array([0.25, 0.75]), [0.25]).tolist() != [1]:
            return False
        if mod.most_probable(np.array([0.1, 0.3, 0.2, 0.3]))[0] != 1:
            return False
        p, e = np.array([0.3, 0.7]), np.array([1.0, -2.0])
        if abs(mod.cvar(p, e, 0.8) - (0.7 * -2.0 + 0.1) / 0.8) > 1e-12:
            return False
        if abs(mod.cvar(np.array([0.25] * 4), np.array([0.0, -1.0, -1.0, 3.0]), 0.5) + 1.0) > 1e-12:
            return False
        ham = wl.pauli_hamiltonian(4, 20, seed=4)
        d = np.real(np.diag(dense.hamiltonian(ham.strings, ham.coeffs)))
        if np.max(np.abs(mod.diagonal_energies(4, ham.strings, ham.coeffs) - d)) > 1e-12:
            return False
        if abs(mod.cvar(np.array([0.6, 1.4]), e, 0.8) - (1.4 * -2.0 + 0.2) / 1.6) > 1e-12:
            return False  # total 2: the tail is alpha of the total mass
        q = np.array([0.5, 0.5]) * 2.0  # total 2: shots must scale u by the total
        if mod.sample(q, [0.75]).tolist() != [1]:
            return False
        return True
    except Exception:
        return False


def test_readout_checks_pass_on_the_oracle():
    assert _readout_checks(readout)


@pytest.mark.parametrize("name", sorted(READOUT_MUTANTS))
def test_readout_mutant_is_caught(name):
    import types

    src = open(readout.__file__).read()
    old, new = READOUT_MUTANTS[name]
    assert old in src, name
    mod = types.ModuleType("readout_mutant")
    exec(compile(src.replace(old, new), "readout_mutant", "exec"), mod.__dict__)
    assert not _readout_checks(mod)
