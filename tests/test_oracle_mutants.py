"""The oracle's pins are sensitive: plausible mistakes planted in a copy of the
oracle source (on the CPU, never in the product) must each fail a pin.

Each mutant is a textual edit of ``oracle/gvqe_oracle.c`` compiled to a
temporary library; the pins run against it and at least one must fail.
"""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from oracle import closed_form, dense
from paper_2607_02749_gb300 import workloads as wl

SRC = os.path.join(os.path.dirname(oracle.__file__), "gvqe_oracle.c")

MUTANTS = {
    "ry_sign": ("psi[x] = c * a - s * b;", "psi[x] = c * a + s * b;"),
    "ry_half_angle": ("const double c = cos(0.5 * theta), s = sin(0.5 * theta);",
                      "const double c = cos(theta), s = sin(theta);"),
    "cx_direction": ("apply_cx(psi, n, q, q + 1);\n}", "apply_cx(psi, n, q + 1, q);\n}"),
    "cx_order": ("for (int q = 0; q + 1 < n; ++q) apply_cx(psi, n, q, q + 1);",
                 "for (int q = n - 2; q >= 0; --q) apply_cx(psi, n, q, q + 1);"),
    "y_phase": ("phase *= b ? -I : I;", "phase *= b ? I : -I;"),
    "z_sign_dropped": ("if (b) phase = -phase;", "(void)b;"),
    "last_term_dropped": ("for (int k = 0; k < n_terms; ++k) {", "for (int k = 0; k + 1 < n_terms; ++k) {"),
    "grad_sign": ("acc += cimag(conj(lam[x]) * ypsi);", "acc -= cimag(conj(lam[x]) * ypsi);"),
    "theta_index": ("apply_ry(psi, n, q, theta[r * n + q]);", "apply_ry(psi, n, q, theta[q * (reps + 1) + r]);"),
    "shift_half": ("grad[p] = 0.5 * (ep - em);", "grad[p] = (ep - em);"),
    "unapply_skipped": ("apply_ry(lam, n, q, -theta[p]);", "(void)0;"),
}


def _pins_pass(lib) -> bool:
    """Run a compact set of pins against a (possibly mutated) oracle library."""
    try:
        n, reps = 5, 2
        rng = np.random.default_rng(1)
        strings = []
        for _ in range(12):
            w = int(rng.integers(1, 4))
            s = ["I"] * n
            for q in rng.choice(n, size=w, replace=False):
                s[int(q)] = "XYZ"[int(rng.integers(0, 3))]
            strings.append("".join(s))
        coeffs = rng.standard_normal(len(strings))
        scale = np.abs(coeffs).sum()
        th = wl.thetas(n, reps, 1, seed=3)[0]
        psi = oracle.state(n, reps, th, lib=lib)
        if np.max(np.abs(psi - dense.state(n, reps, th))) > 1e-12:
            return False
        hp = oracle.apply_hamiltonian(n, strings, coeffs, psi, lib=lib)
        if np.max(np.abs(hp - dense.hamiltonian(strings, coeffs) @ psi)) > 1e-12 * scale:
            return False
        e, g = oracle.energy_grad(n, reps, th, strings, coeffs, lib=lib)
        if abs(e - dense.energy(n, reps, th, strings, coeffs)) > 1e-12 * scale:
            return False
        if np.max(np.abs(g - dense.param_shift_grad(n, reps, th, strings, coeffs))) > 1e-11 * scale:
            return False
        gs = oracle.param_shift_grad(n, reps, th, strings, coeffs, lib=lib)
        if np.max(np.abs(gs - g)) > 1e-11 * scale:
            return False
        ham = wl.z_hamiltonian(n, 15, seed=2)
        t1 = wl.thetas(n, 1, 1, seed=4)[0]
        e1 = oracle.energy(n, 1, t1, ham.strings, ham.coeffs, lib=lib)
        if abs(e1 - closed_form.heisenberg_reps1_energy(n, t1, ham.strings, ham.coeffs)) > 1e-12 * ham.abs_sum():
            return False
        return True
    except RuntimeError:
        return False


def test_unmutated_oracle_passes_compact_pins():
    assert _pins_pass(oracle.load())


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_fails_a_pin(name, tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) >= 1, f"mutation anchor for {name} not found"
    src = tmp_path / "mutant.c"
    src.write_text(text.replace(old, new, 1))
    lib_path = str(tmp_path / "libmutant.so")
    oracle.build(force=True, src=str(src), out=lib_path)
    lib = oracle.load(lib_path)
    assert not _pins_pass(lib), f"mutant {name} survived every pin"
