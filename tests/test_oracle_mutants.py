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
    "cx_direction": ("ctl[k] = q;\n        tgt[k++] = q + 1;", "ctl[k] = q + 1;\n        tgt[k++] = q;"),
    "cx_order": ("for (int g = 0; g < k; ++g) apply_cx(psi, n, ctl[g], tgt[g]);",
                 "for (int g = k - 1; g >= 0; --g) apply_cx(psi, n, ctl[g], tgt[g]);"),
    "circular_wrap_after_chain": (
        "    if ((g_entangler == 1 || g_entangler == 5) && n > 1) {\n        ctl[k] = n - 1;\n        tgt[k++] = 0;\n    }\n"
        "    for (int q = 0; q + 1 < n; ++q) {\n        ctl[k] = q;\n        tgt[k++] = q + 1;\n    }\n",
        "    for (int q = 0; q + 1 < n; ++q) {\n        ctl[k] = q;\n        tgt[k++] = q + 1;\n    }\n"
        "    if ((g_entangler == 1 || g_entangler == 5) && n > 1) {\n        ctl[k] = n - 1;\n        tgt[k++] = 0;\n    }\n"),
    "circular_wrap_direction": ("        ctl[k] = n - 1;\n        tgt[k++] = 0;", "        ctl[k] = 0;\n        tgt[k++] = n - 1;"),
    "full_controls_descending": ("for (int i = 0; i < n; ++i)\n            for (int j = i + 1; j < n; ++j)",
                                 "for (int i = n - 1; i >= 0; --i)\n            for (int j = i + 1; j < n; ++j)"),
    "reverse_linear_ascending": ("for (int q = n - 2; q >= 0; --q) {", "for (int q = 0; q <= n - 2; ++q) {"),
    "pairwise_odd_pairs_first": ("for (int start = 0; start < 2; ++start)", "for (int start = 1; start >= 0; --start)"),
    "pairwise_one_half_only": ("for (int start = 0; start < 2; ++start)", "for (int start = 0; start < 1; ++start)"),
    "sca_rotated_left": ("c2[(g + o) % k] = ctl[g];\n            t2[(g + o) % k] = tgt[g];",
                         "c2[(g + k - o) % k] = ctl[g];\n            t2[(g + k - o) % k] = tgt[g];"),
    "sca_never_swapped": ("const int swap = (layer - 1) & 1;", "const int swap = 0;"),
    "sca_swapped_on_even": ("const int swap = (layer - 1) & 1;", "const int swap = layer & 1;"),
    "sca_offset_from_layer": ("const int o = (layer - 1) % k;", "const int o = layer % k;"),
    "adjoint_wrong_layer_entangler": ("apply_entangler_inverse(psi, n, r);\n            apply_entangler_inverse(lam, n, r);",
                                      "apply_entangler_inverse(psi, n, 1);\n            apply_entangler_inverse(lam, n, 1);"),
    "rz_phase_sign": ("const cplx p0 = cos(0.5 * theta) - I * sin(0.5 * theta);",
                      "const cplx p0 = cos(0.5 * theta) + I * sin(0.5 * theta);"),
    "rz_before_ry": ("    for (int q = 0; q < n; ++q) apply_ry(psi, n, q, theta[base + q]);\n    if (g_gates == 2)\n"
                     "        for (int q = 0; q < n; ++q) apply_rz(psi, n, q, theta[base + n + q]);",
                     "    if (g_gates == 2)\n        for (int q = 0; q < n; ++q) apply_rz(psi, n, q, theta[base + n + q]);\n"
                     "    for (int q = 0; q < n; ++q) apply_ry(psi, n, q, theta[base + q]);"),
    "rz_grad_sign": ("const cplx zpsi = (x & bit) ? -psi[x] : psi[x];", "const cplx zpsi = (x & bit) ? psi[x] : -psi[x];"),
    "rz_param_index": ("const int p = base + n + q;", "const int p = base + q;"),
    "rz_not_unapplied": ("apply_rz(lam, n, q, -theta[p]);", "(void)0;"),
    "y_phase": ("phase *= b ? -I : I;", "phase *= b ? I : -I;"),
    "z_sign_dropped": ("if (b) phase = -phase;", "(void)b;"),
    "last_term_dropped": ("for (int k = 0; k < n_terms; ++k) {", "for (int k = 0; k + 1 < n_terms; ++k) {"),
    "grad_sign": ("acc += cimag(conj(lam[x]) * ypsi);", "acc -= cimag(conj(lam[x]) * ypsi);"),
    "theta_index": ("for (int q = 0; q < n; ++q) apply_ry(psi, n, q, theta[base + q]);",
                    "for (int q = 0; q < n; ++q) apply_ry(psi, n, q, theta[base + n - 1 - q]);"),
    "layer_stride_ignores_rz": ("const int base = r * g_gates * n;\n    for (int q = 0; q < n; ++q) apply_ry",
                                "const int base = r * n;\n    for (int q = 0; q < n; ++q) apply_ry"),
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
        # the other entanglers: the dense model, and the basis-index maps of closed_form
        for ent in (oracle.ENT_CIRCULAR, oracle.ENT_FULL, oracle.ENT_REVERSE_LINEAR, oracle.ENT_PAIRWISE,
                    oracle.ENT_SCA):
            with oracle.entangler(ent, lib=lib):
                if np.max(np.abs(oracle.state(n, reps, th, lib=lib) - dense.state(n, reps, th, ent))) > 1e-12:
                    return False
                flips = np.random.default_rng(ent).integers(0, 2, size=n * (reps + 1))
                psi = oracle.state(n, reps, np.where(flips == 1, math.pi, 0.0), lib=lib)
                if int(np.argmax(np.abs(psi))) != closed_form.basis_state_index(n, reps, flips, ent):
                    return False
                e, g = oracle.energy_grad(n, reps, th, strings, coeffs, lib=lib)
                if np.max(np.abs(g - dense.param_shift_grad(n, reps, th, strings, coeffs, ent))) > 1e-11 * scale:
                    return False
        # the full EfficientSU2 layer (RY then RZ): the dense model and its gradient
        th2 = np.random.default_rng(9).uniform(-3, 3, 2 * n * (reps + 1))
        with oracle.gates(oracle.GATES_RY_RZ, lib=lib):
            if np.max(np.abs(oracle.state(n, reps, th2, lib=lib) - dense.state(n, reps, th2, 0, 2))) > 1e-12:
                return False
            e, g = oracle.energy_grad(n, reps, th2, strings, coeffs, lib=lib)
        if abs(e - dense.energy(n, reps, th2, strings, coeffs, 0, 2)) > 1e-12 * scale:
            return False
        if np.max(np.abs(g - dense.param_shift_grad(n, reps, th2, strings, coeffs, 0, 2))) > 1e-11 * scale:
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
