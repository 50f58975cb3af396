"""Pins for the CPU oracle: it is checked against things other than itself.

* P1 dense brute force (Kronecker-product matrices, n <= 8): state, H psi,
  energy, ground energy of a diagonal H, gradients.
* P2 reps = 0 product-state closed form, any Pauli letters.
* P3 reps = 1 Heisenberg-picture closed form for Z strings.
* P4 theta = 0 and P5 theta in {0, pi}: basis states.
* P6 degree-one trigonometric structure in every angle (Eq. 13 exact,
  central differences equal E' sin(h)/h, 2*pi periodicity).
* P7 invariants: norm, real amplitudes, odd-#Y strings give zero, term order.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import closed_form, dense
from paper_2607_02749_gb300 import workloads as wl


def _rand_paulis(rng, n, m, letters="XYZ", max_w=4):
    strings = []
    for _ in range(m):
        w = int(rng.integers(1, min(max_w, n) + 1))
        qs = rng.choice(n, size=w, replace=False)
        s = ["I"] * n
        for q in qs:
            s[int(q)] = letters[int(rng.integers(0, len(letters)))]
        strings.append("".join(s))
    return strings, rng.standard_normal(m)


@pytest.mark.parametrize("n,reps", [(1, 0), (1, 2), (2, 1), (3, 2), (4, 3), (5, 1), (6, 2), (7, 1)])
def test_state_matches_dense(n, reps):
    th = wl.thetas(n, reps, 1, seed=n * 10 + reps)[0]
    psi = oracle.state(n, reps, th)
    ref = dense.state(n, reps, th)
    assert np.max(np.abs(psi - ref)) < 1e-13


@pytest.mark.parametrize("n", [1, 2, 3, 5, 6])
def test_apply_hamiltonian_matches_dense(n):
    rng = np.random.default_rng(n)
    strings, coeffs = _rand_paulis(rng, n, 12, letters="IXYZ")
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    out = oracle.apply_hamiltonian(n, strings, coeffs, psi)
    ref = dense.hamiltonian(strings, coeffs) @ psi
    assert np.max(np.abs(out - ref)) < 1e-12 * np.abs(coeffs).sum() * np.abs(psi).max()


@pytest.mark.parametrize("n,reps", [(3, 1), (4, 2), (6, 2), (8, 1)])
def test_energy_and_gradient_match_dense(n, reps):
    rng = np.random.default_rng(100 + n)
    strings, coeffs = _rand_paulis(rng, n, 15)
    th = wl.thetas(n, reps, 1, seed=7 + n)[0]
    scale = np.abs(coeffs).sum()
    e, g = oracle.energy_grad(n, reps, th, strings, coeffs)
    assert abs(e - dense.energy(n, reps, th, strings, coeffs)) < 1e-12 * scale
    gd = dense.param_shift_grad(n, reps, th, strings, coeffs)
    assert np.max(np.abs(g - gd)) < 1e-11 * scale
    assert abs(oracle.energy(n, reps, th, strings, coeffs) - e) < 1e-12 * scale


def test_diagonal_ground_energy_is_min_eigenvalue():
    n = 6
    ham = wl.z_hamiltonian(n, 30, seed=3)
    best = math.inf
    for y in range(1 << n):
        flips = [(y >> q) & 1 for q in range(n)]
        th = np.array(flips, dtype=np.float64) * math.pi
        best = min(best, oracle.energy(n, 0, th, ham.strings, ham.coeffs))
    lo = np.linalg.eigvalsh(dense.hamiltonian(ham.strings, ham.coeffs)).min()
    assert abs(best - lo) < 1e-9 * ham.abs_sum()


@pytest.mark.parametrize("n", [1, 4, 9, 12])
def test_product_state_closed_form(n):
    rng = np.random.default_rng(200 + n)
    strings, coeffs = _rand_paulis(rng, n, 40)
    th = wl.thetas(n, 0, 1, seed=n)[0]
    e, g = oracle.energy_grad(n, 0, th, strings, coeffs)
    scale = np.abs(coeffs).sum()
    assert abs(e - closed_form.product_state_energy(th, strings, coeffs)) < 1e-12 * scale
    assert np.max(np.abs(g - closed_form.product_state_grad(th, strings, coeffs))) < 1e-12 * scale


@pytest.mark.parametrize("n", [2, 5, 8, 11])
def test_heisenberg_reps1_closed_form(n):
    ham = wl.z_hamiltonian(n, 25, seed=n)
    th = wl.thetas(n, 1, 1, seed=40 + n)[0]
    e, g = oracle.energy_grad(n, 1, th, ham.strings, ham.coeffs)
    scale = ham.abs_sum()
    fn = lambda t: closed_form.heisenberg_reps1_energy(n, t, ham.strings, ham.coeffs)
    assert abs(e - fn(th)) < 1e-12 * scale
    assert np.max(np.abs(g - closed_form.shift_grad(fn, th))) < 1e-11 * scale


def test_zero_angles_give_all_zero_state():
    n, reps = 7, 3
    rng = np.random.default_rng(5)
    strings, coeffs = _rand_paulis(rng, n, 30)
    th = np.zeros(n * (reps + 1))
    e, g = oracle.energy_grad(n, reps, th, strings, coeffs)
    assert abs(e - closed_form.zero_angle_energy(strings, coeffs)) < 1e-13 * np.abs(coeffs).sum()
    ham = wl.z_hamiltonian(n, 30, seed=1)
    _, gz = oracle.energy_grad(n, reps, th, ham.strings, ham.coeffs)
    assert np.all(gz == 0.0)


@pytest.mark.parametrize("n,reps", [(5, 1), (7, 2), (9, 3)])
def test_basis_state_angles(n, reps):
    rng = np.random.default_rng(n + reps)
    ham = wl.z_hamiltonian(n, 40, seed=n)
    for _ in range(4):
        flips = rng.integers(0, 2, size=n * (reps + 1))
        th = flips.astype(np.float64) * math.pi
        e = oracle.energy(n, reps, th, ham.strings, ham.coeffs)
        ref = closed_form.basis_state_energy(n, reps, flips, ham.strings, ham.coeffs)
        assert abs(e - ref) < 1e-13 * ham.abs_sum()


def test_degree_one_structure_and_exact_shift_rule():
    n, reps = 6, 2
    rng = np.random.default_rng(11)
    strings, coeffs = _rand_paulis(rng, n, 25)
    th = wl.thetas(n, reps, 1, seed=2)[0]
    scale = np.abs(coeffs).sum()
    _, g = oracle.energy_grad(n, reps, th, strings, coeffs)
    gs = oracle.param_shift_grad(n, reps, th, strings, coeffs)
    assert np.max(np.abs(g - gs)) < 1e-12 * scale
    for p in (0, 7, n * (reps + 1) - 1):
        def E(t):
            tt = th.copy()
            tt[p] = t
            return oracle.energy(n, reps, tt, strings, coeffs)
        t0 = th[p]
        # E(t) + E(t + pi) is constant (= 2 gamma)
        assert abs((E(t0) + E(t0 + math.pi)) - (E(t0 + 0.5) + E(t0 + 0.5 + math.pi))) < 1e-12 * scale
        # 2 pi periodicity
        assert abs(E(t0) - E(t0 + 2 * math.pi)) < 1e-12 * scale
        # central difference equals E' sin(h)/h exactly
        h = 1e-1
        fd = (E(t0 + h) - E(t0 - h)) / (2 * h)
        assert abs(fd - g[p] * math.sin(h) / h) < 1e-11 * scale


def test_invariants_norm_real_amplitudes_odd_y():
    n, reps = 8, 3
    th = wl.thetas(n, reps, 1, seed=9)[0]
    for r in range(reps + 1):
        psi = oracle.state(n, r, th[: n * (r + 1)])
        assert abs(np.vdot(psi, psi).real - 1.0) < 1e-12
        assert np.all(psi.imag == 0.0)
    # strings with an odd number of Y letters give exactly zero on a real state
    odd = ["YIIIIIII", "IYZIIIII", "XYIZIIII", "YYYIIIII", "IIIIZXXY"]
    e, ei = oracle.energy(n, reps, th, odd, np.ones(len(odd)), with_imag=True)
    assert e == 0.0 and abs(ei) < 1e-14
    _, g = oracle.energy_grad(n, reps, th, odd, np.ones(len(odd)))
    assert np.max(np.abs(g)) < 1e-14


def test_term_order_invariance_and_string_convention():
    n, reps = 7, 2
    ham = wl.pauli_hamiltonian(n, 40, seed=4)
    th = wl.thetas(n, reps, 1, seed=3)[0]
    e = oracle.energy(n, reps, th, ham.strings, ham.coeffs)
    perm = np.random.default_rng(0).permutation(ham.n_terms)
    ep = oracle.energy(n, reps, th, [ham.strings[i] for i in perm], ham.coeffs[perm])
    assert abs(e - ep) < 1e-12 * ham.abs_sum()
    # character i acts on qubit i: reversing the strings changes the energy
    er = oracle.energy(n, reps, th, [s[::-1] for s in ham.strings], ham.coeffs)
    assert abs(e - er) > 1e-3


def test_duplicate_strings_are_summed():
    n, reps = 5, 1
    th = wl.thetas(n, reps, 1, seed=1)[0]
    s = ["ZZIII", "IXIYI"]
    e1 = oracle.energy(n, reps, th, [s[0], s[0], s[1]], [1.5, 2.0, -0.5])
    e2 = oracle.energy(n, reps, th, [s[0], s[1]], [3.5, -0.5])
    assert abs(e1 - e2) < 1e-13


def test_masked_param_shift_zeroes_inactive_entries():
    n, reps = 4, 1
    ham = wl.z_hamiltonian(n, 10, seed=2)
    th = wl.thetas(n, reps, 1, seed=2)[0]
    mask = np.array([1, 0, 1, 0, 0, 1, 1, 0], dtype=np.uint8)
    g = oracle.param_shift_grad(n, reps, th, ham.strings, ham.coeffs, mask=mask)
    _, full = oracle.energy_grad(n, reps, th, ham.strings, ham.coeffs)
    assert np.all(g[mask == 0] == 0.0)
    assert np.max(np.abs(g[mask == 1] - full[mask == 1])) < 1e-12 * ham.abs_sum()


ALL_ENTS = [oracle.ENT_LINEAR, oracle.ENT_CIRCULAR, oracle.ENT_FULL, oracle.ENT_REVERSE_LINEAR,
            oracle.ENT_PAIRWISE, oracle.ENT_SCA]


@pytest.mark.parametrize("ent", ALL_ENTS)
def test_entangler_pins(ent):
    """Every entangler (Section IV-B, Table 2): the C oracle equals the dense
    matrix model, signed basis states follow the closed-form GF(2) index maps,
    and the adjoint gradient equals the dense parameter-shift gradient."""
    rng = np.random.default_rng(11 + ent)
    for n, reps in ((1, 2), (2, 3), (3, 1), (4, 3), (5, 2), (7, 1)):
        th = wl.thetas(n, reps, 1, seed=n + ent)[0]
        ham = wl.pauli_hamiltonian(n, 10, seed=n)
        with oracle.entangler(ent):
            psi = oracle.state(n, reps, th)
            assert np.max(np.abs(psi - dense.state(n, reps, th, ent))) < 1e-12
            flips = rng.integers(0, 2, size=n * (reps + 1))
            b = oracle.state(n, reps, np.where(flips == 1, math.pi, 0.0))
            assert int(np.argmax(np.abs(b))) == closed_form.basis_state_index(n, reps, flips, ent)
            e, g = oracle.energy_grad(n, reps, th, ham.strings, ham.coeffs)
        scale = ham.abs_sum()
        assert abs(e - dense.energy(n, reps, th, ham.strings, ham.coeffs, ent)) < 1e-12 * scale
        assert np.max(np.abs(g - dense.param_shift_grad(n, reps, th, ham.strings, ham.coeffs, ent))) < 1e-11 * scale


def test_entangler_maps_are_the_cnot_products():
    """The closed-form maps agree with the CNOT lists applied to bit vectors."""
    for n in range(1, 9):
        for ent in ALL_ENTS:
            for layer in (1, 2, 3, 4) if ent == oracle.ENT_SCA else (1,):
                for x in range(1 << n):
                    y = x
                    for c, t in dense.entangler_pairs(n, ent, layer):
                        if (y >> c) & 1:
                            y ^= 1 << t
                    assert y == closed_form.entangler_map(x, n, ent, layer)


def _entangler_unitary(n, ent, layer=1):
    u = np.eye(1 << n)
    for c, t in dense.entangler_pairs(n, ent, layer):
        u = dense.cnot(c, t, n) @ u
    return u


def test_reverse_linear_is_the_full_entangler():
    """A textbook identity: the descending CX chain and the all-pairs CX list in
    lexicographic order are the same unitary."""
    for n in range(2, 7):
        assert np.array_equal(_entangler_unitary(n, oracle.ENT_REVERSE_LINEAR), _entangler_unitary(n, oracle.ENT_FULL))
        assert not np.array_equal(_entangler_unitary(n, oracle.ENT_REVERSE_LINEAR),
                                  _entangler_unitary(n, oracle.ENT_LINEAR)) or n == 2


def _kron_layer(n, pairs):
    """One layer of disjoint nearest-neighbour CNOTs CX(q, q+1) built by Kronecker
    products (qubit q is bit q, so the rightmost factor is qubit 0)."""
    cx = np.array([[1, 0, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0], [0, 1, 0, 0]], dtype=float)  # ctl bit 0, tgt bit 1
    ops, q = [], 0
    starts = {c for c, _ in pairs}
    while q < n:
        if q in starts:
            ops.append(cx)
            q += 2
        else:
            ops.append(np.eye(2))
            q += 1
    u = np.eye(1)
    for op in ops:
        u = np.kron(op, u)
    return u


def test_pairwise_is_two_layers_of_disjoint_cnots():
    for n in range(2, 8):
        even = [(q, q + 1) for q in range(0, n - 1, 2)]
        odd = [(q, q + 1) for q in range(1, n - 1, 2)]
        want = _kron_layer(n, odd) @ _kron_layer(n, even)
        assert np.array_equal(_entangler_unitary(n, oracle.ENT_PAIRWISE), want)


def test_sca_is_the_shifted_circular_entangler_alternating_direction():
    """SCA at offset o = layer - 1 is the circular entangler with every qubit q
    relabelled q - o (mod n); on odd offsets every CNOT is reversed, which is
    conjugation of the whole list by Hadamards on every qubit."""
    for n in range(2, 7):
        circ = _entangler_unitary(n, oracle.ENT_CIRCULAR)
        hn = dense.embed({q: np.array([[1, 1], [1, -1]]) / math.sqrt(2) for q in range(n)}, n).real
        for layer in range(1, 2 * n + 2):
            o = layer - 1
            perm = np.zeros((1 << n, 1 << n))
            for x in range(1 << n):
                xr = 0
                for q in range(n):
                    xr |= ((x >> q) & 1) << ((q - o) % n)
                perm[xr, x] = 1.0
            want = perm @ circ @ perm.T
            if o % 2:
                want = hn @ want @ hn
            assert np.allclose(_entangler_unitary(n, oracle.ENT_SCA, layer), want, atol=1e-12), (n, layer)


# ---------------------------------------------------------- EfficientSU2 --
# The full rotation layer of Eq. 8: RY then RZ on every qubit, P = 2 n (D+1).

@pytest.mark.parametrize("ent", [oracle.ENT_LINEAR, oracle.ENT_CIRCULAR, oracle.ENT_SCA])
def test_su2_oracle_matches_the_dense_model(ent):
    rng = np.random.default_rng(31 + ent)
    for n, reps in ((1, 2), (2, 1), (3, 2), (5, 1), (6, 2)):
        th = rng.uniform(-np.pi, np.pi, 2 * n * (reps + 1))
        ham = wl.pauli_hamiltonian(n, 12, seed=n + 3)
        with oracle.entangler(ent), oracle.gates(oracle.GATES_RY_RZ):
            psi = oracle.state(n, reps, th)
            e, g = oracle.energy_grad(n, reps, th, ham.strings, ham.coeffs)
            gs = oracle.param_shift_grad(n, reps, th, ham.strings, ham.coeffs)
        assert np.max(np.abs(psi - dense.state(n, reps, th, ent, 2))) < 1e-12
        scale = ham.abs_sum()
        assert abs(e - dense.energy(n, reps, th, ham.strings, ham.coeffs, ent, 2)) < 1e-12 * scale
        gd = dense.param_shift_grad(n, reps, th, ham.strings, ham.coeffs, ent, 2)
        assert np.max(np.abs(g - gd)) < 1e-11 * scale
        assert np.max(np.abs(gs - g)) < 1e-11 * scale  # Eq. 13 is exact for RZ too


def test_su2_product_state_closed_form():
    rng = np.random.default_rng(5)
    for n in (1, 4, 9, 12):
        ty, tz = rng.uniform(-np.pi, np.pi, n), rng.uniform(-np.pi, np.pi, n)
        ham = wl.pauli_hamiltonian(n, 40, seed=n)
        with oracle.gates(oracle.GATES_RY_RZ):
            e = oracle.energy(n, 0, np.concatenate([ty, tz]), ham.strings, ham.coeffs)
        want = closed_form.su2_product_state_energy(ty, tz, ham.strings, ham.coeffs)
        assert e == pytest.approx(want, abs=1e-12 * ham.abs_sum())


def test_su2_with_zero_rz_angles_is_the_ry_circuit_and_phases_keep_basis_states():
    n, reps = 6, 2
    rng = np.random.default_rng(8)
    ty = rng.uniform(-np.pi, np.pi, (reps + 1, n))
    th2 = np.concatenate([np.concatenate([ty[r], np.zeros(n)]) for r in range(reps + 1)])
    with oracle.gates(oracle.GATES_RY_RZ):
        psi2 = oracle.state(n, reps, th2)
    assert np.max(np.abs(psi2 - oracle.state(n, reps, ty.reshape(-1)))) < 1e-13
    # RY angles in {0, pi} with arbitrary RZ angles: a basis state up to a phase
    flips = rng.integers(0, 2, size=(reps + 1, n))
    th3 = np.concatenate([np.concatenate([np.pi * flips[r], rng.uniform(-3, 3, n)]) for r in range(reps + 1)])
    with oracle.gates(oracle.GATES_RY_RZ):
        psi3 = oracle.state(n, reps, th3)
    y = closed_form.basis_state_index(n, reps, flips.reshape(-1))
    assert abs(abs(psi3[y]) - 1.0) < 1e-12
    ham = wl.z_hamiltonian(n, 30, seed=1)
    with oracle.gates(oracle.GATES_RY_RZ):
        e = oracle.energy(n, reps, th3, ham.strings, ham.coeffs)
    want = closed_form.basis_state_energy(n, reps, flips.reshape(-1), ham.strings, ham.coeffs)
    assert e == pytest.approx(want, abs=1e-12 * ham.abs_sum())
