"""The full EfficientSU2 rotation layer (RY then RZ on every qubit, Eq. 8;
complex amplitudes) on the GPU against the oracle with gate set 2: energies and
adjoint gradients (RY and RZ entries) in FP32 and FP64, several entanglers, the
whole-register kernel (n <= 8) and tile sizes that force strided passes, reps = 0,
active masks, the parameter-shift comparator, and the calls that refuse the
complex path."""
import numpy as np
import pytest

import oracle
from paper_2607_02749_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2607_02749_gb300 as gv  # noqa: E402

RYRZ = gv.GVQE_GATES_RY_RZ


def _thetas(n, reps, batch, seed):
    return np.random.default_rng(seed).uniform(-np.pi, np.pi, (batch, 2 * n * (reps + 1)))


def _ref(n, reps, th, ham, ent=0):
    es, gs = [], []
    with oracle.entangler(ent), oracle.gates(oracle.GATES_RY_RZ):
        for row in th:
            e, g = oracle.energy_grad(n, reps, row, ham.strings, ham.coeffs)
            es.append(e)
            gs.append(g)
    return np.array(es), np.array(gs)


def _check(e, g, er, gr, scale, fp64):
    if fp64:
        assert np.max(np.abs(e - er)) <= 1e-10 * scale
        assert np.max(np.abs(g - gr)) <= 1e-9 * scale
    else:
        assert np.max(np.abs(e - er)) <= 2e-5 * scale
        for row, ref in zip(g, gr):
            assert np.linalg.norm(row - ref) <= 1e-4 * max(np.linalg.norm(ref), 1e-3 * scale)


@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("n,reps,tb,ent", [(1, 2, 0, 0), (2, 1, 0, 1), (5, 2, 0, 5), (8, 3, 0, 0), (8, 0, 0, 0),
                                           (9, 2, 0, 0), (11, 1, 0, 1), (12, 3, 0, 0), (12, 0, 0, 0),
                                           (14, 2, 0, 5), (14, 2, 10, 0), (17, 2, 11, 2), (16, 1, 12, 4)])
def test_energy_and_gradient_match_the_oracle(n, reps, tb, ent, fp64):
    if fp64 and tb > 12:
        pytest.skip("FP64 tiles are at most 2^12 amplitudes")
    ham = wl.chain_z_hamiltonian(n, 8 * n, seed=n + reps)
    th = _thetas(n, reps, 2, seed=n + 10 * reps + ent)
    a = gv.Ansatz(n, reps, entangler=ent, gates=RYRZ, tile_bits=tb)
    h = gv.Hamiltonian.from_workload(ham)
    t = torch.as_tensor(th, device="cuda")
    e_only = gv.energy(a, h, t, fp64=fp64).cpu().numpy()
    e, g = gv.energy_grad(a, h, t, fp64=fp64)
    er, gr = _ref(n, reps, th, ham, ent)
    scale = ham.abs_sum()
    _check(e_only, g.cpu().numpy(), er, gr, scale, fp64)
    _check(e.cpu().numpy(), g.cpu().numpy(), er, gr, scale, fp64)


@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("n,reps", [(3, 2), (8, 1), (11, 2), (14, 1)])
def test_pauli_hamiltonians_with_odd_y_strings(n, reps, fp64):
    """X/Y strings on complex states: strings with an odd number of Y letters
    now contribute (i^#Y is imaginary), through the complex X-mask group kernel."""
    ham = wl.pauli_hamiltonian(n, 12 * n, seed=n + 40)
    assert any(sum(ch == "Y" for ch in s) % 2 == 1 for s in ham.strings)
    th = _thetas(n, reps, 2, seed=n + 50)
    a = gv.Ansatz(n, reps, gates=RYRZ)
    h = gv.Hamiltonian.from_workload(ham)
    t = torch.as_tensor(th, device="cuda")
    e_only = gv.energy(a, h, t, fp64=fp64).cpu().numpy()
    e, g = gv.energy_grad(a, h, t, fp64=fp64)
    er, gr = _ref(n, reps, th, ham)
    scale = ham.abs_sum()
    _check(e_only, g.cpu().numpy(), er, gr, scale, fp64)
    _check(e.cpu().numpy(), g.cpu().numpy(), er, gr, scale, fp64)


def test_masks_and_parameter_shift():
    n, reps = 11, 2
    ham = wl.z_hamiltonian(n, 90, seed=3)
    th = _thetas(n, reps, 2, seed=4)
    mask = wl.active_mask(2 * n * (reps + 1), 2, seed=5)
    a = gv.Ansatz(n, reps, gates=RYRZ)
    h = gv.Hamiltonian.from_workload(ham)
    t = torch.as_tensor(th, device="cuda")
    m = torch.as_tensor(mask, device="cuda")
    _, g = gv.energy_grad(a, h, t, mask=m, fp64=True)
    _, gs = gv.energy_grad(a, h, t, mask=m, fp64=True, param_shift=True)
    _, gr = _ref(n, reps, th, ham)
    g, gs = g.cpu().numpy(), gs.cpu().numpy()
    scale = ham.abs_sum()
    assert np.all(g[mask == 0] == 0.0) and np.all(gs[mask == 0] == 0.0)
    assert np.max(np.abs(g - gr * mask)) <= 1e-9 * scale
    assert np.max(np.abs(gs - gr * mask)) <= 1e-9 * scale


def test_zero_rz_angles_give_the_ry_ansatz():
    n, reps = 13, 2
    ham = wl.z_hamiltonian(n, 120, seed=6)
    ty = wl.thetas(n, reps, 1, seed=7)[0].reshape(reps + 1, n)
    th2 = np.concatenate([np.concatenate([ty[r], np.zeros(n)]) for r in range(reps + 1)])[None, :]
    a2 = gv.Ansatz(n, reps, gates=RYRZ)
    a1 = gv.Ansatz(n, reps)
    h = gv.Hamiltonian.from_workload(ham)
    e2, g2 = gv.energy_grad(a2, h, torch.as_tensor(th2, device="cuda"), fp64=True)
    e1, g1 = gv.energy_grad(a1, h, torch.as_tensor(ty.reshape(1, -1), device="cuda"), fp64=True)
    assert abs(e2.item() - e1.item()) <= 1e-10 * ham.abs_sum()
    g2 = g2.cpu().numpy()[0].reshape(reps + 1, 2, n)
    assert np.max(np.abs(g2[:, 0, :] - g1.cpu().numpy()[0].reshape(reps + 1, n))) <= 1e-9 * ham.abs_sum()


def test_fullsize_fp32_against_fp64():
    n, reps = 24, 2
    ham = wl.z_hamiltonian(n, 1500, seed=0)
    a = gv.Ansatz(n, reps, gates=RYRZ)
    h = gv.Hamiltonian.from_workload(ham)
    t = torch.as_tensor(_thetas(n, reps, 1, seed=1), device="cuda")
    e32, g32 = gv.energy_grad(a, h, t)
    e64, g64 = gv.energy_grad(a, h, t, fp64=True)
    scale = ham.abs_sum()
    assert abs(e32.item() - e64.item()) <= 2e-5 * scale
    g32, g64 = g32.cpu().numpy()[0], g64.cpu().numpy()[0]
    assert np.linalg.norm(g32 - g64) <= 1e-4 * max(np.linalg.norm(g64), 1e-3 * scale)


def test_unsupported_calls_refuse_the_complex_path():
    n = 10
    a = gv.Ansatz(n, 1, gates=RYRZ)
    t = torch.zeros((1, a.n_params), dtype=torch.float64, device="cuda")
    hz = gv.Hamiltonian.from_workload(wl.z_hamiltonian(n, 30, seed=1))
    with pytest.raises(gv.GvqeError) as e:
        gv._lib.gvqe_energy_static(a.handle, hz.handle, t, torch.empty(1, dtype=torch.float64, device="cuda"), 0, None)
    assert e.value.code == gv._lib.GVQE_EUNSUPPORTED


def test_batch_of_complex_instances():
    insts = wl.cluster_batch(4, qubit_range=(10, 13), reps_range=(1, 2), terms_per_qubit=15)
    ans = [gv.Ansatz(i.n_qubits, i.reps, gates=RYRZ) for i in insts]
    hams = [gv.Hamiltonian.from_workload(i.ham) for i in insts]
    b = gv.Batch(ans, hams, fp64=True)
    params = [torch.as_tensor(_thetas(i.n_qubits, i.reps, 1, seed=k)[0], device="cuda") for k, i in enumerate(insts)]
    grads = [torch.empty_like(p) for p in params]
    e = b.run(params, grads=grads).cpu().numpy()
    for k, i in enumerate(insts):
        er, gr = _ref(i.n_qubits, i.reps, params[k].cpu().numpy()[None, :], i.ham)
        assert abs(e[k] - er[0]) <= 1e-10 * i.ham.abs_sum()
        assert np.max(np.abs(grads[k].cpu().numpy() - gr[0])) <= 1e-9 * i.ham.abs_sum()


@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("n,reps", [(6, 2), (12, 1), (15, 2)])
def test_readout_of_the_complex_state(n, reps, fp64):
    from oracle import readout as ro

    ham = wl.chain_z_hamiltonian(n, 10 * n, seed=n)
    th = _thetas(n, reps, 1, seed=2 * n)[0]
    with oracle.gates(oracle.GATES_RY_RZ):
        p = ro.probabilities(oracle.state(n, reps, th))
    e = ro.diagonal_energies(n, ham.strings, ham.coeffs)
    a = gv.Ansatz(n, reps, gates=RYRZ)
    h = gv.Hamiltonian.from_workload(ham)
    tol = 1e-12 if fp64 else 2e-6
    u = np.random.Generator(np.random.PCG64(0)).random(2048)
    r = gv.readout(a, h, torch.as_tensor(th, device="cuda"), alpha=0.2,
                   uniforms=torch.as_tensor(u, device="cuda"), fp64=fp64)
    assert abs(r.total - 1.0) <= 4 * tol * (1 << n) ** 0.5 + 4 * tol
    xo, po = ro.most_probable(p)
    assert p[r.argmax] >= po - 8 * tol
    assert abs(r.cvar - ro.cvar(p, e, 0.2)) <= (1e-10 if fp64 else 2e-5) * ham.abs_sum()
    s = r.shots.cpu().numpy()
    cdf = np.cumsum(p)
    t = u * cdf[-1]
    slack = 8 * tol * (1 << n) ** 0.5
    lo = np.where(s > 0, cdf[np.maximum(s - 1, 0)], 0.0)
    assert np.all(lo <= t + slack) and np.all(t < cdf[s] + slack)
