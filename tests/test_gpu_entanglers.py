"""Circular, full, reverse-linear, pairwise and SCA entanglers (Section IV-B,
Table 2) on the GPU against the oracle:
energies and adjoint gradients (FP32 and FP64, whole-register and tile paths,
diagonal and X/Y Hamiltonians), the parameter-shift comparator, readout, the
persistent batch with mixed entanglers, and a full-size run against FP64."""
import numpy as np
import pytest

import oracle
from oracle import readout as ro
from paper_2607_02749_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2607_02749_gb300 as gv  # noqa: E402

ENTS = [gv.GVQE_ENT_CIRCULAR, gv.GVQE_ENT_FULL, gv.GVQE_ENT_REVERSE_LINEAR, gv.GVQE_ENT_PAIRWISE, gv.GVQE_ENT_SCA]


def _ref(n, reps, th, ham, ent):
    with oracle.entangler(ent):
        return oracle.energy_grad(n, reps, th, ham.strings, ham.coeffs)


def _check(n, reps, ham, ent, fp64, seed=0, B=2):
    a = gv.Ansatz(n, reps, entangler=ent)
    h = gv.Hamiltonian.from_workload(ham)
    th = wl.thetas(n, reps, B, seed=seed)
    e, g = gv.energy_grad(a, h, torch.as_tensor(th, device="cuda"), fp64=fp64)
    e, g = e.cpu().numpy(), g.cpu().numpy()
    scale = ham.abs_sum()
    for b in range(B):
        er, gr = _ref(n, reps, th[b], ham, ent)
        if fp64:
            assert abs(e[b] - er) <= 1e-10 * scale
            assert np.max(np.abs(g[b] - gr)) <= 1e-9 * scale
        else:
            assert abs(e[b] - er) <= 2e-5 * scale
            assert np.linalg.norm(g[b] - gr) <= 1e-4 * max(np.linalg.norm(gr), 1e-3 * scale)
    a.close()
    h.close()


@pytest.mark.parametrize("ent", ENTS)
@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("n,reps", [(2, 2), (5, 3), (9, 2), (12, 2), (14, 3), (17, 2)])
def test_energy_grad_z(ent, fp64, n, reps):
    _check(n, reps, wl.z_hamiltonian(n, 30 * n, seed=n), ent, fp64, seed=n + ent)


@pytest.mark.parametrize("ent", ENTS)
@pytest.mark.parametrize("fp64", [False, True])
def test_energy_grad_pauli(ent, fp64):
    _check(13, 2, wl.pauli_hamiltonian(13, 200, seed=3), ent, fp64, seed=4)
    _check(8, 1, wl.pauli_hamiltonian(8, 60, seed=5), ent, fp64, seed=5)


@pytest.mark.parametrize("ent", ENTS)
def test_param_shift_and_tile_bits(ent):
    n, reps = 15, 2
    ham = wl.z_hamiltonian(n, 300, seed=1)
    th = wl.thetas(n, reps, 1, seed=2)
    a = gv.Ansatz(n, reps, entangler=ent)
    h = gv.Hamiltonian.from_workload(ham)
    t = torch.as_tensor(th, device="cuda")
    _, gs = gv.energy_grad(a, h, t, fp64=True, param_shift=True)
    _, gref = _ref(n, reps, th[0], ham, ent)
    assert np.max(np.abs(gs.cpu().numpy()[0] - gref)) <= 1e-9 * ham.abs_sum()
    for tb in (10, 11, 12):  # more strided passes per layer
        a.set_tile_bits(tb)
        e, g = gv.energy_grad(a, h, t, fp64=True)
        assert np.max(np.abs(g.cpu().numpy()[0] - gref)) <= 1e-9 * ham.abs_sum()


@pytest.mark.parametrize("ent", ENTS)
def test_readout_with_entangler(ent):
    n, reps = 12, 2
    ham = wl.z_hamiltonian(n, 200, seed=6)
    th = wl.thetas(n, reps, 1, seed=7)[0]
    with oracle.entangler(ent):
        p = ro.probabilities(oracle.state(n, reps, th))
    a = gv.Ansatz(n, reps, entangler=ent)
    h = gv.Hamiltonian.from_workload(ham)
    r = gv.readout(a, h, torch.as_tensor(th, device="cuda"), alpha=0.2, fp64=True)
    assert r.argmax == ro.most_probable(p)[0]
    e = ro.diagonal_energies(n, ham.strings, ham.coeffs)
    assert abs(r.cvar - ro.cvar(p, e, 0.2)) <= 1e-10 * ham.abs_sum()


def test_batch_with_mixed_entanglers():
    insts = wl.cluster_batch(12, qubit_range=(13, 16), reps_range=(1, 3), terms_per_qubit=20)
    ents = [gv.GVQE_ENT_LINEAR] + ENTS
    ents = ents * 2
    ans = [gv.Ansatz(i.n_qubits, i.reps, entangler=e) for i, e in zip(insts, ents)]
    hams = [gv.Hamiltonian.from_workload(i.ham) for i in insts]
    b = gv.Batch(ans, hams, fp64=True)
    params = [torch.as_tensor(i.theta[0], dtype=torch.float64, device="cuda") for i in insts]
    grads = [torch.empty_like(p) for p in params]
    e = b.run(params, grads=grads).cpu().numpy()
    for k, (i, ent) in enumerate(zip(insts, ents)):
        er, gr = _ref(i.n_qubits, i.reps, i.theta[0], i.ham, ent)
        assert abs(e[k] - er) <= 1e-10 * i.ham.abs_sum()
        assert np.max(np.abs(grads[k].cpu().numpy() - gr)) <= 1e-9 * i.ham.abs_sum()


@pytest.mark.parametrize("ent", ENTS)
def test_fullsize_fp32_against_fp64(ent):
    # n = 26 (several strided passes, paired gathers): FP32 adjoint against FP64 mode
    n, reps = 26, 2
    ham = wl.z_hamiltonian(n, 2000, seed=0)
    a = gv.Ansatz(n, reps, entangler=ent)
    h = gv.Hamiltonian.from_workload(ham)
    t = torch.as_tensor(wl.thetas(n, reps, 1, seed=1), device="cuda")
    e32, g32 = gv.energy_grad(a, h, t)
    e64, g64 = gv.energy_grad(a, h, t, fp64=True)
    scale = ham.abs_sum()
    assert abs(e32.item() - e64.item()) <= 2e-5 * scale
    g32, g64 = g32.cpu().numpy()[0], g64.cpu().numpy()[0]
    assert np.linalg.norm(g32 - g64) <= 1e-4 * max(np.linalg.norm(g64), 1e-3 * scale)


@pytest.mark.parametrize("ent", [gv.GVQE_ENT_SCA, gv.GVQE_ENT_PAIRWISE])
def test_deep_circuit_offsets(ent):
    # SCA cycles its offset through every residue mod n (n = 11, reps = 13);
    # FP64 against the oracle, tile passes at 10 tile bits (two strided passes)
    n, reps = 11, 13
    ham = wl.pauli_hamiltonian(n, 120, seed=8)
    th = wl.thetas(n, reps, 1, seed=9)
    a = gv.Ansatz(n, reps, entangler=ent)
    a.set_tile_bits(10)
    h = gv.Hamiltonian.from_workload(ham)
    e, g = gv.energy_grad(a, h, torch.as_tensor(th, device="cuda"), fp64=True)
    er, gr = _ref(n, reps, th[0], ham, ent)
    assert abs(e.item() - er) <= 1e-10 * ham.abs_sum()
    assert np.max(np.abs(g.cpu().numpy()[0] - gr)) <= 1e-9 * ham.abs_sum()
