"""The split strided layout (GVQE_OPT_SPLIT_PASSES): a strided pass whose gate
qubits are two runs, the low ones and the top ones, on the GPU against the
oracle.  Small tiles (2^10, 2^11) force two strided passes per layer at n = 17..20,
where mode 2 splits the first of them; energies and adjoint gradients in FP32 and
FP64, masks, non-linear entanglers, X/Y strings, the complex (RY then RZ) path
and the static energy must all match the oracle, and the split and unsplit
layouts must agree with each other within the FP32 bound."""
import re

import numpy as np
import pytest

import oracle
from paper_2607_02749_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2607_02749_gb300 as gv  # noqa: E402

SPLIT = 2


def _split_runs(a, fp64=False):
    return [tuple(map(int, m)) for m in re.findall(r"split=(\d+),(\d+)", a.describe(fp64=fp64))]


def _ref(n, reps, th, ham, ent=0, gates=1):
    es, gs = [], []
    with oracle.entangler(ent), oracle.gates(gates):
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
@pytest.mark.parametrize("n,reps,tb,ent", [(18, 2, 10, 0), (20, 2, 10, 1), (18, 3, 10, 5), (19, 1, 10, 2),
                                           (18, 0, 10, 0)])
def test_split_layout_matches_the_oracle(n, reps, tb, ent, fp64):
    a = gv.Ansatz(n, reps, entangler=ent, tile_bits=tb, split=SPLIT)
    assert any(k1 > 0 for k1, _ in _split_runs(a, fp64)), a.describe(fp64)
    ham = wl.z_hamiltonian(n, 6 * n + 5, seed=n + reps)
    th = wl.thetas(n, reps, 2, seed=300 + n)
    er, gr = _ref(n, reps, th, ham, ent)
    h = gv.Hamiltonian.from_workload(ham)
    t = torch.as_tensor(th, device="cuda")
    e_only = gv.energy(a, h, t, fp64=fp64).cpu().numpy()
    e, g = gv.energy_grad(a, h, t, fp64=fp64)
    _check(e.cpu().numpy(), g.cpu().numpy(), er, gr, ham.abs_sum(), fp64)
    assert np.max(np.abs(e_only - er)) <= (1e-10 if fp64 else 2e-5) * ham.abs_sum()


def test_split_and_unsplit_layouts_agree_with_masks():
    n, reps, tb = 18, 2, 10
    ham = wl.z_hamiltonian(n, 100, seed=5)
    h = gv.Hamiltonian.from_workload(ham)
    th = wl.thetas(n, reps, 3, seed=6)
    mask = (np.random.default_rng(7).uniform(size=th.shape) < 0.4).astype(np.uint8)
    t = torch.as_tensor(th, device="cuda")
    m = torch.as_tensor(mask, device="cuda")
    out = {}
    for split in (1, SPLIT):
        a = gv.Ansatz(n, reps, tile_bits=tb, split=split)
        e, g = gv.energy_grad(a, h, t, mask=m)
        out[split] = (e.cpu().numpy(), g.cpu().numpy())
    assert _split_runs(gv.Ansatz(n, reps, tile_bits=tb, split=1)) == [(0, 0)] * 3
    (e1, g1), (e2, g2) = out[1], out[SPLIT]
    scale = ham.abs_sum()
    assert np.max(np.abs(e1 - e2)) <= 2e-5 * scale
    assert np.all(g2[mask == 0] == 0.0)
    er, gr = _ref(n, reps, th, ham)
    _check(e2, g2, er, np.where(mask == 1, gr, 0.0), scale, False)


@pytest.mark.parametrize("fp64", [False, True])
def test_split_layout_with_xy_strings(fp64):
    n, reps, tb = 18, 2, 10
    ham = wl.pauli_hamiltonian(n, 60, seed=11)
    a = gv.Ansatz(n, reps, tile_bits=tb, split=SPLIT)
    assert any(k1 > 0 for k1, _ in _split_runs(a, fp64))
    h = gv.Hamiltonian.from_workload(ham)
    th = wl.thetas(n, reps, 1, seed=12)
    er, gr = _ref(n, reps, th, ham)
    e, g = gv.energy_grad(a, h, torch.as_tensor(th, device="cuda"), fp64=fp64)
    _check(e.cpu().numpy(), g.cpu().numpy(), er, gr, ham.abs_sum(), fp64)


@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("n,reps,tb,ent", [(17, 2, 10, 0), (18, 1, 10, 5)])
def test_split_layout_on_the_complex_path(n, reps, tb, ent, fp64):
    a = gv.Ansatz(n, reps, entangler=ent, gates=gv.GVQE_GATES_RY_RZ, tile_bits=tb, split=SPLIT)
    assert any(k1 > 0 for k1, _ in _split_runs(a, fp64))
    ham = wl.chain_z_hamiltonian(n, 8 * n, seed=n)
    th = np.random.default_rng(n + reps).uniform(-np.pi, np.pi, (2, a.n_params))
    er, gr = _ref(n, reps, th, ham, ent, gates=oracle.GATES_RY_RZ)
    h = gv.Hamiltonian.from_workload(ham)
    e, g = gv.energy_grad(a, h, torch.as_tensor(th, device="cuda"), fp64=fp64)
    _check(e.cpu().numpy(), g.cpu().numpy(), er, gr, ham.abs_sum(), fp64)


def test_static_energy_with_the_split_layout():
    n, reps, tb = 18, 2, 10
    ham = wl.z_hamiltonian(n, 80, seed=21)
    a = gv.Ansatz(n, reps, tile_bits=tb, split=SPLIT)
    assert any(k1 > 0 for k1, _ in _split_runs(a, True))
    h = gv.Hamiltonian.from_workload(ham)
    th = torch.as_tensor(wl.thetas(n, reps, 2, seed=22), device="cuda")
    es = torch.empty(2, dtype=torch.float64, device="cuda")
    gv._lib.gvqe_energy_static(a.handle, h.handle, th, es, gv.GVQE_FP64, None)
    er, _ = _ref(n, reps, th.cpu().numpy(), ham)
    assert np.max(np.abs(es.cpu().numpy() - er)) <= 1e-10 * ham.abs_sum()
