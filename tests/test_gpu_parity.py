"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerances (stated per result, scaled by sum_k |c_k|):
  FP64 mode: |dE| <= 1e-10 * sum|c|,  max|dgrad| <= 1e-9 * sum|c|
  FP32 mode: |dE| <= 2e-5  * sum|c|,  ||dgrad||_2 / ||grad||_2 <= 1e-4
Sizes span one tile, several tiles and multi-pass layers (forced small tiles),
the whole-register kernel (n < 10) and the edge cases n = 1 and reps = 0.
"""
import numpy as np
import pytest

import oracle
from paper_2607_02749_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2607_02749_gb300 as gv  # noqa: E402

FP64_E, FP64_G = 1e-10, 1e-9
FP32_E, FP32_G = 2e-5, 1e-4


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _oracle_eg(n, reps, th, ham):
    es, gs = [], []
    for row in th:
        e, g = oracle.energy_grad(n, reps, row, ham.strings, ham.coeffs)
        es.append(e)
        gs.append(g)
    return np.array(es), np.array(gs)


def _check(e, g, e_ref, g_ref, scale, fp64, what=""):
    de = np.max(np.abs(e - e_ref))
    if fp64:
        assert de <= FP64_E * scale, f"{what} |dE|={de:.3e} > {FP64_E * scale:.3e}"
        if g is not None:
            dg = np.max(np.abs(g - g_ref))
            assert dg <= FP64_G * scale, f"{what} max|dg|={dg:.3e} > {FP64_G * scale:.3e}"
    else:
        assert de <= FP32_E * scale, f"{what} |dE|={de:.3e} > {FP32_E * scale:.3e}"
        if g is not None:
            for row, ref in zip(g, g_ref):
                nref = np.linalg.norm(ref)
                rel = np.linalg.norm(row - ref) / max(nref, 1e-300)
                assert rel <= FP32_G, f"{what} grad rel L2={rel:.3e}"


CASES = [
    # (n, reps, tile_bits, batch)
    (1, 0, 0, 2), (1, 3, 0, 2), (2, 1, 0, 2), (5, 2, 0, 3), (9, 3, 0, 2),
    (10, 0, 0, 2), (10, 2, 0, 3), (12, 2, 0, 3), (13, 1, 0, 2), (14, 3, 0, 2),
    (11, 2, 10, 2), (15, 2, 10, 2), (16, 1, 10, 2), (18, 2, 10, 2), (20, 2, 12, 1),
    (17, 3, 11, 2), (19, 0, 10, 2), (16, 2, 13, 1),
]


@pytest.mark.parametrize("n,reps,tb,batch", CASES)
@pytest.mark.parametrize("fp64", [True, False])
def test_energy_and_adjoint_gradient_diagonal(n, reps, tb, batch, fp64):
    if fp64 and tb > 12:
        pytest.skip("FP64 tiles are at most 2^12 amplitudes")
    ham = wl.z_hamiltonian(n, 6 * n + 5, seed=n + reps)
    th = wl.thetas(n, reps, batch, seed=100 + n)
    e_ref, g_ref = _oracle_eg(n, reps, th, ham)
    a = gv.Ansatz(n, reps, tile_bits=tb)
    h = gv.Hamiltonian.from_workload(ham)
    t = _dev(th)
    e_only = gv.energy(a, h, t, fp64=fp64).cpu().numpy()
    e, g = gv.energy_grad(a, h, t, fp64=fp64)
    e, g = e.cpu().numpy(), g.cpu().numpy()
    scale = ham.abs_sum()
    _check(e_only, None, e_ref, None, scale, fp64, "energy")
    _check(e, g, e_ref, g_ref, scale, fp64, "energy_grad")


@pytest.mark.parametrize("n,reps,tb", [(12, 2, 0), (14, 3, 0), (17, 2, 0), (16, 2, 10), (21, 1, 12)])
@pytest.mark.parametrize("fp64", [True, False])
def test_angles_at_and_near_pi(n, reps, tb, fp64):
    """Rotations whose cos(theta/2) is tiny or zero (theta at or near +-pi, and
    beyond the principal range) run the backward pass's two half-angle steps;
    several per pass, mixed with ordinary angles."""
    if fp64 and tb > 12:
        pytest.skip("FP64 tiles are at most 2^12 amplitudes")
    rng = np.random.default_rng(n + 17 * reps)
    th = wl.thetas(n, reps, 2, seed=5 + n)
    special = np.array([np.pi, -np.pi, np.pi - 1e-3, -np.pi + 3e-3, 3 * np.pi, np.pi + 1e-9, 2.9, -3.1])
    pick = rng.uniform(size=th.shape) < 0.4
    th[pick] = rng.choice(special, size=int(pick.sum()))
    ham = wl.z_hamiltonian(n, 6 * n + 5, seed=2 * n)
    e_ref, g_ref = _oracle_eg(n, reps, th, ham)
    a = gv.Ansatz(n, reps, tile_bits=tb)
    h = gv.Hamiltonian.from_workload(ham)
    e, g = gv.energy_grad(a, h, _dev(th), fp64=fp64)
    _check(e.cpu().numpy(), g.cpu().numpy(), e_ref, g_ref, ham.abs_sum(), fp64, "near pi")


@pytest.mark.parametrize("n,reps,tb", [(6, 2, 0), (10, 1, 0), (12, 2, 0), (14, 2, 10), (16, 1, 12), (9, 0, 0), (13, 0, 10)])
@pytest.mark.parametrize("fp64", [True, False])
def test_energy_and_gradient_with_xy_strings(n, reps, tb, fp64):
    ham = wl.pauli_hamiltonian(n, 8 * n, seed=3 * n + reps)
    th = wl.thetas(n, reps, 2, seed=7 + n)
    e_ref, g_ref = _oracle_eg(n, reps, th, ham)
    a = gv.Ansatz(n, reps, tile_bits=tb)
    h = gv.Hamiltonian.from_workload(ham)
    assert h.stats()["groups"] > 0
    t = _dev(th)
    e_only = gv.energy(a, h, t, fp64=fp64).cpu().numpy()
    e, g = gv.energy_grad(a, h, t, fp64=fp64)
    scale = ham.abs_sum()
    _check(e_only, None, e_ref, None, scale, fp64, "energy xy")
    _check(e.cpu().numpy(), g.cpu().numpy(), e_ref, g_ref, scale, fp64, "energy_grad xy")


@pytest.mark.parametrize("xtb", [10, 11, 12, 13])
@pytest.mark.parametrize("fp64", [True, False])
def test_xy_pass_with_its_own_tile_size(xtb, fp64):
    """GVQE_OPT_XY_TILE_BITS: the X-mask pass on 2^10..2^13-amplitude tiles (FP64
    clamps 13 to 12) while the RY passes keep theirs; against the oracle."""
    n, reps = 15, 2
    ham = wl.pauli_hamiltonian(n, 8 * n, seed=21)
    th = wl.thetas(n, reps, 2, seed=22)
    e_ref, g_ref = _oracle_eg(n, reps, th, ham)
    a = gv.Ansatz(n, reps)
    gv.gvqe_ansatz_set_option(a.handle, gv._lib.GVQE_OPT_XY_TILE_BITS, xtb)
    h = gv.Hamiltonian.from_workload(ham)
    t = _dev(th)
    e_only = gv.energy(a, h, t, fp64=fp64).cpu().numpy()
    e, g = gv.energy_grad(a, h, t, fp64=fp64)
    scale = ham.abs_sum()
    _check(e_only, None, e_ref, None, scale, fp64, f"xy tiles {xtb} energy")
    _check(e.cpu().numpy(), g.cpu().numpy(), e_ref, g_ref, scale, fp64, f"xy tiles {xtb} energy_grad")


@pytest.mark.parametrize("n,reps,tb", [(8, 2, 0), (12, 3, 0), (16, 2, 10)])
def test_masks_zero_inactive_and_keep_active(n, reps, tb):
    ham = wl.z_hamiltonian(n, 50, seed=2)
    B = 4
    th = wl.thetas(n, reps, B, seed=5)
    P = n * (reps + 1)
    mask = wl.active_mask(P, B, seed=9)
    mask[1, :] = 0              # nothing active
    mask[2, : n] = 0            # layer 0 inactive
    mask[2, n:] = 1
    mask[3, :] = 0
    mask[3, P - 1] = 1          # only the last parameter
    a = gv.Ansatz(n, reps, tile_bits=tb)
    h = gv.Hamiltonian.from_workload(ham)
    t = _dev(th)
    e_full, g_full = gv.energy_grad(a, h, t, fp64=True)
    e_m, g_m = gv.energy_grad(a, h, t, mask=_dev(mask, torch.uint8), fp64=True)
    e_full, g_full, e_m, g_m = (x.cpu().numpy() for x in (e_full, g_full, e_m, g_m))
    assert np.array_equal(e_full, e_m)
    assert np.all(g_m[mask == 0] == 0.0)
    assert np.array_equal(g_m[mask == 1], g_full[mask == 1])


@pytest.mark.parametrize("n,reps", [(6, 2), (11, 1)])
def test_param_shift_path_matches_oracle(n, reps):
    ham = wl.z_hamiltonian(n, 40, seed=1)
    th = wl.thetas(n, reps, 2, seed=3)
    P = n * (reps + 1)
    mask = wl.active_mask(P, 2, seed=4)
    a = gv.Ansatz(n, reps)
    h = gv.Hamiltonian.from_workload(ham)
    e, g = gv.energy_grad(a, h, _dev(th), mask=_dev(mask, torch.uint8), fp64=True, param_shift=True)
    e, g = e.cpu().numpy(), g.cpu().numpy()
    scale = ham.abs_sum()
    for b in range(2):
        g_ref = oracle.param_shift_grad(n, reps, th[b], ham.strings, ham.coeffs, mask=mask[b])
        assert abs(e[b] - oracle.energy(n, reps, th[b], ham.strings, ham.coeffs)) <= FP64_E * scale
        assert np.max(np.abs(g[b] - g_ref)) <= FP64_G * scale
        assert np.all(g[b][mask[b] == 0] == 0.0)


def test_deterministic_reductions():
    n, reps = 18, 2
    ham = wl.z_hamiltonian(n, 100, seed=0)
    th = _dev(wl.thetas(n, reps, 2, seed=0))
    a = gv.Ansatz(n, reps, tile_bits=10)
    h = gv.Hamiltonian.from_workload(ham)
    r1 = [x.cpu().numpy() for x in gv.energy_grad(a, h, th)]
    r2 = [x.cpu().numpy() for x in gv.energy_grad(a, h, th)]
    assert np.array_equal(r1[0], r2[0]) and np.array_equal(r1[1], r2[1])


def test_batch_api_matches_single_calls():
    insts = wl.cluster_batch(6, qubit_range=(9, 15), reps_range=(1, 3), terms_per_qubit=10)
    ans = [gv.Ansatz(i.n_qubits, i.reps) for i in insts]
    hams = [gv.Hamiltonian.from_workload(i.ham) for i in insts]
    b = gv.Batch(ans, hams)
    b.set_schedule(False)  # the persistent kernel (the staged default is checked in test_gpu_batch.py)
    params = [_dev(i.theta[0]) for i in insts]
    masks = [_dev(i.mask[0], torch.uint8) for i in insts]
    grads = [torch.empty_like(p) for p in params]
    e = b.run(params, masks=masks, grads=grads).cpu().numpy()
    for k, i in enumerate(insts):
        e1, g1 = gv.energy_grad(ans[k], hams[k], params[k], mask=masks[k])
        if i.n_qubits < 12:  # evaluated by a single call inside the run: the same bits
            assert e[k] == e1.item()
            assert np.array_equal(grads[k].cpu().numpy(), g1.cpu().numpy()[0])
        else:  # the persistent launch's 2^12-amplitude tiles sum in another order
            assert abs(e[k] - e1.item()) <= FP32_E * i.ham.abs_sum()
            g1 = g1.cpu().numpy()[0]
            assert np.linalg.norm(grads[k].cpu().numpy() - g1) <= FP32_G * np.linalg.norm(g1)
        e_ref, g_ref = oracle.energy_grad(i.n_qubits, i.reps, i.theta[0], i.ham.strings, i.ham.coeffs)
        g_ref = np.where(i.mask[0] == 1, g_ref, 0.0)
        _check(np.array([e[k]]), grads[k].cpu().numpy()[None], np.array([e_ref]), g_ref[None],
               i.ham.abs_sum(), False, f"batch {k}")


def test_autograd_function_matches_central_differences():
    n, reps = 8, 2
    ham = wl.pauli_hamiltonian(n, 60, seed=2)
    a = gv.Ansatz(n, reps)
    h = gv.Hamiltonian.from_workload(ham)
    th = _dev(wl.thetas(n, reps, 3, seed=1)).requires_grad_(True)
    e = gv.GvqeEnergy.apply(th, a, h, None, True)
    w = torch.tensor([0.5, -1.0, 2.0], dtype=torch.float64, device="cuda")
    (e * w).sum().backward()
    g = th.grad.cpu().numpy()
    base = th.detach()
    hstep = 1e-3
    import math
    for b in range(3):
        for p in (0, 5, 17, n * (reps + 1) - 1):
            tp = base.clone()
            tp[b, p] += hstep
            tm = base.clone()
            tm[b, p] -= hstep
            fd = (gv.energy(a, h, tp, fp64=True)[b] - gv.energy(a, h, tm, fp64=True)[b]).item() / (2 * hstep)
            # E is degree one in each angle, so the central difference is exactly E' sin(h)/h
            fd *= hstep / math.sin(hstep)
            assert abs(w[b].item() * fd - g[b, p]) <= 1e-9 * ham.abs_sum() / hstep
