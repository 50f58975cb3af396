"""Full-size checks at n = 30 (the benchmark's launch configuration: three
2^13-amplitude tile passes per layer), where the CPU oracle cannot run.

Pinned by properties that hold at any size:
  * reps = 0: product-state closed form (energy and every gradient entry);
  * reps = 1: Heisenberg-picture closed form (energy, sampled gradient entries);
  * theta = 0: E = sum of Z-only coefficients, zero gradient;
  * theta in {0, pi}: E = E(y) of the propagated basis state;
  * FP32 mode against FP64 mode at reps = 6 with 20,000 strings;
  * parameter shift (Eq. 13) against the adjoint gradient on sampled entries.
"""
import math

import numpy as np
import pytest

from oracle import closed_form
from paper_2607_02749_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2607_02749_gb300 as gv  # noqa: E402

N = 30


@pytest.fixture(scope="module")
def ham20k():
    return wl.z_hamiltonian(N, 20000, seed=0)


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


@pytest.mark.parametrize("fp64", [False, True])
def test_reps0_product_state_closed_form(ham20k, fp64):
    th = wl.thetas(N, 0, 2, seed=11)
    a = gv.Ansatz(N, 0)
    h = gv.Hamiltonian.from_workload(ham20k)
    e, g = gv.energy_grad(a, h, _dev(th), fp64=fp64)
    e, g = e.cpu().numpy(), g.cpu().numpy()
    scale = ham20k.abs_sum()
    for b in range(2):
        e_ref = closed_form.product_state_energy(th[b], ham20k.strings, ham20k.coeffs)
        g_ref = closed_form.product_state_grad(th[b], ham20k.strings, ham20k.coeffs)
        if fp64:
            assert abs(e[b] - e_ref) <= 1e-10 * scale
            assert np.max(np.abs(g[b] - g_ref)) <= 1e-9 * scale
        else:
            assert abs(e[b] - e_ref) <= 2e-5 * scale
            assert np.linalg.norm(g[b] - g_ref) / np.linalg.norm(g_ref) <= 1e-4


@pytest.mark.parametrize("fp64", [False, True])
def test_reps1_heisenberg_closed_form(fp64):
    ham = wl.z_hamiltonian(N, 1500, seed=5)
    th = wl.thetas(N, 1, 1, seed=12)[0]
    a = gv.Ansatz(N, 1)
    h = gv.Hamiltonian.from_workload(ham)
    e, g = gv.energy_grad(a, h, _dev(th[None]), fp64=fp64)
    e, g = e.item(), g[0].cpu().numpy()
    fn = lambda t: closed_form.heisenberg_reps1_energy(N, t, ham.strings, ham.coeffs)
    scale = ham.abs_sum()
    e_ref = fn(th)
    tol_e = 1e-10 if fp64 else 2e-5
    assert abs(e - e_ref) <= tol_e * scale
    picks = (0, 13, 14, 21, 22, 29, 30, 44, 52, 59)
    g_ref = []
    for p in picks:
        tp = th.copy()
        tp[p] += math.pi / 2
        tm = th.copy()
        tm[p] -= math.pi / 2
        g_ref.append(0.5 * (fn(tp) - fn(tm)))  # Eq. 13, exact for a degree-one angle
    g_ref = np.array(g_ref)
    g_s = g[list(picks)]
    if fp64:
        assert np.max(np.abs(g_s - g_ref)) <= 1e-9 * scale, (g_s, g_ref)
    else:  # the FP32 bound: relative L2 over the sampled entries
        rel = np.linalg.norm(g_s - g_ref) / np.linalg.norm(g_ref)
        print(f"n=30 reps=1 fp32: sampled grad rel L2 = {rel:.3e}")
        assert rel <= 1e-4, (g_s, g_ref)


def test_zero_and_basis_angles_at_reps6(ham20k):
    reps = 6
    P = N * (reps + 1)
    a = gv.Ansatz(N, reps)
    h = gv.Hamiltonian.from_workload(ham20k)
    rng = np.random.default_rng(3)
    flips = rng.integers(0, 2, size=P)
    th = np.stack([np.zeros(P), flips * math.pi])
    for fp64 in (False, True):
        e, g = gv.energy_grad(a, h, _dev(th), fp64=fp64)
        e, g = e.cpu().numpy(), g.cpu().numpy()
        scale = ham20k.abs_sum()
        tol = 1e-12 if fp64 else 2e-6
        assert abs(e[0] - closed_form.zero_angle_energy(ham20k.strings, ham20k.coeffs)) <= tol * scale
        assert np.max(np.abs(g[0])) <= tol * scale
        e_ref = closed_form.basis_state_energy(N, reps, flips, ham20k.strings, ham20k.coeffs)
        assert abs(e[1] - e_ref) <= tol * scale


def test_fp32_matches_fp64_at_benchmark_size(ham20k):
    reps = 6
    a = gv.Ansatz(N, reps)
    h = gv.Hamiltonian.from_workload(ham20k)
    th = _dev(wl.thetas(N, reps, 1, seed=1))
    e32, g32 = gv.energy_grad(a, h, th)
    e32, g32 = e32.item(), g32[0].cpu().numpy()
    e64, g64 = gv.energy_grad(a, h, th, fp64=True)
    e64, g64 = e64.item(), g64[0].cpu().numpy()
    scale = ham20k.abs_sum()
    assert abs(e32 - e64) <= 2e-5 * scale
    assert np.linalg.norm(g32 - g64) / np.linalg.norm(g64) <= 1e-4
    # energy-only path agrees with the energy of the gradient path
    e_only = gv.energy(a, h, th).item()
    assert abs(e_only - e32) <= 1e-6 * scale
    # parameter shift (FP64, Eq. 13) on two sampled parameters
    P = N * (reps + 1)
    mask = torch.zeros(1, P, dtype=torch.uint8, device="cuda")
    mask[0, 17] = 1
    mask[0, P - 5] = 1
    _, gps = gv.energy_grad(a, h, th, mask=mask, fp64=True, param_shift=True)
    gps = gps[0].cpu().numpy()
    for p in (17, P - 5):
        assert abs(gps[p] - g64[p]) <= 1e-9 * scale


def _split_first_strided_pass(a, fp64=False):
    import re

    runs = re.findall(r"split=(\d+),(\d+)", a.describe(fp64=fp64))
    return int(runs[1][0]) > 0


def test_su2_split_layout_at_n30_with_zero_rz_is_the_ry_ansatz(ham20k):
    """n = 30 RY+RZ takes the split strided layout (31 index bits); with every
    RZ angle 0 it must reproduce the RY ansatz (one run per pass) exactly in
    structure: the same energy and RY gradients within the FP32 bound, RZ
    gradients 0 (the amplitudes stay real, so Im<lam|Z|psi> vanishes)."""
    reps = 2
    h = gv.Hamiltonian.from_workload(ham20k)
    ty = wl.thetas(N, reps, 1, seed=3)[0].reshape(reps + 1, N)
    a1 = gv.Ansatz(N, reps)
    assert not _split_first_strided_pass(a1)
    e1, g1 = gv.energy_grad(a1, h, _dev(ty.reshape(1, -1)))
    e1, g1 = e1.item(), g1[0].cpu().numpy().reshape(reps + 1, N)
    a1.close()
    a2 = gv.Ansatz(N, reps, gates=gv.GVQE_GATES_RY_RZ)
    assert _split_first_strided_pass(a2)
    th2 = np.concatenate([np.concatenate([ty[r], np.zeros(N)]) for r in range(reps + 1)])[None, :]
    e2, g2 = gv.energy_grad(a2, h, _dev(th2))
    e2, g2 = e2.item(), g2[0].cpu().numpy().reshape(reps + 1, 2, N)
    a2.close()
    scale = ham20k.abs_sum()
    assert abs(e2 - e1) <= 2e-5 * scale
    assert np.linalg.norm(g2[:, 0, :] - g1) <= 1e-4 * np.linalg.norm(g1)
    assert np.max(np.abs(g2[:, 1, :])) <= 1e-9 * scale


@pytest.mark.parametrize("fp64", [False, True])
def test_su2_reps0_closed_form_at_n30(ham20k, fp64):
    """reps = 0 RY+RZ at n = 30 (FP32: split layout; FP64: three strided passes
    of 2^12 tiles): the Bloch-vector product form gives the energy, and its
    central differences sampled gradient entries."""
    a = gv.Ansatz(N, 0, gates=gv.GVQE_GATES_RY_RZ)
    assert _split_first_strided_pass(a, fp64) == (not fp64)
    h = gv.Hamiltonian.from_workload(ham20k)
    th = np.random.default_rng(5).uniform(-np.pi, np.pi, 2 * N)
    e, g = gv.energy_grad(a, h, _dev(th[None, :]), fp64=fp64)
    e, g = e.item(), g[0].cpu().numpy()
    a.close()
    scale = ham20k.abs_sum()

    def ef(t):
        return closed_form.su2_product_state_energy(t[:N], t[N:], ham20k.strings, ham20k.coeffs)

    assert abs(e - ef(th)) <= (1e-10 if fp64 else 2e-5) * scale
    hstep = 1e-5
    for p in (0, 13, 17, 29, N + 2, N + 16, N + 27):
        tp, tm = th.copy(), th.copy()
        tp[p] += hstep
        tm[p] -= hstep
        fd = (ef(tp) - ef(tm)) / (2 * hstep)
        assert abs(g[p] - fd) <= (1e-8 if fp64 else 2e-5) * scale, p
