"""GPU parity on the benchmark's own workload shapes, against the CPU oracle.

Each test prints the error it measured per result (energy error over sum|c|,
gradient max error over sum|c| or relative L2), so the numbers stand beside the
bounds:
  FP64 mode: |dE| <= 1e-10 * sum|c|,  max|dgrad| <= 1e-9 * sum|c|
  FP32 mode: |dE| <= 2e-5  * sum|c|,  ||dgrad||_2 / ||grad||_2 <= 1e-4

Shapes:
  * n = 24 and n = 26, reps = 6, 2,000 Z-strings (the n = 30 benchmark's depth
    and term mix at a size the oracle finishes): the default plan, 2^13-amplitude
    FP32 tiles and three tile passes per layer, several parameter vectors;
  * n = 24, reps = 4, 2,000 Z-strings, 16 vectors: adjoint (FP32 and FP64)
    against the oracle and the FP64 parameter-shift rule (Eq. 13);
  * 5,000 strings over {I, X, Y, Z} with X/Y letters on about 40% (Eq. 6):
    against the oracle at n = 22, reps = 5; at n = 28, reps = 5 through the
    torch.autograd.Function with 8 vectors, the gradient checked by central
    differences at h = 1e-3 in FP64 mode (E is degree one in every angle, so the
    central difference equals E' sin(h) / h exactly).
"""
import math

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


def _report(what, e, g, e_ref, g_ref, scale, fp64):
    """Assert the bounds on every row and print the errors measured."""
    for b in range(len(e_ref)):
        de = abs(float(e[b]) - float(e_ref[b])) / scale
        line = f"{what} row {b}: |dE|/sum|c| = {de:.3e}"
        if fp64:
            assert de <= FP64_E, line
        else:
            assert de <= FP32_E, line
        if g is not None:
            diff = np.asarray(g[b]) - np.asarray(g_ref[b])
            if fp64:
                dg = np.max(np.abs(diff)) / scale
                line += f", max|dg|/sum|c| = {dg:.3e}"
                assert dg <= FP64_G, line
            else:
                rel = np.linalg.norm(diff) / np.linalg.norm(g_ref[b])
                line += f", grad rel L2 = {rel:.3e}"
                assert rel <= FP32_G, line
        print(line)


def _passes_per_layer(a, fp64=False):
    return a.describe(fp64=fp64).count("layer pass")


@pytest.fixture(scope="module")
def deep24():
    n, reps = 24, 6
    ham = wl.z_hamiltonian(n, 2000, seed=0)
    th = wl.thetas(n, reps, 3, seed=1)
    ref = [oracle.energy_grad(n, reps, row, ham.strings, ham.coeffs) for row in th]
    return n, reps, ham, th, np.array([r[0] for r in ref]), np.array([r[1] for r in ref])


@pytest.fixture(scope="module")
def deep26():
    n, reps = 26, 6
    ham = wl.z_hamiltonian(n, 2000, seed=2)
    th = wl.thetas(n, reps, 1, seed=3)
    e, g = oracle.energy_grad(n, reps, th[0], ham.strings, ham.coeffs)
    return n, reps, ham, th, np.array([e]), g[None, :]


@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("which", ["deep24", "deep26"])
def test_reps6_z2000_against_oracle(which, fp64, request):
    n, reps, ham, th, e_ref, g_ref = request.getfixturevalue(which)
    a = gv.Ansatz(n, reps)
    assert _passes_per_layer(a, fp64) == 3
    assert "tile_bits=13" in a.describe() and "tile_bits=12" in a.describe(fp64=True)
    h = gv.Hamiltonian.from_workload(ham)
    t = _dev(th)
    e, g = gv.energy_grad(a, h, t, fp64=fp64)
    e_only = gv.energy(a, h, t, fp64=fp64)
    scale = ham.abs_sum()
    tag = f"n={n} reps={reps} {'fp64' if fp64 else 'fp32'}"
    _report(tag + " energy", e_only.cpu().numpy(), None, e_ref, None, scale, fp64)
    _report(tag + " energy_grad", e.cpu().numpy(), g.cpu().numpy(), e_ref, g_ref, scale, fp64)


def test_n24_reps4_z2000_adjoint_against_oracle_and_parameter_shift():
    ham, th = wl.make_workload("n24_reps4_z2000")
    n, reps = 24, 4
    assert th.shape == (16, n * (reps + 1))
    a = gv.Ansatz(n, reps)
    h = gv.Hamiltonian.from_workload(ham)
    t = _dev(th)
    scale = ham.abs_sum()
    e32, g32 = (x.cpu().numpy() for x in gv.energy_grad(a, h, t))
    e64, g64 = (x.cpu().numpy() for x in gv.energy_grad(a, h, t, fp64=True))
    # all 16 vectors: FP32 against the FP64 mode
    _report("C2 fp32 vs fp64 mode", e32, g32, e64, g64, scale, False)
    for b in (0, 1):
        e_ref, g_ref = oracle.energy_grad(n, reps, th[b], ham.strings, ham.coeffs)
        _report(f"C2 fp64 vs oracle v{b}", e64[b:b + 1], g64[b:b + 1], [e_ref], [g_ref], scale, True)
        _report(f"C2 fp32 vs oracle v{b}", e32[b:b + 1], g32[b:b + 1], [e_ref], [g_ref], scale, False)
        e_ps, g_ps = gv.energy_grad(a, h, t[b:b + 1], fp64=True, param_shift=True)
        _report(f"C2 param shift vs oracle v{b}", e_ps.cpu().numpy(), g_ps.cpu().numpy(), [e_ref], [g_ref],
                scale, True)
        _report(f"C2 fp32 adjoint vs param shift v{b}", e32[b:b + 1], g32[b:b + 1], e_ps.cpu().numpy(),
                g_ps.cpu().numpy(), scale, False)


@pytest.fixture(scope="module")
def mixed22():
    n, reps = 22, 5
    ham = wl.pauli_hamiltonian(n, 5000, seed=0)
    th = wl.thetas(n, reps, 2, seed=1)
    ref = [oracle.energy_grad(n, reps, row, ham.strings, ham.coeffs) for row in th]
    return n, reps, ham, th, np.array([r[0] for r in ref]), np.array([r[1] for r in ref])


@pytest.mark.parametrize("fp64", [False, True])
def test_mixed_pauli_5000_against_oracle(mixed22, fp64):
    n, reps, ham, th, e_ref, g_ref = mixed22
    a = gv.Ansatz(n, reps)
    h = gv.Hamiltonian.from_workload(ham)
    st = h.stats()
    assert st["groups"] > 0
    t = _dev(th)
    scale = ham.abs_sum()
    e_only = gv.energy(a, h, t, fp64=fp64).cpu().numpy()
    e, g = gv.energy_grad(a, h, t, fp64=fp64)
    tag = f"mixed n={n} {'fp64' if fp64 else 'fp32'}"
    _report(tag + " energy", e_only, None, e_ref, None, scale, fp64)
    _report(tag + " energy_grad", e.cpu().numpy(), g.cpu().numpy(), e_ref, g_ref, scale, fp64)


def test_n28_mixed_pauli_autograd_against_central_differences():
    ham, th = wl.make_workload("n28_reps5_pauli5000")
    n, reps = 28, 5
    P = n * (reps + 1)
    B = th.shape[0]
    assert B == 8
    a = gv.Ansatz(n, reps)
    h = gv.Hamiltonian.from_workload(ham)
    scale = ham.abs_sum()
    # nonzero weights of both signs: backward must scale each row by its own weight
    w = torch.tensor([0.5, -1.0, 2.0, -0.25, 1.5, -2.5, 0.75, 3.0], dtype=torch.float64, device="cuda")
    grads = {}
    for fp64 in (False, True):
        t = _dev(th).requires_grad_(True)
        e = gv.GvqeEnergy.apply(t, a, h, None, fp64)
        (e * w).sum().backward()
        grads[fp64] = (t.grad / w[:, None]).cpu().numpy()
    # FP32 autograd against the FP64 mode over every entry
    g32, g64 = grads[False], grads[True]
    for b in range(B):
        rel = np.linalg.norm(g32[b] - g64[b]) / np.linalg.norm(g64[b])
        print(f"C5 fp32 vs fp64 autograd row {b}: grad rel L2 = {rel:.3e}")
        assert rel <= FP32_G
    # central differences (FP64 energies) on sampled entries of every vector
    hstep = 1e-3
    picks = [0, n - 1, n + 7, 2 * n + 13, P // 2, P - n, P - 1]
    rows = []
    for b in range(B):
        for p in picks:
            for s in (1.0, -1.0):
                r = th[b].copy()
                r[p] += s * hstep
                rows.append(r)
    ef = gv.energy(a, h, _dev(np.array(rows)), fp64=True).cpu().numpy().reshape(B, len(picks), 2)
    fd = (ef[:, :, 0] - ef[:, :, 1]) / (2 * hstep) * (hstep / math.sin(hstep))
    for b in range(B):
        d64 = np.max(np.abs(g64[b, picks] - fd[b])) / scale
        rel32 = np.linalg.norm(g32[b, picks] - fd[b]) / np.linalg.norm(fd[b])
        print(f"C5 central differences row {b}: fp64 max|dg|/sum|c| = {d64:.3e}, fp32 rel L2 = {rel32:.3e}")
        # FD of FP64 energies carries their rounding / h: far below 1e-10 sum|c| / h
        assert d64 <= 1e-10 / hstep
        assert rel32 <= FP32_G
