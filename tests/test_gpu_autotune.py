"""The autotuner on the GPU: it times every distinct tile plan, keeps the
fastest, stores it in the cache, and the tuned plan's energies and gradients
match the CPU oracle within the parity bounds.  A second ansatz with the same
key takes the cached plan without timing."""
import re

import numpy as np
import pytest

import oracle
from paper_2607_02749_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2607_02749_gb300 as gv  # noqa: E402
from paper_2607_02749_gb300 import _lib  # noqa: E402


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("n,reps,fp64", [(17, 2, False), (17, 2, True), (21, 1, False)])
def test_tuned_plan_matches_oracle_and_is_cached(tmp_path, n, reps, fp64):
    cache = str(tmp_path / "tune.json")
    ham = wl.z_hamiltonian(n, 8 * n, seed=n)
    th = wl.thetas(n, reps, 2, seed=3)
    h = gv.Hamiltonian.from_workload(ham)
    a = gv.Ansatz(n, reps)
    rep = a.autotune(h, _dev(th), fp64=fp64, cache=cache)
    print(rep)
    items = re.findall(r"tb=(\d+)/(one run|split y=\d+): ([0-9.]+) ms", rep)
    assert len(items) >= 2, rep  # several distinct plans were timed
    m = re.search(r"measured: tile_bits=(\d+)", rep)
    assert m, rep
    best_tb = int(m.group(1))
    best_ms = min(float(x[2]) for x in items)
    assert any(int(x[0]) == best_tb and float(x[2]) == best_ms for x in items)
    assert "autotune" in a.describe(fp64=fp64)
    assert f"tile_bits={best_tb}" in a.describe(fp64=fp64)
    e, g = gv.energy_grad(a, h, _dev(th), fp64=fp64)
    e, g = e.cpu().numpy(), g.cpu().numpy()
    scale = ham.abs_sum()
    for b in range(2):
        e_ref, g_ref = oracle.energy_grad(n, reps, th[b], ham.strings, ham.coeffs)
        if fp64:
            assert abs(e[b] - e_ref) <= 1e-10 * scale
            assert np.max(np.abs(g[b] - g_ref)) <= 1e-9 * scale
        else:
            assert abs(e[b] - e_ref) <= 2e-5 * scale
            assert np.linalg.norm(g[b] - g_ref) / np.linalg.norm(g_ref) <= 1e-4
    # same key, new handles: the cached plan, no timing
    a2 = gv.Ansatz(n, reps)
    h2 = gv.Hamiltonian.from_workload(ham)
    rep2 = a2.autotune(h2, _dev(th), fp64=fp64, cache=cache)
    assert "cached" in rep2 and f"tile_bits={best_tb}" in rep2, rep2
    key = _lib.gvqe_tune_key(a2.handle, h2.handle, 2, _lib.GVQE_FP64 if fp64 else _lib.GVQE_FP32)
    assert _lib.gvqe_tune_cache_get(cache, key)[0] == best_tb
    e2, g2 = gv.energy_grad(a2, h2, _dev(th), fp64=fp64)
    assert np.array_equal(e2.cpu().numpy(), e) and np.array_equal(g2.cpu().numpy(), g)
    # the other precision keeps its own plan on the tuned ansatz
    e3, _ = gv.energy_grad(a, h, _dev(th), fp64=not fp64)
    tol = (2e-5 if fp64 else 1e-10) * scale
    for b in range(2):
        assert abs(e3[b].item() - oracle.energy(n, reps, th[b], ham.strings, ham.coeffs)) <= tol


def test_energy_only_tuning_with_xy_strings(tmp_path):
    n, reps = 16, 2
    ham = wl.pauli_hamiltonian(n, 6 * n, seed=5)
    th = wl.thetas(n, reps, 1, seed=6)
    h = gv.Hamiltonian.from_workload(ham)
    a = gv.Ansatz(n, reps)
    rep = a.autotune(h, _dev(th), energy_only=True, cache=str(tmp_path / "t.json"))
    assert "(batch 1, energy, fp32)" in rep, rep
    assert "X-mask tiles 2^" in rep, rep  # the X-mask pass's own tile size was swept too
    e = gv.energy(a, h, _dev(th)).item()
    e_ref = oracle.energy(n, reps, th[0], ham.strings, ham.coeffs)
    assert abs(e - e_ref) <= 2e-5 * ham.abs_sum()
