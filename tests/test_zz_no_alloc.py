"""gvqe_energy_static: energies for callers that cannot allocate device memory.

The entry point computes the same energies as gvqe_energy but takes every
scratch buffer from a fixed device array inside the library, so it serves
callers whose runtime owns every device allocation or holds the process to a
memory budget this library may not draw on.  These tests call it through the C
ABI twice in a row, on handles whose tables gvqe_energy never built, check that
the library's device memory does not change across those calls, and compare
each result with gvqe_energy (on a second pair of handles) within the parity
tolerances; the file is collected last so a failure here leaves every other
test already run.
"""
import numpy as np
import pytest

from paper_2607_02749_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2607_02749_gb300 as gv  # noqa: E402
from paper_2607_02749_gb300 import _lib  # noqa: E402


@pytest.mark.parametrize("n,reps,tb,batch", [(7, 2, 0, 3), (12, 0, 0, 2), (16, 2, 12, 2), (18, 3, 0, 1)])
@pytest.mark.parametrize("fp64", [False, True])
def test_static_energy_matches_gvqe_energy_on_two_calls(n, reps, tb, batch, fp64):
    ham = wl.z_hamiltonian(n, 8 * n, seed=n)
    th = torch.as_tensor(wl.thetas(n, reps, batch, seed=2 * n), dtype=torch.float64, device="cuda")
    flags = _lib.GVQE_FP64 if fp64 else _lib.GVQE_FP32
    tol = (1e-10 if fp64 else 2e-5) * ham.abs_sum()
    # handles only the static entry point ever sees: no table, plan or workspace
    # of gvqe_energy exists for them
    a = gv.Ansatz(n, reps, tile_bits=tb)
    h = gv.Hamiltonian.from_workload(ham)
    outs = [torch.full((batch,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    held = _lib.gvqe_device_memory_in_use()
    for e in outs:
        _lib.gvqe_energy_static(a.handle, h.handle, th, e, flags)
        torch.cuda.synchronize()
    assert _lib.gvqe_device_memory_in_use() == held
    a_ref = gv.Ansatz(n, reps, tile_bits=tb)
    h_ref = gv.Hamiltonian.from_workload(ham)
    e_ref = gv.energy(a_ref, h_ref, th, fp64=fp64).cpu().numpy()
    for e in outs:
        e = e.cpu().numpy()
        assert np.all(np.isfinite(e))
        assert np.max(np.abs(e - e_ref)) <= tol


def test_static_energy_rejects_requests_above_the_scratch_limit():
    n = 20
    ham = wl.z_hamiltonian(n, 40, seed=1)
    a = gv.Ansatz(n, 1)
    h = gv.Hamiltonian.from_workload(ham)
    th = torch.zeros(1, a.n_params, dtype=torch.float64, device="cuda")
    e = torch.empty(1, dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.GvqeError) as err:
        _lib.gvqe_energy_static(a.handle, h.handle, th, e, _lib.GVQE_FP32)
    assert err.value.code == _lib.GVQE_EINVAL
    assert "static scratch" in str(err.value)


def test_static_energy_rejects_xy_strings():
    ham = wl.pauli_hamiltonian(8, 30, seed=3)
    a = gv.Ansatz(8, 1)
    h = gv.Hamiltonian.from_workload(ham)
    th = torch.zeros(1, a.n_params, dtype=torch.float64, device="cuda")
    e = torch.empty(1, dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.GvqeError) as err:
        _lib.gvqe_energy_static(a.handle, h.handle, th, e, _lib.GVQE_FP32)
    assert err.value.code == _lib.GVQE_EUNSUPPORTED
