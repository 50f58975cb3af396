"""Failure handling without faulting the GPU: a device memory budget that a
call would exceed returns GVQE_ENOMEM and leaves every handle usable; a batched
call runs fewer vectors per launch to fit a budget; bad handles and arguments
are refused on the host."""
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


def test_memory_limit_refuses_and_recovers():
    n, reps = 20, 2
    ham = wl.z_hamiltonian(n, 200, seed=1)
    th = wl.thetas(n, reps, 1, seed=2)
    a = gv.Ansatz(n, reps)
    h = gv.Hamiltonian.from_workload(ham)
    t = torch.as_tensor(th, device="cuda")
    try:
        _lib.gvqe_set_device_memory_limit(_lib.gvqe_device_memory_in_use() + (8 << 20))
        with pytest.raises(gv.GvqeError) as e:
            gv.energy_grad(a, h, t)
        assert e.value.code == _lib.GVQE_ENOMEM
    finally:
        _lib.gvqe_set_device_memory_limit(0)
    e, g = gv.energy_grad(a, h, t, fp64=True)
    er, gr = oracle.energy_grad(n, reps, th[0], ham.strings, ham.coeffs)
    assert abs(e.item() - er) <= 1e-10 * ham.abs_sum()
    assert np.max(np.abs(g.cpu().numpy()[0] - gr)) <= 1e-9 * ham.abs_sum()


def test_batched_call_shrinks_to_fit_a_budget():
    n, reps, B = 18, 1, 8
    ham = wl.z_hamiltonian(n, 150, seed=3)
    th = wl.thetas(n, reps, B, seed=4)
    a = gv.Ansatz(n, reps)
    h = gv.Hamiltonian.from_workload(ham)
    t = torch.as_tensor(th, device="cuda")
    e_free, g_free = gv.energy_grad(a, h, t, fp64=True)  # all vectors in one launch
    held = _lib.gvqe_device_memory_in_use()
    a2 = gv.Ansatz(n, reps)
    try:
        # one vector's FP64 workspace at n = 18, reps = 1 is 2 stored passes + 2 lambda
        # buffers of 2 MiB: leave room for two vectors (and a little), not eight
        _lib.gvqe_set_device_memory_limit(held + (20 << 20))
        e_lim, g_lim = gv.energy_grad(a2, h, t, fp64=True)
        assert _lib.gvqe_device_memory_in_use() <= held + (20 << 20)
    finally:
        _lib.gvqe_set_device_memory_limit(0)
    assert torch.equal(e_lim, e_free) and torch.equal(g_lim, g_free)


def test_bad_handles_and_arguments_are_refused():
    a = gv.Ansatz(10, 1)
    h = gv.Hamiltonian.from_workload(wl.z_hamiltonian(11, 20, seed=0))
    t = torch.zeros((1, a.n_params), dtype=torch.float64, device="cuda")
    with pytest.raises(gv.GvqeError) as e:
        gv.energy(a, h, t)  # 10 vs 11 qubits
    assert e.value.code == _lib.GVQE_EINVAL
    with pytest.raises(gv.GvqeError):
        _lib.gvqe_energy(0, h.handle, t, torch.zeros(1, dtype=torch.float64, device="cuda"), 0, None)
