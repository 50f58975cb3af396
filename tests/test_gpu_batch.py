"""The persistent batched path (gvqe_batch_*): many independent restricted-update
problems (uneven qubit counts, own Hamiltonians, own active masks) in one
persistent launch replayed from a CUDA graph, checked against single calls and
the oracle, plus the bounded device-side wait returning GVQE_ETIMEOUT."""
import os

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


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _setup(insts, fp64=False, persistent=True):
    ans = [gv.Ansatz(i.n_qubits, i.reps) for i in insts]
    # the batch runs every layer as tile passes; the single calls these tests compare
    # with bit for bit do the same (no closed-form leading layers)
    for a in ans:
        a.set_mps_layers(-1)
    hams = [gv.Hamiltonian.from_workload(i.ham) for i in insts]
    b = gv.Batch(ans, hams, fp64=fp64)
    if persistent:  # most tests here exercise the persistent kernel; the staged one has its own
        b.set_schedule(False)
    params = [_dev(i.theta[0]) for i in insts]
    masks = [_dev(i.mask[0], torch.uint8) for i in insts]
    return ans, hams, b, params, masks


@pytest.mark.parametrize("fp64", [False, True])
def test_persistent_batch_matches_single_calls_and_oracle(fp64):
    insts = wl.cluster_batch(10, qubit_range=(13, 17), reps_range=(1, 3), terms_per_qubit=20)
    ans, hams, b, params, masks = _setup(insts, fp64)
    grads = [torch.full_like(p, float("nan")) for p in params]
    for rep in range(2):  # the graph is replayed
        e = b.run(params, masks=masks, grads=grads).cpu().numpy()
        for k, i in enumerate(insts):
            scale = i.ham.abs_sum()
            e1, g1 = gv.energy_grad(ans[k], hams[k], params[k], mask=masks[k], fp64=fp64)
            g = grads[k].cpu().numpy()
            g1 = g1.cpu().numpy()[0]
            tol_e = (1e-10 if fp64 else 2e-5) * scale
            assert abs(e[k] - e1.item()) <= tol_e
            assert np.all(g[i.mask[0] == 0] == 0.0)
            if fp64:
                assert np.max(np.abs(g - g1)) <= 1e-9 * scale
            else:
                assert np.linalg.norm(g - g1) <= 1e-4 * np.linalg.norm(g1)
            if rep == 0 and k < 3:
                e_ref, g_ref = oracle.energy_grad(i.n_qubits, i.reps, i.theta[0], i.ham.strings, i.ham.coeffs)
                g_ref = np.where(i.mask[0] == 1, g_ref, 0.0)
                assert abs(e[k] - e_ref) <= tol_e
                if fp64:
                    assert np.max(np.abs(g - g_ref)) <= 1e-9 * scale
                else:
                    assert np.linalg.norm(g - g_ref) <= 1e-4 * np.linalg.norm(g_ref)


def test_persistent_batch_energies_only_and_pointer_change():
    insts = wl.cluster_batch(6, qubit_range=(13, 16), reps_range=(2, 3), terms_per_qubit=10)
    ans, hams, b, params, masks = _setup(insts)
    e = b.run(params).cpu().numpy()
    for k in range(len(insts)):
        assert abs(e[k] - gv.energy(ans[k], hams[k], params[k]).item()) <= 2e-5 * insts[k].ham.abs_sum()
    # new parameter buffers between runs are picked up
    params2 = [p.clone() * 0.5 for p in params]
    e2 = b.run(params2).cpu().numpy()
    for k in range(len(insts)):
        assert abs(e2[k] - gv.energy(ans[k], hams[k], params2[k]).item()) <= 2e-5 * insts[k].ham.abs_sum()


@pytest.mark.parametrize("persistent", [True, False])
def test_cluster_workload_256_instances(persistent):
    insts = wl.cluster_batch(256)
    ans, hams, b, params, masks = _setup(insts, persistent=persistent)
    grads = [torch.empty_like(p) for p in params]
    e = b.run(params, masks=masks, grads=grads).cpu().numpy()
    for k in (0, 17, 100, 255):
        i = insts[k]
        e1, g1 = gv.energy_grad(ans[k], hams[k], params[k], mask=masks[k])
        scale = i.ham.abs_sum()
        assert abs(e[k] - e1.item()) <= 2e-5 * scale
        g1 = g1.cpu().numpy()[0]
        assert np.linalg.norm(grads[k].cpu().numpy() - g1) <= 1e-4 * np.linalg.norm(g1)


def test_wave_schedules_give_identical_results_and_autotune_keeps_them():
    """The wave budget only reorders independent items: every budget gives the
    same bits; the batch autotuner times each budget and keeps one."""
    insts = wl.cluster_batch(40, qubit_range=(13, 18), reps_range=(1, 3), terms_per_qubit=10)
    ans, hams, b, params, masks = _setup(insts)
    outs = []
    for wb in (0, 1 << 20, 8 << 20, 48 << 20):
        b.set_wave_bytes(wb)
        grads = [torch.full_like(p, float("nan")) for p in params]
        e = b.run(params, masks=masks, grads=grads).cpu().numpy()
        outs.append((e, [g.cpu().numpy() for g in grads]))
    for e, gs in outs[1:]:
        assert np.array_equal(e, outs[0][0])
        for g, g0 in zip(gs, outs[0][1]):
            assert np.array_equal(g, g0)
    # the staged schedule runs each plan group's passes with the regular kernels,
    # one launch per pass over the group's jobs: the bits of single calls
    b.set_schedule(True)
    grads = [torch.full_like(p, float("nan")) for p in params]
    e = b.run(params, masks=masks, grads=grads).cpu().numpy()
    for k in range(len(insts)):
        e1, g1 = gv.energy_grad(ans[k], hams[k], params[k], mask=masks[k])
        assert e[k] == e1.item()
        assert np.array_equal(grads[k].cpu().numpy(), g1.cpu().numpy()[0])
        assert abs(e[k] - outs[0][0][k]) <= 2e-5 * insts[k].ham.abs_sum()
    b.set_schedule(False)
    # smaller work items (2^11, 2^10 amplitudes) change the summation order only
    for tb in (11, 10):
        b.set_tile_bits(tb)
        b.set_wave_bytes(0)
        grads = [torch.full_like(p, float("nan")) for p in params]
        e = b.run(params, masks=masks, grads=grads).cpu().numpy()
        for k, i in enumerate(insts):
            scale = i.ham.abs_sum()
            assert abs(e[k] - outs[0][0][k]) <= 2e-5 * scale
            g0 = outs[0][1][k]
            assert np.linalg.norm(grads[k].cpu().numpy() - g0) <= 1e-4 * np.linalg.norm(g0)
    grads = [torch.empty_like(p) for p in params]
    rep = b.autotune(params, masks=masks, grads=grads)
    assert "batch autotune: " in rep and rep.count(" ms") >= 6, rep
    e = b.run(params, masks=masks, grads=grads).cpu().numpy()
    if "persistent schedule, tiles 2^12" in rep.splitlines()[0]:
        assert np.array_equal(e, outs[0][0])


def test_bounded_wait_returns_timeout_and_context_survives():
    insts = wl.cluster_batch(3, qubit_range=(13, 14), reps_range=(1, 1), terms_per_qubit=5)
    os.environ["GVQE_TEST_UNSATISFIABLE_WAIT"] = "1"
    os.environ["GVQE_WAIT_TIMEOUT_MS"] = "20"
    try:
        ans, hams, b, params, masks = _setup(insts)
        with pytest.raises(_lib.GvqeError) as err:
            b.run(params)
        assert err.value.code == _lib.GVQE_ETIMEOUT
    finally:
        del os.environ["GVQE_TEST_UNSATISFIABLE_WAIT"]
        del os.environ["GVQE_WAIT_TIMEOUT_MS"]
    # the context is still usable: a fresh batch runs and agrees with single calls
    ans, hams, b, params, masks = _setup(insts)
    e = b.run(params).cpu().numpy()
    for k in range(len(insts)):
        assert abs(e[k] - gv.energy(ans[k], hams[k], params[k]).item()) <= 2e-5 * insts[k].ham.abs_sum()


def test_mixed_batch_small_xy_and_repeated_subproblems():
    """One run over instances the persistent launch takes (n >= 12, diagonal H),
    instances it does not (n < 12, X/Y strings) and one subproblem listed three
    times with different parameter vectors; every slot matches its single call
    and the oracle."""
    insts = wl.cluster_batch(6, qubit_range=(12, 15), reps_range=(1, 2), terms_per_qubit=10)
    small = wl.cluster_batch(3, qubit_range=(6, 11), reps_range=(1, 2), terms_per_qubit=10, base_seed=7000)
    xy_n, xy_reps = 13, 2
    xy_ham = wl.pauli_hamiltonian(xy_n, 60, seed=11)
    ans = [gv.Ansatz(i.n_qubits, i.reps) for i in insts + small]
    hams = [gv.Hamiltonian.from_workload(i.ham) for i in insts + small]
    xa, xh = gv.Ansatz(xy_n, xy_reps), gv.Hamiltonian.from_workload(xy_ham)
    ans.append(xa)
    hams.append(xh)
    rep_a, rep_h = ans[0], hams[0]
    ans += [rep_a, rep_a]
    hams += [rep_h, rep_h]
    thetas = [i.theta[0] for i in insts + small]
    thetas.append(wl.thetas(xy_n, xy_reps, 1, seed=12)[0])
    thetas += [wl.thetas(insts[0].n_qubits, insts[0].reps, 2, seed=13)[k] for k in range(2)]
    b = gv.Batch(ans, hams)
    params = [_dev(t) for t in thetas]
    grads = [torch.full_like(p, float("nan")) for p in params]
    e = b.run(params, grads=grads).cpu().numpy()
    refs = [(i.n_qubits, i.reps, i.ham) for i in insts + small] + [(xy_n, xy_reps, xy_ham)]
    refs += [refs[0], refs[0]]
    for k, (n, reps, ham) in enumerate(refs):
        e1, g1 = gv.energy_grad(ans[k], hams[k], params[k])
        g = grads[k].cpu().numpy()
        scale = ham.abs_sum()
        assert abs(e[k] - e1.item()) <= 2e-5 * scale
        assert np.linalg.norm(g - g1.cpu().numpy()[0]) <= 1e-4 * np.linalg.norm(g1.cpu().numpy()[0])
        e_ref, g_ref = oracle.energy_grad(n, reps, thetas[k], ham.strings, ham.coeffs)
        assert abs(e[k] - e_ref) <= 2e-5 * scale, k
        assert np.linalg.norm(g - g_ref) <= 1e-4 * np.linalg.norm(g_ref), k
    # the repeated subproblem: three different vectors, three different results
    assert len({float(e[0]), float(e[-2]), float(e[-1])}) == 3


@pytest.mark.parametrize("fp64", [False, True])
def test_staged_schedule_takes_every_diagonal_instance(fp64):
    """The staged schedule runs every RY instance with a diagonal H (n < 12
    included) in plan groups; each matches its single call bit for bit and the
    oracle within the bounds; X/Y instances still run as single calls."""
    insts = wl.cluster_batch(12, qubit_range=(7, 15), reps_range=(1, 3), terms_per_qubit=10, base_seed=4000)
    ans, hams, b, params, masks = _setup(insts, fp64)
    xy_ham = wl.pauli_hamiltonian(10, 40, seed=3)
    ans.append(gv.Ansatz(10, 2))
    hams.append(gv.Hamiltonian.from_workload(xy_ham))
    b = gv.Batch(ans, hams, fp64=fp64)  # the staged schedule is the default
    th_xy = wl.thetas(10, 2, 1, seed=4)[0]
    params = params + [_dev(th_xy)]
    masks = masks + [None]
    grads = [torch.full_like(p, float("nan")) for p in params]
    e = b.run(params, masks=[m if m is not None else torch.ones_like(p, dtype=torch.uint8)
                             for m, p in zip(masks, params)], grads=grads).cpu().numpy()
    for k in range(len(params)):
        m = masks[k]
        e1, g1 = gv.energy_grad(ans[k], hams[k], params[k], mask=m, fp64=fp64)
        assert e[k] == e1.item(), k
        assert np.array_equal(grads[k].cpu().numpy(), g1.cpu().numpy()[0]), k
    for k in (0, 5, 11):
        i = insts[k]
        e_ref, g_ref = oracle.energy_grad(i.n_qubits, i.reps, i.theta[0], i.ham.strings, i.ham.coeffs)
        g_ref = np.where(i.mask[0] == 1, g_ref, 0.0)
        scale = i.ham.abs_sum()
        g = grads[k].cpu().numpy()
        if fp64:
            assert abs(e[k] - e_ref) <= 1e-10 * scale
            assert np.max(np.abs(g - g_ref)) <= 1e-9 * scale
        else:
            assert abs(e[k] - e_ref) <= 2e-5 * scale
            assert np.linalg.norm(g - g_ref) <= 1e-4 * np.linalg.norm(g_ref)


def test_staged_schedule_edge_instances():
    """Degenerate instances in one staged batch: n = 1 and 2, reps = 0, n at a
    tile boundary, all-inactive and single-parameter masks; each equals its
    single call bit for bit."""
    specs = [(1, 0), (1, 2), (2, 1), (9, 0), (13, 0), (13, 2), (14, 1), (10, 3)]
    ans, hams, params, masks = [], [], [], []
    for k, (n, reps) in enumerate(specs):
        ham = wl.z_hamiltonian(n, 5 * n + 3, seed=50 + k)
        ans.append(gv.Ansatz(n, reps))
        hams.append(gv.Hamiltonian.from_workload(ham))
        params.append(_dev(wl.thetas(n, reps, 1, seed=60 + k)[0]))
        P = n * (reps + 1)
        m = np.ones(P, dtype=np.uint8)
        if k == 2:
            m[:] = 0  # nothing active
        if k == 5:
            m[:] = 0
            m[P - 1] = 1  # only the last parameter
        masks.append(_dev(m, torch.uint8))
    b = gv.Batch(ans, hams)
    grads = [torch.full_like(p, float("nan")) for p in params]
    e = b.run(params, masks=masks, grads=grads).cpu().numpy()
    for k in range(len(specs)):
        e1, g1 = gv.energy_grad(ans[k], hams[k], params[k], mask=masks[k])
        assert e[k] == e1.item(), specs[k]
        assert np.array_equal(grads[k].cpu().numpy(), g1.cpu().numpy()[0]), specs[k]
    assert np.all(grads[2].cpu().numpy() == 0.0)
