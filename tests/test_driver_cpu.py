"""Host logic of the Graph-VQE driver (Section IV-C to IV-E) on the CPU, with
the oracle's energy and gradient standing in for the GPU: the window early
stop (Eq. 14), lock-step batching of the block optimisers, block restriction
(Eq. 11), fusion, refinement, epochs, and the two-rank round-robin and
Hamiltonian-batching paths (Eq. 12) over gloo."""
import os
import socket

import numpy as np
import pytest

import oracle
from oracle import graph, readout
from paper_2607_02749_gb300 import workloads as wl
from paper_2607_02749_gb300.driver import EarlyStop, GraphVQE, GraphVQEConfig


_ORACLE_THREADS = oracle.max_threads()


class OracleEvaluator:
    """(E, masked dE/dtheta) per row from the CPU oracle (tests only)."""

    def __init__(self, n, reps, strings, coeffs, ent=0, gates=1):
        self.n, self.reps, self.strings, self.coeffs, self.ent = n, reps, list(strings), np.asarray(coeffs), ent
        self.gates = gates
        self.batch_sizes = []

    def __call__(self, th, masks):
        e = np.empty(th.shape[0])
        g = np.empty_like(th)
        oracle.set_threads(1)  # one thread: the same point always gives the same bits
        try:
            with oracle.entangler(self.ent), oracle.gates(self.gates):
                for b in range(th.shape[0]):
                    eb, gb = oracle.energy_grad(self.n, self.reps, th[b], self.strings, self.coeffs)
                    e[b] = eb
                    g[b] = gb if masks is None else gb * (masks[b] != 0)
        finally:
            oracle.set_threads(_ORACLE_THREADS)
        self.batch_sizes.append(th.shape[0])
        return e, g


def test_early_stop_window_and_patience():
    s = EarlyStop(window=3, tol=1e-3, patience=2)
    seq = [10.0, 5.0, 4.0, 4.0, 4.0, 4.0, 4.0, 4.0]
    # diffs 5, 1, 0, 0, 0, 0, 0: the last 3 diffs are all below tol from t = 5 on,
    # and the second such check (t = 6) stops
    stops = [s.update(e) for e in seq]
    assert stops == [False] * 6 + [True, True]
    s = EarlyStop(window=40, tol=1e-4, patience=12)
    assert not any(s.update(1.0) for _ in range(12))  # 11 checks after the first value
    assert s.update(1.0)
    s = EarlyStop(window=2, tol=0.5, patience=1)
    assert [s.update(e) for e in (0.0, 0.1, 1.0, 1.1, 1.2)] == [False, True, False, False, True]


def _problem(n=8, reps=2, seed=1):
    ham = wl.chain_z_hamiltonian(n, 8 * n, seed=seed)
    return ham, OracleEvaluator(n, reps, ham.strings, ham.coeffs), wl.thetas(n, reps, 1, seed=seed + 1)[0]


def test_blocks_and_masks_come_from_the_partition():
    ham, ev, _ = _problem()
    g = GraphVQE(ham, GraphVQEConfig(reps=2), evaluator=ev)
    w = graph.interaction_graph(8, ham.strings, ham.coeffs)
    assert g.labels == graph.partition(w, 1.0, 2)
    assert np.array_equal(g.block_masks(), graph.block_masks(g.labels, 2))


def test_lockstep_blocks_follow_their_solo_trajectories():
    """Batching K block optimisers into one evaluation per step changes nothing
    for any block: each block's result equals optimising it alone."""
    ham, ev, th0 = _problem(n=9, reps=2, seed=3)
    cfg = GraphVQEConfig(reps=2, resolution=1.0, min_block=2, block_maxiter=25)
    g = GraphVQE(ham, cfg, evaluator=ev)
    assert g.n_blocks >= 2
    fused = g.optimize_blocks(th0)
    assert max(ev.batch_sizes) == g.n_blocks and g.block_batches == len(ev.batch_sizes)
    masks = g.block_masks()
    for b in range(g.n_blocks):
        solo = GraphVQE(ham, cfg, evaluator=OracleEvaluator(9, 2, ham.strings, ham.coeffs))
        solo.labels, solo.n_blocks = [0 if l == b else 1 for l in g.labels], 2
        solo_masks = solo.block_masks()
        # run only block b: a lock step of one optimiser
        solo.world, solo.rank = 2, 0  # block 0 of 2 -> this rank's only block
        out = solo.optimize_blocks(th0)
        idx = np.nonzero(masks[b])[0]
        assert np.array_equal(np.nonzero(solo_masks[0])[0], idx)
        assert np.array_equal(out[idx], fused[idx]), b


def test_run_lowers_the_energy_and_keeps_the_best():
    ham, ev, th0 = _problem(n=8, reps=2, seed=5)
    cfg = GraphVQEConfig(reps=2, max_epochs=4, block_maxiter=30, global_maxiter=30)
    g = GraphVQE(ham, cfg, evaluator=ev)
    r = g.run(th0)
    assert r["E"] < r["E_start"]
    assert r["E"] == pytest.approx(min(ep["E"] for ep in r["epochs"]), abs=1e-12) or r["E"] == r["E_start"]
    e_check, _ = ev(r["theta"][None, :], None)
    assert e_check[0] == pytest.approx(r["E"], abs=1e-12)
    # the reachable minimum of a diagonal H is its lowest diagonal entry
    assert r["E"] >= min(readout.diagonal_energies(8, ham.strings, ham.coeffs)) - 1e-9


def test_no_global_ablation_skips_refinement():
    ham, ev, th0 = _problem(n=8, reps=1, seed=7)
    cfg = GraphVQEConfig(reps=1, max_epochs=2, block_maxiter=20, refine=False)
    g = GraphVQE(ham, cfg, evaluator=ev)
    g.run(th0)
    assert {p for _, p, _ in g.history} == {"block"}


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ham, _, th0 = _problem(n=9, reps=2, seed=3)
        cfg = GraphVQEConfig(reps=2, max_epochs=2, block_maxiter=20, global_maxiter=15)
        full = OracleEvaluator(9, 2, ham.strings, ham.coeffs)
        probe = GraphVQE(ham, cfg, evaluator=full, global_evaluator=full)  # for the term slice
        probe.world = world
        lo, hi = probe.term_slice(rank)
        part = OracleEvaluator(9, 2, ham.strings[lo:hi], ham.coeffs[lo:hi])
        g = GraphVQE(ham, cfg, evaluator=full, global_evaluator=part, dist=dist)
        fused = g.optimize_blocks(th0)
        e_global = g.energy(fused)
        out.put((rank, fused, e_global, len(full.batch_sizes)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_round_robin_and_hamiltonian_batching():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, f0, e0, _), (_, f1, e1, _) = res
    assert np.array_equal(f0, f1) and e0 == e1
    # the fused block solution equals the single-process one
    ham, ev, th0 = _problem(n=9, reps=2, seed=3)
    cfg = GraphVQEConfig(reps=2, max_epochs=2, block_maxiter=20, global_maxiter=15)
    single = GraphVQE(ham, cfg, evaluator=ev).optimize_blocks(th0)
    assert np.array_equal(single, f0)
    e_full, _ = ev(single[None, :], None)
    assert e0 == pytest.approx(e_full[0], abs=1e-12 * ham.abs_sum())


def test_full_efficient_su2_layers_in_the_driver():
    """With the RY+RZ layer every block owns the RY and RZ angles of its qubits;
    a short run lowers the energy."""
    n, reps = 7, 1
    ham = wl.chain_z_hamiltonian(n, 8 * n, seed=11)
    cfg = GraphVQEConfig(reps=reps, gates=2, max_epochs=2, block_maxiter=15, global_maxiter=15)
    ev = OracleEvaluator(n, reps, ham.strings, ham.coeffs, gates=2)
    g = GraphVQE(ham, cfg, evaluator=ev)
    m = g.block_masks()
    assert m.shape == (g.n_blocks, 2 * n * (reps + 1)) and np.array_equal(m.sum(axis=0), np.ones(m.shape[1]))
    for b in range(g.n_blocks):
        qs = [q for q in range(n) if g.labels[q] == b]
        want = sorted(r * 2 * n + k * n + q for r in range(reps + 1) for k in range(2) for q in qs)
        assert list(np.nonzero(m[b])[0]) == want
    th0 = np.random.default_rng(3).uniform(-np.pi, np.pi, 2 * n * (reps + 1))
    r = g.run(th0)
    assert r["E"] < r["E_start"]
