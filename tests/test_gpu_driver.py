"""The Graph-VQE driver (Section IV-C to IV-E) on the GPU: the batched masked
evaluator against the oracle, the block phase against the same phase driven
by the oracle, and a short FP32 run that lowers the energy."""
import numpy as np
import pytest

import oracle
from paper_2607_02749_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2607_02749_gb300.driver import GpuEvaluator, GraphVQE, GraphVQEConfig  # noqa: E402

from test_driver_cpu import OracleEvaluator  # noqa: E402


@pytest.mark.parametrize("ent", [0, 1, 5])
def test_batched_masked_evaluator_matches_the_oracle(ent):
    n, reps = 11, 3
    ham = wl.chain_z_hamiltonian(n, 120, seed=2)
    th = wl.thetas(n, reps, 4, seed=3)
    masks = wl.active_mask(n * (reps + 1), 4, seed=4)
    gpu = GpuEvaluator(n, reps, ham.strings, ham.coeffs, ent, fp64=True)
    e, g = gpu(th, masks)
    eo, go = OracleEvaluator(n, reps, ham.strings, ham.coeffs, ent)(th, masks)
    scale = ham.abs_sum()
    assert np.max(np.abs(e - eo)) <= 1e-10 * scale
    assert np.max(np.abs(g - go)) <= 1e-9 * scale
    assert np.all(g[masks == 0] == 0.0)
    gpu.close()


def test_block_phase_follows_the_oracle_driven_phase():
    n, reps = 10, 2
    ham = wl.chain_z_hamiltonian(n, 100, seed=6)
    th0 = wl.thetas(n, reps, 1, seed=7)[0]
    cfg = GraphVQEConfig(reps=reps, block_maxiter=15, fp64=True)
    gpu = GraphVQE(ham, cfg)
    ref = GraphVQE(ham, cfg, evaluator=OracleEvaluator(n, reps, ham.strings, ham.coeffs))
    assert gpu.labels == ref.labels and gpu.n_blocks >= 2
    a, b = gpu.optimize_blocks(th0), ref.optimize_blocks(th0)
    assert np.max(np.abs(a - b)) <= 1e-6
    assert gpu.energy(a) == pytest.approx(ref.energy(b), abs=1e-9 * ham.abs_sum())


def test_fp32_run_lowers_the_energy():
    n, reps = 16, 3
    ham = wl.chain_z_hamiltonian(n, 20 * n, seed=8)
    cfg = GraphVQEConfig(reps=reps, max_epochs=2, block_maxiter=40, global_maxiter=20)
    g = GraphVQE(ham, cfg)
    r = g.run(wl.thetas(n, reps, 1, seed=9)[0])
    assert r["n_blocks"] >= 2
    assert r["E"] < r["E_start"]
    assert g.evaluator.rows > g.evaluator.calls  # block requests went out batched
