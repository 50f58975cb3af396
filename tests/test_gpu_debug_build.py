"""The debug build (GVQE_DEBUG, libgvqe_debug.so): every device workspace sits
between two guard zones.  A child process loads the debug library, runs the
kernels of every path (RY and RY+RZ passes with the split strided layout, FP32
and FP64, masks, X/Y strings, parameter shift, readout, the persistent batch
kernel), then checks the guards; its results must be bit-identical to the
regular library's in this process.  A guard byte overwritten from the host must
be reported as GVQE_ECORRUPT."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKLOADS = r"""
import json, sys
import numpy as np
import torch
import paper_2607_02749_gb300 as gv
from paper_2607_02749_gb300 import _lib
from paper_2607_02749_gb300 import workloads as wl

out = {}
dev = "cuda"
ham = wl.z_hamiltonian(18, 120, seed=1)
h = gv.Hamiltonian.from_workload(ham)
for fp64 in (False, True):
    a = gv.Ansatz(18, 2, tile_bits=10, split=2)
    th = torch.as_tensor(wl.thetas(18, 2, 2, seed=2), device=dev)
    mask = torch.as_tensor((np.arange(th.numel()).reshape(th.shape) % 3 != 0).astype(np.uint8), device=dev)
    e, g = gv.energy_grad(a, h, th, mask=mask, fp64=fp64)
    out[f"ry_{fp64}"] = [e.cpu().tolist(), g.cpu().flatten().tolist()]
    a2 = gv.Ansatz(17, 1, gates=gv.GVQE_GATES_RY_RZ, tile_bits=10, split=2, entangler=gv.GVQE_ENT_SCA)
    h2 = gv.Hamiltonian.from_workload(wl.chain_z_hamiltonian(17, 100, seed=3))
    t2 = torch.as_tensor(np.random.default_rng(4).uniform(-np.pi, np.pi, (1, a2.n_params)), device=dev)
    e, g = gv.energy_grad(a2, h2, t2, fp64=fp64)
    out[f"su2_{fp64}"] = [e.cpu().tolist(), g.cpu().flatten().tolist()]
hp = gv.Hamiltonian.from_workload(wl.pauli_hamiltonian(14, 50, seed=5))
a3 = gv.Ansatz(14, 2, entangler=gv.GVQE_ENT_CIRCULAR)
t3 = torch.as_tensor(wl.thetas(14, 2, 1, seed=6), device=dev)
e, g = gv.energy_grad(a3, hp, t3)
out["xy"] = [e.cpu().tolist(), g.cpu().flatten().tolist()]
m3 = torch.zeros(1, a3.n_params, dtype=torch.uint8, device=dev)
m3[0, 5] = 1
e, g = gv.energy_grad(a3, hp, t3, mask=m3, fp64=True, param_shift=True)
out["shift"] = [e.cpu().tolist(), g.cpu().flatten().tolist()]
a4 = gv.Ansatz(16, 2)
h4 = gv.Hamiltonian.from_workload(wl.z_hamiltonian(16, 80, seed=7))
r = gv.readout(a4, h4, torch.as_tensor(wl.thetas(16, 2, 1, seed=8)[0], device=dev), shots=256)
out["readout"] = [r.argmax, r.p_max, r.cvar, r.shots.cpu().tolist()]
insts = wl.cluster_batch(4, qubit_range=(10, 14), reps_range=(1, 2), terms_per_qubit=10)
b = gv.Batch([gv.Ansatz(i.n_qubits, i.reps) for i in insts], [gv.Hamiltonian.from_workload(i.ham) for i in insts])
params = [torch.as_tensor(i.theta[0], device=dev) for i in insts]
grads = [torch.empty_like(p) for p in params]
e = b.run(params, grads=grads)
out["batch"] = [e.cpu().tolist(), [g.cpu().tolist() for g in grads]]
torch.cuda.synchronize()
if _lib.DEBUG:
    _lib.gvqe_debug_check()
    out["checked"] = True
    _lib.gvqe_debug_poke_guard()
    try:
        _lib.gvqe_debug_check()
        out["poke_detected"] = False
    except _lib.GvqeError as exc:
        out["poke_detected"] = exc.code == _lib.GVQE_ECORRUPT
        out["poke_message"] = str(exc)
    _lib.gvqe_debug_poke_guard(restore=True)
    _lib.gvqe_debug_check()
print(json.dumps(out))
"""


def _run(debug: bool) -> dict:
    env = dict(os.environ, GVQE_DEBUG="1" if debug else "0", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", WORKLOADS], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-4000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_debug_build_guards_hold_and_results_are_bit_identical():
    dbg = _run(True)
    reg = _run(False)
    assert dbg.pop("checked") is True
    assert dbg.pop("poke_detected") is True, dbg.get("poke_message")
    assert "overwritten at byte 0 past the end" in dbg.pop("poke_message")
    assert "checked" not in reg
    assert set(dbg) == set(reg)
    for k in reg:
        assert dbg[k] == reg[k], k
    # and the regular library refuses the check
    from paper_2607_02749_gb300 import _lib

    if not _lib.DEBUG:
        with pytest.raises(_lib.GvqeError) as e:
            _lib.gvqe_debug_check()
        assert e.value.code == _lib.GVQE_EUNSUPPORTED
    assert np.isfinite(reg["ry_False"][0]).all()
