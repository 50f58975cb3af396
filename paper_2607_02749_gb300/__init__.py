"""GB300 (sm_103a) engine for the Graph-VQE hot path (arxiv 2607.02749).

State-vector simulation of the RY+CX hardware-efficient ansatz (Section IV-B),
the expectation of a Pauli-sum Hamiltonian (Eq. 4, Eq. 6) and its adjoint or
parameter-shift (Eq. 13) gradient with active-parameter masks (Eq. 11), all in
hand-written CUDA behind the C ABI of include/gvqe.h.  This package is the
thin Python layer over that ABI plus one torch.autograd.Function.
"""
from __future__ import annotations

from typing import Optional, Sequence

from . import _lib
from ._lib import (GVQE_GATES_RY, GVQE_GATES_RY_RZ, GVQE_ENT_CIRCULAR, GVQE_ENT_FULL, GVQE_ENT_LINEAR, GVQE_ENT_PAIRWISE, GVQE_ENT_REVERSE_LINEAR,
                   GVQE_ENT_SCA, GVQE_FP32, GVQE_FP64, GVQE_GRAD_ADJOINT, GVQE_GRAD_PARAM_SHIFT,
                   GVQE_OPT_SPLIT_PASSES, GVQE_OPT_TILE_BITS, GvqeError, gvqe_ansatz_create, gvqe_ansatz_describe,
                   gvqe_ansatz_set_option, gvqe_batch_create,
                   gvqe_batch_run, gvqe_destroy, gvqe_energy, gvqe_energy_grad, gvqe_hamiltonian_create,
                   gvqe_entangler_inverse, gvqe_hamiltonian_stats, gvqe_interaction_graph, gvqe_last_error,
                   gvqe_partition, gvqe_plan_describe, gvqe_readout, gvqe_version)

__all__ = [
    "Hamiltonian", "Ansatz", "Batch", "GvqeEnergy", "energy", "energy_grad", "readout", "Readout", "GvqeError",
    "GVQE_FP32", "GVQE_FP64", "GVQE_GRAD_ADJOINT", "GVQE_GRAD_PARAM_SHIFT", "GVQE_ENT_LINEAR",
    "GVQE_ENT_CIRCULAR", "GVQE_ENT_FULL", "GVQE_ENT_REVERSE_LINEAR", "GVQE_ENT_PAIRWISE", "GVQE_ENT_SCA",
    "GVQE_GATES_RY", "GVQE_GATES_RY_RZ",
    "gvqe_hamiltonian_create", "gvqe_ansatz_create", "gvqe_ansatz_set_option", "gvqe_energy",
    "gvqe_energy_grad", "gvqe_batch_create", "gvqe_batch_run", "gvqe_destroy", "gvqe_last_error",
    "gvqe_plan_describe", "gvqe_hamiltonian_stats", "gvqe_readout", "gvqe_version", "gvqe_entangler_inverse",
    "gvqe_interaction_graph", "gvqe_partition", "gvqe_ansatz_describe", "GVQE_OPT_SPLIT_PASSES",
]


class _Handle:
    handle: Optional[int] = None

    def close(self) -> None:
        if self.handle:
            gvqe_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Hamiltonian(_Handle):
    """H = sum_k c_k P_k (Eq. 6); strings have one letter per qubit (char i = qubit i)."""

    def __init__(self, n_qubits: int, strings: Sequence[str], coeffs):
        self.n_qubits = n_qubits
        self.handle = gvqe_hamiltonian_create(n_qubits, strings, coeffs)

    @classmethod
    def from_workload(cls, ham) -> "Hamiltonian":
        return cls(ham.n_qubits, ham.strings, ham.coeffs)

    def stats(self) -> dict:
        return gvqe_hamiltonian_stats(self.handle)


class Ansatz(_Handle):
    """Rotation layer + reps x [entangler, rotation layer] (Section IV-B); a rotation
    layer is RY on every qubit (gates=GVQE_GATES_RY, P = n (reps + 1)) or the full
    EfficientSU2 layer RY then RZ (gates=GVQE_GATES_RY_RZ, P = 2 n (reps + 1)).
    entangler: GVQE_ENT_LINEAR (default), GVQE_ENT_CIRCULAR, GVQE_ENT_FULL, GVQE_ENT_REVERSE_LINEAR,
    GVQE_ENT_PAIRWISE or GVQE_ENT_SCA (Section IV-B, Table 2)."""

    def __init__(self, n_qubits: int, reps: int, entangler: int = GVQE_ENT_LINEAR, tile_bits: int = 0,
                 gates: int = _lib.GVQE_GATES_RY, split: int = 0):
        self.n_qubits = n_qubits
        self.reps = reps
        self.entangler = entangler
        self.gates = gates
        self.n_params = gates * n_qubits * (reps + 1)
        self.handle = gvqe_ansatz_create(n_qubits, reps, entangler)
        if gates != _lib.GVQE_GATES_RY:
            gvqe_ansatz_set_option(self.handle, _lib.GVQE_OPT_GATES, gates)
        if tile_bits:
            gvqe_ansatz_set_option(self.handle, GVQE_OPT_TILE_BITS, tile_bits)
        if split:
            gvqe_ansatz_set_option(self.handle, GVQE_OPT_SPLIT_PASSES, split)

    def set_tile_bits(self, bits: int) -> None:
        gvqe_ansatz_set_option(self.handle, GVQE_OPT_TILE_BITS, bits)

    def set_mps_layers(self, layers: int) -> None:
        """Leading layers written in closed form (GVQE_OPT_MPS_LAYERS): 0 auto, -1 none, 1..4."""
        gvqe_ansatz_set_option(self.handle, _lib.GVQE_OPT_MPS_LAYERS, layers)

    def set_mps_tensor(self, mode: int) -> None:
        """Bond-16 closed-form gradient pass (GVQE_OPT_MPS_TENSOR): 0 tensor cores (auto), -1 FP32 pipe."""
        gvqe_ansatz_set_option(self.handle, _lib.GVQE_OPT_MPS_TENSOR, mode)

    def describe(self, fp64: bool = False) -> str:
        """The tile-pass plan of this ansatz (host only), with the last autotune report."""
        return gvqe_ansatz_describe(self.handle, GVQE_FP64 if fp64 else GVQE_FP32)

    def autotune(self, ham: "Hamiltonian", theta, fp64: bool = False, energy_only: bool = False,
                 cache: Optional[str] = None, stream=None) -> str:
        """Time every distinct tile plan on theta (CUDA float64 [B, P]) and keep the
        fastest; `cache` is a JSON file of earlier winners (default: $GVQE_TUNE_CACHE,
        none if unset).  Returns the report."""
        import os

        flags = (GVQE_FP64 if fp64 else GVQE_FP32) | (_lib.GVQE_TUNE_ENERGY if energy_only else 0)
        th = theta.reshape(-1, self.n_params).contiguous()
        path = cache if cache is not None else os.environ.get("GVQE_TUNE_CACHE")
        return _lib.gvqe_autotune(self.handle, ham.handle, th, flags, path, stream)


def _flags(fp64: bool, param_shift: bool = False) -> int:
    return (GVQE_FP64 if fp64 else GVQE_FP32) | (GVQE_GRAD_PARAM_SHIFT if param_shift else 0)


def energy(ansatz: Ansatz, ham: Hamiltonian, theta, fp64: bool = False, stream=None):
    """E[b] for theta[b] (CUDA float64 [B, P]); returns a CUDA float64 tensor [B]."""
    import torch

    th = theta.reshape(-1, ansatz.n_params).contiguous()
    e = torch.empty(th.shape[0], dtype=torch.float64, device=th.device)
    gvqe_energy(ansatz.handle, ham.handle, th, e, _flags(fp64), stream)
    return e


def energy_grad(ansatz: Ansatz, ham: Hamiltonian, theta, mask=None, fp64: bool = False,
                param_shift: bool = False, stream=None):
    """(E[B], dE/dtheta [B, P]); mask uint8 [B, P] (nonzero = active) or None."""
    import torch

    th = theta.reshape(-1, ansatz.n_params).contiguous()
    e = torch.empty(th.shape[0], dtype=torch.float64, device=th.device)
    g = torch.empty_like(th)
    m = None if mask is None else mask.reshape(th.shape).to(torch.uint8).contiguous()
    gvqe_energy_grad(ansatz.handle, ham.handle, th, m, e, g, _flags(fp64, param_shift), stream)
    return e, g


class Readout:
    """Result of readout(): the most probable bitstring, its probability, the
    shots, CVaR_alpha of the outcome energy and the total probability."""

    def __init__(self, argmax: int, p_max: float, cvar: float, total: float, shots, passes: int = 0):
        self.argmax, self.p_max, self.cvar, self.total, self.shots = argmax, p_max, cvar, total, shots
        self.passes = passes  # histogram passes of the CVaR search

    def bitstring(self, n: int) -> str:
        """The most probable x as a string whose character q is qubit q."""
        return "".join("1" if (self.argmax >> q) & 1 else "0" for q in range(n))


def readout(ansatz: Ansatz, ham: Optional[Hamiltonian], theta, alpha: float = 0.2, shots: int = 8192,
            seed: Optional[int] = 0, uniforms=None, fp64: bool = False, stream=None) -> Readout:
    """Read out |psi(theta)> (Section IV-F; 8192 shots with seed 0 and CVaR
    alpha = 0.2 as in Section V-A).  The shots use `uniforms` (CUDA float64, in
    [0, 1)) or, when None, `shots` draws of numpy's PCG64(seed) made on the host.
    alpha = 0 skips the CVaR (ham may then be None)."""
    import numpy as np
    import torch

    th = theta.reshape(-1).to(torch.float64).contiguous()
    dev = th.device
    if uniforms is None and shots > 0:
        u = np.random.Generator(np.random.PCG64(seed)).random(shots)
        uniforms = torch.as_tensor(u, dtype=torch.float64, device=dev)
    n_shots = 0 if uniforms is None else int(uniforms.numel())
    out = torch.empty(max(1, n_shots), dtype=torch.int64, device=dev)
    stats = torch.empty(4, dtype=torch.float64, device=dev)
    amax = torch.empty(1, dtype=torch.int64, device=dev)
    gvqe_readout(ansatz.handle, None if ham is None else ham.handle, th, alpha,
                 None if n_shots == 0 else uniforms.contiguous(), out if n_shots else None, stats, amax,
                 _flags(fp64), stream)
    st = stats.cpu().tolist()
    return Readout(int(amax.item()), st[0], st[1], st[2], out[:n_shots], int(st[3]))


class Batch(_Handle):
    """Many independent (ansatz, Hamiltonian) restricted-update problems run together."""

    def __init__(self, ansatze: Sequence[Ansatz], hams: Sequence[Hamiltonian], fp64: bool = False):
        self._keep = (list(ansatze), list(hams))
        self.handle = gvqe_batch_create([a.handle for a in ansatze], [h.handle for h in hams], _flags(fp64))

    def run(self, params: Sequence, masks: Optional[Sequence] = None, grads: Optional[Sequence] = None,
            energies=None, stream=None):
        import torch

        if energies is None:
            energies = torch.empty(len(params), dtype=torch.float64, device=params[0].device)
        gvqe_batch_run(self.handle, params, masks, energies, grads, stream)
        return energies

    def set_schedule(self, staged: bool) -> None:
        """One launch per stage (True) or one persistent launch (False, the default)."""
        _lib.gvqe_batch_set_option(self.handle, _lib.GVQE_BATCH_OPT_SCHEDULE,
                                   _lib.GVQE_BATCH_STAGED if staged else _lib.GVQE_BATCH_PERSISTENT)

    def set_tile_bits(self, bits: int) -> None:
        """log2 amplitudes of one work item of the persistent launch (10, 11 or 12)."""
        _lib.gvqe_batch_set_option(self.handle, _lib.GVQE_BATCH_OPT_TILE_BITS, bits)

    def set_wave_bytes(self, nbytes: int) -> None:
        """Workspace bytes per wave of the persistent schedule (0: one wave)."""
        _lib.gvqe_batch_set_option(self.handle, _lib.GVQE_BATCH_OPT_WAVE_BYTES, nbytes)

    def autotune(self, params: Sequence, masks: Optional[Sequence] = None, grads: Optional[Sequence] = None,
                 energies=None, stream=None) -> str:
        """Time the batch under each wave budget and keep the fastest; returns the report."""
        import torch

        if energies is None:
            energies = torch.empty(len(params), dtype=torch.float64, device=params[0].device)
        return _lib.gvqe_batch_autotune(self.handle, params, masks, energies, grads, stream)


def _make_function():
    import torch

    class GvqeEnergy(torch.autograd.Function):
        """E = <psi(theta)|H|psi(theta)> per row of theta, differentiable through the adjoint gradient.

        forward(theta [B, P] float64 CUDA, ansatz, ham, mask=None, fp64=False) -> E [B];
        backward returns grad_E[:, None] * dE/dtheta (inactive mask entries give 0).
        """

        @staticmethod
        def forward(ctx, theta, ansatz, ham, mask=None, fp64=False):
            if theta.requires_grad:
                e, g = energy_grad(ansatz, ham, theta.detach(), mask=mask, fp64=fp64)
                ctx.save_for_backward(g)
            else:
                e = energy(ansatz, ham, theta.detach(), fp64=fp64)
                ctx.save_for_backward(None)
            return e

        @staticmethod
        def backward(ctx, grad_e):
            (g,) = ctx.saved_tensors
            gt = None if g is None else grad_e.reshape(-1, 1).to(g.dtype) * g
            return gt, None, None, None, None

    return GvqeEnergy


class _LazyFunction:
    _fn = None

    def __getattr__(self, name):
        if _LazyFunction._fn is None:
            _LazyFunction._fn = _make_function()
        return getattr(_LazyFunction._fn, name)


GvqeEnergy = _LazyFunction()
