"""Graph-VQE host driver (Section IV-C to IV-E): the optimisation loop around
the GPU energy/gradient path.

Each epoch (Section IV-E):
  1. blocks: the weighted qubit interaction graph (Eq. 9) is partitioned by the
     Louvain method (Eq. 10) with small blocks merged (S_min); block B_i owns
     theta_{B_i}, every layer's angle of its qubits;
  2. block phase: every block minimises the full-Hamiltonian energy over its
     own coordinates with all others frozen at the epoch's start (Eq. 11),
     by L-BFGS-B with ftol and gtol = 0.1 ftol and the window early stop of
     Eq. 14; the block solutions are then fused;
  3. global refinement: a short L-BFGS-B run over all P parameters from the
     fused point, with the same early stop;
  4. the epoch's best energy is compared with the best so far; after
     `patience_epoch` epochs without a new best the loop ends, and every epoch
     starts from the best parameters found so far.

GB300 design: the paper spreads blocks round-robin over GPUs (one block per
virtual QPU).  Here the block optimisers of one process run in lock step and
each step's K energy/gradient requests go to the GPU as ONE batched call with
per-row active masks (gvqe_energy_grad, batch = K).  Gradients are adjoint
(exact, one backward sweep) unless `grad="param_shift"` asks for Eq. 13.

With torch.distributed initialised (one process per GPU), blocks are dealt
round-robin to ranks (block i to rank i mod N) and their solutions are summed
across ranks (they are disjoint), and the global phase uses Hamiltonian
batching (Eq. 12): rank r evaluates the r-th contiguous slice of the terms and
the energies and gradients are summed across ranks, so every rank takes the
same optimiser steps.
"""
from __future__ import annotations

import dataclasses
import math
import threading
from typing import Callable, Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import _lib

Evaluator = Callable[[np.ndarray, Optional[np.ndarray]], Tuple[np.ndarray, np.ndarray]]


class EarlyStop:
    """Window criterion of Eq. 14: after each energy E_t, Delta_max is the largest
    |E_s - E_{s-1}| over the last `window` steps; the run stops once
    Delta_max < tol has held for `patience` consecutive checks."""

    def __init__(self, window: int, tol: float, patience: int):
        self.window, self.tol, self.patience = int(window), float(tol), int(patience)
        self.hist: List[float] = []
        self.count = 0

    def update(self, e: float) -> bool:
        self.hist.append(float(e))
        if len(self.hist) < 2:
            return False
        h = self.hist[-(self.window + 1):]
        dmax = max(abs(h[i] - h[i - 1]) for i in range(1, len(h)))
        self.count = self.count + 1 if dmax < self.tol else 0
        return self.count >= self.patience


@dataclasses.dataclass
class GraphVQEConfig:
    """Hyperparameters (defaults from Section V-A and Section VI-C: reps 4,
    tolerance 1e-4, patience 12, window 40, epoch patience 3)."""

    reps: int = 4
    entangler: int = _lib.GVQE_ENT_LINEAR
    gates: int = _lib.GVQE_GATES_RY  # or GVQE_GATES_RY_RZ: the full EfficientSU2 layer (Eq. 8)
    resolution: float = 1.0        # Louvain gamma
    min_block: int = 2             # S_min
    ftol: float = 1e-4             # L-BFGS-B ftol; gtol = 0.1 ftol; also the early-stop tolerance
    window: int = 40               # W of Eq. 14
    patience_block: int = 12
    patience_global: int = 12
    patience_epoch: int = 3
    max_epochs: int = 20
    block_maxiter: int = 200       # L-BFGS-B iterations per block per epoch
    global_maxiter: int = 100      # L-BFGS-B iterations of the refinement per epoch
    refine: bool = True            # False: the no_Global ablation of Section V-A
    fp64: bool = False
    grad: str = "adjoint"          # or "param_shift" (Eq. 13)


class GpuEvaluator:
    """Energies and gradients of rows of theta on this process's GPU through the
    C ABI: one gvqe_energy_grad call per request batch (per-row masks)."""

    def __init__(self, n_qubits: int, reps: int, strings: Sequence[str], coeffs, entangler: int,
                 fp64: bool = False, grad: str = "adjoint", device=None, gates: int = _lib.GVQE_GATES_RY):
        import torch

        from . import Ansatz, Hamiltonian

        self.torch = torch
        self.device = torch.device("cuda") if device is None else torch.device(device)
        self.ansatz = Ansatz(n_qubits, reps, entangler, gates=gates)
        self.ham = Hamiltonian(n_qubits, list(strings), np.asarray(coeffs, dtype=np.float64))
        self.flags = ((_lib.GVQE_FP64 if fp64 else _lib.GVQE_FP32)
                      | (_lib.GVQE_GRAD_PARAM_SHIFT if grad == "param_shift" else 0))
        self.calls = 0
        self.rows = 0

    def __call__(self, thetas: np.ndarray, masks: Optional[np.ndarray]) -> Tuple[np.ndarray, np.ndarray]:
        torch = self.torch
        th = torch.as_tensor(np.ascontiguousarray(thetas, dtype=np.float64), device=self.device)
        b = th.shape[0]
        e = torch.empty(b, dtype=torch.float64, device=self.device)
        g = torch.empty_like(th)
        m = None
        if masks is not None:
            m = torch.as_tensor(np.ascontiguousarray(masks, dtype=np.uint8), device=self.device)
        _lib.gvqe_energy_grad(self.ansatz.handle, self.ham.handle, th, m, e, g, self.flags, None)
        self.calls += 1
        self.rows += b
        return e.cpu().numpy(), g.cpu().numpy()

    def close(self) -> None:
        self.ansatz.close()
        self.ham.close()


class _Stop(Exception):
    pass


class _Objective:
    """f(x) for L-BFGS-B over the coordinates `idx` of theta (others fixed),
    with early stopping and the best point seen kept."""

    def __init__(self, base: np.ndarray, idx: np.ndarray, request, stopper: EarlyStop, record):
        self.base, self.idx, self.request, self.stopper, self.record = base, idx, request, stopper, record
        self.best_e = math.inf
        self.best_x = base[idx].copy()
        self.evals = 0

    def __call__(self, x: np.ndarray):
        th = self.base.copy()
        th[self.idx] = x
        e, g = self.request(th)
        self.evals += 1
        self.record(e)
        if e < self.best_e:
            self.best_e, self.best_x = e, np.array(x, copy=True)
        if self.stopper.update(e):
            raise _Stop()
        return e, g[self.idx]


def _lbfgsb(obj: _Objective, x0: np.ndarray, ftol: float, maxiter: int) -> None:
    from scipy.optimize import minimize

    try:
        minimize(obj, x0, jac=True, method="L-BFGS-B",
                 options={"ftol": ftol, "gtol": 0.1 * ftol, "maxiter": maxiter})
    except _Stop:
        pass


class _Lockstep:
    """K optimisers in K threads; their requests are answered together by one
    batched evaluation once every live optimiser has one pending."""

    def __init__(self, evaluator: Evaluator, masks: np.ndarray):
        self.evaluator, self.masks = evaluator, masks
        self.cv = threading.Condition()
        self.pending: Dict[int, np.ndarray] = {}
        self.results: Dict[int, Tuple[float, np.ndarray]] = {}
        self.live = set(range(masks.shape[0]))
        self.error: Optional[BaseException] = None
        self.batches = 0

    def _flush_locked(self) -> None:
        if not self.pending or not set(self.pending) >= self.live:
            return
        ks = sorted(self.pending)
        try:
            e, g = self.evaluator(np.stack([self.pending[k] for k in ks]), self.masks[ks])
            for i, k in enumerate(ks):
                self.results[k] = (float(e[i]), g[i])
        except BaseException as ex:  # surfaced in every waiting thread
            self.error = ex
        self.pending.clear()
        self.batches += 1
        self.cv.notify_all()

    def request(self, k: int, theta: np.ndarray) -> Tuple[float, np.ndarray]:
        with self.cv:
            self.pending[k] = theta
            self._flush_locked()
            while k not in self.results and self.error is None:
                self.cv.wait()
            if self.error is not None:
                raise RuntimeError("batched evaluation failed") from self.error
            return self.results.pop(k)

    def done(self, k: int) -> None:
        with self.cv:
            self.live.discard(k)
            self._flush_locked()


class GraphVQE:
    """The Graph-VQE optimiser over one Pauli-sum Hamiltonian (see module doc).

    ham: an object with n_qubits, strings, coeffs (workloads.Hamiltonian).
    evaluator: callable (thetas [B, P], masks [B, P] or None) -> (E [B], G [B, P]);
    default a GpuEvaluator on this process's GPU (over this rank's slice of
    the terms for the global phase when torch.distributed is initialised).
    """

    def __init__(self, ham, cfg: Optional[GraphVQEConfig] = None, evaluator: Optional[Evaluator] = None,
                 global_evaluator: Optional[Evaluator] = None, dist=None):
        self.cfg = cfg or GraphVQEConfig()
        self.n = int(ham.n_qubits)
        self.strings = list(ham.strings)
        self.coeffs = np.asarray(ham.coeffs, dtype=np.float64)
        self.P = self.cfg.gates * self.n * (self.cfg.reps + 1)
        self.dist = dist
        self.rank, self.world = 0, 1
        if dist is not None and dist.is_available() and dist.is_initialized():
            self.rank, self.world = dist.get_rank(), dist.get_world_size()
        else:
            self.dist = None
        c = self.cfg
        if evaluator is None:
            evaluator = GpuEvaluator(self.n, c.reps, self.strings, self.coeffs, c.entangler, c.fp64, c.grad,
                                     gates=c.gates)
        self.evaluator = evaluator
        if global_evaluator is None:
            if self.world > 1:
                lo, hi = self.term_slice(self.rank)
                global_evaluator = GpuEvaluator(self.n, c.reps, self.strings[lo:hi], self.coeffs[lo:hi],
                                                c.entangler, c.fp64, c.grad, gates=c.gates)
            else:
                global_evaluator = evaluator
        self.global_evaluator = global_evaluator
        self.history: List[Tuple[int, str, float]] = []  # (epoch, phase, E) per evaluation
        self.epoch = 0
        self.labels, self.n_blocks, self.modularity = self.blocks()

    # -- Section IV-C ------------------------------------------------------
    def term_slice(self, r: int) -> Tuple[int, int]:
        """Terms of rank r under Hamiltonian batching (Eq. 12): ceil(M / N) per rank."""
        m = len(self.strings)
        per = -(-m // self.world)
        return min(m, r * per), min(m, (r + 1) * per)

    def blocks(self) -> Tuple[List[int], int, float]:
        w = _lib.gvqe_interaction_graph(self.n, self.strings, self.coeffs)
        return _lib.gvqe_partition(w, self.cfg.resolution, self.cfg.min_block)

    def block_masks(self) -> np.ndarray:
        """theta_{B_i}: every rotation angle (RY, and RZ with the full layer) of every
        layer on the qubits of block i."""
        g = self.cfg.gates
        m = np.zeros((self.n_blocks, self.P), dtype=np.uint8)
        for r in range(self.cfg.reps + 1):
            for k in range(g):
                for q in range(self.n):
                    m[self.labels[q], r * g * self.n + k * self.n + q] = 1
        return m

    # -- Section IV-D: block phase -----------------------------------------
    def optimize_blocks(self, theta: np.ndarray) -> np.ndarray:
        """Every block of this rank minimises E over theta_{B_i} from `theta`
        (others frozen there); returns the fused point (summed over ranks)."""
        c = self.cfg
        masks_all = self.block_masks()
        mine = [b for b in range(self.n_blocks) if b % self.world == self.rank]
        masks = masks_all[mine]
        lock = _Lockstep(self.evaluator, masks)
        objs = []
        for i, b in enumerate(mine):
            idx = np.nonzero(masks_all[b])[0]
            stop = EarlyStop(c.window, c.ftol, c.patience_block)
            objs.append(_Objective(theta, idx, (lambda i: lambda th: lock.request(i, th))(i), stop,
                                   lambda e: self.history.append((self.epoch, "block", e))))
        errors: List[BaseException] = []

        def work(i: int) -> None:
            try:
                _lbfgsb(objs[i], theta[objs[i].idx], c.ftol, c.block_maxiter)
            except BaseException as ex:
                errors.append(ex)
            finally:
                lock.done(i)

        threads = [threading.Thread(target=work, args=(i,), daemon=True) for i in range(len(mine))]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        if errors:
            raise errors[0]
        self.block_batches = lock.batches
        delta = np.zeros(self.P)
        for o in objs:
            delta[o.idx] = o.best_x - theta[o.idx]
        if self.dist is not None:
            delta = self._allreduce(delta)
        return theta + delta

    # -- Section IV-D: global refinement -----------------------------------
    def refine(self, theta: np.ndarray) -> np.ndarray:
        c = self.cfg
        idx = np.arange(self.P)

        def request(th):
            e, g = self.global_evaluator(th[None, :], None)
            if self.dist is not None:
                eg = self._allreduce(np.concatenate([e[:1], g[0]]))
                return float(eg[0]), eg[1:]
            return float(e[0]), g[0]

        obj = _Objective(theta, idx, request, EarlyStop(c.window, c.ftol, c.patience_global),
                         lambda e: self.history.append((self.epoch, "global", e)))
        _lbfgsb(obj, theta.copy(), c.ftol, c.global_maxiter)
        return obj.best_x

    def _allreduce(self, v: np.ndarray) -> np.ndarray:
        import torch

        backend = self.dist.get_backend()
        dev = torch.device("cuda") if backend == "nccl" else torch.device("cpu")
        t = torch.as_tensor(np.ascontiguousarray(v, dtype=np.float64), device=dev)
        self.dist.all_reduce(t)
        return t.cpu().numpy()

    def energy(self, theta: np.ndarray) -> float:
        e, _ = self.global_evaluator(theta[None, :], None)
        e = np.asarray(e, dtype=np.float64)[:1]
        if self.dist is not None:
            e = self._allreduce(e)
        return float(e[0])

    # -- Section IV-E: epochs ---------------------------------------------
    def run(self, theta0: np.ndarray) -> dict:
        c = self.cfg
        best_theta = np.array(theta0, dtype=np.float64).reshape(-1).copy()
        if best_theta.size != self.P:
            raise ValueError(f"theta0 has {best_theta.size} entries, P = {self.P}")
        best_e = self.energy(best_theta)
        start_e = best_e
        stale = 0
        epochs = []
        for ep in range(c.max_epochs):
            self.epoch = ep
            th = self.optimize_blocks(best_theta)
            e_blocks = self.energy(th)
            if c.refine:
                th = self.refine(th)
            e = self.energy(th)
            epochs.append({"epoch": ep, "E_blocks": e_blocks, "E": e})
            if e < best_e - c.ftol:
                best_e, best_theta, stale = e, th, 0
            else:
                if e < best_e:
                    best_e, best_theta = e, th
                stale += 1
                if stale >= c.patience_epoch:
                    break
        return {"theta": best_theta, "E": best_e, "E_start": start_e, "epochs": epochs,
                "blocks": self.labels, "n_blocks": self.n_blocks, "modularity": self.modularity,
                "evaluations": len(self.history)}
