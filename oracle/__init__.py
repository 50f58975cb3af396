"""CPU oracle for the Graph-VQE energy / gradient path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import this package.  The product library never loads it.

``gvqe_oracle.c`` is the plain complex128 gate-by-gate simulator (Section IV-B,
Eq. 4, 6, 7, 13); ``dense.py`` is an independent dense-matrix model for tiny
registers and ``closed_form.py`` holds closed forms used as pins;
``readout.py`` is the readout of Section IV-F and ``graph.py`` the interaction
graph and Louvain partitioning of Section IV-C.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gvqe_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib: Optional[ctypes.CDLL] = None


def build(force: bool = False, src: str = _SRC, out: str = _LIB_PATH) -> str:
    """Compile the C oracle with gcc + OpenMP into a shared library; returns its path."""
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def load(path: Optional[str] = None) -> ctypes.CDLL:
    """Build (if needed) and load the oracle library."""
    global _lib
    with _lock:
        if path is None and _lib is not None:
            return _lib
        lib = ctypes.CDLL(build() if path is None else path)
        d = ctypes.c_double
        i = ctypes.c_int
        p = ctypes.c_void_p
        lib.oracle_state.argtypes = [i, i, p, p]
        lib.oracle_apply_hamiltonian.argtypes = [i, i, p, p, p, p]
        lib.oracle_energy.argtypes = [i, i, p, i, p, p, p, p]
        lib.oracle_energy_grad.argtypes = [i, i, p, i, p, p, p, p]
        lib.oracle_param_shift_grad.argtypes = [i, i, p, i, p, p, p, p]
        lib.oracle_partial_work.argtypes = [i, i, i, p, p, p, p]
        lib.oracle_sweep_times.argtypes = [i, i, i, p, p, p, p]
        lib.oracle_max_threads.restype = i
        lib.oracle_set_threads.argtypes = [i]
        lib.oracle_set_entangler.argtypes = [i]
        lib.oracle_set_entangler.restype = i
        lib.oracle_set_gates.argtypes = [i]
        lib.oracle_set_gates.restype = i
        for f in ("oracle_state", "oracle_apply_hamiltonian", "oracle_energy",
                  "oracle_energy_grad", "oracle_param_shift_grad", "oracle_partial_work",
                  "oracle_sweep_times"):
            getattr(lib, f).restype = i
        del d
        if path is None:
            _lib = lib
        return lib


def _ptr(a: np.ndarray) -> ctypes.c_void_p:
    return ctypes.c_void_p(a.ctypes.data)


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


class _HamArgs:
    """Flat (strings, coeffs) buffers kept alive for one call."""

    def __init__(self, n: int, strings, coeffs):
        strings = list(strings)
        for s in strings:
            if len(s) != n:
                raise ValueError(f"Pauli string {s!r} has length {len(s)} != {n}")
        self.m = len(strings)
        self.buf = np.frombuffer("".join(strings).encode("ascii") or b"\0", dtype=np.uint8).copy()
        self.c = np.ascontiguousarray(coeffs, dtype=np.float64).reshape(-1).copy()
        if self.c.size == 0:
            self.c = np.zeros(1)


def _ham(ham_or_strings, coeffs=None):
    if coeffs is None:
        return ham_or_strings.n_qubits, ham_or_strings.strings, ham_or_strings.coeffs
    return None, ham_or_strings, coeffs


def set_threads(n: int) -> None:
    load().oracle_set_threads(int(n))


ENT_LINEAR, ENT_CIRCULAR, ENT_FULL = 0, 1, 2
ENT_REVERSE_LINEAR, ENT_PAIRWISE, ENT_SCA = 3, 4, 5


class entangler:
    """Context manager selecting the oracle's entangler (Section IV-B, Table 2):
    ENT_LINEAR (default), ENT_CIRCULAR (CX(n-1,0) first, then the linear chain),
    ENT_FULL (CX(i,j) for all i < j in lexicographic order), ENT_REVERSE_LINEAR
    (the linear chain in descending order), ENT_PAIRWISE (even-start pairs, then
    odd-start pairs) or ENT_SCA (the circular list rotated right by the layer's
    offset r - 1, control and target swapped on odd offsets)."""

    def __init__(self, ent: int, lib: Optional[ctypes.CDLL] = None):
        self.ent = int(ent)
        self.lib = lib

    def __enter__(self):
        _check((self.lib or load()).oracle_set_entangler(self.ent), "set_entangler")
        return self

    def __exit__(self, *exc):
        (self.lib or load()).oracle_set_entangler(ENT_LINEAR)
        return False


GATES_RY, GATES_RY_RZ = 1, 2
_gates = GATES_RY


class gates:
    """Context manager selecting the oracle's rotation layer: GATES_RY (default,
    P = n (D+1)) or GATES_RY_RZ, the full EfficientSU2 layer of Eq. 8 (RY then RZ
    on every qubit, P = 2 n (D+1); layer r's RY angles at 2 r n + q, RZ angles at
    2 r n + n + q)."""

    def __init__(self, g: int, lib: Optional[ctypes.CDLL] = None):
        self.g = int(g)
        self.lib = lib

    def __enter__(self):
        global _gates
        _check((self.lib or load()).oracle_set_gates(self.g), "set_gates")
        _gates = self.g
        return self

    def __exit__(self, *exc):
        global _gates
        (self.lib or load()).oracle_set_gates(GATES_RY)
        _gates = GATES_RY
        return False


def n_params(n: int, reps: int) -> int:
    return _gates * n * (reps + 1)


def max_threads() -> int:
    return int(load().oracle_max_threads())


def state(n: int, reps: int, theta, lib: Optional[ctypes.CDLL] = None) -> np.ndarray:
    """|psi(theta)> as complex128 [2^n] (Section IV-B ansatz)."""
    lib = lib or load()
    th = np.ascontiguousarray(theta, dtype=np.float64).reshape(-1)
    assert th.size == n_params(n, reps)
    out = np.empty(2 << n, dtype=np.float64)
    _check(lib.oracle_state(n, reps, _ptr(th), _ptr(out)), "state")
    return out.view(np.complex128)


def apply_hamiltonian(n: int, strings, coeffs, psi, lib: Optional[ctypes.CDLL] = None) -> np.ndarray:
    """H psi, term by term (Eq. 6)."""
    lib = lib or load()
    h = _HamArgs(n, strings, coeffs)
    v = np.ascontiguousarray(psi, dtype=np.complex128).reshape(-1)
    assert v.size == 1 << n
    out = np.empty(1 << n, dtype=np.complex128)
    _check(lib.oracle_apply_hamiltonian(n, h.m, _ptr(h.buf), _ptr(h.c), _ptr(v), _ptr(out)),
           "apply_hamiltonian")
    return out


def energy(n: int, reps: int, theta, strings, coeffs, lib: Optional[ctypes.CDLL] = None,
           with_imag: bool = False):
    """E = <psi|H|psi> (Eq. 4)."""
    lib = lib or load()
    h = _HamArgs(n, strings, coeffs)
    th = np.ascontiguousarray(theta, dtype=np.float64).reshape(-1)
    e = np.zeros(1)
    ei = np.zeros(1)
    _check(lib.oracle_energy(n, reps, _ptr(th), h.m, _ptr(h.buf), _ptr(h.c), _ptr(e), _ptr(ei)),
           "energy")
    return (float(e[0]), float(ei[0])) if with_imag else float(e[0])


def energy_grad(n: int, reps: int, theta, strings, coeffs,
                lib: Optional[ctypes.CDLL] = None) -> Tuple[float, np.ndarray]:
    """(E, dE/dtheta) by the gate-by-gate adjoint sweep."""
    lib = lib or load()
    h = _HamArgs(n, strings, coeffs)
    th = np.ascontiguousarray(theta, dtype=np.float64).reshape(-1)
    e = np.zeros(1)
    g = np.zeros(th.size)
    _check(lib.oracle_energy_grad(n, reps, _ptr(th), h.m, _ptr(h.buf), _ptr(h.c), _ptr(e), _ptr(g)),
           "energy_grad")
    return float(e[0]), g


def param_shift_grad(n: int, reps: int, theta, strings, coeffs, mask=None,
                     lib: Optional[ctypes.CDLL] = None) -> np.ndarray:
    """dE/dtheta by the parameter-shift rule (Eq. 13); inactive entries are 0."""
    lib = lib or load()
    h = _HamArgs(n, strings, coeffs)
    th = np.ascontiguousarray(theta, dtype=np.float64).reshape(-1)
    g = np.zeros(th.size)
    if mask is None:
        mp = ctypes.c_void_p(0)
    else:
        mk = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
        mp = _ptr(mk)
    _check(lib.oracle_param_shift_grad(n, reps, _ptr(th), h.m, _ptr(h.buf), _ptr(h.c), mp, _ptr(g)),
           "param_shift_grad")
    return g


def partial_work(n: int, n_gates: int, strings, coeffs, theta,
                 lib: Optional[ctypes.CDLL] = None) -> float:
    """Run a bounded slice of one evaluation (n_gates RY gates + len(strings) terms)."""
    lib = lib or load()
    h = _HamArgs(n, strings, coeffs)
    th = np.ascontiguousarray(theta, dtype=np.float64).reshape(-1)
    out = np.zeros(1)
    _check(lib.oracle_partial_work(n, n_gates, h.m, _ptr(h.buf), _ptr(h.c), _ptr(th), _ptr(out)),
           "partial_work")
    return float(out[0])


def sweep_times(n: int, n_gates: int, strings, coeffs, lib: Optional[ctypes.CDLL] = None):
    """Seconds per RY sweep and per Pauli-term sweep of the oracle on a 2^n state."""
    lib = lib or load()
    h = _HamArgs(n, strings, coeffs)
    tg = np.zeros(1)
    tt = np.zeros(1)
    _check(lib.oracle_sweep_times(n, n_gates, h.m, _ptr(h.buf), _ptr(h.c), _ptr(tg), _ptr(tt)), "sweep_times")
    return float(tg[0]), float(tt[0])
