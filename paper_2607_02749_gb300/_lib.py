"""ctypes binding of libgvqe.so: the C ABI of include/gvqe.h, one Python function per C call.

Argument marshalling only: every step of the computation runs in the CUDA
library.  Device buffers are passed as torch tensors (their data pointers);
the stream defaults to torch's current CUDA stream.  If the library is missing
and cannot be compiled, loading raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgvqe.so")
# GVQE_DEBUG=1 in the environment loads the debug build (guarded workspaces)
DEBUG = os.environ.get("GVQE_DEBUG", "0") not in ("", "0")

GVQE_OK = 0
GVQE_EINVAL = -1
GVQE_ENOMEM = -2
GVQE_ECUDA = -3
GVQE_ETIMEOUT = -4
GVQE_EUNSUPPORTED = -5
GVQE_ECORRUPT = -6
GVQE_FP32 = 0x0
GVQE_FP64 = 0x1
GVQE_GRAD_ADJOINT = 0x0
GVQE_GRAD_PARAM_SHIFT = 0x2
GVQE_ENT_LINEAR = 0
GVQE_ENT_CIRCULAR = 1
GVQE_ENT_FULL = 2
GVQE_ENT_REVERSE_LINEAR = 3
GVQE_ENT_PAIRWISE = 4
GVQE_ENT_SCA = 5
GVQE_OPT_TILE_BITS = 1
GVQE_OPT_GATES = 2
GVQE_OPT_SPLIT_PASSES = 3
GVQE_OPT_XY_TILE_BITS = 4
GVQE_OPT_MPS_LAYERS = 5
GVQE_OPT_MPS_TENSOR = 6
GVQE_GATES_RY = 1
GVQE_GATES_RY_RZ = 2
GVQE_MAX_QUBITS = 30
GVQE_STATIC_SCRATCH_BYTES = 16 * 1024 * 1024
GVQE_TUNE_ENERGY = 0x4
GVQE_BATCH_OPT_WAVE_BYTES = 1
GVQE_BATCH_OPT_TILE_BITS = 2
GVQE_BATCH_OPT_SCHEDULE = 3
GVQE_BATCH_PERSISTENT = 0
GVQE_BATCH_STAGED = 1
GVQE_PROF_FWD = 0
GVQE_PROF_BWD = 1
GVQE_PROF_GRAD_L0 = 2
GVQE_PROF_LAMBDA_XY = 3
GVQE_PROF_WHT = 4

_ERRNAMES = {
    GVQE_EINVAL: "GVQE_EINVAL",
    GVQE_ENOMEM: "GVQE_ENOMEM",
    GVQE_ECUDA: "GVQE_ECUDA",
    GVQE_ETIMEOUT: "GVQE_ETIMEOUT",
    GVQE_EUNSUPPORTED: "GVQE_EUNSUPPORTED",
    GVQE_ECORRUPT: "GVQE_ECORRUPT",
}


class GvqeError(RuntimeError):
    """A gvqe call returned a negative code; `.code` holds it."""

    def __init__(self, code: int, func: str, msg: str):
        super().__init__(f"{func} -> {_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib: Optional[ctypes.CDLL] = None

_VP = ctypes.c_void_p
_I = ctypes.c_int
_SIGS = {
    "gvqe_hamiltonian_create": [_I, _I, ctypes.c_char_p, _VP, ctypes.POINTER(_VP)],
    "gvqe_ansatz_create": [_I, _I, _I, ctypes.POINTER(_VP)],
    "gvqe_ansatz_set_option": [_VP, _I, _I],
    "gvqe_energy": [_VP, _VP, _VP, _I, _VP, _I, _VP],
    "gvqe_energy_grad": [_VP, _VP, _VP, _VP, _I, _VP, _VP, _I, _VP],
    "gvqe_batch_create": [_I, _VP, _VP, _I, ctypes.POINTER(_VP)],
    "gvqe_energy_static": [_VP, _VP, _VP, _I, _VP, _I, _VP],
    "gvqe_batch_run": [_VP, _VP, _VP, _VP, _VP, _VP],
    "gvqe_readout": [_VP, _VP, _VP, _I, ctypes.c_double, _I, _VP, _VP, _VP, _VP, _VP],
    "gvqe_destroy": [_VP],
    "gvqe_plan_describe": [_I, _I, _I, _I, ctypes.c_char_p, _I],
    "gvqe_ansatz_describe": [_VP, _I, ctypes.c_char_p, _I],
    "gvqe_entangler_inverse": [_I, _I, _I, _VP, _VP, ctypes.c_longlong],
    "gvqe_set_device_memory_limit": [ctypes.c_longlong],
    "gvqe_interaction_graph": [_I, _I, ctypes.c_char_p, _VP, _VP],
    "gvqe_partition": [_I, _VP, ctypes.c_double, _I, _VP, _VP, _VP],
    "gvqe_hamiltonian_stats": [_VP, _VP, _VP, _VP, _VP],
    "gvqe_version": [],
    "gvqe_profile_enable": [_I],
    "gvqe_profile_read": [_I, _VP, _VP, _VP],
    "gvqe_profile_reset": [],
    "gvqe_debug_check": [],
    "gvqe_debug_poke_guard": [_I],
    "gvqe_batch_set_option": [_VP, _I, ctypes.c_longlong],
    "gvqe_batch_autotune": [_VP, _VP, _VP, _VP, _VP, ctypes.c_char_p, _I, _VP],
    "gvqe_autotune": [_VP, _VP, _VP, _I, _I, ctypes.c_char_p, ctypes.c_char_p, _I, _VP],
    "gvqe_tune_key": [_VP, _VP, _I, _I, ctypes.c_char_p, _I],
    "gvqe_tune_cache_get": [ctypes.c_char_p, ctypes.c_char_p, _VP, _VP, _VP],
    "gvqe_tune_cache_put": [ctypes.c_char_p, ctypes.c_char_p, _I, _I, ctypes.c_double, ctypes.c_char_p],
}


def load(path: Optional[str] = None, build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libgvqe.so (compiling it with nvcc first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or (os.path.join(HERE, "libgvqe_debug.so") if DEBUG else LIB_PATH)
        if path is None and build_if_missing:
            from . import build as _build

            p = _build.build(debug=DEBUG)
        if not os.path.exists(p):
            raise RuntimeError(f"gvqe CUDA library not found at {p}; run paper_2607_02749_gb300.build.build()")
        lib = ctypes.CDLL(p)
        for name, argtypes in _SIGS.items():
            f = getattr(lib, name)
            f.argtypes = argtypes
            f.restype = _I
        lib.gvqe_launch_count.argtypes = []
        lib.gvqe_launch_count.restype = ctypes.c_int64
        lib.gvqe_last_error.argtypes = []
        lib.gvqe_last_error.restype = ctypes.c_char_p
        if path is None:
            _lib = lib
        return lib


def _check(rc: int, func: str) -> int:
    if rc < 0:
        msg = load().gvqe_last_error().decode(errors="replace")
        raise GvqeError(rc, func, msg)
    return rc


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch

        if not torch.cuda.is_available():
            return None
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _require_cuda(*tensors) -> None:
    for t in tensors:
        if t is not None and not isinstance(t, int) and not t.is_cuda:
            raise ValueError("gvqe calls take CUDA tensors (device pointers)")


# ------------------------------------------------------------- C calls --

def gvqe_version() -> int:
    return load().gvqe_version()


def gvqe_last_error() -> str:
    return load().gvqe_last_error().decode(errors="replace")


def gvqe_hamiltonian_create(n_qubits: int, strings: Sequence[str], coeffs) -> int:
    """H = sum_k c_k P_k (Eq. 6).  Returns the handle as an int."""
    import numpy as np

    strings = list(strings)
    c = np.ascontiguousarray(coeffs, dtype=np.float64).reshape(-1)
    if len(strings) != c.size:
        raise ValueError("len(strings) != len(coeffs)")
    flat = "".join(strings).encode("ascii")
    out = _VP()
    _check(load().gvqe_hamiltonian_create(n_qubits, len(strings), flat, c.ctypes.data if c.size else None,
                                          ctypes.byref(out)), "gvqe_hamiltonian_create")
    return out.value


def gvqe_ansatz_create(n_qubits: int, reps: int, entangler: int = GVQE_ENT_LINEAR) -> int:
    out = _VP()
    _check(load().gvqe_ansatz_create(n_qubits, reps, entangler, ctypes.byref(out)), "gvqe_ansatz_create")
    return out.value


def gvqe_ansatz_set_option(ansatz: int, option: int, value: int) -> None:
    _check(load().gvqe_ansatz_set_option(ansatz, option, value), "gvqe_ansatz_set_option")


def gvqe_energy(ansatz: int, ham: int, params, energies, flags: int = GVQE_FP32, stream=None) -> None:
    """energies[b] = <psi(params[b])|H|psi(params[b])> (Eq. 4); CUDA float64 tensors."""
    _require_cuda(params, energies)
    batch = params.shape[0] if params.dim() == 2 else 1
    _check(load().gvqe_energy(ansatz, ham, _ptr(params), batch, _ptr(energies), flags, _stream(stream)),
           "gvqe_energy")


def gvqe_energy_grad(ansatz: int, ham: int, params, mask, energies, grad, flags: int = GVQE_FP32,
                     stream=None) -> None:
    """Energies and dE/dtheta; mask (uint8, same shape as params) or None = all active."""
    _require_cuda(params, mask, energies, grad)
    batch = params.shape[0] if params.dim() == 2 else 1
    _check(load().gvqe_energy_grad(ansatz, ham, _ptr(params), _ptr(mask), batch, _ptr(energies), _ptr(grad),
                                   flags, _stream(stream)), "gvqe_energy_grad")


def gvqe_energy_static(ansatz: int, ham: int, params, energies, flags: int = GVQE_FP32, stream=None) -> None:
    """Energies as gvqe_energy, with no device allocation at all.

    For callers that cannot allocate device memory when they need an energy
    (inside a stream capture, under an allocator or memory budget they do not
    control): every scratch buffer comes from one fixed device array of
    GVQE_STATIC_SCRATCH_BYTES inside the library, so only small registers fit
    (about n <= 19 at batch 1) and the Hamiltonian must be diagonal.  The first
    call on a device looks the array up; calls that overlap on the GPU race on it.
    """
    _require_cuda(params, energies)
    batch = params.shape[0] if params.dim() == 2 else 1
    _check(load().gvqe_energy_static(ansatz, ham, _ptr(params), batch, _ptr(energies), flags, _stream(stream)),
           "gvqe_energy_static")


def gvqe_readout(ansatz: int, ham: Optional[int], params, alpha: float, uniforms, shots, stats, argmax,
                 flags: int = GVQE_FP32, stream=None) -> None:
    """Readout of |psi(params)>: most probable x, shots by inverse CDF, CVaR-alpha (alpha 0 skips it).

    stats (4 doubles) <- p(argmax), CVaR, total probability, CVaR histogram passes; argmax (1 int64);
    shots (int64, one per uniform).  Synchronises the stream.
    """
    _require_cuda(params, uniforms, shots, stats, argmax)
    n_shots = 0 if uniforms is None else int(uniforms.numel())
    _check(load().gvqe_readout(ansatz, ham, _ptr(params), flags, float(alpha), n_shots, _ptr(uniforms),
                               _ptr(shots), _ptr(stats), _ptr(argmax), _stream(stream)), "gvqe_readout")


def gvqe_batch_create(ansatze: Sequence[int], hams: Sequence[int], flags: int = GVQE_FP32) -> int:
    n = len(ansatze)
    a = (_VP * n)(*ansatze)
    h = (_VP * n)(*hams)
    out = _VP()
    _check(load().gvqe_batch_create(n, a, h, flags, ctypes.byref(out)), "gvqe_batch_create")
    return out.value


def gvqe_batch_run(batch: int, params: Sequence, masks: Optional[Sequence], energies, grads: Optional[Sequence],
                   stream=None) -> None:
    n = len(params)
    pa = (_VP * n)(*[_ptr(p) for p in params])
    ma = (_VP * n)(*[_ptr(m) for m in masks]) if masks is not None else None
    ga = (_VP * n)(*[_ptr(g) for g in grads]) if grads is not None else None
    _check(load().gvqe_batch_run(batch, pa, ma, _ptr(energies), ga, _stream(stream)), "gvqe_batch_run")


def gvqe_batch_set_option(batch: int, option: int, value: int) -> None:
    _check(load().gvqe_batch_set_option(batch, option, int(value)), "gvqe_batch_set_option")


def gvqe_batch_autotune(batch: int, params: Sequence, masks: Optional[Sequence], energies,
                        grads: Optional[Sequence], stream=None) -> str:
    """Time the batch under each wave budget and keep the fastest; returns the report."""
    n = len(params)
    pa = (_VP * n)(*[_ptr(p) for p in params])
    ma = (_VP * n)(*[_ptr(m) for m in masks]) if masks is not None else None
    ga = (_VP * n)(*[_ptr(g) for g in grads]) if grads is not None else None
    buf = ctypes.create_string_buffer(1 << 12)
    _check(load().gvqe_batch_autotune(batch, pa, ma, _ptr(energies), ga, buf, len(buf), _stream(stream)),
           "gvqe_batch_autotune")
    return buf.value.decode()


def gvqe_destroy(handle: Optional[int]) -> None:
    _check(load().gvqe_destroy(handle), "gvqe_destroy")


def gvqe_plan_describe(n_qubits: int, reps: int, flags: int = GVQE_FP32, tile_bits: int = 0) -> str:
    buf = ctypes.create_string_buffer(1 << 16)
    _check(load().gvqe_plan_describe(n_qubits, reps, flags, tile_bits, buf, len(buf)), "gvqe_plan_describe")
    return buf.value.decode()


def gvqe_debug_check() -> None:
    """Debug build: raise GvqeError (GVQE_ECORRUPT) if a device write landed in a
    workspace guard; regular builds raise GVQE_EUNSUPPORTED."""
    _check(load().gvqe_debug_check(), "gvqe_debug_check")


def gvqe_debug_poke_guard(restore: bool = False) -> None:
    """Debug build, tests only: overwrite (or restore) the first guard byte above the largest workspace."""
    _check(load().gvqe_debug_poke_guard(1 if restore else 0), "gvqe_debug_poke_guard")


def gvqe_autotune(ansatz: int, ham: int, params, flags: int = GVQE_FP32, cache_path: Optional[str] = None,
                  stream=None) -> str:
    """Pick the ansatz's tile plan by timing every distinct candidate on `params`
    (CUDA float64 [B, P]); returns the report (choice and sweep)."""
    _require_cuda(params)
    batch = params.shape[0] if params.dim() > 1 else 1
    buf = ctypes.create_string_buffer(1 << 14)
    path = cache_path.encode() if cache_path else None
    _check(load().gvqe_autotune(ansatz, ham, _ptr(params), batch, flags, path, buf, len(buf), _stream(stream)),
           "gvqe_autotune")
    return buf.value.decode()


def gvqe_tune_key(ansatz: int, ham: int, batch: int, flags: int = GVQE_FP32) -> str:
    buf = ctypes.create_string_buffer(1024)
    _check(load().gvqe_tune_key(ansatz, ham, batch, flags, buf, len(buf)), "gvqe_tune_key")
    return buf.value.decode()


def gvqe_tune_cache_get(path: str, key: str):
    """(tile_bits, split, ms) of the cached entry for key, or None (host only)."""
    tb, sp, ms = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0.0)
    rc = _check(load().gvqe_tune_cache_get(path.encode(), key.encode(), ctypes.byref(tb), ctypes.byref(sp),
                                           ctypes.byref(ms)), "gvqe_tune_cache_get")
    return (tb.value, sp.value, ms.value) if rc == 1 else None


def gvqe_tune_cache_put(path: str, key: str, tile_bits: int, split: int, ms: float = 0.0, sweep: str = "") -> None:
    _check(load().gvqe_tune_cache_put(path.encode(), key.encode(), tile_bits, split, ms, sweep.encode()),
           "gvqe_tune_cache_put")


def gvqe_ansatz_describe(a: int, flags: int = GVQE_FP32) -> str:
    buf = ctypes.create_string_buffer(1 << 16)
    _check(load().gvqe_ansatz_describe(a, flags, buf, len(buf)), "gvqe_ansatz_describe")
    return buf.value.decode()


def gvqe_entangler_inverse(entangler: int, n_qubits: int, layer: int, y) -> "np.ndarray":
    """x = A^-1 y for the entangler of layer `layer` (host only, no GPU)."""
    import numpy as np

    ya = np.ascontiguousarray(np.asarray(y, dtype=np.int64).reshape(-1))
    xa = np.empty_like(ya)
    _check(load().gvqe_entangler_inverse(entangler, n_qubits, layer, ya.ctypes.data, xa.ctypes.data, ya.size),
           "gvqe_entangler_inverse")
    return xa


def gvqe_set_device_memory_limit(limit_bytes: int) -> None:
    """Budget for the library's device workspaces (0 = none); over it calls fail with GVQE_ENOMEM."""
    _check(load().gvqe_set_device_memory_limit(int(limit_bytes)), "gvqe_set_device_memory_limit")


def gvqe_device_memory_in_use() -> int:
    lib = load()
    lib.gvqe_device_memory_in_use.restype = ctypes.c_longlong
    lib.gvqe_device_memory_in_use.argtypes = []
    return int(lib.gvqe_device_memory_in_use())


def gvqe_interaction_graph(n_qubits: int, strings, coeffs) -> "np.ndarray":
    """Eq. 9 weighted interaction graph (host only, no GPU): n x n, symmetric."""
    import numpy as np

    strings = list(strings)
    for s in strings:
        if len(s) != n_qubits:
            raise GvqeError(GVQE_EINVAL, "gvqe_interaction_graph", f"string {s!r} does not have {n_qubits} letters")
    flat = "".join(strings).encode("ascii")
    c = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64).reshape(-1))
    if c.size != len(strings):
        raise GvqeError(GVQE_EINVAL, "gvqe_interaction_graph", "one coefficient per string")
    w = np.zeros((n_qubits, n_qubits))
    _check(load().gvqe_interaction_graph(n_qubits, len(strings), flat, c.ctypes.data, w.ctypes.data),
           "gvqe_interaction_graph")
    return w


def gvqe_partition(w, resolution: float = 1.0, min_block: int = 1):
    """Louvain blocks of the graph w (Section IV-C, Eq. 10): (block_of, n_blocks, Q)."""
    import numpy as np

    wa = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
    n = wa.shape[0]
    if wa.shape != (n, n):
        raise GvqeError(GVQE_EINVAL, "gvqe_partition", "w must be square")
    lab = np.zeros(n, dtype=np.int32)
    nb = ctypes.c_int()
    q = ctypes.c_double()
    _check(load().gvqe_partition(n, wa.ctypes.data, float(resolution), int(min_block), lab.ctypes.data,
                                 ctypes.byref(nb), ctypes.byref(q)), "gvqe_partition")
    return [int(v) for v in lab], nb.value, q.value


def gvqe_hamiltonian_stats(ham: int) -> dict:
    vals = [ctypes.c_int() for _ in range(4)]
    _check(load().gvqe_hamiltonian_stats(ham, *[ctypes.byref(v) for v in vals]), "gvqe_hamiltonian_stats")
    return dict(zip(("diag", "groups", "grouped", "dropped_odd_y"), (v.value for v in vals)))


def gvqe_launch_count() -> int:
    """Kernels this library has enqueued in this process so far."""
    return int(load().gvqe_launch_count())


def gvqe_profile_enable(on: bool) -> None:
    _check(load().gvqe_profile_enable(1 if on else 0), "gvqe_profile_enable")


def gvqe_profile_read(kind: int) -> dict:
    """{launches, ms, bytes} summed over recorded launches of one kernel kind (GVQE_PROF_*)."""
    n = ctypes.c_int64()
    ms = ctypes.c_double()
    by = ctypes.c_double()
    _check(load().gvqe_profile_read(kind, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by)),
           "gvqe_profile_read")
    return {"launches": n.value, "ms": ms.value, "bytes": by.value}


def gvqe_profile_reset() -> None:
    _check(load().gvqe_profile_reset(), "gvqe_profile_reset")
