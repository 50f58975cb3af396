"""C-ABI checks that need no GPU: the library loads, exports every symbol that
include/gvqe.h declares, validates arguments on the host, and plans passes."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2607_02749_gb300 import _lib
from paper_2607_02749_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gvqe.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gvqe_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    names = _declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), f"{name} declared in gvqe.h but not exported"


def test_every_declared_symbol_has_a_python_binding():
    for name in _declared_functions():
        assert hasattr(_lib, name), f"no Python binding named {name}"


def test_version_and_empty_error():
    assert _lib.gvqe_version() >= 100
    assert isinstance(_lib.gvqe_last_error(), str)


def test_hamiltonian_parsing_and_stats():
    n = 6
    strings = ["ZZIIII", "ZZIIII", "IIIIII", "XIXIII", "YYIIII", "YIIIII", "IXZYII", "XIXZII"]
    coeffs = [1.0, 2.0, 0.5, 1.5, -1.0, 3.0, 0.7, 0.2]
    h = _lib.gvqe_hamiltonian_create(n, strings, coeffs)
    try:
        st = _lib.gvqe_hamiltonian_stats(h)
        # diagonal: ZZ (merged) and the identity; X groups: mask 0b101 (XIX, XIXZ) and 0b11 (YY);
        # odd-Y strings YIIIII and IXZYII are dropped
        assert st == {"diag": 2, "groups": 2, "grouped": 3, "dropped_odd_y": 2}
    finally:
        _lib.gvqe_destroy(h)


@pytest.mark.parametrize("bad", ["ZZA", "zzI", "Z Z"])
def test_bad_letters_rejected(bad):
    with pytest.raises(_lib.GvqeError) as e:
        _lib.gvqe_hamiltonian_create(3, [bad], [1.0])
    assert e.value.code == _lib.GVQE_EINVAL
    assert "letter" in str(e.value)


def test_size_checks():
    for n in (0, 31, -1):
        with pytest.raises(_lib.GvqeError) as e:
            _lib.gvqe_hamiltonian_create(n, [], [])
        assert e.value.code == _lib.GVQE_EINVAL
        with pytest.raises(_lib.GvqeError):
            _lib.gvqe_ansatz_create(n, 1)
    with pytest.raises(_lib.GvqeError):
        _lib.gvqe_ansatz_create(4, -1)
    with pytest.raises(_lib.GvqeError) as e:
        _lib.gvqe_ansatz_create(4, 1, entangler=7)
    assert e.value.code == _lib.GVQE_EINVAL
    for ent in ALL_ENTS:
        _lib.gvqe_destroy(_lib.gvqe_ansatz_create(4, 1, entangler=ent))
    with pytest.raises(_lib.GvqeError):
        _lib.gvqe_hamiltonian_create(3, ["ZZ"], [1.0])  # string shorter than n is caught by length


def test_destroy_null_and_bad_handle():
    _lib.gvqe_destroy(None)
    junk = ctypes.create_string_buffer(64)
    with pytest.raises(_lib.GvqeError):
        _lib.gvqe_destroy(ctypes.addressof(junk))


def test_tile_bits_option_validation():
    a = _lib.gvqe_ansatz_create(12, 2)
    try:
        _lib.gvqe_ansatz_set_option(a, _lib.GVQE_OPT_TILE_BITS, 12)
        _lib.gvqe_ansatz_set_option(a, _lib.GVQE_OPT_TILE_BITS, 0)
        with pytest.raises(_lib.GvqeError):
            _lib.gvqe_ansatz_set_option(a, _lib.GVQE_OPT_TILE_BITS, 9)
        with pytest.raises(_lib.GvqeError):
            _lib.gvqe_ansatz_set_option(a, 99, 1)
    finally:
        _lib.gvqe_destroy(a)


def _layer_passes(text):
    """(tile bits, carry, high start, [qubits of the pass's gates]) per layer pass."""
    out = []
    for m in re.finditer(r"layer pass \d+: tile_bits=(\d+) carry=(\d+) high_start=(\d+) qubits=(\S+)", text):
        qs = []
        for lo, hi in re.findall(r"\[(-?\d+),(-?\d+)\]", m.group(4)):
            qs.extend(range(int(lo), int(hi) + 1))
        out.append((int(m.group(1)), int(m.group(2)), int(m.group(3)), qs))
    return out


@pytest.mark.parametrize("n,flags,tb,expect", [
    (30, 0, 0, 3), (30, 1, 0, 3), (24, 0, 0, 3), (24, 0, 12, 3), (28, 0, 0, 3), (13, 0, 0, 1), (14, 0, 0, 2), (12, 1, 0, 1),
    (20, 0, 10, 3), (16, 0, 10, 2), (9, 0, 0, 1), (1, 0, 0, 1),
])
def test_plan_covers_every_qubit_once(n, flags, tb, expect):
    text = _lib.gvqe_plan_describe(n, 2, flags, tb)
    passes = _layer_passes(text)
    assert len(passes) == expect
    covered = []
    for tbits, carry, start, qs in passes:
        covered.extend(qs)
        assert carry >= min(3 if flags else 4, tbits) or carry == tbits
    assert sorted(covered) == list(range(n))


def test_plan_step_sequence_for_gradient():
    text = _lib.gvqe_plan_describe(20, 3, 0, 10)
    kinds = re.findall(r"^\s+(fwd|bwd|grad_l0|lambda_xy)\s", text, flags=re.M)
    p = 3
    assert kinds.count("fwd") == 3 * p
    assert kinds.count("bwd") == 3 * p
    assert kinds[-1] == "grad_l0"
    assert kinds.index("bwd") == 3 * p  # backward starts after the forward


def test_workload_generators_shapes():
    ham = wl.z_hamiltonian(12, 200, seed=0)
    assert ham.n_terms == 200 and all(len(s) == 12 for s in ham.strings)
    assert all(set(s) <= {"I", "Z"} for s in ham.strings)
    assert (ham.coeffs[:150] < 0).all() and (ham.coeffs[150:] == 10.0).all()
    w = [sum(ch != "I" for ch in s) for s in ham.strings]
    assert min(w) >= 1 and max(w) <= 4
    ph = wl.pauli_hamiltonian(28, 5000, seed=0)
    xy = sum(any(ch in "XY" for ch in s) for s in ph.strings)
    assert 0.35 < xy / 5000 < 0.45
    th = wl.thetas(30, 6, 4)
    assert th.shape == (4, 210) and abs(th).max() <= 3.1416
    batch = wl.cluster_batch(8)
    for inst in batch:
        assert 14 <= inst.n_qubits <= 20 and 2 <= inst.reps <= 4
        frac = inst.mask.mean()
        assert 0.25 <= frac <= 0.65


ALL_ENTS = (_lib.GVQE_ENT_LINEAR, _lib.GVQE_ENT_CIRCULAR, _lib.GVQE_ENT_FULL, _lib.GVQE_ENT_REVERSE_LINEAR,
            _lib.GVQE_ENT_PAIRWISE, _lib.GVQE_ENT_SCA)


def test_every_entangler_creates_at_every_size():
    # creation checks that the layer-1 gather of every tile size splits its product-state tables
    for ent in ALL_ENTS:
        for n in range(1, _lib.GVQE_MAX_QUBITS + 1):
            _lib.gvqe_destroy(_lib.gvqe_ansatz_create(n, 3, entangler=ent))


def test_entangler_inverse_matches_the_oracle_maps():
    """The library's closed forms of A^-1 (the ones its gathers and scatters use)
    invert the oracle's closed-form entangler maps, for every layer offset."""
    from oracle import closed_form

    rng = np.random.default_rng(3)
    for ent in ALL_ENTS:
        for n in (1, 2, 3, 5, 8, 13, 14, 21, 30):
            for layer in (1, 2, 3, 4, n + 1, n + 2):
                xs = rng.integers(0, 1 << n, size=64) if n > 6 else np.arange(1 << n)
                ys = np.array([closed_form.entangler_map(int(x), n, ent, layer) for x in xs])
                got = _lib.gvqe_entangler_inverse(ent, n, layer, ys)
                assert np.array_equal(got, xs), (ent, n, layer)


def test_entangler_inverse_rejects_bad_arguments():
    for args in ((6, 4, 1, [0]), (0, 0, 1, [0]), (0, 4, 0, [0]), (0, 4, 1, [16]), (0, 4, 1, [-1])):
        with pytest.raises(_lib.GvqeError) as e:
            _lib.gvqe_entangler_inverse(*args)
        assert e.value.code == _lib.GVQE_EINVAL


def test_gate_set_option():
    a = _lib.gvqe_ansatz_create(10, 2)
    _lib.gvqe_ansatz_set_option(a, _lib.GVQE_OPT_GATES, _lib.GVQE_GATES_RY_RZ)
    _lib.gvqe_ansatz_set_option(a, _lib.GVQE_OPT_GATES, _lib.GVQE_GATES_RY)
    with pytest.raises(_lib.GvqeError) as e:
        _lib.gvqe_ansatz_set_option(a, _lib.GVQE_OPT_GATES, 3)
    assert e.value.code == _lib.GVQE_EINVAL
    _lib.gvqe_destroy(a)


def test_device_memory_limit_setter():
    _lib.gvqe_set_device_memory_limit(1 << 30)
    _lib.gvqe_set_device_memory_limit(0)
    assert _lib.gvqe_device_memory_in_use() >= 0
    with pytest.raises(_lib.GvqeError) as e:
        _lib.gvqe_set_device_memory_limit(-1)
    assert e.value.code == _lib.GVQE_EINVAL


def test_split_layout_option_and_plans():
    """GVQE_OPT_SPLIT_PASSES: auto splits only where the top strided pass would
    span more than 2^8 large pages (n = 30 RY+RZ in FP32, n = 30 RY in FP64), never
    keeps one run per pass, always splits any layer with two strided passes; the
    split qubit runs still cover every qubit once."""
    import re

    import paper_2607_02749_gb300 as gv

    def runs(a, fp64=False):
        d = a.describe(fp64=fp64)
        out = []
        for m in re.finditer(r"carry=(\d+) high_start=(\d+) qubits=\S+ split=(\d+),(\d+)", d):
            out.append(tuple(map(int, m.groups())))
        return d, out

    _, r = runs(gv.Ansatz(30, 6))
    assert all(k1 == 0 and gap == 0 for _, _, k1, gap in r)  # FP32 RY: top pass spans 2^8 pages
    _, r = runs(gv.Ansatz(30, 6), fp64=True)
    assert r[1][2:] == (5, 9) and r[2][1] == 17  # [12,17) + [26,30), then [17,26)
    _, r = runs(gv.Ansatz(30, 6, gates=gv.GVQE_GATES_RY_RZ))
    assert r[1][2:] == (5, 9) and r[2][1] == 18  # [13,18) + [27,31), then [18,27)
    _, r = runs(gv.Ansatz(30, 6, gates=gv.GVQE_GATES_RY_RZ, split=1))
    assert all(k1 == 0 and gap == 0 for _, _, k1, gap in r)
    d, r = runs(gv.Ansatz(17, 2, tile_bits=10, split=2))
    assert r[1][2] > 0
    # every qubit is a gate bit of exactly one pass of the layer
    c1, a1, k1, gap = r[1]
    first = list(range(a1, a1 + k1)) + list(range(a1 + k1 + gap, a1 + gap + 10 - c1))
    c2, a2, _, _ = r[2]
    second = list(range(a2, a2 + 10 - c2))
    assert sorted(list(range(10)) + first + second) == list(range(17))
    assert [p[3] for p in _layer_passes(d)] == [list(range(10)), first, second]
    a = gv.Ansatz(12, 1)
    for bad in (-1, 33):
        with pytest.raises(gv.GvqeError) as e:
            gv.gvqe_ansatz_set_option(a.handle, gv.GVQE_OPT_SPLIT_PASSES, bad)
        assert e.value.code == gv._lib.GVQE_EINVAL
    # 2 + y: the first strided pass takes y top qubits (capped below its gate count)
    for y in (1, 3, 6):
        _, r = runs(gv.Ansatz(30, 6, split=2 + y))
        c1, a1, k1, gap = r[1]
        g1 = 13 - c1
        ye = min(y, g1 - 1)
        assert k1 == g1 - ye and a1 + k1 + gap == 30 - ye  # low run [13, 13 + k1), top run [30 - y, 30)


def test_debug_entry_points_refuse_in_the_regular_build():
    if _lib.DEBUG:
        pytest.skip("the debug library is loaded")
    for f in (_lib.gvqe_debug_check, _lib.gvqe_debug_poke_guard):
        with pytest.raises(_lib.GvqeError) as e:
            f()
        assert e.value.code == _lib.GVQE_EUNSUPPORTED


@pytest.mark.parametrize("gates", [1, 2])
@pytest.mark.parametrize("fp64", [False, True])
def test_split_rule_over_register_sizes(gates, fp64):
    """For every size with two strided passes per layer: auto mode splits exactly
    when the top pass would span more than 2^8 large pages (gate index bits whose
    stride is at least 2 MiB), and then moves the fewest top qubits that leave the
    other pass at 2^8; every index bit of the layer is covered once."""
    import re

    import paper_2607_02749_gb300 as gv

    pb = 18 if fp64 else 19  # index bits with a stride of at least 2 MiB
    seen_split = False
    for n in range(14, 31):
        a = gv.Ansatz(n, 1, gates=gates)
        d = a.describe(fp64=fp64)
        nb = int(re.search(r"n=(\d+)", d).group(1))
        passes = _layer_passes(d)
        runs = [tuple(map(int, m)) for m in re.findall(r"split=(\d+),(\d+)", d)]
        covered = sorted(q for p in passes for q in p[3])
        first = 1 if gates == 2 else 0  # index bit 0 is the channel on the complex path
        assert covered == list(range(first, nb)), (n, d)
        if len(passes) != 3:
            assert all(r == (0, 0) for r in runs)
            continue
        tb = passes[0][0]
        ga = tb - passes[1][1]
        top_unsplit = max(0, nb - max(tb + ga, pb))
        split = runs[1][0] > 0
        assert split == (top_unsplit > 8), (n, fp64, gates, d)
        pages_second = sum(1 for q in passes[2][3] if q >= pb)
        if split:
            seen_split = True
            assert pages_second <= 8
            y = ga - runs[1][0]
            # one fewer top qubit would leave the second pass above 2^8 pages
            lo, hi = tb + ga - (y - 1), nb - (y - 1)
            assert y == 1 or max(0, hi - max(lo, pb)) > 8
    assert seen_split == (gates == 2 or fp64)


def test_closed_form_layer_option_and_plans():
    """GVQE_OPT_MPS_LAYERS: FP32 plans with n >= 14, reps >= 2 and a linear,
    full or reverse-linear entangler write layers 1..min(4, reps - 1) in closed
    form (one table build and one write per stored state); everything else keeps
    every layer as tile passes."""
    def desc(n, reps, ent=_lib.GVQE_ENT_LINEAR, mps=None, flags=_lib.GVQE_FP32):
        a = _lib.gvqe_ansatz_create(n, reps, ent)
        try:
            if mps is not None:
                _lib.gvqe_ansatz_set_option(a, _lib.GVQE_OPT_MPS_LAYERS, mps)
            return _lib.gvqe_ansatz_describe(a, flags)
        finally:
            _lib.gvqe_destroy(a)

    def steps_of(d):
        return [ln.split()[0] for ln in d.splitlines()[1:] if ln.startswith("  ")
                and not ln.startswith("  layer pass") and not ln.startswith("  closed-form")]

    d = desc(30, 6)
    assert ("closed-form layers 1..4 (bond dimension up to 16), 245760 table floats per job; their gradients "
            "from lambda and the matrix product (tensor cores, TF32 split)") in d
    # layer 4's final state in closed form, layers 5..6 as tile passes and their backward, then the
    # gradients of layers 0..4 from lambda_4 (no backward passes and no layer-0 pass below layer 5)
    assert steps_of(d) == (["mps_tab", "mps"] + ["fwd"] * 6 + ["bwd"] * 6
                           + ["mps_grad", "mps_ghigh", "mps_gred", "mps_genv"])
    d3 = desc(30, 6, mps=3)
    assert ("closed-form layers 1..3 (bond dimension up to 8), 59136 table floats per job; their gradients "
            "from lambda and the matrix product\n") in d3  # bond 8: FP32 pipe
    # GVQE_OPT_MPS_TENSOR: -1 keeps the bond-16 gradient pass on the FP32 pipe; same steps
    a = _lib.gvqe_ansatz_create(30, 6)
    try:
        _lib.gvqe_ansatz_set_option(a, _lib.GVQE_OPT_MPS_TENSOR, -1)
        d_fp32 = _lib.gvqe_ansatz_describe(a, _lib.GVQE_FP32)
        assert "matrix product\n" in d_fp32 and "tensor cores" not in d_fp32
        assert steps_of(d_fp32) == steps_of(d)
        _lib.gvqe_ansatz_set_option(a, _lib.GVQE_OPT_MPS_TENSOR, 0)
        assert "(tensor cores, TF32 split)" in _lib.gvqe_ansatz_describe(a, _lib.GVQE_FP32)
        for bad in (-2, 1):
            with pytest.raises(_lib.GvqeError):
                _lib.gvqe_ansatz_set_option(a, _lib.GVQE_OPT_MPS_TENSOR, bad)
    finally:
        _lib.gvqe_destroy(a)
    assert steps_of(d3).count("fwd") == 9 and steps_of(d3).count("bwd") == 9
    for ent in (_lib.GVQE_ENT_FULL, _lib.GVQE_ENT_REVERSE_LINEAR):
        assert "closed-form layers 1..4 " in desc(20, 5, ent)
        assert "closed-form layers 1..2 " in desc(20, 3, ent)
    assert "closed-form layers 1..1 " in desc(14, 2)
    assert "closed-form layers 1..2 " in desc(14, 6, mps=2)
    for args in [dict(n=13, reps=4), dict(n=20, reps=1), dict(n=20, reps=4, mps=-1),
                 dict(n=20, reps=4, flags=_lib.GVQE_FP64), dict(n=20, reps=4, ent=_lib.GVQE_ENT_CIRCULAR),
                 dict(n=20, reps=4, ent=_lib.GVQE_ENT_PAIRWISE), dict(n=20, reps=4, ent=_lib.GVQE_ENT_SCA)]:
        assert "closed-form" not in desc(**args), args
    a = _lib.gvqe_ansatz_create(16, 3)
    try:
        for v in (-1, 0, 1, 2, 3, 4):
            _lib.gvqe_ansatz_set_option(a, _lib.GVQE_OPT_MPS_LAYERS, v)
        for v in (-2, 5):
            with pytest.raises(_lib.GvqeError):
                _lib.gvqe_ansatz_set_option(a, _lib.GVQE_OPT_MPS_LAYERS, v)
    finally:
        _lib.gvqe_destroy(a)
