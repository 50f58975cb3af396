"""Parity of gvqe_readout (most probable bitstring, inverse-CDF shots, CVaR-alpha)
with the readout oracle on the oracle's state, through the C ABI."""
import math

import numpy as np
import pytest

import oracle
from oracle import readout as ro
from paper_2607_02749_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2607_02749_gb300 as gv  # noqa: E402


def _tol(fp64):
    return 1e-12 if fp64 else 2e-6


def _check_against_oracle(n, reps, th, ham, fp64, alphas=(0.05, 0.2, 0.5, 1.0), shots=4096, seed=0):
    a = gv.Ansatz(n, reps)
    h = gv.Hamiltonian.from_workload(ham)
    tht = torch.as_tensor(th, dtype=torch.float64, device="cuda")
    p = ro.probabilities(oracle.state(n, reps, th))
    e = ro.diagonal_energies(n, ham.strings, ham.coeffs)
    tol = _tol(fp64)
    scale = ham.abs_sum()
    u = np.random.Generator(np.random.PCG64(seed)).random(shots)
    for k, alpha in enumerate(alphas):
        r = gv.readout(a, h, tht, alpha=alpha, uniforms=torch.as_tensor(u, device="cuda"), fp64=fp64)
        # total probability and the most probable bitstring
        assert abs(r.total - p.sum()) <= 4 * tol
        xo, po = ro.most_probable(p)
        assert abs(r.p_max - po) <= 4 * tol * max(po, 1.0)
        assert p[r.argmax] >= po - 4 * tol
        second = np.partition(p, -2)[-2] if p.size > 1 else -1.0
        if po - second > 8 * tol:
            assert r.argmax == xo
        # CVaR of the diagonal energy
        want = ro.cvar(p, e, alpha)
        assert abs(r.cvar - want) <= (1e-10 if fp64 else 2e-5) * scale, (alpha, r.cvar, want)
        if k == 0:
            # shots: each lands where the oracle's cumulative probability crosses u*T
            s = r.shots.cpu().numpy()
            so = ro.sample(p, u)
            cdf = np.cumsum(p)
            t = u * cdf[-1]
            lo = np.where(s > 0, cdf[np.maximum(s - 1, 0)], 0.0)
            hi = cdf[s]
            slack = 4 * tol * max(1.0, cdf[-1])
            assert np.all(p[s] > 0)
            assert np.all(lo <= t + slack) and np.all(t < hi + slack)
            # and equals the oracle's shot wherever t is not within the slack of a boundary
            d_lo = np.abs(t - np.where(so > 0, cdf[np.maximum(so - 1, 0)], 0.0))
            d_hi = np.abs(cdf[so] - t)
            clear = (d_lo > slack) & (d_hi > slack)
            assert np.array_equal(s[clear], so[clear])
    a.close()
    h.close()


@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("n,reps", [(4, 2), (9, 1), (12, 2), (14, 2), (16, 1)])
def test_readout_matches_oracle_z(n, reps, fp64):
    ham = wl.z_hamiltonian(n, 40 * n, seed=n)
    th = wl.thetas(n, reps, 1, seed=n + reps)[0]
    _check_against_oracle(n, reps, th, ham, fp64)


@pytest.mark.parametrize("fp64", [False, True])
def test_readout_matches_oracle_pauli_and_product_state(fp64):
    ham = wl.pauli_hamiltonian(12, 300, seed=5)
    _check_against_oracle(12, 2, wl.thetas(12, 2, 1, seed=6)[0], ham, fp64)
    ham = wl.z_hamiltonian(13, 200, seed=2)
    _check_against_oracle(13, 0, wl.thetas(13, 0, 1, seed=3)[0], ham, fp64, alphas=(0.2,))


@pytest.mark.parametrize("fp64", [False, True])
def test_basis_state_readout(fp64):
    # theta in {0, pi}: a signed basis state |y>; every shot is y, p(y) = 1, CVaR = E(y) for every alpha
    n, reps = 11, 2
    rng = np.random.default_rng(7)
    flips = rng.integers(0, 2, size=n * (reps + 1))
    th = np.where(flips == 1, math.pi, 0.0)
    psi = oracle.state(n, reps, th)
    y = int(np.argmax(np.abs(psi)))
    ham = wl.z_hamiltonian(n, 100, seed=4)
    e = ro.diagonal_energies(n, ham.strings, ham.coeffs)
    a, h = gv.Ansatz(n, reps), gv.Hamiltonian.from_workload(ham)
    tht = torch.as_tensor(th, dtype=torch.float64, device="cuda")
    for alpha in (1e-9, 0.3, 1.0):
        r = gv.readout(a, h, tht, alpha=alpha, shots=512, seed=1, fp64=fp64)
        assert r.argmax == y
        assert abs(r.p_max - 1.0) <= 1e-6
        assert set(r.shots.cpu().tolist()) == {y}
        assert abs(r.cvar - e[y]) <= 1e-9 * ham.abs_sum()


def test_readout_alpha_zero_and_no_shots():
    n, reps = 10, 1
    a = gv.Ansatz(n, reps)
    tht = torch.as_tensor(wl.thetas(n, reps, 1, seed=1)[0], device="cuda")
    r = gv.readout(a, None, tht, alpha=0.0, shots=0)
    assert math.isnan(r.cvar)
    assert r.shots.numel() == 0
    p = ro.probabilities(oracle.state(n, reps, tht.cpu().numpy()))
    assert r.argmax == ro.most_probable(p)[0]


def test_readout_rejects_bad_arguments():
    n = 10
    a = gv.Ansatz(n, 1)
    tht = torch.zeros(a.n_params, dtype=torch.float64, device="cuda")
    with pytest.raises(gv.GvqeError):
        gv.readout(a, None, tht, alpha=0.5)  # CVaR needs a Hamiltonian
    h = gv.Hamiltonian.from_workload(wl.z_hamiltonian(n, 20, seed=0))
    with pytest.raises(gv.GvqeError):
        gv.readout(a, h, tht, alpha=1.5)


@pytest.mark.parametrize("fp64", [False, True])
def test_readout_large_register_properties(fp64):
    # n = 24 (16 Mi amplitudes, larger than one readout chunk): properties that hold at any size
    n, reps = 24, 2
    ham = wl.z_hamiltonian(n, 2000, seed=0)
    a, h = gv.Ansatz(n, reps), gv.Hamiltonian.from_workload(ham)
    tht = torch.as_tensor(wl.thetas(n, reps, 1, seed=1)[0], device="cuda")
    energy = gv.energy(a, h, tht, fp64=fp64).item()
    vals = []
    for alpha in (0.01, 0.2, 0.6, 1.0):
        r = gv.readout(a, h, tht, alpha=alpha, shots=2048, seed=3, fp64=fp64)
        vals.append(r.cvar)
        assert abs(r.total - 1.0) <= (1e-12 if fp64 else 1e-4)
        s = r.shots.cpu().numpy()
        assert s.min() >= 0 and s.max() < (1 << n)
    assert all(b >= a_ - 1e-9 * ham.abs_sum() for a_, b in zip(vals, vals[1:]))
    assert abs(vals[-1] - energy) <= (1e-10 if fp64 else 2e-5) * ham.abs_sum()
    # deterministic: the same call gives the same bits
    r1 = gv.readout(a, h, tht, alpha=0.2, shots=1024, seed=9, fp64=fp64)
    r2 = gv.readout(a, h, tht, alpha=0.2, shots=1024, seed=9, fp64=fp64)
    assert r1.cvar == r2.cvar and r1.argmax == r2.argmax
    assert torch.equal(r1.shots, r2.shots)
