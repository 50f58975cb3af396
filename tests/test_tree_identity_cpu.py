"""The regrouping behind the high-qubit gradient tree (k_mps_gtree), on the CPU.

The gradient of site q = 13 + t (layer k) is sum_c l_c A_13[c_0] .. dA^k_q[c_t] ..
A_{n-1}[c_{K-1}] 1 over the chunk index c (K = n - 13 bits).  The kernel regroups it
level by level: with E_t(j) the left environments summed over the low t bits and
R_t(j') the right environments of the bits above t,
g(k, 13 + t) = sum_j E_t(j) dA^k[j & 1] R_t(j >> 1), E_{t+1}(j) = E_t(2j) A[0] +
E_t(2j + 1) A[1]; stage 1 takes blocks of 2^8 chunks from their own right
environment, stage 2 the block vectors E_8.  This test replays that index
arithmetic (block and level offsets, the stage-2 vector stride 2^8) on random
matrices and compares it with the direct per-chunk sum, so a mistake in the
regrouping fails here without a GPU.
"""
import numpy as np
import pytest


def _direct(l, A, dA, K, D, r):
    chunks = 1 << K
    idx = np.arange(chunks)
    g = np.zeros((K, r + 1))
    for t in range(K):
        U = l.copy()
        for tt in range(t):
            bit = ((idx >> tt) & 1)[:, None]
            U = np.where(bit == 0, U @ A[tt][0], U @ A[tt][1])
        S = np.ones((chunks, D))
        for tt in range(K - 1, t, -1):
            bit = ((idx >> tt) & 1)[:, None]
            S = np.where(bit == 0, S @ A[tt][0].T, S @ A[tt][1].T)
        y = ((idx >> t) & 1)[:, None]
        for k in range(r + 1):
            W = np.where(y == 0, S @ dA[k][t][0].T, S @ dA[k][t][1].T)
            g[t, k] = np.sum(U * W)
    return g


def _stage(vecs, A, dA, K, r, t0, L, sh, blk, g):
    E = np.array([vecs[((blk << L) + v) << sh] for v in range(1 << L)])
    x = np.ones(E.shape[1])
    for t in range(K - 1, t0 + L - 1, -1):  # the right environment of the block's own bits
        x = A[t][(blk >> (t - t0 - L)) & 1] @ x
    R = {L - 1: [x]}
    for lt in range(L - 2, -1, -1):
        t = t0 + lt
        R[lt] = [A[t + 1][jp & 1] @ R[lt + 1][jp >> 1] for jp in range(1 << (L - 1 - lt))]
    for lt in range(L):
        t, nv = t0 + lt, 1 << (L - lt)
        for k in range(r + 1):
            g[t, k] += sum(E[2 * jj + y] @ (dA[k][t][y] @ R[lt][jj]) for jj in range(nv // 2) for y in range(2))
        E = np.array([E[2 * j] @ A[t][0] + E[2 * j + 1] @ A[t][1] for j in range(nv // 2)])
    return E[0]


@pytest.mark.parametrize("K,D,r", [(5, 4, 2), (9, 2, 1), (11, 2, 1)])
def test_tree_regrouping_matches_direct_sum(K, D, r):
    rng = np.random.default_rng(K * 10 + D)
    l = rng.standard_normal((1 << K, D))
    A = [[rng.standard_normal((D, D)) * 0.7 for _ in range(2)] for _ in range(K)]
    dA = [[[rng.standard_normal((D, D)) for _ in range(2)] for _ in range(K)] for _ in range(r + 1)]
    B = min(8, K)
    g = np.zeros((K, r + 1))
    vecs = l.copy()
    for blk in range(1 << (K - B)):  # stage 1: E_B of each block into its first chunk vector
        vecs[blk << B] = _stage(vecs, A, dA, K, r, 0, B, 0, blk, g)
    if K > B:  # stage 2 over the block vectors, stride 2^B
        _stage(vecs, A, dA, K, r, B, K - B, B, 0, g)
    ref = _direct(l, A, dA, K, D, r)
    assert np.max(np.abs(g - ref)) <= 1e-12 * np.max(np.abs(ref))
