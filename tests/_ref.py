"""Small independent re-derivations used by the tests (numpy only).

These do not call the oracle or the CUDA path; they restate definitions from the
paper with library primitives so that the oracle can be pinned to something other
than itself.
"""
import math

import numpy as np

M64 = (1 << 64) - 1


def numpy_philox_block(ctr, key):
    """Philox4x64-10 block for counter ``ctr`` from numpy's own Philox bit generator
    (numpy advances the counter by one before producing each block of four words)."""
    c = sum(int(x) << (64 * i) for i, x in enumerate(ctr))
    bg = np.random.Philox(counter=(c - 1) % (1 << 256), key=[int(key[0]), int(key[1])])
    return np.array(bg.random_raw(4), dtype=np.uint64)


def svd_leverage(A, tol=1e-12):
    """l_i = ||U(i,:)||^2 with U the left singular vectors of the numerical range."""
    U, s, _ = np.linalg.svd(A, full_matrices=False)
    k = int(np.sum(s > tol * s[0])) if s.size and s[0] > 0 else 0
    return np.sum(U[:, :k] ** 2, axis=1)


def khatri_rao(mats):
    """Z with Z(key, :) = prod_t mats[t](i_t, :), key = sum_t i_t prod_{u<t} n_u."""
    Z = mats[0]
    for A in mats[1:]:
        Z = np.einsum("ir,jr->jir", Z, A).reshape(-1, Z.shape[1])
    return Z


def product_probs(ps):
    """Full p vector over linear keys (first mode fastest), multiplied in mode order."""
    p = ps[0]
    for q in ps[1:]:
        p = (p[None, :] * q[:, None]).reshape(-1)  # p_prev * q_t, prev index fastest
    return p


def draw_ref(C, T, u):
    t = (int(u) * int(T)) >> 64
    return int(np.searchsorted(C, np.uint64(t), side="right"))


def unfold(X, k):
    """Mode-k unfolding with the other modes in ascending order, first fastest."""
    D = X.ndim
    others = [m for m in range(D) if m != k]
    Y = np.transpose(X, [k] + others[::-1])
    return Y.reshape(X.shape[k], -1)


def dense_mttkrp(X, factors, k):
    others = [m for m in range(X.ndim) if m != k]
    Z = khatri_rao([factors[m] for m in others])
    return unfold(X, k) @ Z, Z


def cp_dense(lam, factors):
    r = lam.shape[0]
    X = np.zeros(tuple(F.shape[0] for F in factors))
    for j in range(r):
        T = lam[j]
        for F in factors:
            T = np.multiply.outer(T, F[:, j])
        X = X + T
    return X
