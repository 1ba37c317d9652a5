"""Oracle: second-quantised operators as dense matrices in the occupation basis.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

This module does NOT use the Jordan-Wigner map.  It builds a_p directly from the
definition of a fermionic annihilation operator on occupation-number states,
a_p |..., n_p = 1, ...> = (-1)^(sum_{q<p} n_q) |..., n_p = 0, ...>,
so that it can pin the Pauli-string construction in `oracle.pauli`
(Sec. 2, Eq. ham-pbc) and the compiled UCC excitation unitaries
(Sec. 2, Eq. uccansatz).

Basis order: index = sum_s n_s 2^(n-1-s), i.e. orbital/site 0 is the most
significant bit, the same order as the MPS coefficient tensor c_{i1 i2 ... iN}.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def annihilation(p: int, n: int) -> np.ndarray:
    dim = 2 ** n
    a = np.zeros((dim, dim))
    for idx in range(dim):
        occ = [(idx >> (n - 1 - s)) & 1 for s in range(n)]
        if occ[p] == 0:
            continue
        sign = (-1) ** sum(occ[:p])
        a[idx & ~(1 << (n - 1 - p)), idx] = sign
    return a


def hamiltonian(h: np.ndarray, eri: np.ndarray) -> np.ndarray:
    """sum_pq h_pq a+_p a_q + 1/2 sum_pqrs (pq|rs) a+_p a+_r a_s a_q (chemist notation)."""
    n = h.shape[0]
    a = [annihilation(p, n) for p in range(n)]
    ad = [m.T for m in a]
    H = np.zeros((2 ** n, 2 ** n))
    for p in range(n):
        for q in range(n):
            if h[p, q] != 0.0:
                H += h[p, q] * ad[p] @ a[q]
    for (p, q, r, s) in np.argwhere(eri != 0.0):
        H += 0.5 * eri[p, q, r, s] * ad[p] @ ad[r] @ a[s] @ a[q]
    return H


def excitation_operator(exc, n: int) -> np.ndarray:
    """T for exc = (i, j, a, b): a+_a a_i (single, j = b = -1) or a+_a a+_b a_j a_i."""
    i, j, a_, b = exc
    a = [annihilation(p, n) for p in range(n)]
    if j < 0:
        return a[a_].T @ a[i]
    return a[a_].T @ a[b].T @ a[j] @ a[i]


def excitation_unitary(exc, theta: float, n: int) -> np.ndarray:
    """exp(theta (T - T+)) (Sec. 2, Eq. uccansatz for one excitation)."""
    T = excitation_operator(exc, n)
    return scipy.linalg.expm(theta * (T - T.T))


def number_operator(n: int) -> np.ndarray:
    a = [annihilation(p, n) for p in range(n)]
    return sum(m.T @ m for m in a)


def sz_operator(n: int) -> np.ndarray:
    """S_z = 1/2 (N_alpha - N_beta), alpha = even orbitals."""
    a = [annihilation(p, n) for p in range(n)]
    return sum((0.5 if p % 2 == 0 else -0.5) * (a[p].T @ a[p]) for p in range(n))


def basis_state(bits) -> np.ndarray:
    n = len(bits)
    v = np.zeros(2 ** n)
    v[sum(int(b) << (n - 1 - s) for s, b in enumerate(bits))] = 1.0
    return v
