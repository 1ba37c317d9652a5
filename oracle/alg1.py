"""Oracle: the paper's memory-efficient back-propagation (Sec. 4, Algorithm 1) on MPS, with the
Hamiltonian split into groups.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Paper passages followed:
* Sec. 4, Algorithm 1: starting from Psi = Psi_M (the final state) and phi = H Psi_M, walk the
  gates backwards; per gate j: Psi <- U_j^+ Psi, grads[j] = Re <phi| dU_j |Psi>, then
  phi <- U_j^+ phi.  Every U^+ is applied with the same two-site update and truncation to D as
  the forward pass (Sec. 3).
* Sec. 4, grouping: H = sum_j H^j in m groups; the gradient is the sum of the groups'
  gradients (exact whenever nothing is truncated, whatever the split).
* Sec. 4: H^j Psi is a sum of Pauli-string images of Psi; adding k MPS of bond dimension D gives
  bond dimension up to k D, which is compressed back to D.

Readings:
* A Pauli string acts site by site on the physical index, so P Psi keeps Psi's tensors' shapes
  and its right-canonical form (Pauli matrices are unitary).
* Addition is the direct sum of the bond spaces (the coefficients multiply the first site).
* Compression (the paper does not say how): left-to-right QR, then a right-to-left SVD sweep
  truncated with the forward pass's rule, k = max(1, min(D, #{s_i/||s|| > eps and
  s_i > 1e-13 s_1})).  The result is right-canonical with the state's norm in site 0 and
  normalised Schmidt vectors on every bond, the form the two-site update expects.
* dE/dphi_j = 2 Re <phi| dU_j/dphi |Psi> for gate j's Rz angle (the factor 2 of the complex
  derivative convention, App. A), as in the state-vector form.  The normalisation of E is not
  differentiated: with unitary gates and nothing truncated, <psi|psi> does not depend on theta.
* Groups are consecutive chunks of the canonically ordered strings (the identity string with
  the first group), m groups of sizes differing by at most one.
"""
from __future__ import annotations

import math

import numpy as np

from . import pauli
from .mps import MPS, apply_gate, truncation_rank


def apply_pauli(mps: MPS, x: int, z: int) -> MPS:
    """P |mps> for the Pauli string (x, z): each site tensor gets O_s on its physical index."""
    out = mps.copy()
    for s in range(mps.n):
        O = pauli.site_matrix(x, z, s)
        out.B[s] = np.einsum("ij,ajb->aib", O, mps.B[s])
    return out


def add(terms) -> list:
    """sum_k c_k |mps_k> as site tensors of the direct-sum bond spaces (not canonical)."""
    n = terms[0][1].n
    out = []
    for s in range(n):
        blocks = [c * m.B[s] if s == 0 else m.B[s] for c, m in terms]
        Dl = 1 if s == 0 else sum(b.shape[0] for b in blocks)
        Dr = 1 if s == n - 1 else sum(b.shape[2] for b in blocks)
        A = np.zeros((Dl, 2, Dr), dtype=complex)
        l = r = 0
        for b in blocks:
            dl, dr = b.shape[0], b.shape[2]
            ls = slice(0, 1) if s == 0 else slice(l, l + dl)
            rs = slice(0, 1) if s == n - 1 else slice(r, r + dr)
            if s == 0 or s == n - 1:
                A[ls, :, rs] += b
            else:
                A[ls, :, rs] = b
            l += dl
            r += dr
        out.append(A)
    return out


def compress(A: list, D: int, eps: float) -> MPS:
    """Site tensors of any MPS -> right-canonical MPS truncated to D (see the module readings)."""
    n = len(A)
    A = [a.copy() for a in A]
    for s in range(n - 1):                       # left-canonical sweep
        Dl, _, Dr = A[s].shape
        Q, R = np.linalg.qr(A[s].reshape(Dl * 2, Dr))
        A[s] = Q.reshape(Dl, 2, Q.shape[1])
        A[s + 1] = np.einsum("km,mjc->kjc", R, A[s + 1])
    lam = [None] * (n - 1)
    for s in range(n - 1, 0, -1):               # right-to-left truncated SVD sweep
        Dl, _, Dr = A[s].shape
        U, S, Vh = np.linalg.svd(A[s].reshape(Dl, 2 * Dr), full_matrices=False)
        k = truncation_rank(S, D, eps)
        A[s] = Vh[:k].reshape(k, 2, Dr)
        A[s - 1] = np.einsum("aim,mk->aik", A[s - 1], U[:, :k] * S[:k])
        Sk = S[:k]
        lam[s - 1] = Sk / math.sqrt(float(np.sum(Sk * Sk)))
    return MPS(A, lam)


def overlap_with_two_site_operator(phi: MPS, psi: MPS, bond: int, O: np.ndarray) -> complex:
    """<phi| O_(bond, bond+1) |psi> by a left-to-right contraction (O: 4 x 4, index 2 i_b + i_b+1)."""
    L = np.ones((1, 1), dtype=complex)
    s = 0
    n = psi.n
    while s < n:
        if s == bond:
            tp = np.einsum("aim,mjc->aijc", psi.B[s], psi.B[s + 1])
            Dl, Dr = tp.shape[0], tp.shape[3]
            tp = np.einsum("xy,ayc->axc", O, tp.reshape(Dl, 4, Dr))
            tf = np.einsum("aim,mjc->aijc", phi.B[s], phi.B[s + 1])
            tf = tf.reshape(tf.shape[0], 4, tf.shape[3])
            L = np.einsum("ab,axc,bxd->cd", L, tf.conj(), tp)
            s += 2
        else:
            L = np.einsum("ab,aic,bid->cd", L, phi.B[s].conj(), psi.B[s])
            s += 1
    return complex(L[0, 0])


def groups(ham: pauli.PauliHamiltonian, m: int) -> list:
    """m consecutive chunks of the canonically ordered strings (indices)."""
    idx = np.arange(len(ham))
    return [g for g in np.array_split(idx, m) if len(g)]


def gradient(final: MPS, gates, theta, ham: pauli.PauliHamiltonian, D: int, eps: float, m: int = 1):
    """Algorithm 1 with m Hamiltonian groups; returns (dE/dtheta, dE/dphi per gate)."""
    theta = np.asarray(theta, dtype=float)
    gate_grad = np.zeros(len(gates))
    for grp in groups(ham, m):
        terms = [(float(ham.coeff[k]), apply_pauli(final, ham.x[k], ham.z[k])) for k in grp]
        phi = compress(add(terms), D, eps)
        Psi = final.copy()
        for t in range(len(gates) - 1, -1, -1):
            g = gates[t]
            G = g.matrix(theta)
            apply_gate(Psi, g.bond, G.conj().T, D, eps)
            if g.parametric:
                gate_grad[t] += 2.0 * np.real(overlap_with_two_site_operator(phi, Psi, g.bond, g.dmatrix(theta)))
            apply_gate(phi, g.bond, G.conj().T, D, eps)
    grad = np.zeros(len(theta))
    for t, g in enumerate(gates):
        if g.parametric:
            grad[g.theta_idx] += g.scale * gate_grad[t]
    return grad, gate_grad
