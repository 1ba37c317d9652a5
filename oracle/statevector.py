"""Oracle: dense state-vector simulator ("brute force method", Sec. 1).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Stores all 2^n amplitudes (site 0 = most significant index bit) and is exact up
to rounding: no truncation.  It provides the pins for the MPS oracle when n is
small: amplitudes, Schmidt values, <psi|H|psi>, and the exact gradient by
Algorithm 1 (Sec. 4) run on the state vector, where the memory-efficient
back-propagation is exact (no MPS compression of H|psi>):

    Psi <- psi_M, phi <- H psi_M
    for j = M..1:  Psi <- U_j^+ Psi;  dE/dphi_j = 2 Re <phi| dU_j/dphi |Psi>;  phi <- U_j^+ phi
"""
from __future__ import annotations

import numpy as np

from . import pauli


def product_state(bits) -> np.ndarray:
    n = len(bits)
    v = np.zeros(2 ** n, dtype=complex)
    v[sum(int(b) << (n - 1 - s) for s, b in enumerate(bits))] = 1.0
    return v


def apply_two_site(psi: np.ndarray, n: int, bond: int, G: np.ndarray) -> np.ndarray:
    t = psi.reshape(2 ** bond, 4, 2 ** (n - bond - 2))
    return np.einsum("xy,ayc->axc", G, t).reshape(-1)


def run(bits, gates, theta, phi_override=None) -> np.ndarray:
    n = len(bits)
    psi = product_state(bits)
    for t, g in enumerate(gates):
        phi = None if phi_override is None else phi_override.get(t)
        psi = apply_two_site(psi, n, g.bond, g.matrix(theta, phi=phi))
    return psi


def apply_pauli(psi: np.ndarray, n: int, x: int, z: int) -> np.ndarray:
    t = psi.reshape([2] * n)
    for s in range(n):
        O = pauli.site_matrix(x, z, s)
        t = np.moveaxis(np.tensordot(O, t, axes=([1], [s])), 0, s)
    return t.reshape(-1)


def apply_hamiltonian(psi: np.ndarray, ham: pauli.PauliHamiltonian) -> np.ndarray:
    out = np.zeros_like(psi)
    for x, z, c in zip(ham.x, ham.z, ham.coeff):
        out += c * apply_pauli(psi, ham.n, x, z)
    return out


def energy(psi: np.ndarray, ham: pauli.PauliHamiltonian) -> float:
    return float(np.real(np.vdot(psi, apply_hamiltonian(psi, ham))) / np.real(np.vdot(psi, psi)))


def gradient(bits, gates, theta, ham: pauli.PauliHamiltonian):
    """Algorithm 1 on the state vector; returns (E, dE/dtheta, dE/dphi per gate)."""
    n = len(bits)
    theta = np.asarray(theta, dtype=float)
    psi = run(bits, gates, theta)
    phi = apply_hamiltonian(psi, ham)
    E = float(np.real(np.vdot(psi, phi)))
    Psi = psi
    gate_grad = np.zeros(len(gates))
    for t in range(len(gates) - 1, -1, -1):
        g = gates[t]
        G = g.matrix(theta)
        Psi = apply_two_site(Psi, n, g.bond, G.conj().T)
        if g.parametric:
            gate_grad[t] = 2.0 * np.real(np.vdot(phi, apply_two_site(Psi, n, g.bond, g.dmatrix(theta))))
        phi = apply_two_site(phi, n, g.bond, G.conj().T)
    grad = np.zeros(len(theta))
    for t, g in enumerate(gates):
        if g.parametric:
            grad[g.theta_idx] += g.scale * gate_grad[t]
    return E, grad, gate_grad


def schmidt_values(psi: np.ndarray, n: int, bond: int) -> np.ndarray:
    """Singular values of the (sites 0..bond) x (sites bond+1..n-1) reshaping."""
    return np.linalg.svd(psi.reshape(2 ** (bond + 1), -1), compute_uv=False)
