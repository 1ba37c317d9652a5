"""The parameter-shift gradient (Sec. 4, Eq. psr) on the GPU, as the baseline of the adjoint.

Each Rz gate of the circuit, G(phi) = post Rz(phi) pre with Rz(phi) = diag(e^{-i phi/2},
e^{i phi/2}), has dE/dphi = [E(phi + pi/2) - E(phi - pi/2)] / 2 exactly when nothing is truncated,
and dE/dtheta_t sums theta_scale * dE/dphi over the gates that share theta_t.  That costs two
forward passes plus two energies per Rz gate, 2 M evaluations for M gates, against one forward,
one energy and one reverse pass for the adjoint whatever M is.  Here the 2 M shifted circuits run
as instances of batched states: every gate gets its own angle slot (phi directly), and each
instance shifts one slot.
"""
from __future__ import annotations

import time

import numpy as np

from . import api
from ._lib import GATE_DTYPE


def per_gate_circuit(gates: np.ndarray, theta: np.ndarray):
    """The same gates with one angle slot per Rz gate: (gates', phi0, parametric gate indices)."""
    g = np.array(gates, dtype=GATE_DTYPE, copy=True)
    par = np.flatnonzero(g["theta_idx"] >= 0)
    phi0 = g["theta_scale"][par] * np.asarray(theta, dtype=np.float64)[g["theta_idx"][par]]
    g["theta_idx"][par] = np.arange(len(par), dtype=np.int32)
    g["theta_scale"][par] = 1.0
    return g, phi0, par


def parameter_shift(n: int, bits, gates: np.ndarray, theta, ham: "api.Hamiltonian", D: int, eps: float,
                    batch: int = 128, stream=None, precision: str = "fp64"):
    """dE/dtheta (and dE/dphi per gate) by parameter shift, 2 M evaluations in batches of `batch`.

    Returns (grad, gate_grad, evaluations, seconds).
    """
    gates1, phi0, par = per_gate_circuit(gates, theta)
    M = len(par)
    circ = api.Circuit(n, gates1)
    rows = np.repeat(phi0[None, :], 2 * M, axis=0)
    for j in range(M):
        rows[2 * j, j] += np.pi / 2
        rows[2 * j + 1, j] -= np.pi / 2
    E = np.zeros(2 * M)
    t0 = time.perf_counter()
    for lo in range(0, 2 * M, batch):
        hi = min(2 * M, lo + batch)
        st = api.State.product_batch(np.stack([bits] * (hi - lo)), D, eps, stream=stream, precision=precision)
        api.apply_circuit(st, circ, np.ascontiguousarray(rows[lo:hi]))
        e = api.energy(st, ham)
        E[lo:hi] = np.atleast_1d(e)
        st.free()
    seconds = time.perf_counter() - t0
    dphi = 0.5 * (E[0::2] - E[1::2])
    gate_grad = np.zeros(len(gates))
    gate_grad[par] = dphi
    grad = np.zeros(len(np.atleast_1d(theta)))
    np.add.at(grad, np.asarray(gates["theta_idx"])[par], np.asarray(gates["theta_scale"])[par] * dphi)
    return grad, gate_grad, 2 * M, seconds
