"""Pins for the oracle's UCCSD compiler (Sec. 2, Eq. uccansatz; Sec. 3, gate fusion)."""
import numpy as np
import pytest
import scipy.linalg

import synthetic as S
from oracle import ansatz, fermion, pauli


def test_excitation_counts():
    assert len(S.sd_excitations(4, 2)) == 3
    assert len(S.sd_excitations(12, 6)) == 117      # 18 singles + 99 doubles
    assert len(S.sd_excitations(20, 10)) == 875


def test_rz_convention():
    Z = np.diag([1.0, -1.0])
    for phi in (0.3, -1.7, 2.9):
        assert np.allclose(ansatz.rz(phi), scipy.linalg.expm(-0.5j * phi * Z), atol=1e-15)
        h = 1e-6
        fd = (ansatz.rz(phi + h) - ansatz.rz(phi - h)) / (2 * h)
        assert np.allclose(ansatz.drz(phi), fd, atol=1e-9)


def test_basis_changes():
    X = np.array([[0, 1], [1, 0]])
    Y = np.array([[0, -1j], [1j, 0]])
    Z = np.diag([1.0, -1.0])
    assert np.allclose(ansatz.HAD @ Z @ ansatz.HAD, X)
    assert np.allclose(ansatz.RXP.conj().T @ Z @ ansatz.RXP, Y)
    assert np.allclose(ansatz.RXM @ ansatz.RXP, np.eye(2))


@pytest.mark.parametrize("n,n_e", [(4, 2), (6, 3), (6, 2)])
def test_each_excitation_matches_expm(n, n_e):
    rng = np.random.default_rng(n * 10 + n_e)
    for exc in S.sd_excitations(n, n_e):
        th = rng.uniform(-np.pi, np.pi)
        U = ansatz.circuit_unitary_dense(n, ansatz.compile_circuit(n, [exc]), [th])
        assert np.abs(U - fermion.excitation_unitary(exc, th, n)).max() < 1e-12


def test_whole_circuit_matches_product_of_exponentials():
    n, n_e = 6, 3
    excs = S.sd_excitations(n, n_e)
    th = np.random.default_rng(2).uniform(-np.pi, np.pi, len(excs))
    U = ansatz.circuit_unitary_dense(n, ansatz.compile_circuit(n, excs), th)
    Ue = np.eye(2 ** n)
    for t, e in enumerate(excs):
        Ue = fermion.excitation_unitary(e, th[t], n) @ Ue
    assert np.abs(U - Ue).max() < 1e-12


def test_peephole_rules_preserve_the_unitary():
    n, n_e = 6, 3
    excs = S.sd_excitations(n, n_e)[:6]
    th = np.random.default_rng(4).uniform(-np.pi, np.pi, len(excs))
    prims = ansatz.primitive_circuit(n, excs)
    raw = ansatz.absorb_single_qubit(prims, n)                 # no cancellation, no merge
    full = ansatz.compile_circuit(n, excs)
    assert len(full) < len(raw)
    U1 = ansatz.circuit_unitary_dense(n, raw, th)
    U2 = ansatz.circuit_unitary_dense(n, full, th)
    assert np.abs(U1 - U2).max() < 1e-12


def test_gate_list_structure():
    p = S.make_problem(1)
    gates = ansatz.compile_circuit(p.n, p.excitations)
    n_strings = sum(2 if e[1] < 0 else 8 for e in p.excitations)
    assert sum(g.parametric for g in gates) == n_strings       # one Rz per string rotation
    assert {g.theta_idx for g in gates if g.parametric} == set(range(len(p.excitations)))
    assert all(0 <= g.bond < p.n - 1 for g in gates)
    for g in gates[:200]:
        G = g.matrix(p.theta)
        assert np.abs(G @ G.conj().T - np.eye(4)).max() < 1e-13
    # per-excitation coefficients: singles +-1/2, doubles +-1/8 (scale = -2c)
    for e in p.excitations[:30]:
        cs = sorted(abs(c) for (_, _, c) in ansatz.excitation_strings(e, p.n))
        assert cs == ([0.5] * 2 if e[1] < 0 else [0.125] * 8)
