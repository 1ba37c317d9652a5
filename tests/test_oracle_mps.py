"""Pins for the oracle's MPS forward pass and energy (Sec. 3; Sec. 2, Eq. expect-val)."""
import math

import numpy as np
import pytest

import synthetic as S
from oracle import ansatz, mps as M, pauli, statevector as SV


def small_problem(n=8, n_e=4, D=64, eps=1e-12, n_exc=None, seed_cfg=90):
    spec = S.ConfigSpec(f"n{n}_D{D}", n=n, n_e=n_e, D=D, eps=eps, decay=2.0)
    p = S.make_problem(seed_cfg, spec=spec)
    excs = p.excitations if n_exc is None else p.excitations[:n_exc]
    gates = ansatz.compile_circuit(n, excs)
    ham = pauli.jw_hamiltonian(p.h, p.eri)
    return p, gates, p.theta[: len(excs)], ham


def test_product_state():
    bits = [1, 0, 1, 1, 0]
    m = M.init_product(bits)
    assert np.array_equal(M.to_dense(m), SV.product_state(bits))


@pytest.mark.parametrize("cfg", ["cfg0", "n8"])
def test_forward_matches_statevector(cfg):
    if cfg == "cfg0":
        p = S.make_problem(0)
        gates = ansatz.compile_circuit(p.n, p.excitations)
        th, D, eps = p.theta, p.spec.D, p.spec.eps
    else:
        p, gates, th, _ = small_problem()
        D, eps = p.spec.D, p.spec.eps
    m = M.apply_circuit(M.init_product(p.bits), gates, th, D, eps)
    psi = SV.run(p.bits, gates, th)
    assert np.abs(M.to_dense(m) - psi).max() < 1e-12
    for b in range(p.n - 1):
        sv = SV.schmidt_values(psi, p.n, b)
        lam = m.lam[b]
        assert np.abs(lam - sv[: len(lam)]).max() < 1e-12
        assert np.sum(sv[len(lam):] ** 2) < 1e-24
    assert M.right_canonical_residual(m) < 1e-13
    assert abs(np.vdot(M.to_dense(m), M.to_dense(m)).real - 1.0) < 1e-12


def test_energy_matches_dense_and_imaginary_parts_vanish():
    p, gates, th, ham = small_problem()
    m = M.apply_circuit(M.init_product(p.bits), gates, th, p.spec.D, p.spec.eps)
    E = M.energy(m, ham)
    Ed = SV.energy(SV.run(p.bits, gates, th), ham)
    assert abs(E - Ed) < 1e-12 * max(1.0, abs(Ed))
    e, Z = M.string_expectations(m, ham)
    assert np.abs(e.imag).max() < 1e-13


def test_energy_closed_form_at_theta_zero():
    p = S.make_problem(1)
    ham = pauli.jw_hamiltonian(p.h, p.eri)
    gates = ansatz.compile_circuit(p.n, p.excitations[:20])
    m = M.apply_circuit(M.init_product(p.bits), gates, np.zeros(20), p.spec.D, p.spec.eps)
    occ = range(p.spec.n_e)
    closed = math.fsum(p.h[i, i] for i in occ) + math.fsum(
        0.5 * (p.eri[i, i, j, j] - p.eri[i, j, j, i]) for i in occ for j in occ)
    assert abs(M.energy(m, ham) - closed) < 1e-12 * max(1.0, abs(closed))


def test_product_state_rule():
    bits = [1, 1, 0, 1, 0, 0]
    m = M.init_product(bits)
    p = S.make_problem(90, spec=S.ConfigSpec("n6", n=6, n_e=3, D=8, eps=1e-12))
    ham = pauli.jw_hamiltonian(p.h, p.eri)
    e, _ = M.string_expectations(m, ham)
    for ek, x, z in zip(e, ham.x, ham.z):
        want = 0.0 if x else (-1.0) ** sum(bits[s] for s in range(6) if (z >> s) & 1)
        assert abs(ek - want) < 1e-15


def test_regauge_invariance():
    p, gates, th, ham = small_problem(n_exc=25)
    m = M.apply_circuit(M.init_product(p.bits), gates, th, p.spec.D, p.spec.eps)
    E0 = M.energy(m, ham)
    rng = np.random.default_rng(5)
    for b in range(p.n - 1):
        d = m.B[b].shape[2]
        X = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d)) + 3 * np.eye(d)
        assert abs(M.energy(M.regauge(m, b, X), ham) - E0) < 1e-12 * max(1, abs(E0))


def test_particle_number_and_sz_conserved():
    p, gates, th, _ = small_problem(n_exc=40)
    n = p.n
    m = M.apply_circuit(M.init_product(p.bits), gates, th, p.spec.D, p.spec.eps)
    # N = sum_p (1 - Z_p)/2 and S_z = sum_p (+-1/2)(1 - Z_p)/2 as Pauli sums
    zs = [1 << s for s in range(n)]
    N = pauli.PauliHamiltonian(n, [0] * (n + 1), [0] + zs, [n / 2] + [-0.5] * n)
    sz_c = [0.0] + [-0.25 if s % 2 == 0 else 0.25 for s in range(n)]
    Sz = pauli.PauliHamiltonian(n, [0] * (n + 1), [0] + zs, sz_c)
    assert abs(M.energy(m, N) - p.spec.n_e) < 1e-12
    assert abs(M.energy(m, Sz)) < 1e-12


def test_truncation_loses_norm_by_the_discarded_weight():
    p, gates, th, ham = small_problem(D=4, eps=1e-10, n_exc=12)
    m = M.init_product(p.bits)
    discarded = 0.0
    for g in gates:
        tape = M.apply_gate(m, g.bond, g.matrix(th), p.spec.D, p.spec.eps, keep_tape=True)
        s = tape["s"]
        discarded += float(np.sum(s[tape["k"]:] ** 2) / np.sum(s ** 2))
    assert discarded > 1e-6                       # the case really truncates
    norm = np.vdot(M.to_dense(m), M.to_dense(m)).real
    assert abs((1.0 - norm) - discarded) < 0.25 * discarded
