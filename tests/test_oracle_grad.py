"""Pins for the oracle's reverse-mode gradient (Sec. 4; App. A)."""
import numpy as np
import pytest

import synthetic as S
from oracle import ansatz, mps as M, pauli, statevector as SV

from test_oracle_mps import small_problem


@pytest.mark.parametrize("cfg", ["cfg0", "n8"])
def test_gradient_matches_algorithm1_on_statevector(cfg):
    if cfg == "cfg0":
        p = S.make_problem(0)
        gates = ansatz.compile_circuit(p.n, p.excitations)
        th, ham = p.theta, pauli.jw_hamiltonian(p.h, p.eri)
    else:
        p, gates, th, ham = small_problem(n_exc=30)
    r = M.energy_grad(M.init_product(p.bits), gates, th, ham, p.spec.D, p.spec.eps,
                      checkpoint_every=11)
    E, g, gg = SV.gradient(p.bits, gates, th, ham)
    assert abs(r.E - E) < 1e-11
    assert np.linalg.norm(r.grad - g) < 1e-10 * max(1.0, np.linalg.norm(g))
    assert np.abs(r.gate_grad - gg).max() < 1e-10


def test_checkpoint_interval_does_not_change_the_result():
    p, gates, th, ham = small_problem(D=4, eps=1e-10, n_exc=10)
    r1 = M.energy_grad(M.init_product(p.bits), gates, th, ham, 4, 1e-10, checkpoint_every=1000)
    r2 = M.energy_grad(M.init_product(p.bits), gates, th, ham, 4, 1e-10, checkpoint_every=3)
    assert r1.E == r2.E
    assert np.array_equal(r1.grad, r2.grad)


def kept_profile(p, gates, th, D, eps):
    m = M.init_product(p.bits)
    ks = []
    for g in gates:
        ks.append(M.apply_gate(m, g.bond, g.matrix(th), D, eps, keep_tape=True)["k"])
    return ks


def test_gradient_matches_finite_differences_under_truncation():
    p, gates, th, ham = small_problem(D=4, eps=1e-10, n_exc=10)
    D, eps = 4, 1e-10
    r = M.energy_grad(M.init_product(p.bits), gates, th, ham, D, eps)
    k0 = kept_profile(p, gates, th, D, eps)
    h = 1e-5
    checked = 0
    for t in range(len(th)):
        tp, tm = th.copy(), th.copy()
        tp[t] += h
        tm[t] -= h
        if kept_profile(p, gates, tp, D, eps) != k0 or kept_profile(p, gates, tm, D, eps) != k0:
            continue
        Ep = M.energy(M.apply_circuit(M.init_product(p.bits), gates, tp, D, eps), ham)
        Em = M.energy(M.apply_circuit(M.init_product(p.bits), gates, tm, D, eps), ham)
        fd = (Ep - Em) / (2 * h)
        assert abs(fd - r.grad[t]) < 1e-7 * max(1.0, abs(fd))
        checked += 1
    assert checked >= 8


def test_parameter_shift_rule_per_gate():
    """Eq. (psr): dE/dphi = 1/2 [E(phi + pi/2) - E(phi - pi/2)], exact without truncation."""
    p, gates, th, ham = small_problem(n_exc=15)
    r = M.energy_grad(M.init_product(p.bits), gates, th, ham, p.spec.D, p.spec.eps)
    par = [t for t, g in enumerate(gates) if g.parametric]
    for t in par[:: max(1, len(par) // 8)][:8]:
        phi = gates[t].phi(th)
        Ep = M.energy(M.apply_circuit(M.init_product(p.bits), gates, th, p.spec.D, p.spec.eps,
                                      phi_override={t: phi + np.pi / 2}), ham)
        Em = M.energy(M.apply_circuit(M.init_product(p.bits), gates, th, p.spec.D, p.spec.eps,
                                      phi_override={t: phi - np.pi / 2}), ham)
        assert abs(0.5 * (Ep - Em) - r.gate_grad[t]) < 1e-11


def test_single_angle_sinusoid():
    """Without truncation E(phi) of one Rz angle is a + b cos(phi) + c sin(phi)."""
    p, gates, th, ham = small_problem(n_exc=8)
    t = [u for u, g in enumerate(gates) if g.parametric][3]
    phis = np.linspace(-3, 3, 7)
    Es = [M.energy(M.apply_circuit(M.init_product(p.bits), gates, th, p.spec.D, p.spec.eps,
                                   phi_override={t: f}), ham) for f in phis]
    A = np.stack([np.ones_like(phis), np.cos(phis), np.sin(phis)], axis=1)
    coef, res, *_ = np.linalg.lstsq(A, np.array(Es), rcond=None)
    assert np.abs(A @ coef - Es).max() < 1e-12


@pytest.mark.parametrize("shape,k", [((12, 8), 5), ((8, 12), 5), ((10, 10), 10), ((6, 16), 3)])
def test_svd_adjoint_against_finite_differences(shape, k):
    """f(C~) = Re<X, C~ V_k V_k^+> + <b, s_k/||s_k||>, a gauge-invariant function of the SVD."""
    rng = np.random.default_rng(sum(shape) + k)
    m, ncol = shape
    Ct = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    X = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    b = rng.standard_normal(k)

    def f(C):
        U, s, Vh = np.linalg.svd(C, full_matrices=True)
        Vk = Vh.conj().T[:, :k]
        sk = s[:k]
        return np.real(np.vdot(X, C @ Vk @ Vk.conj().T)) + b @ (sk / np.linalg.norm(sk))

    U, s, Vh = np.linalg.svd(Ct, full_matrices=True)
    V = Vh.conj().T
    Vk = V[:, :k]
    lam = s[:k] / np.linalg.norm(s[:k])
    sbar = (b - lam * (lam @ b)) / np.linalg.norm(s[:k])
    Vbar = 0.5 * (Ct.conj().T @ X @ Vk + X.conj().T @ Ct @ Vk)
    Cbar = 0.5 * X @ Vk @ Vk.conj().T + M.svd_adjoint(Ct, s, V, k, sbar, Vbar)
    h = 1e-6
    for _ in range(4):
        dC = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
        fd = (f(Ct + h * dC) - f(Ct - h * dC)) / (2 * h)
        assert abs(fd - 2 * np.real(np.vdot(Cbar, dC))) < 1e-6 * max(1, abs(fd))


def test_energy_seed_against_finite_differences():
    p, gates, th, ham = small_problem(D=4, eps=1e-10, n_exc=10)
    m = M.apply_circuit(M.init_product(p.bits), gates, th, 4, 1e-10)
    E, Bbar = M.energy_seed(m, ham)
    rng = np.random.default_rng(9)
    h = 1e-6
    for s in range(p.n):
        dB = rng.standard_normal(m.B[s].shape) + 1j * rng.standard_normal(m.B[s].shape)
        mp, mm = m.copy(), m.copy()
        mp.B[s] = mp.B[s] + h * dB
        mm.B[s] = mm.B[s] - h * dB
        fd = (M.energy(mp, ham) - M.energy(mm, ham)) / (2 * h)
        assert abs(fd - 2 * np.real(np.vdot(Bbar[s], dB))) < 1e-7 * max(1, abs(fd))
