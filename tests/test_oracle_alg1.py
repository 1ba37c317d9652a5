"""Pins for the oracle's Algorithm 1 with Hamiltonian groups (Sec. 4), the paper's own gradient.

Without truncation, Algorithm 1 on MPS equals Algorithm 1 on the dense state vector, whatever
the grouping; its building blocks (Pauli images, MPS addition, compression) are checked against
dense linear algebra.  With truncation it is an approximation, and its distance R from the
exact adjoint (Eq. meanerror) is only bounded loosely.
"""
import numpy as np
import pytest

import synthetic as S
from oracle import alg1, ansatz, mps as M, pauli, statevector as SV

from test_oracle_mps import small_problem


def _final(p, gates, th, D, eps):
    return M.apply_circuit(M.init_product(p.bits), gates, th, D, eps)


def test_pauli_image_addition_and_compression_against_dense():
    p, gates, th, ham = small_problem(n_exc=12)
    psi = _final(p, gates, th, p.spec.D, p.spec.eps)
    dense = M.to_dense(psi)
    rng = np.random.default_rng(3)
    ks = rng.choice(len(ham), size=5, replace=False)
    want = np.zeros_like(dense)
    terms = []
    for k in ks:
        img = alg1.apply_pauli(psi, ham.x[k], ham.z[k])
        d = SV.apply_pauli(dense, p.n, ham.x[k], ham.z[k])
        assert np.abs(M.to_dense(img) - d).max() < 1e-13          # P|psi> exactly
        assert M.right_canonical_residual(M.MPS(img.B[1:], img.lam[1:])) < 1e-12
        terms.append((float(ham.coeff[k]), img))
        want = want + float(ham.coeff[k]) * d
    out = alg1.compress(alg1.add(terms), 10 ** 6, 0.0)
    assert np.abs(M.to_dense(out) - want).max() < 1e-12 * np.abs(want).max()
    # right-canonical from site 1 on, Schmidt vectors of the normalised state on every bond
    assert M.right_canonical_residual(M.MPS(out.B[1:], out.lam[1:])) < 1e-12
    wn = want / np.linalg.norm(want)
    for b in range(p.n - 1):
        sv = SV.schmidt_values(wn, p.n, b)
        assert np.abs(out.lam[b] - sv[: len(out.lam[b])]).max() < 1e-12


@pytest.mark.parametrize("m", [1, 3])
def test_algorithm1_on_mps_equals_the_state_vector_form_without_truncation(m):
    p, gates, th, ham = small_problem(n_exc=20)
    final = _final(p, gates, th, p.spec.D, p.spec.eps)
    g, gg = alg1.gradient(final, gates, th, ham, p.spec.D, p.spec.eps, m=m)
    E, gs, ggs = SV.gradient(p.bits, gates, th, ham)
    assert np.linalg.norm(g - gs) < 1e-10 * max(1.0, np.linalg.norm(gs))
    assert np.abs(gg - ggs).max() < 1e-10


def test_algorithm1_under_truncation_is_finite_and_exact_once_D_suffices():
    """n = 8 needs D = 16.  With D = 8 the three middle bonds are truncated and Algorithm 1 is an
    approximation (R, Eq. meanerror, against the exact adjoint of the truncated forward); with
    D = 16 nothing is truncated and R vanishes for any grouping."""
    for D, exact in ((8, False), (16, True)):
        p, gates, th, ham = small_problem(D=D, eps=1e-10, n_exc=12)
        final = _final(p, gates, th, D, 1e-10)
        g_ad = M.energy_grad(M.init_product(p.bits), gates, th, ham, D, 1e-10).grad
        for m in (1, 4):
            g_bp, _ = alg1.gradient(final, gates, th, ham, D, 1e-10, m=m)
            R = np.linalg.norm(g_bp - g_ad) / np.linalg.norm(g_ad)
            assert np.isfinite(R)
            if exact:
                assert R < 1e-10
