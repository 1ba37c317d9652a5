"""Pins for the oracle's Pauli algebra and Jordan-Wigner Hamiltonian (Sec. 2, Eq. ham-pbc)."""
import math
import os
import random

import numpy as np
import pytest

import synthetic as S
from oracle import fermion, pauli

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_pauli_product_matches_matrices():
    rng = random.Random(1)
    n = 3
    for _ in range(200):
        x1, z1, x2, z2 = (rng.randrange(8) for _ in range(4))
        e, x3, z3 = pauli.mul(x1, z1, x2, z2)
        lhs = pauli.pauli_dense(x1, z1, n) @ pauli.pauli_dense(x2, z2, n)
        rhs = (1j ** e) * pauli.pauli_dense(x3, z3, n)
        assert np.allclose(lhs, rhs, atol=0)


def test_jw_single_mode_operators_match_fermionic_definition():
    n = 4
    for p in range(n):
        A = sum((1j ** k) * 0.5 * pauli.pauli_dense(x, z, n) for (k, x, z) in pauli.jw_annihilation(p))
        assert np.allclose(A, fermion.annihilation(p, n), atol=1e-15)
        Ad = sum((1j ** k) * 0.5 * pauli.pauli_dense(x, z, n) for (k, x, z) in pauli.jw_creation(p))
        assert np.allclose(Ad, fermion.annihilation(p, n).T, atol=1e-15)


def _random_integrals(n_spatial, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    hS, eS = S.spatial_integrals(n_spatial, rng)
    return S.spin_orbital_integrals(hS, eS)


@pytest.mark.parametrize("case", ["cfg0", "random6"])
def test_jw_hamiltonian_equals_occupation_basis_matrix(case):
    if case == "cfg0":
        p = S.make_problem(0)
        h, eri = p.h, p.eri
    else:
        h, eri = _random_integrals(3, 7)
    ham = pauli.jw_hamiltonian(h, eri)
    Hjw = pauli.hamiltonian_dense(ham)
    Hf = fermion.hamiltonian(h, eri)
    assert np.abs(Hjw - Hf).max() < 1e-12 * max(1.0, np.abs(Hf).max())


def test_hermitian_and_symmetries():
    h, eri = _random_integrals(3, 11)
    n = h.shape[0]
    H = pauli.hamiltonian_dense(pauli.jw_hamiltonian(h, eri))
    assert np.abs(H - H.conj().T).max() < 1e-13
    N = fermion.number_operator(n)
    Sz = fermion.sz_operator(n)
    assert np.abs(H @ N - N @ H).max() < 1e-12
    assert np.abs(H @ Sz - Sz @ H).max() < 1e-12


def slater_condon(h, eri, n_e):
    """<HF|H|HF> = sum_i h_ii + 1/2 sum_ij [(ii|jj) - (ij|ji)] over occupied spin orbitals."""
    occ = range(n_e)
    e1 = math.fsum(h[i, i] for i in occ)
    e2 = math.fsum(0.5 * (eri[i, i, j, j] - eri[i, j, j, i]) for i in occ for j in occ)
    return e1 + e2


@pytest.mark.parametrize("case", ["cfg0", "random6"])
def test_hf_energy_closed_form(case):
    if case == "cfg0":
        p = S.make_problem(0)
        h, eri, n_e = p.h, p.eri, p.spec.n_e
    else:
        h, eri = _random_integrals(3, 5)
        n_e = 3
    ham = pauli.jw_hamiltonian(h, eri)
    n = h.shape[0]
    hf = fermion.basis_state([1] * n_e + [0] * (n - n_e))
    e_dense = float(hf @ pauli.hamiltonian_dense(ham).real @ hf)
    assert abs(e_dense - slater_condon(h, eri, n_e)) < 1e-12


def test_h2_structure_has_the_papers_15_strings():
    p = S.make_problem(0)
    ham = pauli.jw_hamiltonian(p.h, p.eri)
    with open(os.path.join(GOLDEN, "h2_like_strings.txt")) as f:
        want = {ln.strip() for ln in f if ln.strip() and not ln.startswith("#")}
    assert len(want) == 15
    assert set(ham.labels()) == want


def test_canonical_order_and_batches():
    p = S.make_problem(1)
    ham = pauli.jw_hamiltonian(p.h, p.eri)
    keys = [pauli.sort_key(x, z, ham.n) for x, z in zip(ham.x, ham.z)]
    assert keys == sorted(keys) and len(set(keys)) == len(keys)
    starts = [pauli.support_range(x, z)[0] for x, z in zip(ham.x, ham.z)]
    off = ham.batch_offsets
    for b in range(len(off) - 1):
        assert len(set(starts[off[b]:off[b + 1]])) == 1
        if b > 0:
            assert starts[off[b]] != starts[off[b] - 1]
    assert 500 <= len(ham) <= 700          # ~600 strings at n = 12


def test_merge_is_order_independent():
    p = S.make_problem(1)
    acc = pauli.accumulate_hamiltonian(p.h, p.eri)
    ref = acc.merged()
    rng = random.Random(3)
    for key in list(acc.re)[:200]:
        rng.shuffle(acc.re[key])
    for key in list(acc.im)[:200]:
        rng.shuffle(acc.im[key])
    again = acc.merged()
    assert all(ref[k] == again[k] for k in ref)
