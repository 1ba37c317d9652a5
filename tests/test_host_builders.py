"""The library's native host builders (step S0) against the oracle, and the ABI surface.

CPU only: these entry points do not touch the GPU.
"""
import ctypes

import numpy as np
import pytest

import synthetic as S
from oracle import ansatz, pauli


@pytest.fixture(scope="module")
def lib():
    from paper_2211_07983_gb300 import build, _lib
    build.build()
    return _lib


def test_library_exports_every_header_symbol(lib):
    so = lib.load()
    names = lib.header_symbols()
    assert "mps_energy_grad" in names and "mps_init_product" in names
    for name in names:
        assert hasattr(so, name), name


@pytest.mark.parametrize("cfg", [0, 1, 2])
def test_hamiltonian_bit_exact_with_oracle(lib, cfg):
    import paper_2211_07983_gb300 as M
    p = S.make_problem(cfg)
    x, z, c = M.build_hamiltonian(p.h, p.eri)
    H = pauli.jw_hamiltonian(p.h, p.eri)
    assert list(x) == H.x and list(z) == H.z
    assert np.array_equal(c, H.coeff)          # bit for bit: both are correctly rounded exact sums


@pytest.mark.parametrize("cfg", [0, 1])
def test_gate_list_matches_oracle(lib, cfg):
    import paper_2211_07983_gb300 as M
    p = S.make_problem(cfg)
    g = M.compile_excitations(p.n, p.excitations)
    og = ansatz.compile_circuit(p.n, p.excitations)
    assert len(g) == len(og)
    for a, b in zip(g, og):
        assert int(a["bond"]) == b.bond and int(a["theta_idx"]) == b.theta_idx
        if b.parametric:
            assert int(a["rz_site"]) == b.rz_site and a["theta_scale"] == b.scale
            for fld, arr in (("pre", b.pre), ("post", b.post)):
                assert np.abs(a[fld].view(np.complex128).reshape(4, 4) - arr).max() < 1e-14
        else:
            assert np.abs(a["mat"].view(np.complex128).reshape(4, 4) - b.mat).max() < 1e-14


def test_builders_reject_bad_input(lib):
    import paper_2211_07983_gb300 as M
    from paper_2211_07983_gb300._lib import MpsError
    with pytest.raises(MpsError):
        M.compile_excitations(4, [(0, -1, 9, -1)])          # orbital out of range
    h = np.zeros((2, 2))
    h[0, 1] = 1.0                                           # not symmetric -> non-Hermitian H
    with pytest.raises(MpsError):
        M.build_hamiltonian(h, np.zeros((2, 2, 2, 2)))


def test_capacity_protocol(lib):
    so = lib.load()
    p = S.make_problem(0)
    h = np.ascontiguousarray(p.h)
    e = np.ascontiguousarray(p.eri)
    cnt = ctypes.c_int64(0)
    P = ctypes.POINTER
    code = so.mps_build_hamiltonian(p.n, h.ctypes.data_as(P(ctypes.c_double)), e.ctypes.data_as(P(ctypes.c_double)),
                                    3, None, None, None, ctypes.byref(cnt))
    assert code == 1 and cnt.value == 15
