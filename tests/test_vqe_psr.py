"""The variational loop (Sec. 5) and the parameter-shift baseline (Sec. 4, Eq. psr).

CPU: the loop's stopping rules on known functions, and the per-gate angle slots of the
parameter-shift circuit.  GPU: parameter shift through the library equals the adjoint gradient
when nothing is truncated; the loop on the n = 4 workload reaches a stationary point that
respects the variational bound of the exact ground energy in its particle-number sector.
"""
import numpy as np
import pytest

import synthetic as S


def test_minimize_stops_on_the_gradient_rule_for_a_quadratic():
    import torch
    from paper_2211_07983_gb300 import vqe
    A = torch.tensor([[3.0, 0.5, 0.0], [0.5, 2.0, 0.3], [0.0, 0.3, 1.0]], dtype=torch.float64)
    b = torch.tensor([1.0, -2.0, 0.5], dtype=torch.float64)
    f = lambda x: 0.5 * x @ A @ x - b @ x
    r = vqe.minimize(f, np.zeros(3), method="lbfgs")
    x_star = torch.linalg.solve(A, b)
    assert r.reason in ("gradient", "energy") and r.iterations <= 5
    assert torch.allclose(r.theta, x_star, atol=1e-6)
    assert r.grad_norm < 1e-5 or abs(r.history[-1][0] - r.history[-2][0]) < 1e-6


def test_minimize_stops_on_the_energy_rule_and_on_the_iteration_cap():
    import torch
    from paper_2211_07983_gb300 import vqe
    f = lambda x: (x ** 2).sum()
    r = vqe.minimize(f, np.ones(4), method="adam", lr=0.05, max_iter=1000, e_tol=1e-6, g_tol=1e-12)
    assert r.reason == "energy"
    assert abs(r.history[-1][0] - r.history[-2][0]) < 1e-6
    r2 = vqe.minimize(f, np.ones(4), method="adam", lr=1e-4, max_iter=7, e_tol=0.0, g_tol=0.0)
    assert r2.reason == "iterations" and r2.iterations == 7 and len(r2.history) == 7
    with pytest.raises(ValueError):
        vqe.minimize(f, np.ones(2), method="sgd")


def test_parameter_shift_circuit_gives_every_rz_gate_its_own_slot():
    from paper_2211_07983_gb300 import psr
    from paper_2211_07983_gb300._lib import GATE_DTYPE
    g = np.zeros(5, dtype=GATE_DTYPE)
    g["theta_idx"] = [-1, 0, 1, 0, -1]
    g["theta_scale"] = [0.0, 0.5, -2.0, 0.25, 0.0]
    theta = np.array([0.3, -1.1])
    g1, phi0, par = psr.per_gate_circuit(g, theta)
    assert list(par) == [1, 2, 3]
    assert np.allclose(phi0, [0.15, 2.2, 0.075])
    assert list(g1["theta_idx"]) == [-1, 0, 1, 2, -1] and list(g1["theta_scale"][par]) == [1.0, 1.0, 1.0]
    assert list(g["theta_idx"]) == [-1, 0, 1, 0, -1]          # the input is not modified


@pytest.mark.gpu
@pytest.mark.parametrize("case", ["cfg0", "n8"])
def test_parameter_shift_equals_the_adjoint_without_truncation(case):
    import torch
    assert torch.cuda.is_available()
    from paper_2211_07983_gb300 import build
    build.build()
    import paper_2211_07983_gb300 as M
    from paper_2211_07983_gb300 import psr
    if case == "cfg0":
        p = S.make_problem(0)
    else:
        p = S.make_problem(90, spec=S.ConfigSpec("n8_D64", n=8, n_e=4, D=64, eps=1e-12, decay=2.0))
    x, z, c = M.build_hamiltonian(p.h, p.eri)
    gates = M.compile_excitations(p.n, p.excitations)
    ham = M.Hamiltonian(p.n, x, z, c)
    st = M.State.product(p.bits, p.spec.D, p.spec.eps)
    E, g, gg = M.energy_grad(st, M.Circuit(p.n, gates), p.theta, ham, gate_grad=True)
    gp, ggp, n_eval, _ = psr.parameter_shift(p.n, p.bits, gates, p.theta, ham, p.spec.D, p.spec.eps, batch=64)
    assert n_eval == 2 * int(np.count_nonzero(gates["theta_idx"] >= 0))
    assert np.abs(ggp - gg).max() <= 1e-9 * max(1.0, np.abs(gg).max())
    assert np.linalg.norm(gp - g) <= 1e-9 * max(1.0, np.linalg.norm(g))


@pytest.mark.gpu
def test_vqe_loop_on_the_n4_workload_respects_the_variational_bound():
    import torch
    assert torch.cuda.is_available()
    from paper_2211_07983_gb300 import build
    build.build()
    import paper_2211_07983_gb300 as M
    from paper_2211_07983_gb300 import vqe
    from oracle import fermion, pauli
    p = S.make_problem(0)
    x, z, c = M.build_hamiltonian(p.h, p.eri)
    circ = M.Circuit(p.n, M.compile_excitations(p.n, p.excitations))
    ham = M.Hamiltonian(p.n, x, z, c)
    st = M.State.product(p.bits, p.spec.D, p.spec.eps)
    f = vqe.mps_objective(st, circ, ham)
    E_hf = float(f(torch.zeros(len(p.theta), dtype=torch.float64, device="cuda")))
    r = vqe.minimize(f, np.full(len(p.theta), 0.1), method="lbfgs", device="cuda")
    assert r.reason in ("gradient", "energy"), r.reason
    # exact ground energy in the sector of the reference state: n_e electrons, S_z = 0
    H = pauli.hamiltonian_dense(pauli.jw_hamiltonian(p.h, p.eri)).real
    N = np.diag(fermion.number_operator(p.n))
    Sz = np.diag(fermion.sz_operator(p.n))
    sector = np.flatnonzero((np.abs(N - p.spec.n_e) < 1e-9) & (np.abs(Sz) < 1e-9))
    E_exact = np.linalg.eigvalsh(H[np.ix_(sector, sector)])[0]
    assert r.energy <= E_hf + 1e-12
    assert r.energy >= E_exact - 1e-9
    energies = [e for e, _ in r.history]
    assert all(b <= a + 1e-9 for a, b in zip(energies, energies[1:]))   # line-search steps never go up
