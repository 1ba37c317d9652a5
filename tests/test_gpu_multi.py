"""mps_energy_grad_multi: independent problems of uneven (n, D) evaluated together.

Instances of the 64-problem batch workload (each its own qubit count, bond dimension,
Hamiltonian and a seeded sample of its singles-and-doubles ansatz) must give, through the
concurrent call, exactly the results of one mps_energy_grad_dev call each, on the eager, the
capturing and the replaying calls, with either SVD policy; the small ones are checked against
the oracle.
"""
import numpy as np
import pytest

import synthetic as S
from oracle import ansatz, mps as OM, pauli

pytestmark = pytest.mark.gpu

E_TOL, G_TOL = 1e-10, 1e-9
# batch instances: n8 D16, n12 D32, n12 D64, n16 D64, n20 D64, n16 D128, n24 D256
INSTANCES = (1, 0, 2, 25, 5, 6, 33)
N_SINGLE, N_DOUBLE = 4, 2


@pytest.fixture(scope="module")
def M():
    import torch
    assert torch.cuda.is_available()
    from paper_2211_07983_gb300 import build
    build.build()
    import paper_2211_07983_gb300 as M
    return M


def problem(i):
    p = S.make_problem(3, i)
    excs = S.sampled_excitations(p.excitations, N_SINGLE, N_DOUBLE, S.seed_for(3, 20_000 + i))
    return p, excs, p.theta[: len(excs)]


def build(M, i, one_cta):
    p, excs, th = problem(i)
    x, z, c = M.build_hamiltonian(p.h, p.eri)
    st = M.State.product(p.bits, p.spec.D, p.spec.eps)
    st.set_svd_policy(one_cta)
    return st, M.Circuit(p.n, M.compile_excitations(p.n, excs)), th, M.Hamiltonian(p.n, x, z, c)


@pytest.mark.parametrize("one_cta", [True, False])
def test_multi_equals_single_calls(M, one_cta):
    probs = [build(M, i, one_cta) for i in INSTANCES]
    single = [M.energy_grad(st, c, th, h) for st, c, th, h in probs]
    states, circs, thetas, hams = zip(*probs)
    for call in range(3):   # eager, capturing, replaying (per-problem graphs)
        Es, gs = M.energy_grad_multi(list(states), list(circs), list(thetas), list(hams))
        for k, (E1, g1) in enumerate(single):
            assert Es[k] == E1, (INSTANCES[k], call)
            assert np.array_equal(gs[k], g1), (INSTANCES[k], call)


def test_multi_against_oracle(M):
    """The problems with n <= 16 against the oracle's E and dE/dtheta."""
    picked = [i for i in INSTANCES if S.batch_spec(i).n <= 16]
    probs = [build(M, i, True) for i in picked]
    states, circs, thetas, hams = zip(*probs)
    Es, gs = M.energy_grad_multi(list(states), list(circs), list(thetas), list(hams))
    for k, i in enumerate(picked):
        p, excs, th = problem(i)
        ref = OM.energy_grad(OM.init_product(p.bits), ansatz.compile_circuit(p.n, excs), th,
                             pauli.jw_hamiltonian(p.h, p.eri), p.spec.D, p.spec.eps)
        assert abs(Es[k] - ref.E) <= E_TOL * max(1.0, abs(ref.E)), i
        assert np.linalg.norm(gs[k] - ref.grad) <= G_TOL * max(1.0, np.linalg.norm(ref.grad)), i


def test_multi_device_outputs_and_errors(M):
    import torch
    from paper_2211_07983_gb300._lib import MpsError
    probs = [build(M, i, True) for i in INSTANCES[:3]]
    states, circs, thetas, hams = zip(*probs)
    outs = [(torch.zeros(1, dtype=torch.float64, device="cuda"),
             torch.zeros(len(th), dtype=torch.float64, device="cuda")) for th in thetas]
    M.energy_grad_multi(list(states), list(circs), list(thetas), list(hams), outs=outs)
    Es, gs = M.energy_grad_multi(list(states), list(circs), list(thetas), list(hams))
    for k in range(3):
        assert float(outs[k][0][0]) == Es[k]
        assert np.array_equal(outs[k][1].cpu().numpy(), gs[k])
    # the same state twice is rejected before any work
    with pytest.raises(MpsError):
        M.energy_grad_multi([states[0], states[0]], [circs[0]] * 2, [thetas[0]] * 2, [hams[0]] * 2)
    # a bad angle index in one problem is reported, and the others are still waited for
    bad = np.array(thetas[1])[:-1]
    with pytest.raises(MpsError):
        M.energy_grad_multi(list(states), list(circs), [thetas[0], bad, thetas[2]], list(hams))
    Es2, gs2 = M.energy_grad_multi(list(states), list(circs), list(thetas), list(hams))
    assert Es2 == Es
