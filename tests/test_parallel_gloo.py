"""Multi-rank paths on CPU with the gloo backend, world size 2.

* string sharding: per-rank E_r and dE_r/dB* summed by all_reduce equal the full energy and
  cotangent (per-rank values computed by the oracle, the reduction by the library's helpers);
* the timing combiner takes the maximum over ranks.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import synthetic as S
        from oracle import ansatz, mps as OM, pauli
        from paper_2211_07983_gb300 import parallel
        p = S.make_problem(90, spec=S.ConfigSpec("n8", n=8, n_e=4, D=4, eps=1e-10, decay=2.0))
        ham = pauli.jw_hamiltonian(p.h, p.eri)
        gates = ansatz.compile_circuit(p.n, p.excitations[:10])
        m = OM.apply_circuit(OM.init_product(p.bits), gates, p.theta[:10], 4, 1e-10)
        shards = parallel.shard_terms(ham.x, ham.z, ham.coeff, world)
        mine = shards[rank]
        sub = pauli.PauliHamiltonian(ham.n, [ham.x[k] for k in mine], [ham.z[k] for k in mine],
                                     ham.coeff[mine])
        Er, Bbar_r = OM.energy_seed(m, sub)
        flat = torch.tensor(np.concatenate([b.ravel() for b in Bbar_r]).view(np.float64))
        E_t = torch.tensor([Er], dtype=torch.float64)
        parallel.allreduce_sum([E_t, flat])
        t_max = parallel.max_over_ranks(1.0 + rank)
        if rank == 0:
            E, Bbar = OM.energy_seed(m, ham)
            full = np.concatenate([b.ravel() for b in Bbar]).view(np.float64)
            q.put((abs(E_t.item() - E), float(np.abs(flat.numpy() - full).max()), t_max,
                   sorted(np.concatenate(shards).tolist()) == list(range(len(ham)))))
    finally:
        dist.destroy_process_group()


def test_string_sharding_and_timing_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(timeout=300)
    assert all(pr.exitcode == 0 for pr in procs)
    dE, dB, t_max, covers = q.get(timeout=10)
    assert covers
    assert dE < 1e-13
    assert dB < 1e-13
    assert t_max == 2.0


def test_shard_terms_balances_and_keeps_batches_whole():
    import synthetic as S
    from oracle import pauli
    from paper_2211_07983_gb300 import parallel
    p = S.make_problem(1)
    ham = pauli.jw_hamiltonian(p.h, p.eri)
    shards = parallel.shard_terms(ham.x, ham.z, ham.coeff, 3)
    assert sorted(np.concatenate(shards).tolist()) == list(range(len(ham)))
    firsts = [{pauli.support_range(ham.x[k], ham.z[k])[0] for k in sh} - {-1} for sh in shards]
    for i in range(3):
        for j in range(i + 1, 3):
            assert not (firsts[i] & firsts[j])


def _worker_sharded(rank, world, port, q):
    """parallel.energy_grad_sharded over gloo ranks, with the library's two halves replaced by the
    oracle: begin -> (E_r, dE_r/dB*) of the shard's strings, end -> returns the cotangent it was
    given, so that rank 0 can check the allreduced cotangent against the unsharded one."""
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import synthetic as S
        from oracle import ansatz, mps as OM, pauli
        from paper_2211_07983_gb300 import api, parallel
        p = S.make_problem(90, spec=S.ConfigSpec("n8", n=8, n_e=4, D=4, eps=1e-10, decay=2.0))
        ham = pauli.jw_hamiltonian(p.h, p.eri)
        gates = ansatz.compile_circuit(p.n, p.excitations[:10])
        m = OM.apply_circuit(OM.init_product(p.bits), gates, p.theta[:10], 4, 1e-10)

        class FakeHam:
            def __init__(self, n, x, z, c):
                self.h = pauli.PauliHamiltonian(n, [int(v) for v in x], [int(v) for v in z], np.asarray(c))

        def begin(state0, circuit, theta, h):
            E, Bbar = OM.energy_seed(m, h.h)
            return (torch.tensor([E], dtype=torch.float64),
                    torch.tensor(np.concatenate([b.ravel() for b in Bbar]).view(np.float64)))

        api.Hamiltonian = FakeHam
        api.energy_grad_shard_begin = begin
        api.energy_grad_shard_end = lambda state0, circuit, n_theta, Bbar: Bbar.numpy().copy()
        state = type("St", (), {"n": p.n, "n_inst": 1})()
        E, g = parallel.energy_grad_sharded(state, None, p.theta[:10], np.array(ham.x, dtype=np.uint64),
                                            np.array(ham.z, dtype=np.uint64), ham.coeff, rank, world)
        if rank == 0:
            E_full, B_full = OM.energy_seed(m, ham)
            full = np.concatenate([b.ravel() for b in B_full]).view(np.float64)
            q.put((abs(E.item() - E_full), float(np.abs(g - full).max())))
    finally:
        dist.destroy_process_group()


def test_sharded_energy_grad_orchestration_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_sharded, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(timeout=300)
    assert all(pr.exitcode == 0 for pr in procs)
    dE, dB = q.get(timeout=10)
    assert dE < 1e-13 and dB < 1e-13
