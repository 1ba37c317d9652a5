"""Multi-rank helpers (one process per GPU).

Two ways the hot path spreads over ranks:

* independent instances (different circuits, states or angles): each rank runs its own, no
  collective on the data path; timings are combined with `max_over_ranks`;
* one instance with its Pauli strings sharded: E and dE/dB* are linear in the string
  coefficients once divided by the common <psi|psi>, so with H = sum_r H_r (H_r = the strings
  of rank r, the identity string on rank 0)
      E = sum_r E_r,   dE/dB* = sum_r [env_{H_r} - E_r env_I] / <psi|psi>,
  and a single sum-allreduce of (E_r, dE_r/dB*) gives the full cotangent.  The gate chain is
  replicated (every rank runs the forward pass), as it is one sequential dependency chain.
"""
from __future__ import annotations

import numpy as np


def _first_last(x: int, z: int):
    s = int(x) | int(z)
    if s == 0:
        return -1, -1
    return (s & -s).bit_length() - 1, s.bit_length() - 1


def shard_terms(x, z, c, world: int):
    """Split strings over `world` ranks: whole first-site batches (they share trie prefixes),
    greedily by estimated sweep cost (the string lengths), the identity string on rank 0.
    Returns one index array per rank."""
    x = np.asarray(x, dtype=np.uint64)
    z = np.asarray(z, dtype=np.uint64)
    batches = {}
    ident = []
    for k in range(len(x)):
        a, b = _first_last(x[k], z[k])
        if a < 0:
            ident.append(k)
            continue
        batches.setdefault(a, []).append((k, b - a + 1))
    load = [0.0] * world
    out = [[] for _ in range(world)]
    out[0].extend(ident)
    for a in sorted(batches, key=lambda q: -sum(w for _, w in batches[q])):
        r = min(range(world), key=lambda q: load[q])
        out[r].extend(k for k, _ in batches[a])
        load[r] += sum(w for _, w in batches[a])
    return [np.array(sorted(o), dtype=np.int64) for o in out]


def energy_grad_sharded(state0, circuit, theta, x, z, c, rank: int, world: int, allreduce=None):
    """E and dE/dtheta of one instance with the strings split over `world` ranks (this is rank
    `rank`): the forward and reverse passes are replicated, each rank sweeps its own strings, and
    one sum-allreduce of (E_r, dE_r/dB*) joins them (mps_energy_grad_shard_begin / _end).

    allreduce(list of tensors) sums in place over the ranks (default: torch.distributed SUM)."""
    from . import api
    idx = shard_terms(x, z, c, world)[rank]
    x, z, c = np.asarray(x), np.asarray(z), np.asarray(c)
    ham = api.Hamiltonian(state0.n, x[idx], z[idx], c[idx])
    E, Bbar = api.energy_grad_shard_begin(state0, circuit, theta, ham)
    (allreduce or allreduce_sum)([E, Bbar])
    n_theta = int(np.asarray(theta).shape[-1]) if not hasattr(theta, "shape") else int(theta.shape[-1])
    g = api.energy_grad_shard_end(state0, circuit, n_theta, Bbar)
    return E, g


def allreduce_sum(values, group=None):
    """Sum a list of torch tensors (or numpy arrays) over all ranks, in place for tensors."""
    import torch
    import torch.distributed as dist
    out = []
    for v in values:
        t = v if isinstance(v, torch.Tensor) else torch.as_tensor(np.asarray(v))
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        out.append(t)
    return out


def max_over_ranks(value: float, device=None, group=None) -> float:
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
