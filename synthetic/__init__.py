"""Seeded synthetic inputs shaped like the paper's molecular problems.

This module is the one place that both the CPU oracle and the GPU library's
tests/benchmarks draw their inputs from.  It holds *no* arithmetic of the
simulation method itself (no Jordan-Wigner transform, no circuit compilation,
no MPS algebra): it only produces

* one- and two-electron integrals h_pq and (pq|rs) in a spin-orbital basis
  (the inputs of the second-quantised Hamiltonian, Sec. 2, Eq. ham-pbc),
* the list of spin-conserving single/double excitations that defines a UCCSD
  ansatz (Sec. 2, Eq. uccansatz and the cluster operator T below it),
* the Hartree-Fock occupation bits (Sec. 3, Eq. hf) and
* variational angles theta ~ U(-pi, pi).

The paper's molecules (PySCF integrals, Table tab:info / tab:large) are not
available; these random integrals stand in for them with the same shapes:
qubit counts, electron counts, Pauli-string counts and excitation counts.

Conventions
-----------
* spin-orbital p = 2*P + sigma (interleaved: even = alpha, odd = beta),
* chemist notation (pq|rs), real orbitals, 8-fold permutational symmetry,
* HF reference = the first n_e spin-orbitals occupied (bits 1...10...0).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 221107983


def seed_for(config: int, instance: int = 0) -> int:
    """Seed of one problem instance: base + 1000*config + instance."""
    return SEED_BASE + 1000 * config + instance


@dataclass
class ConfigSpec:
    """Shape parameters of one synthetic workload."""
    name: str
    n: int                      # qubits = spin orbitals
    n_e: int                    # electrons
    D: int                      # maximal bond dimension
    eps: float                  # relative singular-value cutoff
    tau: float = 0.0            # two-electron integrals with |v| < tau are zeroed
    decay: float | None = None  # (PQ|RS) *= exp(-|P-R|/decay) (spatial indices)
    z2_parity: bool = False     # H2-like orbital parity selection rule
    keep: int | None = None     # keep the `keep` largest-scored excitations
    note: str = ""


# The five workloads.  tau values were chosen once (by counting the merged
# Jordan-Wigner strings with the oracle) so that N_h lands near the target
# string counts of the workloads: ~15, ~600, ~2.5k, ~20k.
CONFIGS: dict[int, ConfigSpec] = {
    0: ConfigSpec("n4_D16", n=4, n_e=2, D=16, eps=1e-12, z2_parity=True,
                  note="H2-like, exact (no truncation)"),
    1: ConfigSpec("n12_D64", n=12, n_e=6, D=64, eps=1e-12, tau=0.065, decay=2.0,
                  note="exact: maximal bond dimension 2^6 = 64"),
    2: ConfigSpec("n20_D128", n=20, n_e=10, D=128, eps=1e-10, tau=0.068, decay=2.0),
    4: ConfigSpec("n40_D256", n=40, n_e=20, D=256, eps=1e-10, tau=0.067, decay=2.0,
                  keep=2000),
}

# config 3: 64 independent instances of uneven size
BATCH_NS = (8, 12, 16, 20, 24, 28)
BATCH_DS = (32, 64, 128, 256)
BATCH_TAU = {8: 0.0, 12: 0.065, 16: 0.066, 20: 0.068, 24: 0.068, 28: 0.07}


def batch_spec(instance: int) -> ConfigSpec:
    """Shape of instance `instance` of the 64-instance batch workload."""
    rng = np.random.Generator(np.random.PCG64(seed_for(3, 10_000 + instance)))
    n = int(rng.choice(BATCH_NS))
    D = int(rng.choice(BATCH_DS))
    D = min(D, 2 ** (n // 2))
    return ConfigSpec(f"batch{instance}_n{n}_D{D}", n=n, n_e=n // 2, D=D, eps=1e-10,
                      tau=BATCH_TAU[n], decay=2.0)


def spatial_integrals(nS: int, rng: np.random.Generator, *, decay=None, tau=0.0,
                      z2_parity=False):
    """Random real symmetric h_PQ ~ N(0,1) and 8-fold symmetric (PQ|RS) ~ N(0, 0.1^2).

    One value is drawn per 8-fold orbit and written to all of its images, so the
    symmetry is exact.  The distance decay and the sparsification are applied to
    the orbit's canonical representative (P>=Q, R>=S, PQ>=RS), so every image of
    an orbit shares one value.
    """
    h = np.zeros((nS, nS))
    for P in range(nS):
        for Q in range(P, nS):
            v = rng.standard_normal()
            h[P, Q] = h[Q, P] = v
    eri = np.zeros((nS, nS, nS, nS))
    pairs = [(P, Q) for P in range(nS) for Q in range(P + 1)]
    for ia, (P, Q) in enumerate(pairs):
        for (R, S) in pairs[: ia + 1]:
            v = 0.1 * rng.standard_normal()
            if decay is not None:
                v *= math.exp(-abs(P - R) / decay)
            if abs(v) < tau:
                v = 0.0
            if z2_parity and (P + Q + R + S) % 2 == 1:
                v = 0.0
            for (a, b, c, d) in ((P, Q, R, S), (Q, P, R, S), (P, Q, S, R), (Q, P, S, R),
                                 (R, S, P, Q), (S, R, P, Q), (R, S, Q, P), (S, R, Q, P)):
                eri[a, b, c, d] = v
    if z2_parity:
        for P in range(nS):
            for Q in range(nS):
                if (P + Q) % 2 == 1:
                    h[P, Q] = 0.0
    return h, eri


def spin_orbital_integrals(h: np.ndarray, eri: np.ndarray):
    """Expand spatial integrals to spin orbitals p = 2P + sigma (spin-conserving)."""
    nS = h.shape[0]
    n = 2 * nS
    sp = np.arange(n) // 2
    sg = np.arange(n) % 2
    same = (sg[:, None] == sg[None, :]).astype(float)
    hs = h[np.ix_(sp, sp)] * same
    es = eri[np.ix_(sp, sp, sp, sp)] * same[:, :, None, None] * same[None, None, :, :]
    return np.ascontiguousarray(hs), np.ascontiguousarray(es)


def sd_excitations(n: int, n_e: int):
    """Spin-conserving singles then doubles, lexicographic.

    Each excitation is (i, j, a, b) with occupied i<j and virtual a<b; a single
    excitation i->a is stored as (i, -1, a, -1).
    """
    occ = range(n_e)
    vir = range(n_e, n)
    out = []
    for i in occ:
        for a in vir:
            if i % 2 == a % 2:
                out.append((i, -1, a, -1))
    for i in occ:
        for j in occ:
            if j <= i:
                continue
            for a in vir:
                for b in vir:
                    if b <= a:
                        continue
                    if (i % 2) + (j % 2) == (a % 2) + (b % 2):
                        out.append((i, j, a, b))
    return out


def sampled_excitations(excs, n_single: int, n_double: int, seed: int):
    """A seeded random choice of n_single singles and n_double doubles of `excs`, kept in list
    order (singles first): the reduced circuit of a batch instance."""
    rng = np.random.Generator(np.random.PCG64(seed))
    singles = [e for e in excs if e[1] < 0]
    doubles = [e for e in excs if e[1] >= 0]
    ps = np.sort(rng.choice(len(singles), size=min(n_single, len(singles)), replace=False))
    pd = np.sort(rng.choice(len(doubles), size=min(n_double, len(doubles)), replace=False))
    return [singles[t] for t in ps] + [doubles[t] for t in pd]


def mp2_like_scores(excs, hs, es):
    """Score |(ia|jb) - (ib|ja)| / max(|e_a + e_b - e_i - e_j|, 0.1), e_p = h_pp.

    A single i->a is scored |h_ia| / max(|e_a - e_i|, 0.1).
    """
    e = np.diag(hs)
    sc = []
    for (i, j, a, b) in excs:
        if j < 0:
            sc.append(abs(hs[i, a]) / max(abs(e[a] - e[i]), 0.1))
        else:
            num = abs(es[i, a, j, b] - es[i, b, j, a])
            sc.append(num / max(abs(e[a] + e[b] - e[i] - e[j]), 0.1))
    return np.array(sc)


def prune(excs, hs, es, keep: int):
    """Keep the `keep` highest-scoring excitations, ordered by rank (ties: index order)."""
    sc = mp2_like_scores(excs, hs, es)
    order = sorted(range(len(excs)), key=lambda t: (-sc[t], excs[t]))
    return [excs[t] for t in order[:keep]]


@dataclass
class Problem:
    """One synthetic VQE problem: Hamiltonian integrals, ansatz and angles."""
    spec: ConfigSpec
    seed: int
    h: np.ndarray           # (n, n) spin-orbital one-electron integrals
    eri: np.ndarray         # (n, n, n, n) spin-orbital (pq|rs)
    bits: np.ndarray        # (n,) uint8 HF occupation
    excitations: list = field(default_factory=list)
    theta: np.ndarray = None

    @property
    def n(self):
        return self.spec.n


def make_problem(config: int, instance: int = 0, spec: ConfigSpec | None = None) -> Problem:
    """Build the seeded problem of a workload (config 3 = batch instance `instance`)."""
    if spec is None:
        spec = batch_spec(instance) if config == 3 else CONFIGS[config]
    seed = seed_for(config, instance)
    rng = np.random.Generator(np.random.PCG64(seed))
    hS, eS = spatial_integrals(spec.n // 2, rng, decay=spec.decay, tau=spec.tau,
                               z2_parity=spec.z2_parity)
    hs, es = spin_orbital_integrals(hS, eS)
    excs = sd_excitations(spec.n, spec.n_e)
    if spec.keep is not None and spec.keep < len(excs):
        excs = prune(excs, hs, es, spec.keep)
    theta = rng.uniform(-math.pi, math.pi, size=len(excs))
    bits = np.zeros(spec.n, dtype=np.uint8)
    bits[: spec.n_e] = 1
    return Problem(spec=spec, seed=seed, h=hs, eri=es, bits=bits, excitations=excs,
                   theta=theta)


def random_theta(seed: int, m: int) -> np.ndarray:
    """Angles ~ U(-pi, pi) from their own seeded generator."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-math.pi, math.pi, size=m)
