"""Write tests/golden/config4_prefix.json: the oracle's E and dE/dtheta on a prefix of the
n = 40, D = 256 workload, with the full Hamiltonian.

Only `oracle/` computes (and `synthetic/` supplies the seeded inputs).  The prefix is the first 12
excitations of the pruned list (singles that take the middle bonds to D = 64) followed by five
short-span doubles; together they take bonds 16-18 to 256 or just below, so the 512 x 512 gate
SVDs, truncation by D and the doubles' gate patterns are all exercised, while most bonds stay at
64 and the oracle's per-string energy cotangent stays affordable on a CPU.

    python tests/golden/make_config4_prefix.py      # about an hour on 8 cores
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synthetic as S  # noqa: E402
from oracle import ansatz, mps as OM, pauli  # noqa: E402

# indices into the workload's (pruned, ranked) excitation list
PREFIX = list(range(12)) + [825, 189, 824, 920, 1172]
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "config4_prefix.json")


def main():
    p = S.make_problem(4)
    excs = [p.excitations[t] for t in PREFIX]
    theta = np.array([p.theta[t] for t in PREFIX])
    ham = pauli.jw_hamiltonian(p.h, p.eri)
    gates = ansatz.compile_circuit(p.n, excs)
    t0 = time.time()
    r = OM.energy_grad(OM.init_product(p.bits), gates, theta, ham, p.spec.D, p.spec.eps, checkpoint_every=512)
    dt = time.time() - t0
    out = {"workload": "n40_D256", "prefix": PREFIX, "excitations": [list(e) for e in excs],
           "theta": theta.tolist(), "n_gates": len(gates), "n_strings": len(ham),
           "bond_dims": r.final.bond_dims(), "E": r.E, "grad": r.grad.tolist(),
           "gate_grad": r.gate_grad.tolist(), "oracle_seconds": dt,
           "source": "oracle.mps.energy_grad (checkpoint_every=512)"}
    with open(OUT, "w") as f:
        json.dump(out, f)
    print(f"E = {r.E!r}, |g| = {np.linalg.norm(r.grad):.6e}, max bond {max(r.final.bond_dims())}, "
          f"{len(gates)} gates, {len(ham)} strings, {dt:.0f} s")


if __name__ == "__main__":
    main()
