"""Write tests/golden/config2_doubles.json: the oracle's E and dE/dtheta on a subset of the
n = 20, D = 128, eps = 1e-10 differentiation workload that includes double excitations.

Only `oracle/` computes (and `synthetic/` supplies the seeded inputs).  The subset is sixteen
single excitations with wide spans across the middle of the chain followed by six doubles on the
middle orbitals: 985 gates, bonds 10-12 reach D = 128 and the truncation acts, so the reverse
pass with checkpoint segments of 512 gates crosses a segment boundary.

It also stores the oracle's own rounding spread on this case: the relative change of dE/dtheta
when LAPACK's gesvd driver replaces the default gesdd for every SVD of the same computation.
Gates here keep Schmidt values near 1e-9 s_1, whose SVD adjoint divides by w_k = s_k^2, so two
correct FP64 evaluations differ by about 1e-9 relative.

    python tests/golden/make_config2_doubles.py      # a few minutes on 8 cores
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np
import scipy.linalg as sla

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synthetic as S  # noqa: E402
from oracle import ansatz, mps as OM, pauli  # noqa: E402

# indices into the workload's excitation list (singles first, then doubles, lexicographic)
SUBSET = [24, 29, 23, 28, 34, 39, 22, 27, 33, 38, 44, 49, 21, 26, 32, 37, 755, 756, 760, 761, 764, 768]
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "config2_doubles.json")


def main():
    p = S.make_problem(2)
    excs = [p.excitations[t] for t in SUBSET]
    theta = np.array([p.theta[t] for t in SUBSET])
    ham = pauli.jw_hamiltonian(p.h, p.eri)
    gates = ansatz.compile_circuit(p.n, excs)
    t0 = time.time()
    r = OM.energy_grad(OM.init_product(p.bits), gates, theta, ham, p.spec.D, p.spec.eps, checkpoint_every=512)
    dt = time.time() - t0
    orig = np.linalg.svd
    np.linalg.svd = lambda a, full_matrices=True, compute_uv=True: sla.svd(
        a, full_matrices=full_matrices, compute_uv=compute_uv, lapack_driver="gesvd")
    try:
        alt = OM.energy_grad(OM.init_product(p.bits), gates, theta, ham, p.spec.D, p.spec.eps, checkpoint_every=512)
    finally:
        np.linalg.svd = orig
    spread = float(np.linalg.norm(alt.grad - r.grad) / np.linalg.norm(r.grad))
    out = {"workload": "n20_D128", "subset": SUBSET, "excitations": [list(e) for e in excs],
           "theta": theta.tolist(), "n_gates": len(gates), "n_strings": len(ham),
           "bond_dims": r.final.bond_dims(), "E": r.E, "grad": r.grad.tolist(),
           "gate_grad": r.gate_grad.tolist(), "oracle_seconds": dt, "grad_spread_gesvd": spread,
           "source": "oracle.mps.energy_grad (checkpoint_every=512)"}
    with open(OUT, "w") as f:
        json.dump(out, f)
    print(f"E = {r.E!r}, |g| = {np.linalg.norm(r.grad):.6e}, bonds {r.final.bond_dims()}, {len(gates)} gates, "
          f"{dt:.0f} s, gesvd spread {spread:.2e}")


if __name__ == "__main__":
    main()
