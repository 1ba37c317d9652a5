"""Study: the paper's Algorithm 1 with m Hamiltonian groups under truncation (Sec. 4, Eq. meanerror).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): it runs the oracle alone.

On a small seeded problem (n = 8, 4 electrons, the first 12 singles-and-doubles excitations; the
exact state needs D = 16), for bond dimensions D that truncate and for m = 1, 2, 4, 8, ..., N_h
groups (N_h = the number of Pauli strings), it prints
  R_AD    = |g_BP - g_AD| / |g_AD|: Algorithm 1 against the exact derivative of the truncated
            forward pass (the hot path's gradient), the paper's relative error R;
  R_exact = |g_BP - g_exact| / |g_exact|: against the gradient of the untruncated circuit;
  the discarded weight 1 - <psi|psi> of the truncated forward pass, and the oracle's seconds.
Each group's H^j|psi> is compressed to D, so more groups mean fewer strings per compression.

    python oracle/alg1_grouping_study.py
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import synthetic as S  # noqa: E402
from oracle import alg1, ansatz, mps as M, pauli, statevector as SV  # noqa: E402


def problem(n=8, n_e=4, n_exc=12, seed_cfg=90):
    spec = S.ConfigSpec(f"n{n}_study", n=n, n_e=n_e, D=64, eps=1e-12, decay=2.0)
    p = S.make_problem(seed_cfg, spec=spec)
    excs = p.excitations[:n_exc]
    return p, ansatz.compile_circuit(n, excs), p.theta[: len(excs)], pauli.jw_hamiltonian(p.h, p.eri)


def main():
    p, gates, th, ham = problem()
    nh = len(ham)
    _, g_exact, _ = SV.gradient(p.bits, gates, th, ham)
    ms = sorted({1, 2, 4, 8, 16, 32, nh} - {m for m in (16, 32) if m >= nh})
    print(f"n = {p.n}, {len(gates)} gates, N_h = {nh} strings; |g_exact| = {np.linalg.norm(g_exact):.4f}")
    print("| D | discarded weight | m | N_h/m | R_AD | R_exact | s |")
    print("|---|---|---|---|---|---|---|")
    for D in (8, 12):
        eps = 1e-10
        final = M.apply_circuit(M.init_product(p.bits), gates, th, D, eps)
        dw = 1.0 - float(np.real(np.vdot(M.to_dense(final), M.to_dense(final))))
        g_ad = M.energy_grad(M.init_product(p.bits), gates, th, ham, D, eps).grad
        for m in ms:
            t0 = time.perf_counter()
            g_bp, _ = alg1.gradient(final, gates, th, ham, D, eps, m=m)
            dt = time.perf_counter() - t0
            r_ad = np.linalg.norm(g_bp - g_ad) / np.linalg.norm(g_ad)
            r_ex = np.linalg.norm(g_bp - g_exact) / np.linalg.norm(g_exact)
            print(f"| {D} | {dw:.2e} | {m} | {nh / m:.1f} | {r_ad:.3f} | {r_ex:.3f} | {dt:.1f} |", flush=True)
        print(f"| {D} | | (g_AD) | | 0 | {np.linalg.norm(g_ad - g_exact) / np.linalg.norm(g_exact):.3f} | |")


if __name__ == "__main__":
    main()
