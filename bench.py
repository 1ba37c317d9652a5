#!/usr/bin/env python3
"""Energy + gradient evaluations per second of the differentiable-MPS VQE hot path on GB300.

One step = one full evaluation of E(theta) and dE/dtheta (forward gates with truncated SVDs,
trie-shared Pauli sweeps, energy cotangent, exact reverse pass) for each of B independent
instances of the workload.  The instances live in one batched state: every kernel launch of
the evaluation serves all B of them (the gate SVD runs one CTA per instance, so B = 152 fills
the GPU), on one stream, replayed as one CUDA graph.  `value` = instances / device time of a
step, summed over ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--instances B] [--impl ours|reference]

Under torchrun every rank runs its own B instances on its own GPU (weak scaling; no data-path
collective: the instances are independent problems).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthetic as S  # noqa: E402

METRIC = "energy+gradient evals/s at n=40,D=256; Pauli-term expectations/s vs roofline"
WORKLOADS = {
    # name: (config, excitation prefix or None)
    "n12_D64": (1, None),
    "n4_D16": (0, None),
    # prefixes of the n12_D64 circuit (same shapes; used for profiler captures)
    "n12_D64_p10": (1, 10),
    "n12_D64_p40": (1, 40),
}
# Per-SM ALU peaks used for the single-CTA SVD kernel (recipe nominal figures, per SM):
# FP64 1.25 TFLOP/s / 152 SMs; FP32 152 SMs x 128 FMA/clk x 2 x 2.07 GHz = 80.5 TFLOP/s / 152.
N_SM = 152
P64_SM = 1.25e12 / N_SM
P32_SM = 128 * 2 * 2.07e9


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--instances", type=int, default=152)
    ap.add_argument("--workload", default="n12_D64", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision comparison")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---- clocks sampled during the timed region -------------------------------------------------
class ClockSampler:
    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        fd, self.path = tempfile.mkstemp(prefix=f"clocks_rank{gpu_index}_", suffix=".csv")
        os.close(fd)

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        try:
            return self._read()
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass

    def _read(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---- oracle baseline ------------------------------------------------------------------------
def _cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


def oracle_full(cfg: int):
    """Time the oracle's whole E+gradient evaluation of one instance of the workload."""
    from oracle import ansatz, mps as OM, pauli
    p = S.make_problem(cfg)
    ham = pauli.jw_hamiltonian(p.h, p.eri)
    gates = ansatz.compile_circuit(p.n, p.excitations)
    t0 = time.perf_counter()
    OM.energy_grad(OM.init_product(p.bits), gates, p.theta, ham, p.spec.D, p.spec.eps)
    dt = time.perf_counter() - t0
    return {"value": 1.0 / dt, "unit": "evals/s", "cores": _cores(), "kind": "oracle",
            "sample": f"one full oracle E+grad evaluation of the workload ({len(gates)} gates, {len(ham)} strings, "
                      f"one instance) took {dt:.2f} s, timed end to end"}


def oracle_sample(cfg: int, n_exc: int = 40):
    """Time the oracle's E+gradient on a prefix of the workload's circuit (full Hamiltonian)."""
    from oracle import ansatz, mps as OM, pauli
    p = S.make_problem(cfg)
    ham = pauli.jw_hamiltonian(p.h, p.eri)
    full = ansatz.compile_circuit(p.n, p.excitations)
    excs = p.excitations[:n_exc]
    gates = ansatz.compile_circuit(p.n, excs)
    t0 = time.perf_counter()
    OM.energy_grad(OM.init_product(p.bits), gates, p.theta[: len(excs)], ham, p.spec.D, p.spec.eps)
    dt = time.perf_counter() - t0
    # evaluation time scales with the gate count (the sweeps and reverse pass are per gate)
    t_full = dt * len(full) / len(gates)
    return {"value": 1.0 / t_full, "unit": "evals/s", "cores": _cores(), "kind": "oracle",
            "sample": f"oracle E+grad on the first {len(excs)} excitations ({len(gates)} of {len(full)} gates, "
                      f"all {len(ham)} strings) took {dt:.2f} s; scaled by gate count to the full circuit "
                      f"({t_full:.1f} s per evaluation)"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    cfg, _ = WORKLOADS[args.workload]
    t0 = time.perf_counter()
    vals = []
    for _ in range(args.warmup + args.steps):
        vals.append(oracle_sample(cfg, n_exc=40))
    base = vals[-1]
    tot = [1.0 / v["value"] for v in vals[args.warmup:]]
    val = args.steps / sum(tot)
    line = {"metric": METRIC, "value": val, "unit": "evals/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(tot) / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": f"{args.workload} (one instance, oracle on host cores)"},
            "cpu_baseline": {"value": val, "unit": "evals/s", "cores": base["cores"], "kind": "oracle",
                             "sample": base["sample"]},
            "e2e": {"value": val, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t0}
    print(json.dumps(line), flush=True)


# ---- our implementation ---------------------------------------------------------------------
def run_ours(args, rank, world, local):
    import torch
    import paper_2211_07983_gb300 as M
    from paper_2211_07983_gb300 import build

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    cfg, n_exc = WORKLOADS[args.workload]
    p = S.make_problem(cfg)
    excs = p.excitations if n_exc is None else p.excitations[:n_exc]
    x, z, c = M.build_hamiltonian(p.h, p.eri)
    gates = M.compile_excitations(p.n, excs)
    circ = M.Circuit(p.n, gates)
    ham = M.Hamiltonian(p.n, x, z, c)
    B = args.instances
    n_theta = len(excs)
    stream = torch.cuda.Stream()
    state = M.State.product_batch(np.stack([p.bits] * B), p.spec.D, p.spec.eps, checkpoint_every=0,
                                  stream=stream)
    # per-instance angles: the workload's theta for instance 0, fresh seeded angles for the others
    thetas_h = np.ascontiguousarray(np.stack(
        [p.theta[:n_theta] if i == 0 else S.random_theta(S.seed_for(1, 500 + 1000 * rank + i), n_theta)
         for i in range(B)]))
    with torch.cuda.stream(stream):
        thetas_d = torch.tensor(thetas_h, dtype=torch.float64, device="cuda")
        E_d = torch.zeros(B, dtype=torch.float64, device="cuda")
        g_d = torch.zeros((B, n_theta), dtype=torch.float64, device="cuda")
        flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # 512 MB > L2
    torch.cuda.synchronize()

    def sync_all():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
            torch.cuda.synchronize()

    # SVD launches are bracketed by CUDA events on the state's stream (captured into the graph)
    state.profile(True)
    # warm-up: the first call runs eagerly, the second captures the whole evaluation as a CUDA
    # graph, later calls replay it
    for _ in range(args.warmup):
        M.energy_grad(state, circ, thetas_d, ham, out=(E_d, g_d))
    state.profile_read()          # reset the counters
    clocks = ClockSampler(local)
    launches0 = M.kernel_launches()
    sync_all()
    clocks.start()
    dev_ms = 0.0
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)                   # L2 flush between timed steps
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        M.energy_grad(state, circ, thetas_d, ham, out=(E_d, g_d))
        e1.record(stream)
        e1.synchronize()
        dev_ms += e0.elapsed_time(e1)
    sync_all()
    clk = clocks.stop()
    launches = M.kernel_launches() - launches0
    prof = state.profile_read()
    t_step = dev_ms / 1e3 / args.steps
    if world > 1:
        import torch.distributed as dist
        tt = torch.tensor([t_step], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_step = float(tt.item())
    value = B * world / t_step
    # ---- end to end: host angles in, host E and gradient out, through the public API ----
    e2e = None
    if not args.no_e2e:
        sync_all()
        walls = []
        for _ in range(max(1, min(args.steps, 2))):
            t0 = time.perf_counter()
            M.energy_grad(state, circ, thetas_h, ham)
            walls.append(time.perf_counter() - t0)
        t_e2e = sum(walls) / len(walls)
        if world > 1:
            import torch.distributed as dist
            tt = torch.tensor([t_e2e], dtype=torch.float64, device="cuda")
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            t_e2e = float(tt.item())
        e2e = {"value": B * world / t_e2e, "unit": "evals/s", "h2d_bytes_per_step": 8 * n_theta * B,
               "d2h_bytes_per_step": 8 * (1 + n_theta) * B}
    # ---- Pauli-term expectations per second on the final states (energy pass alone) ----
    st_f = state.clone()
    M.apply_circuit(st_f, circ, thetas_d)
    M.energy(st_f, ham)                                  # builds the sweep plan
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    n_rep = 3
    for _ in range(n_rep):
        M.energy(st_f, ham)
    t_energy = (time.perf_counter() - t0) / n_rep
    terms_per_s = len(x) * B / t_energy
    st_f.free()
    # algorithmic work of one energy pass (per instance): every transfer step of the sweep trie
    # and of the two identity chains costs 2 Dl Dr (Dl + Dr) complex MACs at the bond caps
    cap = [min(2 ** min(i, p.n - i), p.spec.D) for i in range(p.n + 1)]
    nodes = set()
    for xm, zm in zip(x.tolist(), z.tolist()):
        sup = xm | zm
        if not sup:
            continue
        a, b = (sup & -sup).bit_length() - 1, sup.bit_length() - 1
        sym = tuple((((xm >> q) & 1) | (((zm >> q) & 1) << 1)) for q in range(a, b + 1))
        for e in range(1, len(sym) + 1):
            nodes.add((a, sym[:e]))
    step_mac = lambda site: 2 * cap[site] * cap[site + 1] * (cap[site] + cap[site + 1])
    mac = sum(step_mac(a + len(sym) - 1) for a, sym in nodes) + 2 * sum(step_mac(q) for q in range(p.n))
    energy_flops = 8.0 * mac * B
    energy_roof = {"bound": "alu", "achieved": energy_flops / t_energy / 1e12, "peak": P64_SM * N_SM / 1e12,
                   "unit": "TFLOP/s", "frac": energy_flops / t_energy / (P64_SM * N_SM),
                   "work": f"{len(nodes)} trie nodes + 2 x {p.n} identity steps per instance, "
                           "2 Dl Dr (Dl + Dr) complex MACs each at the bond caps; host-clock time of the "
                           "whole energy call"}
    # ---- the mixed-precision path on the same instances (3xTF32 contractions and sweeps) ----
    mixed = None
    if not args.no_mixed:
        E64, g64 = E_d.cpu().numpy().copy(), g_d.cpu().numpy().copy()
        state.free()
        torch.cuda.synchronize()
        st_m = M.State.product_batch(np.stack([p.bits] * B), p.spec.D, p.spec.eps, checkpoint_every=0,
                                     stream=stream, precision="mixed")
        for _ in range(2):                      # eager, then captured
            M.energy_grad(st_m, circ, thetas_d, ham, out=(E_d, g_d))
        torch.cuda.synchronize()
        ms_m = 0.0
        n_m = max(5, min(args.steps, 5))        # five timed steps
        for _ in range(n_m):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            M.energy_grad(st_m, circ, thetas_d, ham, out=(E_d, g_d))
            e1.record(stream)
            e1.synchronize()
            ms_m += e0.elapsed_time(e1)
        Em, gm = E_d.cpu().numpy(), g_d.cpu().numpy()
        t_m = ms_m / 1e3 / n_m
        g_rel = np.linalg.norm(gm - g64, axis=1) / np.maximum(1.0, np.linalg.norm(g64, axis=1))
        mixed = {"value": B * world / t_m, "unit": "evals/s", "ms_per_step": 1e3 * t_m,
                 "speedup_vs_fp64": t_step / t_m,
                 "max_rel_E_err_vs_fp64": float(np.max(np.abs(Em - E64) / np.maximum(1.0, np.abs(E64)))),
                 "rel_grad_err_vs_fp64": {"median": float(np.median(g_rel)),
                                          "p90": float(np.percentile(g_rel, 90)), "max": float(g_rel.max()),
                                          "fraction_within_1e-5": float(np.mean(g_rel <= 1e-5))},
                 "grad_note": "large differences come from rare ill-conditioned instances that keep Schmidt "
                              "values just above eps",
                 "precision": "energy Pauli sweeps and recomputed two-site tensors in 3xTF32 on tensor cores "
                              "(mma.sync, FP32 accumulation); gate contractions, energy cotangent, SVD, SVD "
                              "adjoint, sums FP64"}
        st_m.free()
    # ---- roofline of the dominant kernel (the gate SVD: one CTA per instance per launch) ----
    roof = None
    n_launch = prof["svd_launches"]
    if n_launch:
        t_launch = prof["svd_ms"] / 1e3 / n_launch                   # CUDA events, timed region
        f64_l, f32_l = prof["fp64_flops"] / n_launch, prof["fp32_flops"] / n_launch
        achieved = (f64_l + f32_l * P64_SM / P32_SM) / t_launch       # FP64-equivalent rate
        peak = P64_SM * N_SM
        roof = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "kernel": f"svd_kernel (gate SVD; {B} CTAs per launch, one per instance)",
                "per_launch": {"ms": 1e3 * t_launch, "fp64_flops": f64_l, "fp32_flops": f32_l,
                               "launches": n_launch},
                "note": "achieved = (F64 + F32*P64/P32) flops per launch, counted on the device, / the "
                        "launch's CUDA-event duration on the state's stream over the timed steps; peak = "
                        "recipe nominal FP64 1.25 TFLOP/s for the GPU (fallback: FP64 is not in the measured "
                        "peaks); FP32 converted at 152 SMs x 128 FMA/clk x 2 x 2.07 GHz",
                "svd_share_of_step": prof["svd_ms"] / 1e3 / (t_step * args.steps)}
    if rank == 0:
        cpu = None if args.no_cpu_baseline else (oracle_full(cfg) if n_exc is None else oracle_sample(cfg))
        line = {"metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * t_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": f"{args.workload}: n={p.n} qubits, {p.spec.n_e} electrons, D={p.spec.D}, "
                                       f"eps={p.spec.eps}, {n_theta} theta, {len(gates)} gates, {len(x)} Pauli "
                                       f"strings; {B} instances per GPU batched into every launch",
                           "instances_per_gpu": B, "l2": "512 MB buffer written between timed steps; "
                                                         "per-instance tape ~0.9 GB > L2",
                           "precision": "FP64 contractions; SVD FP32-preconditioned, FP64-finished"},
                "e2e": e2e, "gpu_launches": launches, "roofline": roof, "cpu_baseline": cpu, "clocks": clk,
                "mixed_precision": mixed,
                "pauli_terms_per_s": {"value": terms_per_s, "unit": "Pauli-term expectations/s",
                                      "roofline": energy_roof,
                                      "note": f"energy pass alone on the {B} final states "
                                              f"({len(x)} strings each), host clock over {n_rep} calls"}}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
