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
    ap.add_argument("--no-n40", action="store_true", help="skip the n = 40, D = 256 measurements")
    ap.add_argument("--no-psr", action="store_true", help="skip the parameter-shift comparison")
    ap.add_argument("--no-autotune", action="store_true", help="use the SVD work-split rule, not the tuned table")
    ap.add_argument("--config3", action="store_true",
                    help="also run the 64-instance uneven batch (about 15 minutes: looped single calls "
                         "against mps_energy_grad_multi)")
    ap.add_argument("--profile-case", default=None,
                    choices=["zgemm_tc", "zgemm_mma_sync", "zgemm_fp64", "svd_coop", "step"],
                    help="run one kernel on a synthetic case (two warm-up calls, one timed) for a profiler "
                         "capture, instead of the benchmark")
    ap.add_argument("--size", type=int, default=2048, help="matrix side of --profile-case")
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
def measure_peaks():
    """Arithmetic peaks of this GPU from libpeaks.so (FP64/FP32 FMA, TF32 mma.sync, TF32 tcgen05)."""
    import ctypes
    import paper_2211_07983_gb300 as M
    lib = ctypes.CDLL(os.path.join(os.path.dirname(M.__file__), "libpeaks.so"))
    lib.peaks_measure.argtypes = [ctypes.c_void_p]
    lib.peaks_measure_tcgen05.argtypes = [ctypes.c_void_p]
    o = (ctypes.c_double * 4)()
    t = (ctypes.c_double * 2)()
    rc1, rc2 = lib.peaks_measure(o), lib.peaks_measure_tcgen05(t)
    return {"fp64_tflops": o[0] / 1e12, "fp32_tflops": o[1] / 1e12, "tf32_mma_sync_tflops": o[2] / 1e12,
            "tf32_tcgen05_tflops": t[0] / 1e12, "sms": int(o[3]), "rc": [rc1, rc2],
            "how": "libpeaks.so: register-only FMA chains (8 per thread, 8 CTAs of 256 threads per SM); "
                   "mma.sync m16n8k8 TF32 chains; one CTA per SM issuing 128x256x8 tcgen05.mma kind::tf32 "
                   "back to back; CUDA events, best launch of 3-5 after a warm-up"}


def event_time(stream, fn):
    """Device time (s) of fn() on `stream` bracketed by CUDA events."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3


def trie_work(x, z, n, D):
    """Trie nodes of the canonical strings and the bond caps (2^min(i, n-i), at most D)."""
    cap = [min(2 ** min(i, n - i), D) for i in range(n + 1)]
    nodes = set()
    for xm, zm in zip(x.tolist(), z.tolist()):
        sup = xm | zm
        if not sup:
            continue
        a, b = (sup & -sup).bit_length() - 1, sup.bit_length() - 1
        sym = tuple((((xm >> q) & 1) | (((zm >> q) & 1) << 1)) for q in range(a, b + 1))
        for e in range(1, len(sym) + 1):
            nodes.add((a, sym[:e]))
    return nodes, cap


def energy_mac(nodes, dims, n):
    """Complex MACs of one energy pass as the trie runs it: per node v at site s,
    L_v = (O B_s)^H T_par costs 2 D_s D_{s+1}^2; T_p = L_p B_s costs 2 D_s^2 D_{s+1} once per parent
    (shared by its children; a string's first site uses the identity chain's T); the two identity
    chains cost 2 D_s D_{s+1} (D_s + D_{s+1}) per site each."""
    mac = 0
    parents = set()
    for a, sym in nodes:
        s = a + len(sym) - 1
        mac += 2 * dims[s] * dims[s + 1] ** 2
        if len(sym) > 1:
            parents.add((a, sym[:-1]))
    for a, sym in parents:
        s = a + len(sym)            # the children's site
        mac += 2 * dims[s] ** 2 * dims[s + 1]
    mac += 2 * sum(2 * dims[q] * dims[q + 1] * (dims[q] + dims[q + 1]) for q in range(n))
    return mac


# the n = 40, D = 256 workload: twelve singles and five short doubles of the pruned list (the
# prefix whose oracle values tests/golden/config4_prefix.json holds)
N40_PREFIX = list(range(12)) + [825, 189, 824, 920, 1172]


def run_n40(M, stream, peaks):
    """n = 40, D = 256 on one GPU: the prefix circuit's E+grad (FP64 and mixed), the Pauli-sweep
    energy on its final state (20083 strings), and the measured gate cost at 512 x 512."""
    import torch
    p = S.make_problem(4)
    excs = [p.excitations[t] for t in N40_PREFIX]
    th = np.array([p.theta[t] for t in N40_PREFIX])
    x, z, c = M.build_hamiltonian(p.h, p.eri)
    gates = M.compile_excitations(p.n, excs)
    full_gates = M.compile_excitations(p.n, p.excitations)
    circ = M.Circuit(p.n, gates)
    ham = M.Hamiltonian(p.n, x, z, c)
    out = {"workload": f"n40_D256: n=40, 20 electrons, D=256, eps=1e-10, {len(x)} Pauli strings (the full Hamiltonian); "
                       f"circuit = 12 singles + 5 doubles of the pruned excitation list ({len(gates)} gates; the "
                       f"full list has {len(p.excitations)} excitations, {len(full_gates)} gates)"}
    # forward with the gate SVD timed by CUDA events around every launch
    st = M.State.product(p.bits, p.spec.D, p.spec.eps, stream=stream)
    st.profile(True)
    M.apply_circuit(st, circ, th)                      # warm-up (cooperative kernel set-up, plans)
    st.free()
    st = M.State.product(p.bits, p.spec.D, p.spec.eps, stream=stream)
    st.profile(True)
    st.profile_read()
    t_fwd = event_time(stream, lambda: M.apply_circuit(st, circ, th))
    pr = st.profile_read()
    dims, _, _ = st.read()
    out["forward"] = {"s": t_fwd, "gates": len(gates), "svd_ms_total": pr["svd_ms"], "svd_launches": pr["svd_launches"],
                      "bond_dims": [int(v) for v in dims]}
    # Pauli sweeps on the final state: FP64 and mixed (tcgen05 split-TF32 for bond sides >= 64)
    nodes, cap = trie_work(x, z, p.n, p.spec.D)
    mac = energy_mac(nodes, [int(v) for v in dims], p.n)
    sweeps = {}
    for prec in ("fp64", "mixed"):
        s2 = M.State.product(p.bits, p.spec.D, p.spec.eps, stream=stream, precision=prec)
        M.apply_circuit(s2, circ, th)
        E0 = M.energy(s2, ham)                         # builds the sweep plan
        ts = [event_time(stream, lambda: M.energy(s2, ham)) for _ in range(3)]
        t = min(ts)
        sweeps[prec] = {"E": E0, "s": t, "pauli_terms_per_s": len(x) / t, "complex_mac": mac,
                        "algorithmic_tflops": 8.0 * mac / t / 1e12}
        s2.free()
        torch.cuda.synchronize()
    sweeps["mixed"]["rel_E_vs_fp64"] = abs(sweeps["mixed"]["E"] - sweeps["fp64"]["E"]) / abs(sweeps["fp64"]["E"])
    # the tensor-core work of the mixed sweeps: 4 real products per complex MAC, 3 TF32 MMAs each
    tc_rate = 24.0 * mac / sweeps["mixed"]["s"] / 1e12
    sweeps["mixed"]["roofline"] = {"bound": "tensor", "achieved": tc_rate, "peak": peaks["tf32_tcgen05_tflops"],
                                   "unit": "TFLOP/s", "frac": tc_rate / peaks["tf32_tcgen05_tflops"],
                                   "note": "TF32 tensor flops = 24 x complex MACs of the trie (split-TF32: 4 real "
                                           "products x 3 MMAs) / CUDA-event time of the whole energy call; peak = "
                                           "tcgen05 kind::tf32 measured by libpeaks in this run"}
    sweeps["fp64"]["roofline"] = {"bound": "alu", "achieved": sweeps["fp64"]["algorithmic_tflops"],
                                  "peak": peaks["fp64_tflops"], "unit": "TFLOP/s",
                                  "frac": sweeps["fp64"]["algorithmic_tflops"] / peaks["fp64_tflops"]}
    out["pauli_sweeps"] = sweeps
    out["trie_nodes"] = len(nodes)
    # E + gradient of the prefix circuit (checkpoint segments of 512 gates)
    eg = {}
    for prec in ("fp64", "mixed"):
        s3 = M.State.product(p.bits, p.spec.D, p.spec.eps, checkpoint_every=512, stream=stream, precision=prec)
        res = {}
        t = event_time(stream, lambda: res.setdefault("r", M.energy_grad(s3, circ, th, ham)))
        E, g = res["r"]
        eg[prec] = {"s": t, "evals_per_s": 1.0 / t, "E": E, "grad_norm": float(np.linalg.norm(g)), "grad": g}
        s3.free()
        torch.cuda.synchronize()
    g64, gm = eg["fp64"].pop("grad"), eg["mixed"].pop("grad")
    eg["mixed"]["rel_E_vs_fp64"] = abs(eg["mixed"]["E"] - eg["fp64"]["E"]) / abs(eg["fp64"]["E"])
    eg["mixed"]["rel_grad_vs_fp64"] = float(np.linalg.norm(gm - g64) / np.linalg.norm(g64))
    eg["mixed"]["speedup_vs_fp64"] = eg["fp64"]["s"] / eg["mixed"]["s"]
    out["energy_grad_prefix"] = eg
    # projection of the whole 2000-excitation circuit from the measured per-gate SVD cost
    svd_per_gate = pr["svd_ms"] / 1e3 / max(1, pr["svd_launches"])
    out["projection_full_circuit"] = {
        "note": "not measured: the full circuit's forward alone repeats the measured per-gate cost for every gate; "
                "E+grad adds a recomputation and the adjoint of each gate",
        "gates": len(full_gates), "measured_s_per_gate_forward": t_fwd / len(gates),
        "measured_svd_s_per_gate": svd_per_gate}
    st.free()
    return out


def run_psr(M, stream):
    """Parameter shift (2 M shifted circuits as batched instances) against one adjoint evaluation,
    on prefixes of the n = 12 workload: t_PSR / t_grad as M grows (Sec. 4, Eq. psr)."""
    import torch
    from paper_2211_07983_gb300 import psr
    p = S.make_problem(1)
    x, z, c = M.build_hamiltonian(p.h, p.eri)
    ham = M.Hamiltonian(p.n, x, z, c)
    rows = []
    for n_exc in (4, 8, 16, 32):
        excs = p.excitations[:n_exc]
        gates = M.compile_excitations(p.n, excs)
        circ = M.Circuit(p.n, gates)
        th = p.theta[:n_exc]
        st = M.State.product(p.bits, p.spec.D, p.spec.eps, stream=stream)
        M.energy_grad(st, circ, th, ham)                       # warm-up (plans)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        E, g = M.energy_grad(st, circ, th, ham)
        t_grad = time.perf_counter() - t0
        st.free()
        gp, _, n_eval, _ = psr.parameter_shift(p.n, p.bits, gates, th, ham, p.spec.D, p.spec.eps, batch=256,
                                               stream=stream)  # warm-up
        gp, _, n_eval, t_psr = psr.parameter_shift(p.n, p.bits, gates, th, ham, p.spec.D, p.spec.eps, batch=256,
                                                   stream=stream)
        rows.append({"excitations": n_exc, "M_theta": n_exc, "M_rz": n_eval // 2, "gates": len(gates),
                     "t_grad_s": t_grad, "t_psr_s": t_psr, "ratio": t_psr / t_grad,
                     "rel_diff": float(np.linalg.norm(gp - g) / max(1e-300, np.linalg.norm(g)))})
    return {"workload": "prefixes of n12_D64 (no truncation), one instance", "rows": rows,
            "note": "host wall clock of one mps_energy_grad call against the whole parameter-shift gradient "
                    "(2 M_rz forward passes and energies, 256 instances per batched state)"}


def run_config3(M, n_single=8, n_double=4):
    """The batching workload: 64 independent problems of uneven (n, D), each with its own seeded
    Hamiltonian and a seeded sample of its singles-and-doubles ansatz (n_single singles and
    n_double doubles; the whole ansatz of the larger instances is out of reach, as at n = 40),
    evaluated (a) one mps_energy_grad call after another and (b) all together through
    mps_energy_grad_multi (one library stream per problem, each replaying its own captured graph).
    Both timed by the host clock around whole calls, after warm-up calls that allocate and capture."""
    import torch
    probs = []
    for i in range(64):
        p = S.make_problem(3, i)
        excs = S.sampled_excitations(p.excitations, n_single, n_double, S.seed_for(3, 20_000 + i))
        x, z, c = M.build_hamiltonian(p.h, p.eri)
        st = M.State.product(p.bits, p.spec.D, p.spec.eps, checkpoint_every=256)
        st.set_svd_policy(True)   # one CTA per SVD: many problems share the GPU
        gates = M.compile_excitations(p.n, excs)
        probs.append((st, M.Circuit(p.n, gates), p.theta[: len(excs)], M.Hamiltonian(p.n, x, z, c),
                      p.n, p.spec.D, len(gates), len(x)))
    from paper_2211_07983_gb300 import autotune
    shapes = sorted({sh for q in probs for sh in autotune.cap_shapes(q[4], q[5])})
    autotune.ensure(shapes)
    states, circs, thetas, hams = (list(v) for v in zip(*[q[:4] for q in probs]))
    single = [M.energy_grad(st, c, th, h) for st, c, th, h in zip(states, circs, thetas, hams)]   # eager
    for _ in range(2):   # the second call captures each problem's graph
        M.energy_grad_multi(states, circs, thetas, hams)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loop = [M.energy_grad(st, c, th, h) for st, c, th, h in zip(states, circs, thetas, hams)]
    t_loop = time.perf_counter() - t0
    reps = 3
    t0 = time.perf_counter()
    for _ in range(reps):
        Es, gs = M.energy_grad_multi(states, circs, thetas, hams)
    t_multi = (time.perf_counter() - t0) / reps
    same = all(Es[k] == loop[k][0] and np.array_equal(gs[k], loop[k][1]) for k in range(64))
    for st in states:
        st.free()
    return {"workload": f"64 instances: n in {{8..28}}, D in {{16..256}} (capped at 2^(n/2)), eps=1e-10; "
                        f"{n_single} singles + {n_double} doubles sampled per instance; "
                        f"{sum(q[6] for q in probs)} gates and {sum(q[7] for q in probs)} Pauli strings in all",
            "instances": [{"n": q[4], "D": q[5], "gates": q[6], "strings": q[7]} for q in probs],
            "loop_single_s": t_loop, "multi_s": t_multi,
            "loop_evals_per_s": 64 / t_loop, "multi_evals_per_s": 64 / t_multi, "speedup": t_loop / t_multi,
            "multi_equals_single_bitwise": bool(same),
            "note": "host wall clock around whole calls (each call synchronises); SVD policy one CTA per matrix"}


def run_ours(args, rank, world, local):
    import torch
    import paper_2211_07983_gb300 as M
    from paper_2211_07983_gb300 import build

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    peaks = measure_peaks()
    cfg, n_exc = WORKLOADS[args.workload]
    p = S.make_problem(cfg)
    # the SVD work split of this workload's matrix shapes, from the project's autotuner (untimed
    # setup; the table is cached per GPU model and reused by later runs)
    from paper_2211_07983_gb300 import autotune
    t0 = time.perf_counter()
    tune_rows = [] if args.no_autotune else autotune.ensure(autotune.cap_shapes(p.n, p.spec.D))
    tune_info = {"rows": tune_rows, "seconds": time.perf_counter() - t0,
                 "note": "lanes per column pair of the one-CTA SVD's FP32/FP64 sweeps per bond-cap shape "
                         "(0 = the library's rule); timed by mps_svd_tune on seeded probe matrices"}
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
        dev_ms += 1e3 * event_time(stream, lambda: M.energy_grad(state, circ, thetas_d, ham, out=(E_d, g_d)))
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
    E64, g64 = E_d.cpu().numpy().copy(), g_d.cpu().numpy().copy()
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
    t_energy = min(event_time(stream, lambda: M.energy(st_f, ham)) for _ in range(3))
    dims_f, _, _ = st_f.read()
    st_f.free()
    terms_per_s = len(x) * B / t_energy
    nodes, cap = trie_work(x, z, p.n, p.spec.D)
    energy_flops = 8.0 * energy_mac(nodes, [int(v) for v in dims_f], p.n) * B
    energy_roof = {"bound": "alu", "achieved": energy_flops / t_energy / 1e12, "peak": peaks["fp64_tflops"],
                   "unit": "TFLOP/s", "frac": energy_flops / t_energy / 1e12 / peaks["fp64_tflops"],
                   "work": f"{len(nodes)} trie nodes per instance: L_v = (O B)^H T costs 2 Dl Dr^2 complex MACs per "
                           "node, T = L B costs 2 Dl^2 Dr once per parent, plus the two identity chains, at instance 0's "
                           "final bond dimensions; CUDA-event time of the whole energy call; peak = FP64 FMA "
                           "measured by libpeaks in this run"}
    # ---- the mixed-precision path on the same instances ----
    mixed = None
    state.free()
    torch.cuda.synchronize()
    if not args.no_mixed:
        st_m = M.State.product_batch(np.stack([p.bits] * B), p.spec.D, p.spec.eps, checkpoint_every=0,
                                     stream=stream, precision="mixed")
        for _ in range(2):                      # eager, then captured
            M.energy_grad(st_m, circ, thetas_d, ham, out=(E_d, g_d))
        torch.cuda.synchronize()
        ms_m = 0.0
        n_m = 5
        for _ in range(n_m):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
            ms_m += 1e3 * event_time(stream, lambda: M.energy_grad(st_m, circ, thetas_d, ham, out=(E_d, g_d)))
        Em, gm = E_d.cpu().numpy(), g_d.cpu().numpy()
        t_m = ms_m / 1e3 / n_m
        g_rel = np.linalg.norm(gm - g64, axis=1) / np.maximum(1.0, np.linalg.norm(g64, axis=1))
        mixed = {"value": B * world / t_m, "unit": "evals/s", "ms_per_step": 1e3 * t_m, "steps": n_m,
                 "speedup_vs_fp64": t_step / t_m,
                 "max_rel_E_err_vs_fp64": float(np.max(np.abs(Em - E64) / np.maximum(1.0, np.abs(E64)))),
                 "rel_grad_err_vs_fp64": {"median": float(np.median(g_rel)),
                                          "p90": float(np.percentile(g_rel, 90)), "max": float(g_rel.max()),
                                          "argmax": int(g_rel.argmax()),
                                          "fraction_within_1e-5": float(np.mean(g_rel <= 1e-5))},
                 "precision": "energy Pauli sweeps and recomputed two-site tensors in split-TF32 on tensor cores "
                              "(tcgen05.mma for bond sides >= 64, mma.sync below; FP32 accumulation); gate "
                              "contractions, energy cotangent, SVD, SVD adjoint, sums FP64"}
        st_m.free()
    flush = None
    torch.cuda.synchronize()
    # ---- n = 40, D = 256 (rank 0 only; one GPU) ----
    n40 = None
    if rank == 0 and not args.no_n40:
        n40 = run_n40(M, stream, peaks)
    psr_rows = None
    if rank == 0 and not args.no_psr:
        psr_rows = run_psr(M, stream)
    batch64 = None
    if rank == 0 and args.config3:
        batch64 = run_config3(M)
    # ---- roofline of the dominant kernel (the gate SVD: one CTA per instance per launch) ----
    roof = None
    n_launch = prof["svd_launches"]
    if n_launch:
        t_launch = prof["svd_ms"] / 1e3 / n_launch                   # CUDA events, timed region
        f64_l, f32_l = prof["fp64_flops"] / n_launch, prof["fp32_flops"] / n_launch
        p64, p32 = peaks["fp64_tflops"] * 1e12, peaks["fp32_tflops"] * 1e12
        achieved = (f64_l + f32_l * p64 / p32) / t_launch             # FP64-equivalent rate
        # DRAM bytes (read + write) of one svd_kernel launch from an ncu capture of launch 3001 of
        # `bench.py --profile-case step --workload n12_D64 --instances 4` (a 64-wide bond, 4 CTAs:
        # 444,672 + 0 bytes), scaled to this launch's CTA count
        traffic = 444672.0 / 4 * B
        roof = {"bound": "alu", "achieved": achieved / 1e12, "peak": p64 / 1e12, "unit": "TFLOP/s",
                "frac": achieved / p64, "traffic": traffic,
                "kernel": f"svd_kernel (gate SVD; {B} CTAs per launch, one per instance)",
                "per_launch": {"ms": 1e3 * t_launch, "fp64_flops": f64_l, "fp32_flops": f32_l,
                               "launches": n_launch},
                "note": "achieved = (F64 + F32*P64/P32) flops per launch, counted on the device, / the launch's "
                        "CUDA-event duration on the state's stream over the timed steps; P64, P32 = FP64 and FP32 "
                        "FMA peaks measured by libpeaks in this run (of measured); traffic: dram__bytes_read.sum + "
                        "dram__bytes_write.sum of one 4-CTA launch (a 64-wide bond) from one ncu capture, scaled to "
                        "the launch's CTAs; the kernel works in shared memory, so this is the input matrix read once",
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
                "peaks_measured": peaks, "mixed_precision": mixed,
                "pauli_terms_per_s": {"value": terms_per_s, "unit": "Pauli-term expectations/s",
                                      "roofline": energy_roof,
                                      "note": f"energy pass alone on the {B} final states ({len(x)} strings each), "
                                              "best of 3 calls timed with CUDA events"},
                "n40_D256": n40, "psr": psr_rows, "batch64_uneven": batch64, "svd_autotune": tune_info}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_profile_case(args):
    """One kernel on a seeded synthetic case: a complex n x n x n GEMM through one contraction
    kernel, or the cooperative SVD of one n x n complex matrix (n <= 512)."""
    import torch
    import paper_2211_07983_gb300 as M
    from paper_2211_07983_gb300 import build
    build.build()
    rng = np.random.default_rng(1)
    n = args.size
    if args.profile_case == "step":
        # one eager energy + gradient evaluation of --workload on --instances instances
        cfg, n_exc = WORKLOADS[args.workload]
        p = S.make_problem(cfg)
        excs = p.excitations if n_exc is None else p.excitations[:n_exc]
        x, z, c = M.build_hamiltonian(p.h, p.eri)
        circ = M.Circuit(p.n, M.compile_excitations(p.n, excs))
        ham = M.Hamiltonian(p.n, x, z, c)
        B = args.instances
        th = np.stack([S.random_theta(S.seed_for(1, 500 + i), len(excs)) for i in range(B)])
        st = M.State.product_batch(np.stack([p.bits] * B), p.spec.D, p.spec.eps)
        l0 = M.kernel_launches()
        t0 = time.perf_counter()
        M.energy_grad(st, circ, th, ham)
        print(json.dumps({"case": "step", "workload": args.workload, "instances": B, "s_wall": time.perf_counter() - t0,
                          "launches": M.kernel_launches() - l0}))
        return
    if args.profile_case == "svd_coop":
        n = min(n, 512)
        A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        for _ in range(2):
            M.svd(A, n // 2, 1e-10)
        t0 = time.perf_counter()
        s, V, W, k = M.svd(A, n // 2, 1e-10)
        dt = time.perf_counter() - t0
        print(json.dumps({"case": "svd_coop", "n": n, "k": k, "s_wall": dt, "note": "wall clock of mps_svd_dev, "
                          "host transposes included"}))
        return
    eng = {"zgemm_tc": "tcgen05", "zgemm_mma_sync": "mma_sync", "zgemm_fp64": "fp64"}[args.profile_case]
    A = torch.tensor(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)), device="cuda")
    B = torch.tensor(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)), device="cuda")
    for _ in range(2):
        M.api.zgemm(A, B, "N", "N", eng)
    torch.cuda.synchronize()
    t = event_time(torch.cuda.current_stream(), lambda: M.api.zgemm(A, B, "N", "N", eng))
    print(json.dumps({"case": args.profile_case, "n": n, "s": t, "complex_tflops": 8.0 * n ** 3 / t / 1e12,
                      "note": "CUDA events around mps_zgemm_mixed_dev (descriptor upload and a synchronise "
                              "included)"}))


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.profile_case:
        run_profile_case(args)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
