#!/usr/bin/env python
"""Benchmark of the Axilrod-Teller three-body engine on one GB300.

Headline step: one exhaustive FP32-bulk solve of Phi for the N = 32 768
uniform workload (cube of side 32, minimum pair distance 0.5, seed 2), i.e.
all C(N,3) = 5.8635e12 unordered triples. The metric is triples/s.

The JSON line also carries, for context (each time-bounded):
  fp64_exhaustive : plain FP64 exhaustive rate (N = 8 192, same density);
  tree            : multi-tree particles/s at eps = 1e-2 and 1e-1, alpha = 0.05,
                    on 65 536 points from the 2^20 Gaussian-mixture generator
                    (4 components of 16 384 points at the same component
                    density); % within eps on sampled particles against the
                    exact sum; speedup over plain FP64 exhaustive particles/s;
  forces          : adjoint (force) rate at N = 16 384, force-workload density;
  serving         : Poisson stream of the serving mix (potential 70 % / forces
                    30 %, uniform and Gaussian-mixture systems) with p50/p99;
plus the roofline of the dominant kernel, the CPU oracle baseline, an
end-to-end number through the host-buffer C entry point, and the SM clocks
sampled during the timed region.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs an independent replica (the exhaustive sum of
one system needs no exchange); value = all ranks' triples / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "AT triples/s (exhaustive) & particles/s at eps=1e-2 vs plain FP64; p50/p99 ms"
WORKLOAD = "exh32_n32768"
N_MAIN = 32768
FLOPS_PER_TRIPLE_FP32 = 23   # counted from the inner loop (FMA = 2), see csrc/tile_fp32.cuh
# adjoint (gather form): 43 FLOPs per evaluation of grad_i phi (9 dot-product
# operations = 15 FLOPs, products and coefficients 22, accumulations 6; FMA = 2,
# csrc/adjoint.cu), three evaluations per unordered triple
FLOPS_PER_TRIPLE_ADJOINT = 3 * 43
FP32_LANES_PER_SM = 128
# dram__bytes_read.sum + dram__bytes_write.sum of one exh_fp32_pt_kernel launch on
# the N = 32 768 set (ncu, one pass; the command is in
# profiles/exh_fp32_n32768_launches.md). Valid for the kernel as committed with it.
EXH_FP32_TRAFFIC_BYTES = 4088735832064 + 14698218240
N_CONFIG3 = 1 << 20


def triples(n):
    return n * (n - 1) * (n - 2) // 6


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def aggregate(local_ms: float, units: float, dist=None):
    """Whole-job rate over ranks: units of all ranks / max time (weak scaling).
    Returns (value, max_ms); with dist None or world size 1 it is local."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return units / (local_ms / 1e3), local_ms
    import torch
    t = torch.tensor([local_ms, units], dtype=torch.float64)
    if dist.get_backend() == "nccl":
        t = t.cuda()
    m = t.clone()
    dist.all_reduce(m[0:1], op=dist.ReduceOp.MAX)
    dist.all_reduce(m[1:2], op=dist.ReduceOp.SUM)
    max_ms, tot = float(m[0]), float(m[1])
    return tot / (max_ms / 1e3), max_ms


class ClockSampler:
    """nvidia-smi clock/throttle sampling every 200 ms during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu_index = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
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
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_oracle_rate(X, n_particles, seed=2024):
    """Oracle Phi for a bounded seeded sample of particles on all host cores;
    returns (triples/s of the whole job, seconds, particles, threads)."""
    import oracle
    from paper_1105_2769_gb300 import inputs
    oracle.build()
    nt = oracle.max_threads()
    m = n_particles or nt
    idx = inputs.sample_indices(len(X), m, seed)
    t0 = time.perf_counter()
    oracle.phi(X, idx, nthreads=nt)
    dt = time.perf_counter() - t0
    n = len(X)
    evals = m * (n - 1) * (n - 2) / 2          # phi evaluations done
    return evals / 3.0 / dt, dt, m, nt        # full job = 3 C(N,3) evaluations


def run_reference(args):
    """The oracle as it stands, timed on the host cores (rank 0 only)."""
    if int(os.environ.get("RANK", "0")) != 0:
        return 0
    from paper_1105_2769_gb300 import inputs
    X = inputs.workload(WORKLOAD)
    import oracle
    oracle.build()
    nt = oracle.max_threads()
    cpu_oracle_rate(X, nt)  # warm-up (page-in, thread start)
    rates, total_t = [], 0.0
    for _ in range(args.steps):
        r, dt, m, nt = cpu_oracle_rate(X, nt)
        rates.append(r)
        total_t += dt
    value = sum(rates) / len(rates)
    sample = (f"{nt} seeded particles per step of the N={N_MAIN} set (each a full "
              f"C(N-1,2) sum); job-equivalent triples = evaluations/3")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "triples/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_t / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N_MAIN,
                   "distribution": "uniform [0,32]^3, d_min 0.5, seed 2"},
        "cpu_baseline": {"value": value, "unit": "triples/s", "cores": nt, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "triples/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }))
    return 0


def bench_fp64(api, inputs, torch, dev):
    n64 = 8192
    X = inputs.uniform_cube(n64, 32.0 * (n64 / N_MAIN) ** (1 / 3), 0.5, 2)
    Xd = torch.from_numpy(X).to(dev)
    api.potential(Xd, mode="fp64")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    api.potential(Xd, mode="fp64")
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return {"n": n64, "triples_per_s": triples(n64) / dt, "s": dt}


def bench_tree(api, inputs, torch, dev, r64, np, workload="gmm4_n65536", eps_list=(1e-2, 1e-1),
               warm=True, n_sample=256, progress=False, exact_file=None):
    """Tree solves (relative eps, alpha 0.05) timed end to end from device-resident X;
    accuracy on n_sample seeded particles against the exact sampled sum (read
    from exact_file when it holds this workload's sample, else computed and,
    with exact_file given, saved there)."""
    X = inputs.workload(workload)
    n = len(X)
    Xd = torch.from_numpy(X).to(dev)
    idx = inputs.sample_indices(n, n_sample, 11)
    exact = None
    if exact_file and os.path.exists(exact_file):
        saved = np.load(exact_file)
        if saved["n"] == n and np.array_equal(saved["idx"], idx):
            exact = saved["exact"]
    if exact is None:
        t0 = time.perf_counter()
        exact = api.potential_sampled(Xd, idx).cpu().numpy()
        if progress:
            print(json.dumps({"progress": workload, "sampled_exact_s": time.perf_counter() - t0}),
                  flush=True)
        if exact_file:
            np.savez(exact_file, n=n, idx=idx, exact=exact)
    out = {"workload": workload, "n": n, "alpha": 0.05, "sampled_particles": len(idx)}
    fp64_pps = n * r64 / triples(n)                       # plain FP64 exhaustive particles/s
    fp64_pps_config3 = N_CONFIG3 * r64 / triples(N_CONFIG3)
    for eps in eps_list:
        if warm:
            api.potential(Xd, eps=eps, alpha=0.05, mode="tree")  # warm-up
        torch.cuda.synchronize()
        sampler = ClockSampler(dev.index or 0) if progress else None
        if sampler:
            sampler.start()
        t0 = time.perf_counter()
        phi, st = api.potential(Xd, eps=eps, alpha=0.05, mode="tree", stats=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        clocks = sampler.stop() if sampler else None
        rel = np.abs(phi.cpu().numpy()[idx] - exact) / np.abs(exact)
        out[f"eps_{eps:g}"] = {
            "particles_per_s": n / dt, "s": dt, "within_eps": float(np.mean(rel <= eps)),
            "max_rel_err": float(rel.max()), "speedup_vs_fp64_exhaustive": n / dt / fp64_pps,
            "phase_ms": {k: round(st[k], 2) for k in
                         ("ms_build", "ms_traverse", "ms_base", "ms_finalize")},
            "det_prunes": st["det_prunes"], "mc_prunes": st["mc_prunes"],
            "base_triples": st["base_triples"], "mc_samples": st["mc_samples"]}
        if clocks:
            out[f"eps_{eps:g}"]["clocks"] = clocks
        if progress:
            print(json.dumps({"progress": workload, f"eps_{eps:g}": out[f"eps_{eps:g}"]}),
                  flush=True)
    out["fp64_exhaustive_particles_per_s"] = fp64_pps
    out["fp64_exhaustive_particles_per_s_n1048576"] = fp64_pps_config3
    return out


def fp32_peak_tflops(torch, dev):
    props = torch.cuda.get_device_properties(dev)
    sm_max = float(_peaks().get("sm_max_mhz", 2070.0))
    return props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12


def forces_roofline(rate, torch, dev):
    peak = fp32_peak_tflops(torch, dev)
    achieved = rate * FLOPS_PER_TRIPLE_ADJOINT / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "kernel": "adjoint_kernel<float>",
            "flops_per_triple": FLOPS_PER_TRIPLE_ADJOINT, "traffic": None}


def bench_forces(api, inputs, torch, dev):
    n = 16384
    X = inputs.uniform_cube(n, 32.0 * (n / 65536) ** (1 / 3), 0.5, 4)
    Xd = torch.from_numpy(X).to(dev)
    api.forces(Xd, mode="fp32")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    api.forces(Xd, mode="fp32")
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return {"n": n, "triples_per_s": triples(n) / dt, "s": dt,
            "roofline": forces_roofline(triples(n) / dt, torch, dev),
            "note": "gather form: each unordered triple evaluated once per member"}


def bench_serving(api, inputs, np, duration=6.0, rate=200.0):
    """Poisson arrivals of the serving mix with N log-uniform in [1 024, 4 096]."""
    rng = np.random.default_rng(5)
    systems = []
    for q in range(24):
        n = int(np.exp(rng.uniform(np.log(1024), np.log(4096))))
        if q % 2:
            X = inputs.uniform_cube(n, n ** (1 / 3), 0.5, 500 + q)
        else:
            X = inputs.gaussian_mixture(n, max(1, n // 16384 + 1), 100.0 * (n / N_CONFIG3) ** (1 / 3),
                                        0.5, 3.0, 0.05, 500 + q)
        systems.append(X)
    srv = api.Server(0, hbm_budget_bytes=120 << 30, slots=8)
    # warm the slots
    for X in systems[:8]:
        srv.poll(srv.submit(X, mode="fp32"))
    n_req = int(duration * rate)
    gaps = rng.exponential(1.0 / rate, size=n_req)
    kinds = rng.uniform(size=n_req) < 0.7
    picks = rng.integers(0, len(systems), size=n_req)
    tickets, parts = [], 0
    t_start = time.perf_counter()
    t_next = t_start
    for q in range(n_req):
        t_next += gaps[q]
        while time.perf_counter() < t_next:
            time.sleep(0.0002)
        X = systems[picks[q]]
        parts += len(X)
        if kinds[q]:
            tickets.append(srv.submit(X, mode="tree", eps=1e-2, alpha=0.05,
                                      system_id=int(picks[q]) + 1))
        else:
            tickets.append(srv.submit(X, kind="forces", mode="fp32"))
    lat, comp_tree, comp_forces = [], [], []
    for q, t in enumerate(tickets):
        st, res, _ = srv.poll(t)
        lat.append(res["latency_ms"])
        (comp_tree if kinds[q] else comp_forces).append(res["compute_ms"])
    wall = time.perf_counter() - t_start
    stats = srv.stats()
    srv.close()
    return {"offered_req_per_s": rate, "requests": n_req, "served_req_per_s": n_req / wall,
            "particles_per_s": parts / wall, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "wall_s": wall, "slots": 8,
            "n_range": [1024, 4096], "admitted": stats["admitted"],
            "rejected": stats["rejected"],
            "compute_ms_p50": {"tree": float(np.percentile(comp_tree, 50)) if comp_tree else None,
                               "forces": float(np.percentile(comp_forces, 50))
                               if comp_forces else None},
            "mix": "70% tree Phi (eps 1e-2, alpha 0.05, resident systems), 30% FP32 forces"}


def _config5_system(n, q):
    """One system of the serving workload: uniform at density 1 (d_min 0.5) for
    even q, else the Gaussian-mixture generator of the N = 2^20 set scaled to
    n (components of 16 384 points at the same component density)."""
    from paper_1105_2769_gb300 import inputs
    if q % 2 == 0:
        return inputs.uniform_cube(n, n ** (1 / 3), 0.5, 700 + q)
    comps = max(1, n // 16384)
    return inputs.gaussian_mixture(n, comps, 100.0 * (comps / 64) ** (1 / 3), 0.5, 3.0, 0.05,
                                   700 + q)


def run_serving_only(args):
    """The serving workload as specified: Poisson arrivals at 200 req/s for 60 s,
    N log-uniform in [1 024, 262 144] (a pool of seeded systems, half uniform,
    half mixture), 70 % Phi / 30 % forces, both by the tree method at eps = 1e-2,
    alpha = 0.05, systems kept resident, 120 GB budget, 8 slots. After the
    offered window the server drains for at most `drain` s; requests still
    queued then are reported, not waited for."""
    import numpy as np
    import torch  # noqa: F401  (CUDA context for the library)

    from paper_1105_2769_gb300 import api
    rate, duration, drain = args.serve_rate, args.serve_seconds, args.serve_drain
    rng = np.random.default_rng(5)
    pool_n = [int(np.exp(rng.uniform(np.log(1024), np.log(262144)))) for _ in range(args.serve_pool)]
    t0 = time.perf_counter()
    pool = [_config5_system(n, q) for q, n in enumerate(pool_n)]
    gen_s = time.perf_counter() - t0
    srv = api.Server(0, hbm_budget_bytes=120 << 30, slots=8)
    n_req = int(duration * rate)
    gaps = rng.exponential(1.0 / rate, size=n_req)
    is_phi = rng.uniform(size=n_req) < 0.7
    picks = rng.integers(0, len(pool), size=n_req)
    tickets = []
    t_start = time.perf_counter()
    t_next = t_start
    for q in range(n_req):
        t_next += gaps[q]
        while time.perf_counter() < t_next:
            time.sleep(0.0002)
        X = pool[picks[q]]
        kind = "potential" if is_phi[q] else "forces"
        try:
            tickets.append((q, srv.submit(X, kind=kind, mode="tree", eps=1e-2, alpha=0.05,
                                          system_id=int(picks[q]) + 1)))
        except Exception:  # rejected by the budget
            tickets.append((q, None))
    t_offer = time.perf_counter() - t_start
    lat, comp, parts_done, done_kinds, iv = [], [], 0, [], []
    deadline = t_start + duration + drain
    pending = 0
    for q, t in tickets:
        if t is None:
            continue
        left = deadline - time.perf_counter()
        st, res, _ = srv.poll(t, timeout_us=max(0, int(left * 1e6)))
        if res is None:
            pending += 1
            continue
        lat.append(res["latency_ms"])
        comp.append(res["compute_ms"])
        parts_done += len(pool[picks[q]])
        done_kinds.append(bool(is_phi[q]))
        iv.append((res["dev_start_ns"], res["dev_end_ns"]))
    wall = time.perf_counter() - t_start
    stats = srv.stats()
    # device concurrency: the largest number of requests whose device intervals overlap
    ev = sorted([(a, 1) for a, b in iv if b > a] + [(b, -1) for a, b in iv if b > a])
    cur = peak = 0
    for _, d in ev:
        cur += d
        peak = max(peak, cur)
    srv.close()
    rep = {"report": "serving", "offered_req_per_s": rate, "offered_s": t_offer,
           "requests_offered": n_req, "drain_s": drain, "completed": len(lat),
           "not_completed_at_deadline": pending,
           "rejected": stats["rejected"], "admitted": stats["admitted"],
           "served_req_per_s": len(lat) / wall, "particles_per_s": parts_done / wall,
           "p50_ms": float(np.percentile(lat, 50)) if lat else None,
           "p99_ms": float(np.percentile(lat, 99)) if lat else None,
           "compute_ms_p50": float(np.percentile(comp, 50)) if comp else None,
           "completed_phi": int(sum(done_kinds)), "completed_forces": len(done_kinds) - int(sum(done_kinds)),
           "max_requests_overlapping_on_device": peak, "slots": 8, "budget_gb": 120,
           "pool": {"systems": len(pool), "n_min": min(pool_n), "n_max": max(pool_n),
                    "generation_s": gen_s},
           "mix": "70% Phi / 30% forces, tree eps 1e-2 alpha 0.05, resident systems"}
    print(json.dumps(rep))
    return 0


def run_forces_only(args):
    """Forces of the N = 65 536 force workload (uniform [0,32]^3, d_min 0.5,
    seed 4): the exhaustive FP32-bulk adjoint timed once, and the tree forces
    at eps = 1e-2 (alpha 0.05) of the same set, with accuracy on sampled
    particles against the exhaustive result."""
    import numpy as np
    import torch

    from paper_1105_2769_gb300 import api, inputs
    dev = torch.device("cuda", 0)
    n = args.forces_n
    X = inputs.workload("forces_n65536") if n == 65536 else \
        inputs.uniform_cube(n, 32.0 * (n / 65536) ** (1 / 3), 0.5, 4)
    Xd = torch.from_numpy(X).to(dev)
    rep = {"report": "forces", "n": n, "workload": "uniform [0,32]^3 density 2, d_min 0.5, seed 4"}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    F = api.forces(Xd, mode="fp32")
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    rep["exhaustive_fp32"] = {"s": dt, "triples_per_s": triples(n) / dt,
                              "roofline": forces_roofline(triples(n) / dt, torch, dev)}
    print(json.dumps({"progress": rep}), flush=True)
    Fe = F.cpu().numpy()
    for eps in (1e-2,):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Ft, st = api.forces(Xd, eps=eps, alpha=0.05, mode="tree", stats=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        d = np.abs(Ft.cpu().numpy() - Fe).max(axis=1) / np.linalg.norm(Fe, axis=1)
        rep[f"tree_eps_{eps:g}"] = {
            "s": dt, "particles_per_s": n / dt, "speedup_vs_exhaustive_fp32": rep["exhaustive_fp32"]["s"] / dt,
            "phase_ms": {k: round(st[k], 2) for k in ("ms_build", "ms_traverse", "ms_base")},
            "det_prunes": st["det_prunes"], "mc_prunes": st["mc_prunes"],
            "base_triples": st["base_triples"],
            "max_dev_over_abs_force": float(d.max()), "median_dev_over_abs_force": float(np.median(d))}
    print(json.dumps(rep))
    return 0


def farfield_flops_per_query(p):
    """FP32 operations of one query point in ff_eval_kernel<p>, counted from its
    loops: 14 Taylor recurrences (per coefficient of degree k >= 1: the v_d t
    products and their sum, the t_{a - 2e_d} sum, and the scaled combination)
    and 10 contractions (per padded row of L columns: L multiply-adds, the two
    partial sums, and the multiply-add with t_{a12})."""
    def n(k):
        return 0 if k < 0 else (k + 1) * (k + 2) * (k + 3) // 6

    taylor = 0
    for k in range(1, p + 1):
        taylor += 2  # the two coefficients of the level
        for i in range(k, -1, -1):
            for j in range(k - i, -1, -1):
                l = k - i - j
                na = (i > 0) + (j > 0) + (l > 0)
                nb = (i > 1) + (j > 1) + (l > 1)
                taylor += 2 * na - 1 + max(nb - 1, 0) + (3 if nb else 1)
    contract = 0
    for d in range(p + 1):
        L = n(p - d)
        contract += (d + 1) * (d + 2) // 2 * (2 * L + 3)
    return 14 * taylor + 10 * contract


def bench_farfield(orders, n_exact):
    """The three-body far-field expansion (mbm_farfield3) on 2^20 query points
    against two source clusters of 4 096 points each (Gaussian, radius 0.35,
    centre distances 4-6.4: the separations of pruned node triples): the
    whole call and the query sweep alone timed with CUDA events on the
    launching stream; accuracy of n_exact sampled queries against the exact
    double sum (FP64 oracle) and against the oracle's expansion."""
    import numpy as np
    import torch

    import oracle
    from oracle import farfield as off
    from paper_1105_2769_gb300 import api
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(22)
    n_src, nq = 4096, 1 << 20
    Y2 = rng.normal(size=(n_src, 3)) * 0.35 + np.array([4.0, 0.3, -0.2])
    Y3 = rng.normal(size=(n_src, 3)) * 0.35 + np.array([0.5, 4.0, 1.6])
    Xq = rng.normal(size=(nq, 3)) * 0.35
    d = [torch.from_numpy(a).to(dev) for a in (Xq, Y2, Y3)]
    idx = rng.choice(nq, n_exact, replace=False)
    t0 = time.perf_counter()
    exact = off.pairset_sum(Xq[idx], Y2, Y3)
    t_exact = time.perf_counter() - t0
    peak = fp32_peak_tflops(torch, dev)
    ctx = api.default_context(0)
    rows = []
    for p in orders:
        out = api.farfield3(*d, p)
        for _ in range(3):
            api.farfield3(*d, p)
        s = torch.cuda.current_stream()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 10
        ev0.record(s)
        for _ in range(reps):
            api.farfield3(*d, p, validate=False)
        ev1.record(s)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / reps
        ctx.set_timing(True)  # events around the query sweep alone
        sweep = []
        for _ in range(reps):
            api.farfield3(*d, p, validate=False)
            sweep.append(ctx.last_kernel_ms())
        ctx.set_timing(False)
        k_ms = float(np.median(sweep))
        got = out.cpu().numpy()[idx]
        ref = off.farfield3(Xq[idx], Y2, Y3, p)
        rate = nq / (ms * 1e-3)
        fl = farfield_flops_per_query(p)
        achieved = nq * fl / (k_ms * 1e-3) / 1e12
        rows.append({"p": p, "ms": ms, "queries_per_s": rate, "sweep_ms": k_ms,
                     "max_rel_err_vs_exact": float(np.max(np.abs(got - exact) / np.abs(exact))),
                     "max_rel_dev_vs_oracle_expansion": float(np.max(np.abs(got - ref) / np.abs(ref))),
                     "roofline": {"bound": "alu", "achieved": achieved, "peak": peak,
                                  "unit": "TFLOP/s", "frac": achieved / peak,
                                  "kernel": f"ff_eval_kernel<{p}>",
                                  "flops_per_query": fl, "traffic": None}})
    return {"queries": nq, "sources": [n_src, n_src], "sampled_queries": n_exact,
            "workload": "Gaussian clusters radius 0.35 at centre distances 4-6.4, seed 22",
            "exact_pairs_per_s_cpu_oracle": n_exact * n_src * n_src / t_exact,
            "exact_cores": oracle.max_threads(), "rows": rows}


def run_farfield_only(args):
    """bench_farfield at every order 0..6, 64 sampled queries."""
    rep = bench_farfield(range(7), 64)
    for r in rep["rows"]:
        print(json.dumps({"progress": r}), flush=True)
    print(json.dumps({"report": "farfield", **rep}))
    return 0


def run_paper_shape(args):
    """The paper's experiment shapes (Sec. 6) on this GPU: uniform cube, unit
    ball and thin shell ("annulus"), tree solves at eps 1e-1/1e-2/1e-3 and
    alpha 0 / 0.1, against the FP64 exhaustive solve of the same set: speed-up
    and the fraction of particles within eps (the statistics of Tables 1-3)."""
    import numpy as np
    import torch

    from paper_1105_2769_gb300 import api, inputs
    dev = torch.device("cuda", 0)
    sets = {"uniform": lambda n: inputs.uniform_cube(n, 1.0, 1e-3, 41),
            "ball": lambda n: inputs.unit_ball(n, 1e-3, 42),
            "shell": lambda n: inputs.spherical_shell(n, 0.95, 1.0, 1e-3, 43)}
    rows = []
    for name, gen in sets.items():
        for n in args.paper_n:
            X = gen(n)
            Xd = torch.from_numpy(X).to(dev)
            api.potential(Xd, mode="fp64")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ex = api.potential(Xd, mode="fp64").cpu().numpy()
            t_ex = time.perf_counter() - t0
            for eps in (1e-1, 1e-2, 1e-3):
                for alpha in (0.0, 0.1):
                    api.potential(Xd, eps=eps, alpha=alpha, mode="tree")
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    phi = api.potential(Xd, eps=eps, alpha=alpha, mode="tree").cpu().numpy()
                    dt = time.perf_counter() - t0
                    rel = np.abs(phi - ex) / np.abs(ex)
                    rows.append({"set": name, "n": n, "eps": eps, "alpha": alpha,
                                 "tree_s": dt, "fp64_exhaustive_s": t_ex,
                                 "speedup": t_ex / dt, "within_eps": float(np.mean(rel <= eps)),
                                 "mean_rel_err": float(rel.mean()),
                                 "var_rel_err": float(rel.var()),
                                 "max_rel_err": float(rel.max())})
                    print(json.dumps(rows[-1]), flush=True)
    print(json.dumps({"report": "paper_shape", "rows": len(rows)}))
    return 0


def run_tree_only(args):
    import numpy as np
    import torch

    from paper_1105_2769_gb300 import api, inputs
    dev = torch.device("cuda", 0)
    fp64 = bench_fp64(api, inputs, torch, dev)
    eps_list = tuple(float(e) for e in args.tree_eps.split(","))
    rep = bench_tree(api, inputs, torch, dev, fp64["triples_per_s"], np, workload=args.tree_only,
                     eps_list=eps_list, warm=False, n_sample=args.tree_sample, progress=True,
                     exact_file=args.tree_exact_file)
    rep["fp64_exhaustive"] = fp64
    print(json.dumps({"report": "tree", **rep}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip FP64/tree/forces/serving")
    ap.add_argument("--tree-only", metavar="WORKLOAD", default=None,
                    help="only time tree solves of this workload (e.g. gmm_n1048576), one "
                         "solve per eps without warm-up, and print their JSON report")
    ap.add_argument("--tree-eps", default="1e-2,1e-1")
    ap.add_argument("--tree-sample", type=int, default=256)
    ap.add_argument("--tree-exact-file", default=None,
                    help="npz cache of the sampled exact sums used by --tree-only")
    ap.add_argument("--paper-shape", action="store_true",
                    help="tree vs FP64 exhaustive on the paper's uniform/ball/shell shapes")
    ap.add_argument("--paper-n", type=int, nargs="+", default=list(range(1000, 10001, 1000)))
    ap.add_argument("--serving-only", action="store_true",
                    help="the serving workload as specified (60 s Poisson stream, N up to 2^18)")
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-drain", type=float, default=60.0)
    ap.add_argument("--serve-pool", type=int, default=32)
    ap.add_argument("--forces-only", action="store_true",
                    help="exhaustive and tree forces of the N = 65 536 force workload")
    ap.add_argument("--forces-n", type=int, default=65536)
    ap.add_argument("--farfield-only", action="store_true",
                    help="far-field expansion orders 0..6 on 2^20 queries")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.tree_only:
        return run_tree_only(args)
    if args.paper_shape:
        return run_paper_shape(args)
    if args.serving_only:
        return run_serving_only(args)
    if args.forces_only:
        return run_forces_only(args)
    if args.farfield_only:
        return run_farfield_only(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1105_2769_gb300 import api, inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    X = inputs.workload(WORKLOAD)
    Xd = torch.from_numpy(X).to(dev)
    ctx = api.default_context(local)
    ctx.set_timing(True)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    phi = torch.empty(len(X), dtype=torch.float64, device=dev)

    for _ in range(args.warmup):
        api.potential(Xd, mode="fp32", out=phi)
    torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    kernel_ms = []
    sampler = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    for s in range(args.steps):
        flush.zero_()                      # evict L2 between steps
        starts[s].record(stream)
        api.potential(Xd, mode="fp32", out=phi)
        ends[s].record(stream)
        kernel_ms.append(ctx.last_kernel_ms())
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if world > 1:
        dist.barrier()
    tot_ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends))
    n_trip = triples(len(X))
    value, tot_ms = aggregate(tot_ms, float(n_trip * args.steps), dist if world > 1 else None)

    props = torch.cuda.get_device_properties(dev)
    sm_max = float(_peaks().get("sm_max_mhz", 2070.0))
    peak_tflops = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    k_ms = sum(kernel_ms) / len(kernel_ms)
    achieved = FLOPS_PER_TRIPLE_FP32 * n_trip / (k_ms / 1e3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops,
                "traffic": EXH_FP32_TRAFFIC_BYTES if len(X) == N_MAIN else None,
                "traffic_note": ("ncu dram bytes per launch of the sweep (read 4.089e12, write "
                                 "1.47e10): it streams the pair table's (i,k) blocks, 16 B per "
                                 "pair term (0.7 B per triple), by design: the table replaces "
                                 "FP32 pair set-up in the sweep; algorithmic input+output is "
                                 "1.0 MB"),
                "peak_note": (f"derived: {props.multi_processor_count} SMs x 128 FP32 lanes x 2 "
                              f"x {sm_max:.0f} MHz (maximum SM clock)"),
                "kernel": "exh_fp32_pt_kernel", "flops_per_triple": FLOPS_PER_TRIPLE_FP32,
                "kernel_ms": k_ms}
    if clocks.get("sm_mhz"):
        roofline["frac_at_sampled_clock"] = achieved / (peak_tflops * clocks["sm_mhz"] / sm_max)

    # end to end through the host-buffer entry point (pinned host memory)
    Xh = torch.from_numpy(X).pin_memory().numpy()
    ph = torch.empty(len(X), dtype=torch.float64).pin_memory().numpy()
    api.potential_host(Xh, mode="fp32", out=ph)
    t0 = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 3))
    for _ in range(e2e_steps):
        api.potential_host(Xh, mode="fp32", out=ph)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e = {"value": world * n_trip / e2e_s, "unit": "triples/s",
           "h2d_bytes_per_step": int(X.nbytes), "d2h_bytes_per_step": int(ph.nbytes)}

    line = {
        "metric": METRIC, "value": value, "unit": "triples/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": len(X), "triples_per_step": n_trip,
                   "distribution": "uniform [0,32]^3, d_min 0.5, seed 2",
                   "precision": "FP32 triple arithmetic, FP64 accumulation",
                   "l2": "flushed between steps (256 MiB write)", "parallelism": f"replicas x{world}"},
        "roofline": roofline,
        "e2e": e2e,
        "gpu_launches": 2 * args.steps,
        "clocks": clocks,
    }
    if not args.no_extras and rank == 0:
        fp64 = bench_fp64(api, inputs, torch, dev)
        fp64["fp32_over_fp64"] = value / world / fp64["triples_per_s"]
        line["fp64_exhaustive"] = fp64
        line["tree"] = bench_tree(api, inputs, torch, dev, fp64["triples_per_s"], np)
        line["forces"] = bench_forces(api, inputs, torch, dev)
        line["farfield"] = bench_farfield((2, 4), 16)
        line["serving"] = bench_serving(api, inputs, np)
        # the same mix at an offered load the server keeps up with
        line["serving_at_100_req_s"] = bench_serving(api, inputs, np, rate=100.0)
    if rank == 0 and not args.no_cpu_baseline:
        r, dt, m, nt = cpu_oracle_rate(X, 0)
        line["cpu_baseline"] = {"value": r, "unit": "triples/s", "cores": nt, "kind": "oracle",
                                "sample": f"{m} seeded particles of the N={len(X)} set, "
                                          f"{dt:.1f} s; job-equivalent triples = evaluations/3"}
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
