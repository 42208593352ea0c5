#!/usr/bin/env python3
"""Benchmark of the entropy-stable DGSEM shallow-water hot path on GB300.

One step = one five-stage LSRK4(5) time step of the whole path on the
degree-sweep dam-break workload (N=7, 256x256 curved periodic quads, 4.19M
LGL nodes, FP64): per stage the primitives, the entropy-stable interface
flux, the artificial-viscosity indicator and BR1 gradients, the viscous
interface average, the volume kernel (flux differencing, source, lifts,
viscous divergence, 1/J) and the stage update with the positivity limiter;
per step the device-side CFL/positivity time step, and the mass and entropy
integrals read back to the host. Each step starts from the same input state
(one batch). The metric is RHS node-updates per second: 5 right-hand sides x
K (N+1)^2 nodes per step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun with N > 1 every rank runs an independent replica on its own
GPU (the method needs no cross-GPU exchange for independent problems), the
time is the maximum over ranks and the value the sum of the ranks' work.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

RK_STAGES = 5


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--N", type=int, default=7)
    ap.add_argument("--K1", type=int, default=None)
    ap.add_argument("--rhs-reps", type=int, default=1000,
                    help="right-hand sides per RHS-alone rate (mean and median of one call)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--no-developed", action="store_true",
                    help="skip the leg timed from the developed state (200 steps after the dam release)")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the split-form vs standard-form comparison")
    ap.add_argument("--ensemble", type=int, default=0,
                    help="members of the uneven ensemble (e.g. 256): one JSON line comparing the batched "
                         "ensemble with stepping every member through its own context")
    ap.add_argument("--adjoint", action="store_true",
                    help="gauge-misfit gradient by the adjoint (N=4, 64x64 quads, 200 steps, 64 gauges, "
                         "checkpoints every 20 steps): one JSON line against the plain forward path")
    ap.add_argument("--case", default=None, choices=["rhs", "step", "ensemble", "rhs_adjoint"],
                    help="one small, untimed invocation for profiler captures (no JSON line): "
                         "rhs = --reps right-hand sides of the ES+AV dam break at --N on --K1 x --K1 quads; "
                         "step = one warm-up step and one step with its integrals (every kernel class); "
                         "ensemble = one warm-up step (graph capture) and --steps steps of the 256-member "
                         "ensemble; rhs_adjoint = --reps right-hand-side adjoints of the dam break")
    ap.add_argument("--reps", type=int, default=3, help="repetitions of a --case invocation")
    ap.add_argument("--sweep", default=None,
                    help="comma-separated degrees: one JSON line per degree at ~4.2M nodes "
                         "(step rate, right-hand-side rates, volume-kernel roofline)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload_config(N, K1):
    return {"workload": f"dam_break N={N} {K1}x{K1} curved periodic quads, ES flux + AV + limiter, LSRK4(5)",
            "N": N, "K": K1 * K1, "nodes": K1 * K1 * (N + 1) ** 2, "eps0": 0.025, "cfl": 0.5,
            "rk": "LSRK4(5)", "l2": "inputs larger than L2 (state 0.1 GB + geometry 0.4 GB per step)"}


# ---------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index, enabled=True):
        self.index, self.p, self.out = index, None, None
        if not enabled:
            return
        try:
            self.out = open(os.devnull, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            txt, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            txt = ""
        rows = [r.split(",") for r in txt.strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return None
        sm = sorted(float(r[1]) for r in rows)
        mx = max(float(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[5 + j].strip().lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].strip() not in ("", "[N/A]"))}


# ---------------------------------------------------------------------------
# Algorithmic work of the volume kernel (flux differencing + per-node terms,
# entropy-stable path; the viscous divergence of the few viscous elements is
# not counted, so the figure is a lower bound)
# ---------------------------------------------------------------------------

def volume_flops_per_node(N):
    """28 flops per symmetric pair (2 metric sums, 4 state sums, Q: 3,
    P: 1, X2: 3, X3: 3, two-sided accumulation of 3 components: 12), N pairs
    per node (N(N+1)/2 per line, 2(N+1) lines per element); per node 9 flops
    (2gh, the three rescalings and the two source products) and the interface
    lift, 3 fused multiply-adds on each of the 4(N+1) side nodes."""
    n = N + 1
    return 28 * N + 9 + 6 * 4 * n / (n * n)


def volume_flops_per_node_direct(N):
    """Flops of the two-point form as written, per node: the averaged
    metrics and fluxes formed for every pair, 40 per pair (N pairs per node
    over its two lines) plus 20 per node for the lifts, source and scaling. The
    kernel evaluates the same right-hand side with fewer (the symmetric pair
    once, with host-precomputed pair constants); its time over this count
    reads as the rate of the direct form."""
    return 40 * N + 20


def volume_bytes_per_node(N):
    """Compulsory DRAM bytes: W (24), velocities (16), per-pair metric
    constants (2 doubles per pair, N pairs per node: 16N), -1/(w w J) and
    -2/(w w J) (16), source coefficients (16), R (24), interface flux traces
    3 x 4(N+1) doubles per element."""
    n = N + 1
    return 96 + 16 * N + 3 * 8 * 4 * n / (n * n)


def volume_traffic(N, nodes):
    """DRAM bytes per launch of the volume kernel from the committed ncu
    summary (dram__bytes_read.sum + dram__bytes_write.sum per node, measured
    on a smaller case of the same kernel and scaled by the node count), or
    None when the kernel source changed since the counters were taken."""
    import hashlib
    src = os.path.join(ROOT, "paper_1804_02221_gb300", "csrc", "k_volume.cuh")
    summ = os.path.join(ROOT, "profiles", "volume_kernel_dam_break_N7.txt")
    if not os.path.exists(summ):
        return None
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    vals = {}
    for line in open(summ):
        if "=" in line and line.strip().startswith("traffic."):
            k, v = line.strip().split("=", 1)
            vals[k.strip()] = v.strip()
    if vals.get("traffic.kernel_sha256_16") != sha or int(vals.get("traffic.N", -1)) != N:
        return None
    return float(vals["traffic.dram_bytes_per_node"]) * nodes


def volume_adjoint_flops_per_node(N):
    """Algorithmic flops of the adjoint of the volume kernel (inviscid part):
    per symmetric pair 38 (the three cotangent differences 3, the pair's
    flux Q 5, its cotangent Q^ = 2 d1 + (u_i+u_q) d2 + (v_i+v_q) d3 7, the
    pressure cotangent P^ = Sx d2 + Sy d3 3, ten cotangent accumulations
    20), N pairs per node; per node 10 (the cotangents of R scaled by
    -1/(w w J) 3, the h cotangent with the source terms 5, the source
    coefficients' cotangents 2) and the interface-flux cotangents, 3
    products on each of the 4(N+1) side nodes of an element."""
    n = N + 1
    return 38 * N + 10 + 3 * 4 * n / (n * n)


def fp64_peak_gflops(sm_mhz):
    """152 SMs x 2 FP64 fused multiply-adds per clock (measured: 1.9 DFMA/clk/SM
    with independent chains at 2070 MHz nominal) x 2 flops."""
    return 152 * 2 * 2 * sm_mhz * 1e6 / 1e9


def combine_ranks(ms_step, e2e_ms, nodes, world_size, dist=None, device="cpu"):
    """Replicas: every rank advanced its own mesh of `nodes` nodes. The step
    time is the maximum over ranks and the value the work of all ranks over
    that time. Returns (ms_step, e2e_ms, value, e2e_value)."""
    import torch
    if dist is not None and world_size > 1:
        t = torch.tensor([ms_step, e2e_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step, e2e_ms = float(t[0]), float(t[1])
    value = world_size * RK_STAGES * nodes / (ms_step * 1e-3)
    e2e_value = world_size * RK_STAGES * nodes / (e2e_ms * 1e-3)
    return ms_step, e2e_ms, value, e2e_value


# ---------------------------------------------------------------------------
# Oracle timing (CPU baseline and reference arm)
# ---------------------------------------------------------------------------

def oracle_rate(N, K1, steps, warmup=0, variant=None, prob=None):
    from oracle import oracle as O
    from paper_1804_02221_gb300 import inputs as I
    p = prob if prob is not None else I.dam_break(N=N, K1=K1)
    o = O.Oracle(p, flux=1, av=True, eps0=0.025, limiter=True, rk=0, cfl=0.5, variant=variant)
    for _ in range(warmup):
        o.step(p.W, 0.0, 1)
        o.entropy(p.W)
    t0 = time.perf_counter()
    for _ in range(steps):
        W, rc, _ = o.step(p.W, 0.0, 1)
        o.entropy(W)
        o.mass(W)
    t = (time.perf_counter() - t0) / max(steps, 1)
    return RK_STAGES * p.nodes / t, t, O.threads(variant), p.nodes


def cpu_model():
    """The host CPU's model name (from /proc/cpuinfo, else the platform)."""
    import platform
    try:
        for line in open("/proc/cpuinfo"):
            key = line.split(":")[0].strip().lower()
            if key in ("model name", "cpu model", "hardware"):
                return line.split(":", 1)[1].strip()
        parts = {"0xd4f": "Arm Neoverse V2", "0xd40": "Arm Neoverse V1", "0xd49": "Arm Neoverse N2",
                 "0xd0c": "Arm Neoverse N1"}
        for line in open("/proc/cpuinfo"):
            if line.split(":")[0].strip().lower() == "cpu part":
                part = line.split(":", 1)[1].strip().lower()
                return f"{platform.machine()} {parts.get(part, 'cpu part ' + part)}"
    except OSError:
        pass
    return platform.machine()


def run_reference(args):
    """The oracle on the host cores, on the GPU arm's own workload (the full
    N=7 256x256 dam break unless --N/--K1 say otherwise): `steps` full
    LSRK4(5) steps after `warmup` untimed ones, each step followed by the
    mass and entropy of the new state."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    N = args.N
    K1 = args.K1 or int(round(2048 / (N + 1)))
    rate, t, cores, nodes = oracle_rate(N, K1, args.steps, args.warmup)
    sample = (f"dam_break N={N} on {K1}x{K1} quads ({nodes} nodes, the GPU arm's workload), "
              f"{args.steps} full LSRK4(5) steps after {args.warmup} untimed, {t:.2f} s per step")
    line = {"impl": "reference", "metric": "RHS node-updates/s (FP64)", "value": rate,
            "unit": "node-updates/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": workload_config(N, K1),
            "cpu_baseline": {"value": rate, "unit": "node-updates/s", "cores": cores, "kind": "oracle",
                             "sample": sample, "cpu_model": cpu_model()},
            "e2e": {"value": rate, "unit": "node-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def kernel_ms(ctx, W0, R, which="volume", reps=10):
    """Mean event time of one launch of kernel class `which` over `reps`
    right-hand sides (after two untimed ones)."""
    import torch
    for _ in range(2):
        ctx.rhs(W0, R)
    torch.cuda.synchronize()
    ctx.timing(True, classes=(which,))
    for _ in range(reps):
        ctx.rhs(W0, R)
    torch.cuda.synchronize()
    ms, cnt = ctx.timing_read(which)
    ctx.timing(False)
    return ms / max(cnt, 1)


def rhs_rate(ctx, W0, R, nodes, reps=10):
    import torch
    stream = torch.cuda.current_stream()
    for _ in range(2):
        ctx.rhs(W0, R)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        ctx.rhs(W0, R)
    b.record(stream)
    torch.cuda.synchronize()
    return nodes / (a.elapsed_time(b) / reps * 1e-3)


def rhs_stats(ctx, W0, R, nodes, reps):
    """`reps` right-hand sides back to back after two untimed ones, an event
    between consecutive calls: node-updates/s from the mean time, and the
    mean and median time of one call (the paper's protocol: the mean of
    1000 evaluations)."""
    import torch
    stream = torch.cuda.current_stream()
    for _ in range(2):
        ctx.rhs(W0, R)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
    ev[0].record(stream)
    for i in range(reps):
        ctx.rhs(W0, R)
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    t = sorted(ev[i].elapsed_time(ev[i + 1]) for i in range(reps))
    mean = ev[0].elapsed_time(ev[reps]) / reps
    med = t[reps // 2] if reps % 2 else 0.5 * (t[reps // 2 - 1] + t[reps // 2])
    return {"node_updates_per_s": nodes / (mean * 1e-3), "ms_mean": mean, "ms_median": med, "reps": reps}


def split_vs_standard(prob, W0, R):
    """The paper's GPU comparison (Eq. VolInt): the split-form volume kernel
    against the standard one on the same state (ES interface flux, no AV, so
    both kernels do only their volume work), and the full right-hand sides
    with ES flux + AV in both forms."""
    from paper_1804_02221_gb300 import swedg
    out = {}
    for name, vol in (("split", 0), ("standard", 1)):
        c = swedg.SweContext.from_problem(prob, flux=1, volume=vol)
        out[f"volume_ms_{name}"] = kernel_ms(c, W0, R)
        c.close()
        c = swedg.SweContext.from_problem(prob, flux=1, av=True, eps0=0.025, volume=vol)
        out[f"rhs_es_av_node_updates_per_s_{name}"] = rhs_rate(c, W0, R, prob.nodes)
        c.close()
    out["volume_ratio_split_over_standard"] = out["volume_ms_split"] / out["volume_ms_standard"]
    out["rhs_ratio_split_over_standard"] = (out["rhs_es_av_node_updates_per_s_standard"] /
                                            out["rhs_es_av_node_updates_per_s_split"])
    return out


def sweep(args):
    """Degree sweep of the same workload recipe at ~4.2M nodes per degree."""
    import torch

    from paper_1804_02221_gb300 import inputs as I
    from paper_1804_02221_gb300 import swedg
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    for N in [int(v) for v in args.sweep.split(",")]:
        K1 = int(round(2048 / (N + 1)))
        prob = I.dam_break(N=N, K1=K1)
        kw = dict(flux=1, av=True, eps0=0.025, limiter=True, rk=0, cfl=0.5)
        ctx = swedg.SweContext.from_problem(prob, **kw)
        W0 = torch.from_numpy(prob.W).cuda()
        W = torch.empty_like(W0)
        for _ in range(args.warmup):
            W.copy_(W0)
            ctx.step(W, 0.0, 1)
        torch.cuda.synchronize()
        ctx.timing(True, classes=("volume",))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            W.copy_(W0)
            ctx.step_integrals(W, 0.0, 1)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        vol_ms, vol_n = ctx.timing_read("volume")
        ctx.timing(False)
        rates, med = {}, {}
        R = torch.empty_like(W0)
        for name, kk in (("ES+AV", kw), ("EC", dict(flux=0))):
            c2 = ctx if name == "ES+AV" else swedg.SweContext.from_problem(prob, **kk)
            st = rhs_stats(c2, W0, R, prob.nodes, args.rhs_reps)
            rates[name] = st["node_updates_per_s"]
            med[name] = st["ms_median"]
            if c2 is not ctx:
                c2.close()
        vol = vol_ms / vol_n
        achieved = volume_flops_per_node(N) * prob.nodes / (vol * 1e-3) / 1e12
        peak = fp64_peak_gflops(2070.0) / 1e3
        cmp = split_vs_standard(prob, W0, R)
        print(json.dumps({"sweep": True, "N": N, "K": prob.K, "nodes": prob.nodes, "ms_per_step": ms,
                          "node_updates_per_s": RK_STAGES * prob.nodes / (ms * 1e-3),
                          "rhs_node_updates_per_s": rates, "rhs_ms_median": med, "rhs_reps": args.rhs_reps,
                          "volume_ms": vol,
                          "volume_tflops": achieved, "volume_frac_at_2070MHz": achieved / peak,
                          "volume_gbs_algorithmic": volume_bytes_per_node(N) * prob.nodes / (vol * 1e-3) / 1e9,
                          "split_vs_standard": cmp}), flush=True)
        ctx.close()


def ensemble_bench(args):
    """The uneven ensemble (16x16..96x96 quads, N in {3, 5, 7}): `steps`
    adaptive LSRK4(5) steps of all members in one swe_ens_step call (one graph
    replay per step) against the plain path, every member advanced by its own
    context in its own swe_step call. Same members, same parameters, the same
    results bit for bit."""
    import torch

    from paper_1804_02221_gb300 import inputs as I
    from paper_1804_02221_gb300 import swedg
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    probs = I.ensemble(args.ensemble)
    t_gen = time.perf_counter() - t0
    kw = dict(flux=1, av=True, eps0=0.01, limiter=True, rk=0, cfl=0.5)
    nodes = sum(p.nodes for p in probs)
    t0 = time.perf_counter()
    ens = swedg.SweEnsemble(probs, **kw)
    t_create = time.perf_counter() - t0
    W0 = ens.pack([p.W for p in probs])
    W = torch.empty_like(W0)

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    W.copy_(W0)
    ens.step(W, 0.0, args.warmup)
    W.copy_(W0)
    l0 = ens.launches()
    ms_ens = timed(lambda: ens.step(W, 0.0, args.steps)) / args.steps
    launches_ens = ens.launches() - l0
    Wens = W.clone()
    R = torch.empty_like(W0)
    ens.rhs(W0, R)
    ms_rhs_ens = timed(lambda: [ens.rhs(W0, R) for _ in range(5)]) / 5

    groups_default = ens.groups()
    groups_tuned = ens.autotune(W0)
    W.copy_(W0)
    ens.step(W, 0.0, 1)
    W.copy_(W0)
    ms_tuned = timed(lambda: ens.step(W, 0.0, args.steps)) / args.steps
    same_tuned = torch.equal(W, Wens)

    ctxs = [swedg.SweContext.from_problem(p, **kw) for p in probs]
    Ws = [torch.from_numpy(p.W).cuda() for p in probs]
    for c, w in zip(ctxs, Ws):
        c.step(w, 0.0, args.warmup)
    for w, p in zip(Ws, probs):
        w.copy_(torch.from_numpy(p.W))
    l0 = sum(c.launches() for c in ctxs)
    ms_plain = timed(lambda: [c.step(w, 0.0, args.steps) for c, w in zip(ctxs, Ws)]) / args.steps
    launches_plain = sum(c.launches() for c in ctxs) - l0
    same = all(torch.equal(ens.view(Wens, i), Ws[i]) for i in range(len(probs)))
    Rs = [torch.empty_like(w) for w in Ws]
    Wi = [torch.from_numpy(p.W).cuda() for p in probs]
    ms_rhs_plain = timed(lambda: [[c.rhs(w, r) for c, w, r in zip(ctxs, Wi, Rs)] for _ in range(5)]) / 5
    rate = lambda ms: RK_STAGES * nodes / (ms * 1e-3)
    line = {
        "ensemble": True, "metric": "RHS node-updates/s (FP64)", "unit": "node-updates/s",
        "members": len(probs), "nodes": nodes, "groups": ens.ngroups,
        "degrees": {str(N): sum(1 for p in probs if p.N == N) for N in sorted({p.N for p in probs})},
        "steps": args.steps, "warmup": args.warmup,
        "batched": {"value": rate(ms_ens), "ms_per_step": ms_ens, "gpu_launches": launches_ens,
                    "rhs_node_updates_per_s": nodes / (ms_rhs_ens * 1e-3)},
        "plain": {"value": rate(ms_plain), "ms_per_step": ms_plain, "gpu_launches": launches_plain,
                  "rhs_node_updates_per_s": nodes / (ms_rhs_plain * 1e-3)},
        "batched_autotuned": {"value": rate(ms_tuned), "ms_per_step": ms_tuned, "bitwise_equal": same_tuned,
                              "groups": [{"N": g[0], "members": g[1], "volume_threads_per_block": g[2],
                                          "update_warps_per_block": g[3]} for g in groups_tuned],
                              "default_groups": [list(g) for g in groups_default]},
        "speedup": ms_plain / ms_ens, "speedup_autotuned": ms_plain / ms_tuned, "bitwise_equal": same,
        "setup_s": {"inputs": t_gen, "create": t_create},
        "config": {"workload": f"uneven ensemble: {len(probs)} members, 16x16..96x96 curved periodic quads, "
                               "N in {3,5,7}, seeded 8-Gaussian bathymetry + Gaussian hump, ES+AV(eps0=0.01)"
                               "+limiter, adaptive LSRK4(5) CFL 0.5",
                   "l2": "inputs larger than L2 (~0.95 GB state)"},
    }
    print(json.dumps(line), flush=True)


def adjoint_bench(args):
    """The adjoint workload: N = 4 on 64 x 64 curved periodic quads (lake at rest
    with a hump, ES flux, AV in every element, LSRK4(5) at CFL 0.5), 200
    adaptive steps, loss = squared h misfit at 64 seeded gauges against a run
    over a perturbed bathymetry, gradients with respect to the initial state
    and the bathymetry by the library's adjoint with checkpoints every 20
    steps. Reported against the plain forward path on the same run."""
    import numpy as np
    import torch

    from paper_1804_02221_gb300 import inputs as I
    from paper_1804_02221_gb300 import swedg
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    N, K1, T, G, C = 4, 64, 200, 64, 20
    p = I.lake_hump(N=N, K1=K1, amp=0.05)
    kw = dict(flux=1, av=True, eps0=0.01, sigma_min=-301.0, sigma_max=-300.0, rk=0, cfl=0.5)
    ctx = swedg.SweContext.from_problem(p, **kw)
    rng = np.random.default_rng(3)
    pts = rng.uniform(0.1, 1.9, size=(G, 2))
    gw = I.gauge_weights(p, pts)
    elem = torch.tensor([k for k, _ in gw], dtype=torch.int32, device="cuda")
    wts = torch.tensor(np.stack([w.reshape(-1) for _, w in gw]), dtype=torch.float64, device="cuda")
    q = I.Problem(p.name, p.N, p.Kx, p.Ky, p.x, p.y, p.b + 0.02 * np.sin(np.pi * p.x) * np.sin(np.pi * p.y),
                  p.W, p.EToE, p.EToF, p.flip, p.g)
    ctx_t = swedg.SweContext.from_problem(q, **kw)
    target = torch.zeros(T, G, dtype=torch.float64, device="cuda")
    swedg.GaugeLoss(ctx_t, elem, wts, torch.zeros_like(target), T).forward(torch.from_numpy(p.W).cuda(),
                                                                           record=target)
    W0 = torch.from_numpy(p.W).cuda()

    def timed(fn):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        out = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b), out

    run = swedg.GaugeLoss(ctx, elem, wts, target, T, checkpoint=C)
    run.forward(W0)
    run.backward()
    ms_fwd, loss = timed(lambda: run.forward(W0))
    ms_bwd, (Wbar, bbar) = timed(lambda: run.backward())
    # the reverse sweep that recomputes every step inside its step adjoint
    ms_bwd_rc, (Wbar_rc, bbar_rc) = timed(lambda: run.backward(recorded=False))
    same = bool(torch.equal(Wbar, Wbar_rc) and torch.equal(bbar, bbar_rc))
    # plain forward path: the same 200 steps without the gauges
    W = W0.clone()
    ms_plain, _ = timed(lambda: [ctx.step(W, dt, 1) for dt in run.dts])
    # one right-hand side and its adjoint
    R = torch.empty_like(W0)
    Rbar = torch.randn_like(W0)
    ms_rhs, _ = timed(lambda: [ctx.rhs(W0, R) for _ in range(20)])
    Wb, bb = torch.zeros_like(W0), torch.zeros_like(W0[0])
    ms_rhs_adj, _ = timed(lambda: [ctx.rhs_adjoint(W0, Rbar, Wb, bb) for _ in range(20)])
    nodes = p.nodes
    # launch shapes on this mesh (4096 elements: 164 blocks of the default
    # 128-thread volume shape for 152 SMs): the tuner's choice against the
    # defaults, on the plain forward path and one right-hand side
    ctx.autotune(W0)
    tuned = ctx.tuning()
    W = W0.clone()
    ms_plain_t, _ = timed(lambda: [ctx.step(W, dt, 1) for dt in run.dts])
    ms_rhs_t, _ = timed(lambda: [ctx.rhs(W0, R) for _ in range(20)])
    ctx.set_tuning(128, 4)
    # one right-hand side and its adjoint at the main workload's size (N=7, 4.19M nodes)
    big = I.dam_break(N=7)
    cb = swedg.SweContext.from_problem(big, flux=1, av=True, eps0=0.025)
    Wd = torch.from_numpy(big.W).cuda()
    Rd, Rbd = torch.empty_like(Wd), torch.randn_like(Wd)
    Wbd, bbd = torch.zeros_like(Wd), torch.zeros_like(Wd[0])
    cb.rhs(Wd, Rd)
    cb.rhs_adjoint(Wd, Rbd, Wbd, bbd)
    ms_big, _ = timed(lambda: [cb.rhs(Wd, Rd) for _ in range(5)])
    ms_big_adj, _ = timed(lambda: [cb.rhs_adjoint(Wd, Rbd, Wbd, bbd) for _ in range(5)])
    # the launch time of every kernel class within one right-hand-side adjoint
    # (events around every launch: a pass of its own), and the reverse volume
    # kernel against its algorithmic flops
    cb.timing(True)
    for _ in range(5):
        cb.rhs_adjoint(Wd, Rbd, Wbd, bbd)
    torch.cuda.synchronize()
    adj_classes = {}
    for name in swedg.KERNEL_CLASSES:
        t, n_l = cb.timing_read(name)
        if n_l:
            adj_classes[name] = {"ms_per_rhs_adjoint": t / 5, "launches_per_rhs_adjoint": n_l / 5}
    cb.timing(False)
    vol_adj_ms = adj_classes["adjoint_volume"]["ms_per_rhs_adjoint"] / adj_classes["adjoint_volume"][
        "launches_per_rhs_adjoint"]
    vol_fwd_ms = kernel_ms(cb, Wd, Rd, "volume", reps=5)
    fl_adj = volume_adjoint_flops_per_node(7) * big.nodes / (vol_adj_ms * 1e-3) / 1e12
    peak = fp64_peak_gflops(2070.0) / 1e3
    cb.close()
    line = {
        "adjoint": True, "metric": "RHS node-updates/s (FP64)", "unit": "node-updates/s",
        "config": {"workload": f"gauge-misfit gradient, N={N} {K1}x{K1} curved periodic quads ({nodes} nodes), "
                               f"{T} LSRK4(5) steps, {G} gauges, checkpoints every {C}, ES+AV"},
        "loss": float(loss),
        "forward": {"ms_per_step": ms_fwd / T, "value": RK_STAGES * nodes / (ms_fwd / T * 1e-3)},
        "plain_forward": {"ms_per_step": ms_plain / T, "value": RK_STAGES * nodes / (ms_plain / T * 1e-3)},
        "backward": {"ms_per_step": ms_bwd / T, "value": RK_STAGES * nodes / (ms_bwd / T * 1e-3),
                     "note": "per step: one recorded recomputation of the step (checkpoint segments), "
                             "5 stage adjoints"},
        "gradient_over_plain": (ms_fwd + ms_bwd) / ms_plain,
        "backward_recomputing": {"ms_per_step": ms_bwd_rc / T,
                                 "gradient_over_plain": (ms_fwd + ms_bwd_rc) / ms_plain,
                                 "bitwise_equal": same,
                                 "note": "the step adjoint recomputes its step again (no records)"},
        "rhs": {"ms": ms_rhs / 20, "value": nodes / (ms_rhs / 20 * 1e-3)},
        "rhs_adjoint": {"ms": ms_rhs_adj / 20, "value": nodes / (ms_rhs_adj / 20 * 1e-3),
                        "note": "includes the forward recomputation of the right-hand side"},
        "grad_norms": {"W0": float(Wbar.norm()), "b": float(bbar.norm())},
        "autotune": {"volume_threads_per_block": tuned[0], "update_warps_per_block": tuned[1],
                     "default": [128, 4],
                     "plain_forward_ms_per_step": {"default": ms_plain / T, "tuned": ms_plain_t / T},
                     "rhs_ms": {"default": ms_rhs / 20, "tuned": ms_rhs_t / 20},
                     "note": "swe_autotune on this mesh's state; every shape computes bitwise the same"},
        "large": {"workload": f"dam_break N=7 256x256 ({big.nodes} nodes), ES+AV",
                  "rhs_ms": ms_big / 5, "rhs_adjoint_ms": ms_big_adj / 5,
                  "rhs_value": big.nodes / (ms_big / 5 * 1e-3),
                  "rhs_adjoint_value": big.nodes / (ms_big_adj / 5 * 1e-3),
                  "ratio": ms_big_adj / ms_big,
                  "rhs_adjoint_kernels": adj_classes,
                  "volume_adjoint": {"ms_per_launch": vol_adj_ms, "forward_volume_ms_per_launch": vol_fwd_ms,
                                     "ratio_to_forward": vol_adj_ms / vol_fwd_ms,
                                     "flops_per_node": volume_adjoint_flops_per_node(7),
                                     "roofline": {"bound": "alu", "achieved": fl_adj, "peak": peak,
                                                  "unit": "TFLOP/s", "frac": fl_adj / peak,
                                                  "peak_note": "152 SMs x 2 DFMA/clk x 2 flops at 2070 MHz"}}},
    }
    print(json.dumps(line), flush=True)


def e2e_pipelined(ctx, Wh, W, steps, res, res_h, barrier):
    """End to end through the C ABI from pinned host memory: each step's
    state uploaded on a copy stream into the other of two device buffers
    while the previous step computes (the upload into a buffer waits for the
    step that last read it), the step's integrals, step size and status
    copied back to pinned host memory. Returns ms per step (host clock)."""
    import torch
    stream = torch.cuda.current_stream()
    Wb = [W, torch.empty_like(W)]
    cs = torch.cuda.Stream()
    arrived = [torch.cuda.Event(), torch.cuda.Event()]
    freed = [torch.cuda.Event(), torch.cuda.Event()]
    res_h.zero_()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    with torch.cuda.stream(cs):
        Wb[0].copy_(Wh, non_blocking=True)
        arrived[0].record(cs)
    for i in range(steps):
        cur = i % 2
        stream.wait_event(arrived[cur])
        if i + 1 < steps:
            with torch.cuda.stream(cs):
                if i >= 1:
                    cs.wait_event(freed[1 - cur])
                Wb[1 - cur].copy_(Wh, non_blocking=True)
                arrived[1 - cur].record(cs)
        ctx.step_async(Wb[cur], 0.0, 1, out=res[i])
        res_h[i].copy_(res[i], non_blocking=True)
        freed[cur].record(stream)
    torch.cuda.synchronize()
    return (time.perf_counter() - t0) * 1e3 / steps


def viscous_fraction(ctx, W, R):
    """Share of the elements with a nonzero viscosity in the right-hand side of W."""
    ctx.rhs(W, R)
    return float((ctx.epsilon() > 0).double().mean())


def developed_leg(prob, W0, args, shapes, barrier, advance=200, cfl_visc=0.25, all_viscous=False):
    """The same workload in a developed state: the dam break advanced
    `advance` adaptive steps under the viscous time-step restriction
    (cfl_visc; under the paper's rule alone this run's time step collapses),
    then `steps` timed steps each restarting from that state, with the same
    device-timed and end-to-end loops as the t = 0 line. all_viscous: the
    indicator thresholds set so that every element carries eps0 (the upper
    bound of the viscous work), timed from the start state (advance 0)."""
    import torch

    from paper_1804_02221_gb300 import swedg
    stream = torch.cuda.current_stream()
    kw = dict(flux=1, av=True, eps0=0.025, limiter=True, rk=0, cfl=0.5, cfl_visc=cfl_visc)
    if all_viscous:
        kw.update(sigma_min=-301.0, sigma_max=-300.0)
    ctx = swedg.SweContext.from_problem(prob, **kw)
    ctx.set_tuning(*shapes)
    Wd = W0.clone()
    adv = torch.zeros((max(advance, 1), 6), dtype=torch.float64, device="cuda")
    for i in range(advance):
        ctx.step_async(Wd, 0.0, 1, out=adv[i])
    torch.cuda.synchronize()
    a = adv[:advance].cpu()
    if int((a[:, 5] != 0).sum()):
        raise RuntimeError("the developed state's advance failed")
    R = torch.empty_like(W0)
    frac = viscous_fraction(ctx, Wd, R)
    W = torch.empty_like(W0)
    for _ in range(args.warmup):
        W.copy_(Wd)
        ctx.step_async(W, 0.0, 1)
    res = torch.zeros((args.steps, 6), dtype=torch.float64, device="cuda")
    res_h = torch.zeros((args.steps, 6), dtype=torch.float64).pin_memory()
    ctx.timing(True, classes=("volume",))
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        W.copy_(Wd)
        ctx.step_async(W, 0.0, 1, out=res[i])
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    r = res.cpu()
    if int((r[:, 5] != 0).sum()):
        raise RuntimeError("a timed step from the developed state failed")
    ms = e0.elapsed_time(e1) / args.steps
    vol_ms, vol_n = ctx.timing_read("volume")
    ctx.timing(False)
    Wh = Wd.cpu().pin_memory()
    e2e_ms = e2e_pipelined(ctx, Wh, W, args.steps, res, res_h, barrier)
    if int((res_h[:, 5] != 0).sum()):
        raise RuntimeError("an end-to-end step from the developed state failed")
    out = {"ms_per_step": ms, "volume_ms_per_launch": vol_ms / max(vol_n, 1),
           "viscous_element_fraction": frac, "advanced_steps": advance,
           "t": float(a[:, 4].sum()), "dt": float(r[0, 4]), "cfl_visc": cfl_visc,
           "e2e_ms_per_step": e2e_ms}
    ctx.close()
    return out


def profile_case(args):
    """Small invocations that ncu captures; they print a check value, not a rate."""
    import torch

    from paper_1804_02221_gb300 import inputs as I
    from paper_1804_02221_gb300 import swedg

    torch.cuda.set_device(0)
    if args.case == "ensemble":
        probs = I.ensemble(256)
        ens = swedg.SweEnsemble(probs, flux=1, av=True, eps0=0.01, limiter=True, rk=0, cfl=0.5)
        W = ens.pack([p.W for p in probs])
        ens.step(W, 0.0, 1)
        ens.step(W, 0.0, args.steps)
        torch.cuda.synchronize()
        print("ok", float(W.abs().max()), "launches", ens.launches())
        ens.close()
        return
    N = args.N
    K1 = args.K1 or int(round(2048 / (N + 1)))
    p = I.dam_break(N=N, K1=K1)
    if args.case == "step":
        ctx = swedg.SweContext.from_problem(p, flux=1, av=True, eps0=0.025, limiter=True, rk=0, cfl=0.5)
    else:
        ctx = swedg.SweContext.from_problem(p, flux=1, av=True, eps0=0.025)
    W0 = torch.from_numpy(p.W).cuda()
    if args.case == "rhs":
        R = torch.empty_like(W0)
        for _ in range(args.reps):
            ctx.rhs(W0, R)
        check = float(R.abs().max())
    elif args.case == "step":
        W = W0.clone()
        ctx.step(W, 0.0, 1)
        W.copy_(W0)
        check = ctx.step_integrals(W, 0.0, 1)
    else:
        gen = torch.Generator(device="cuda").manual_seed(1)
        Rb = torch.randn(W0.shape, dtype=W0.dtype, device="cuda", generator=gen)
        Wb, bb = torch.zeros_like(W0), torch.zeros_like(W0[0])
        for _ in range(args.reps):
            ctx.rhs_adjoint(W0, Rb, Wb, bb)
        check = float(Wb.abs().max())
    torch.cuda.synchronize()
    print("ok", check)
    ctx.close()


def main():
    args = parse()
    if args.case:
        profile_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    if args.sweep:
        sweep(args)
        return
    if args.ensemble:
        ensemble_bench(args)
        return
    if args.adjoint:
        adjoint_bench(args)
        return
    import numpy as np
    import torch

    from paper_1804_02221_gb300 import inputs as I
    from paper_1804_02221_gb300 import swedg

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    N = args.N
    K1 = args.K1 or int(round(2048 / (N + 1)))
    prob = I.dam_break(N=N, K1=K1)
    kw = dict(flux=1, av=True, eps0=0.025, limiter=True, rk=0, cfl=0.5)
    ctx = swedg.SweContext.from_problem(prob, **kw)
    W0 = torch.from_numpy(prob.W).cuda()
    W = torch.empty_like(W0)
    nodes = prob.nodes
    stream = torch.cuda.current_stream()

    def one_step(Wd):
        # the step, and the mass, momenta and entropy of the new state read
        # back to the host (one synchronisation for both)
        ctx.step_integrals(Wd, 0.0, 1)

    # Timed loops: the step and its integrals enqueued without a host
    # synchronisation (swe_step_async); every step's integrals, step size and
    # status land in a row of `res`, checked after the loop.
    res = torch.zeros((args.steps, 6), dtype=torch.float64, device="cuda")
    res_h = torch.zeros((args.steps, 6), dtype=torch.float64).pin_memory()

    def check_steps(rows):
        bad = int((rows[:, 5] != 0).sum())
        if bad:
            raise RuntimeError(f"{bad} timed steps failed (status bits {rows[:, 5].max().item():.0f})")

    # launch shapes only: results are bitwise the same for every shape
    shapes = ctx.tuning() if args.no_autotune else ctx.autotune(W0)

    for _ in range(args.warmup):
        W.copy_(W0)
        one_step(W)
    torch.cuda.synchronize()

    # ---- device-resident timed region ----
    clocks = Clocks(local, enabled=not args.no_clocks)
    time.sleep(0.3)
    # events around the volume kernel's launches only: the roofline's launch
    # time; the other classes are timed in a pass of their own below
    ctx.timing(True, classes=("volume",))
    l0 = ctx.launches()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        W.copy_(W0)
        ctx.step_async(W, 0.0, 1, out=res[i])
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    check_steps(res.cpu())
    launches = ctx.launches() - l0
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    vol_ms, vol_n = ctx.timing_read("volume")
    ctx.timing(False)

    # ---- per-class kernel times: events around every launch, own pass ----
    ctx.timing(True)
    for _ in range(min(args.steps, 10)):
        W.copy_(W0)
        one_step(W)
    torch.cuda.synchronize()
    kernels = {}
    for name in swedg.KERNEL_CLASSES:
        t, c = ctx.timing_read(name)
        if c:
            kernels[name] = {"ms_total": t, "launches": c, "ms_per_launch": t / c}
    ctx.timing(False)

    # ---- end to end through the C ABI with host buffers ----
    Wh = torch.from_numpy(prob.W).pin_memory()
    for _ in range(2):
        W.copy_(Wh, non_blocking=True)
        one_step(W)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for i in range(args.steps):
        W.copy_(Wh, non_blocking=True)
        ctx.step_async(W, 0.0, 1, out=res[i])
        res_h[i].copy_(res[i], non_blocking=True)  # the step's results to the host
    torch.cuda.synchronize()
    e2e_serial_ms = (time.perf_counter() - t0) * 1e3 / args.steps
    check_steps(res_h)

    # pipelined: the next step's input uploaded on a copy stream (e2e_pipelined)
    e2e_ms = e2e_pipelined(ctx, Wh, W, args.steps, res, res_h, barrier)
    check_steps(res_h)

    # ---- RHS alone: entropy-conservative vs entropy-stable + AV ----
    rhs_rates, rhs_median = {}, {}
    R = torch.empty_like(W0)
    for name, kk in (("ES+AV", kw), ("EC", dict(flux=0))):
        c2 = ctx if name == "ES+AV" else swedg.SweContext.from_problem(prob, **kk)
        st = rhs_stats(c2, W0, R, nodes, args.rhs_reps)
        rhs_rates[name] = st["node_updates_per_s"]
        rhs_median[name] = st["ms_median"]

    # ---- the paper's comparison: split-form vs standard volume kernel ----
    cmp = None if args.no_compare else split_vs_standard(prob, W0, R)

    # ---- the viscous share of the t = 0 state, and the developed state ----
    visc0 = viscous_fraction(ctx, W0, R)
    dev = None if args.no_developed else developed_leg(prob, W0, args, shapes, barrier)
    allv = None if args.no_developed else developed_leg(prob, W0, args, shapes, barrier, advance=0,
                                                         all_viscous=True)

    # ---- reduce over ranks ----
    t_step, e2e_ms, value, e2e_value = combine_ranks(ms, e2e_ms, nodes, ws, dist, "cuda")
    _, e2e_serial_ms, _, e2e_serial_value = combine_ranks(ms, e2e_serial_ms, nodes, ws, dist, "cuda")
    for leg in (dev, allv):
        if leg is not None:
            leg["ms_per_step"], leg["e2e_ms_per_step"], leg["value"], leg["e2e_value"] = combine_ranks(
                leg["ms_per_step"], leg["e2e_ms_per_step"], nodes, ws, dist, "cuda")

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    sm_mhz = clk["sm_mhz"] if clk else 2070.0
    vol_avg_ms = vol_ms / vol_n if vol_n else float("nan")
    flops = volume_flops_per_node(N) * nodes
    achieved = flops / (vol_avg_ms * 1e-3) / 1e12
    peak = fp64_peak_gflops(sm_mhz) / 1e3
    traffic = volume_traffic(N, nodes)
    line = {
        "metric": "RHS node-updates/s (FP64)", "value": value, "unit": "node-updates/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": dict(workload_config(N, K1), viscous_element_fraction=visc0),
        "roofline": {"bound": "alu", "kernel": "volume", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                     "ms_per_launch": vol_avg_ms, "flops_per_launch": flops,
                     "flops_per_node": volume_flops_per_node(N),
                     "direct_form": {"flops_per_node": volume_flops_per_node_direct(N),
                                     "achieved": volume_flops_per_node_direct(N) * nodes / (vol_avg_ms * 1e-3) / 1e12,
                                     "frac": volume_flops_per_node_direct(N) * nodes / (vol_avg_ms * 1e-3) / 1e12 / peak,
                                     "note": "the same launch time over the flops of the two-point form as written "
                                             "(averaged metrics and fluxes per pair); frac above 1 only says the "
                                             "kernel does fewer operations than that form"},
                     "bytes_per_launch": volume_bytes_per_node(N) * nodes,
                     "peak_note": "FP64 ALU: 152 SMs x 2 DFMA/clk x 2 flops at the median SM clock sampled "
                                  "during the timed region (MEASURED_PEAKS has no FP64 figure)"},
        "e2e": {"value": e2e_value, "unit": "node-updates/s", "h2d_bytes_per_step": int(W0.numel() * 8),
                "d2h_bytes_per_step": 6 * 8, "ms_per_step": e2e_ms,
                "note": "host wall clock; each step's state uploaded from pinned host memory on a copy stream "
                        "into a second device buffer while the previous step computes, the step's "
                        "integrals, step size and status copied back to pinned host memory; steps "
                        "enqueued without a host synchronisation (swe_step_async), one at the end",
                "serial": {"value": e2e_serial_value, "ms_per_step": e2e_serial_ms,
                           "note": "the upload on the compute stream before each step (no overlap)"}},
        "gpu_launches": launches,
        "clocks": clk,
        "kernels": kernels,
        "kernels_note": "per-class event times from a pass of its own (every launch bracketed by events); "
                        "the timed steps carry events around the volume kernel only",
        "rhs_only_node_updates_per_s": rhs_rates,
        "rhs_only_ms_median": rhs_median, "rhs_only_reps": args.rhs_reps,
        "launch_shapes": {"volume_threads_per_block": shapes[0], "update_warps_per_block": shapes[1]},
        "split_vs_standard": cmp,
        "scalar_updates_per_s": 3 * value,
    }
    if dev is not None:
        # the same workload 200 steps after the dam release (viscous time-step
        # restriction on, which keeps that run stable); the headline stays t = 0
        dvol = dev["volume_ms_per_launch"]
        line["developed"] = {
            "value": dev["value"], "unit": "node-updates/s",
            "ms_per_step": dev["ms_per_step"],
            "e2e": {"value": dev["e2e_value"],
                    "ms_per_step": dev["e2e_ms_per_step"], "h2d_bytes_per_step": int(W0.numel() * 8),
                    "d2h_bytes_per_step": 6 * 8},
            "viscous_element_fraction": dev["viscous_element_fraction"],
            "roofline": {"bound": "alu", "kernel": "volume", "ms_per_launch": dvol,
                         "achieved": flops / (dvol * 1e-3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                         "frac": flops / (dvol * 1e-3) / 1e12 / peak,
                         "note": "algorithmic flops of the inviscid pair loop; the viscous divergence of "
                                 "the viscous elements is extra work not counted"},
            "state": {"advanced_steps": dev["advanced_steps"], "t": dev["t"], "dt": dev["dt"],
                      "cfl_visc": dev["cfl_visc"]},
            "config": {"workload": workload_config(N, K1)["workload"] + ", 200 steps after the dam release, "
                                                                         "viscous time-step restriction cfl_visc=0.25"}}
    if allv is not None:
        avol = allv["volume_ms_per_launch"]
        line["all_viscous"] = {
            "value": allv["value"], "unit": "node-updates/s", "ms_per_step": allv["ms_per_step"],
            "e2e": {"value": allv["e2e_value"], "ms_per_step": allv["e2e_ms_per_step"],
                    "h2d_bytes_per_step": int(W0.numel() * 8), "d2h_bytes_per_step": 6 * 8},
            "viscous_element_fraction": allv["viscous_element_fraction"],
            "roofline": {"bound": "alu", "kernel": "volume", "ms_per_launch": avol,
                         "achieved": flops / (avol * 1e-3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                         "frac": flops / (avol * 1e-3) / 1e12 / peak,
                         "note": "inviscid algorithmic flops only (a lower bound of the work done)"},
            "config": {"workload": workload_config(N, K1)["workload"] + ", every element at eps0 (upper bound "
                                                                         "of the viscous work), cfl_visc=0.25"}}
    if not args.no_cpu_baseline and ws == 1:
        from oracle import oracle as O
        rate, t, cores, n_s = oracle_rate(N, K1, 1, prob=prob)
        # the same oracle on one thread, on a bounded sample (64x64 quads)
        O.set_threads(1)
        rate1, t1, _, n_1 = oracle_rate(N, 64, 1)
        O.set_threads(cores)
        # the same source built for speed only (timing; its results are not used)
        tuned = None
        try:
            rate_t, t_t, cores_t, _ = oracle_rate(N, K1, 1, variant="tuned", prob=prob)
            tuned = {"value": rate_t, "unit": "node-updates/s", "cores": cores_t,
                     "flags": " ".join(O._flags("tuned")),
                     "sample": f"one LSRK4(5) step of the same workload, {t_t:.2f} s"}
        except Exception as exc:  # a host compiler without these flags: report why
            tuned = {"unavailable": str(exc).splitlines()[0][:200]}
        line["cpu_baseline"] = {"value": rate, "unit": "node-updates/s", "cores": cores, "kind": "oracle",
                                "sample": f"one LSRK4(5) step of the same workload ({n_s} nodes), "
                                          f"{t:.1f} s on {cores} OpenMP threads",
                                "cpu_model": cpu_model(),
                                "flags": " ".join(O._flags(None)),
                                "single_thread": {"value": rate1, "unit": "node-updates/s",
                                                  "sample": f"one LSRK4(5) step, dam_break N={N} on 64x64 "
                                                            f"quads ({n_1} nodes), {t1:.1f} s on 1 thread"},
                                "tuned_build": tuned}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
