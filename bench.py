"""Throughput benchmark of the GF(4) BP decoder on the toric d = 15 workload.

Workload (one "step"): the toric code d = 15 (450 qubits, 450 checks, 1800
edges), i.i.d. depolarising noise at p = 0.02, 0.04, ..., 0.16 (8 values),
10^6 shots per p (per rank), EWAInit-BP (alpha = 0.5), at most 100
iterations, flooding schedule, fp32 messages: 8 decode launches, one per p.
Syndromes are sampled on the device before timing (480 MB per rank, larger
than the 129 MB L2, so no flush is needed between steps).

Reported: shots/s and edge-updates/s of EWAInit-BP (the headline) and of
plain/Momentum/AdaGrad BP on the same inputs, p50/p99 launch latency,
the roofline of the decode kernel, an end-to-end figure through the C-ABI
host-buffer entry point (bpq_decode_host), the FP64 oracle timed on the
host cores as a CPU baseline, and the logical error rate per p on the
uniform priors and (untimed) on priors with a 2^-16 per-qubit jitter, which
breaks the exact symmetric ties that uniform priors leave on the torus.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank decodes its own Philox shot range (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "EWAInit-BP decoded shots/s & edge-updates/s vs plain kernel; p99 latency"
P_SWEEP = [0.02, 0.04, 0.06, 0.08, 0.10, 0.12, 0.14, 0.16]
SEED = 0xB9E00001
CODE, DIST, MAX_ITER = "toric", 15, 100
VARIANT_PARAMS = {"ewainit": dict(alpha=0.5), "plain": {}, "momentum": dict(alpha=0.5, gamma=0.0),
                  "adagrad": dict(alpha=5.0), "aewa": dict()}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--shots-per-p", type=int, default=1_000_000)
    ap.add_argument("--variants", default="ewainit,plain,momentum,adagrad")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-latency", action="store_true")
    ap.add_argument("--no-probe", action="store_true")
    ap.add_argument("--no-jitter-ler", action="store_true")
    ap.add_argument("--workload", default="toric15", choices=["toric15", "mixed", "serve", "train", "aewa", "serial"],
                    help="toric15: the headline sweep; mixed: many codes in one batched launch; "
                         "serve: continuous-batching server on a Poisson request stream; "
                         "train: differentiable unrolled EWAInit-BP (forward + backward kernels); "
                         "aewa: EWAInit-BP vs AEWA-BP on planar L = 3, 7, 11 (Appendix C); "
                         "serial: serial vs parallel schedule on planar d=7 and toric d=15")
    ap.add_argument("--loads", default="1e4,1e5,1e6,1e7", help="offered loads (requests/s) for --workload serve")
    ap.add_argument("--train-loss", default="coset", choices=["coset", "posterior"],
                    help="train: coset (every iteration's checks and logicals) or posterior (final cross-entropy)")
    ap.add_argument("--train-model", default="ewainit", choices=["ewainit", "momentum"],
                    help="unrolled model for --workload train")
    ap.add_argument("--shots-per-thread", type=int, default=0, choices=[0, 1, 2],
                    help="decode kernel: 1 or 2 shots per thread (0: the library's choice, 2 on the toric codes)")
    ap.add_argument("--launch", default="0,0", help="threads per shot group, shot groups per CTA (0,0: automatic)")
    ap.add_argument("--prior-jitter", type=float, default=0.0,
                    help="relative per-qubit prior perturbation of the timed toric15 sweep (0: the uniform "
                         "channel); an untimed EWAInit-BP pass on 2^-16-jittered priors is always reported")
    return ap.parse_args()


def workload_config(args):
    return {
        "workload": f"toric d={DIST} (N=450, M=450, E=1800), depolarising p in {P_SWEEP}, "
                    f"{args.shots_per_p} shots per p per rank, max_iter {MAX_ITER}, flooding schedule",
        "code": f"toric d={DIST}", "p_sweep": P_SWEEP, "shots_per_p": args.shots_per_p,
        "max_iter": MAX_ITER, "headline_variant": "ewainit alpha=0.5",
        "l2": "inputs larger than L2 (syndromes 60 B/shot x 8e6 shots = 480 MB per rank); no flush",
        "parallelism": f"replicas x{args.gpus}: disjoint Philox shot ranges, no data-path collective",
        "seed": SEED, "prior": ("uniform depolarising channel" if not args.prior_jitter else
                                f"depolarising channel, per-qubit relative jitter {args.prior_jitter}"),
    }


def kernel_code_hash(src: str) -> str:
    """First 16 hex digits of the SHA-256 of a CUDA source with its comments
    and all whitespace removed: it changes when the code does, not when a
    comment does."""
    import hashlib
    import re
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return hashlib.sha256("".join(src.split()).encode()).hexdigest()[:16]


# ------------------------------------------------------------------ dist

def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        local = int(os.environ.get("LOCAL_RANK", "0"))
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return rank, world


def shot_offset(rank, shots_per_p):
    """First Philox shot index of a rank: ranks decode disjoint consecutive
    shot ranges of every p value (weak scaling, no data-path collective)."""
    return rank * shots_per_p


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return None
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------------ CPU baseline

def cpu_baseline(args, seconds):
    """The FP64 oracle, as it stands, on the host cores: rounds of `cores`
    shots per p value (EWAInit-BP, the same seeds and shot indices as the GPU
    run) until `seconds` of wall time have been spent."""
    import oracle
    from oracle import codes

    oracle.build()
    cores = os.cpu_count() or 1
    H, _ = codes.build_code(CODE, DIST)
    inputs = {}
    for p in P_SWEEP:
        inputs[p] = oracle.sample(H, *oracle.depolarizing(p), seed=SEED + P_SWEEP.index(p), shot0=0,
                                  B=cores * 64)[1]
    done, it_sum, rounds = 0, 0, 0
    t0 = time.perf_counter()
    while True:
        for p in P_SWEEP:
            prior = np.tile(np.asarray(oracle.depolarizing(p), dtype=np.float32).astype(np.float64), (H.shape[1], 1))
            syn = inputs[p][rounds * cores:(rounds + 1) * cores]
            _, _, iters = oracle.decode(H, syn, prior, "ewainit", max_iter=MAX_ITER, alpha=0.5, nthreads=cores)
            done += syn.shape[0]
            it_sum += int(iters.sum())
        rounds += 1
        el = time.perf_counter() - t0
        if el >= seconds or (rounds + 1) * cores > cores * 64:
            break
    import platform
    ld = {"x86_64": "x87 80-bit", "AMD64": "x87 80-bit", "aarch64": "software IEEE binary128",
          "arm64": "software IEEE binary128"}.get(platform.machine(), "the platform's long double")
    return {"value": done / el, "unit": "shots/s", "cores": cores, "kind": "oracle",
            "edge_updates_per_s": it_sum * 1800 / el,
            "sample": f"{rounds} rounds x {cores} shots x {len(P_SWEEP)} p values = {done} shots of the same "
                      f"workload (EWAInit-BP, shot indices from 0), {el:.1f} s wall, FP64 oracle with "
                      f"{cores} threads on {platform.machine()}; its check update is evaluated in long double "
                      f"({ld} here), which dominates its time where long double is software arithmetic",
            "long_double": ld}


# ------------------------------------------------------------------ reference arm

def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle on the host cores, each step a
    bounded sample of the same workload (rank 0 only)."""
    if rank != 0:
        return
    vals, secs = [], []
    cb = None
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        cb = cpu_baseline(args, max(2.0, min(args.cpu_seconds, 20.0) / 2))
        if s >= args.warmup:
            vals.append(cb["value"])
            secs.append(time.perf_counter() - t0)
    v = statistics.median(vals) if vals else cb["value"]
    line = {"metric": METRIC, "value": v, "unit": "shots/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(secs) if secs else None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": workload_config(args),
            "cpu_baseline": {"value": v, "unit": "shots/s", "cores": cb["cores"], "kind": "oracle",
                             "sample": cb["sample"]},
            "e2e": {"value": v, "unit": "shots/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm

def run_ours(args, rank, world):
    import torch

    import paper_2407_11523_gb300 as bpq

    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    t = bpq.Tanner(CODE, DIST).upload()
    t.set_shots_per_thread(args.shots_per_thread)
    t.set_launch(*[int(x) for x in args.launch.split(",")])
    B = args.shots_per_p
    shot0 = shot_offset(rank, B)
    syns, errs, priors = [], [], []
    for k, p in enumerate(P_SWEEP):
        err, syn = bpq.sample(t, *[p / 3] * 3, seed=SEED + k, shot0=shot0, B=B)
        syns.append(syn)
        errs.append(err)  # kept for the logical error rates, computed after timing
        priors.append(bpq.prior_tensor(t, p / 3, p / 3, p / 3, jitter=args.prior_jitter))
    outs = [(torch.empty((B, t.N), dtype=torch.uint8, device=dev), torch.empty(B, dtype=torch.uint8, device=dev),
             torch.empty(B, dtype=torch.uint8, device=dev)) for _ in P_SWEEP]
    work = bpq.workspace(dev)
    torch.cuda.synchronize()

    results = {}
    clocks = None
    for v in args.variants.split(","):
        params = bpq.make_params(v, **VARIANT_PARAMS[v])

        def step(ev=None):
            for k in range(len(P_SWEEP)):
                if ev is not None:
                    ev[k][0].record(stream)
                bpq.decode(t, syns[k], priors[k], v, params=params, max_iter=MAX_ITER, out=outs[k], work=work)
                if ev is not None:
                    ev[k][1].record(stream)

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        launch_ms = []
        sampler = ClockSampler(dev.index) if v == "ewainit" else None
        if sampler:
            sampler.__enter__()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        evs = [[[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in P_SWEEP] for _ in range(args.steps)]
        e0.record(stream)
        for s in range(args.steps):
            step(evs[s])
        e1.record(stream)
        e1.synchronize()
        torch.cuda.synchronize()
        barrier(world)
        if sampler:
            sampler.__exit__()
            clocks = sampler.summary()
        ms = e0.elapsed_time(e1)
        for s in range(args.steps):
            for k in range(len(P_SWEEP)):
                launch_ms.append(evs[s][k][0].elapsed_time(evs[s][k][1]))
        iters_total = sum(int(o[2].sum(dtype=torch.int64).item()) for o in outs)
        conv = sum(int(o[1].sum(dtype=torch.int64).item()) for o in outs)
        # iteration histogram over the last step's shots, in bins 1-5, 6-10, ..., 96-100
        hist = sum(torch.bincount((o[2].long() - 1).clamp(min=0) // 5, minlength=MAX_ITER // 5) for o in outs)
        # logical error rate per p (Sec. IV: failure = not converged, or a logical error), with the
        # detected / undetected split and a 2-sigma binomial half-width; not timed
        ler = []
        for k, p in enumerate(P_SWEEP):
            f = bpq.check_logical(t, errs[k], outs[k][0])
            det = reduce_sum(float((f == 1).sum().item()), world)
            und = reduce_sum(float((f == 2).sum().item()), world)
            n = float(B * world)
            r = (det + und) / n
            ler.append({"p": p, "ler": r, "two_sigma": 2.0 * float(np.sqrt(max(r * (1 - r), 1.0 / n) / n)),
                        "detected": det / n, "undetected": und / n})
        sec = reduce_max(ms / 1e3, world)
        shots = reduce_sum(float(B * len(P_SWEEP) * args.steps), world)
        eu = reduce_sum(float(iters_total) * t.E * args.steps, world)
        results[v] = {"shots_per_s": shots / sec, "edge_updates_per_s": eu / sec, "ms_per_step": sec * 1e3 / args.steps,
                      "avg_iterations": iters_total / (B * len(P_SWEEP)), "converged_frac": conv / (B * len(P_SWEEP)),
                      "launch_ms_mean": float(np.mean(launch_ms)), "launches": len(launch_ms),
                      "iteration_histogram_5": [int(x) for x in hist.tolist()], "ler": ler,
                      "edge_updates_per_step": iters_total * t.E}
    head = results.get("ewainit") or next(iter(results.values()))

    # untimed EWAInit-BP pass on priors jittered by 2^-16 per qubit: uniform
    # priors put trapping sets into nearly symmetric oscillations that the
    # parallel schedule leaves only through asymmetries below binary32
    # resolution (Sec. IV-A), so part of the uniform-prior failures are
    # decided by the working precision; the jitter puts the asymmetry into
    # the input
    if "ewainit" in results and not args.no_jitter_ler:
        rel = 2.0 ** -16
        params = bpq.make_params("ewainit", **VARIANT_PARAMS["ewainit"])
        jl, jit_iters = [], 0
        for k, p in enumerate(P_SWEEP):
            pj = bpq.prior_tensor(t, p / 3, p / 3, p / 3, jitter=rel)
            bpq.decode(t, syns[k], pj, "ewainit", params=params, max_iter=MAX_ITER, out=outs[k], work=work)
            f = bpq.check_logical(t, errs[k], outs[k][0])
            n = float(B * world)
            r = reduce_sum(float((f > 0).sum().item()), world) / n
            jit_iters += int(outs[k][2].sum(dtype=torch.int64).item())
            jl.append({"p": p, "ler": r, "two_sigma": 2.0 * float(np.sqrt(max(r * (1 - r), 1.0 / n) / n)),
                       "unconverged": reduce_sum(float((outs[k][1] == 0).sum().item()), world) / n})
        results["ewainit"]["prior_jitter_2^-16"] = {"ler": jl, "avg_iterations": jit_iters / (B * len(P_SWEEP)),
                                                    "timed": False}

    # p50/p99 launch latency at p = 0.08, EWAInit-BP, batches of 1 and 1024 shots
    lat = {}
    k8 = P_SWEEP.index(0.08)
    params = bpq.make_params("ewainit", alpha=0.5)
    for nb in (() if args.no_latency else (1, 1024)):
        sub = syns[k8][:nb].contiguous()
        o = tuple(x[:nb] for x in outs[k8])
        times = []
        for r in range(230):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            bpq.decode(t, sub, priors[k8], "ewainit", params=params, max_iter=MAX_ITER, out=o, work=work)
            b.record(stream)
            b.synchronize()
            if r >= 30:
                times.append(a.elapsed_time(b))
        lat[f"batch_{nb}"] = {"p50_ms": float(np.percentile(times, 50)), "p99_ms": float(np.percentile(times, 99)),
                              "launches": len(times)}

    # roofline of the decode kernel: in-SM arithmetic.  DRAM traffic per shot
    # and the issue-slot share come from the ncu summary recorded beside the
    # profile (profiles/*.json), used only while the kernel's code (comments
    # and whitespace aside) still matches the profiled one.
    traffic = issue_pct = prof_rec = None
    pair = t.shots_per_thread("ewainit") == 2
    kname = "decode_pair_kernel" if pair else "decode_kernel"
    try:
        prof_rec = json.load(open(os.path.join(ROOT, "profiles", f"{kname}_toric15_ewainit.json")))
        csrc = os.path.join(ROOT, "paper_2407_11523_gb300", "csrc")
        src = "".join(open(os.path.join(csrc, f)).read()
                      for f in (["decode_kernel.cuh", "decode_pair.cuh"] if pair else ["decode_kernel.cuh"]))
        if kernel_code_hash(src) == prof_rec["kernel_code_sha256_16"]:
            traffic = float(prof_rec["dram_bytes_per_shot"]) * args.shots_per_p
            issue_pct = float(prof_rec["issue_active_pct"])
    except (OSError, KeyError, ValueError):
        traffic = issue_pct = None
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    try:
        hbm_peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        hbm_peak = None
    sfu_peak = float("nan") if args.no_probe else bpq.probe_peak("sfu", blocks=sms * 8, threads=256, iters=4096)
    fma_peak = float("nan") if args.no_probe else bpq.probe_peak("fma", blocks=sms * 8, threads=256, iters=4096)
    # algorithmic work per edge-update (one c->v and one v->c message on one
    # edge in one iteration) in the literal form of eqs. (h_update), (lambda):
    # tanh + atanh on the check side (2 transcendental + 2 reciprocal) and a
    # softplus and a two-term log-sum-exp on the variable side (2 ex2 + 2
    # lg2): 8 SFU operations.  The kernel's delta form needs 5 (check side rcp
    # + lg2, variable side ex2 + rcp per edge, 4 ex2 per degree-4 qubit).
    sfu_per_edge_update, impl_sfu_per_edge_update = 8.0, 5.0
    ew = results.get("ewainit", head)
    kernel_sec = ew["launch_ms_mean"] / 1e3
    eu_per_launch = ew["edge_updates_per_step"] / len(P_SWEEP)
    achieved = sfu_per_edge_update * eu_per_launch / kernel_sec
    impl_achieved = impl_sfu_per_edge_update * eu_per_launch / kernel_sec
    roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": sfu_peak / 1e12, "unit": "TSFUop/s",
                "frac": achieved / sfu_peak, "traffic": traffic,
                "kernel": f"{kname}<EWAINIT>", "per_unit": f"{sfu_per_edge_update:g} SFU ops per edge-update "
                "(the literal form's tanh, atanh, softplus and log-sum-exp)",
                "edge_updates_per_launch": eu_per_launch, "launch_ms": ew["launch_ms_mean"],
                "impl_sfu_per_edge_update": impl_sfu_per_edge_update,
                "impl_achieved": impl_achieved / 1e12, "impl_frac": impl_achieved / sfu_peak,
                "ncu_issue_active_pct": issue_pct,
                "ncu_summary": None if prof_rec is None else {k: prof_rec.get(k) for k in (
                    "instructions_per_launch", "issue_active_pct", "dram_bytes_per_shot", "shots", "command")},
                "ncu_summary_current": traffic is not None,
                "note": "issue-bound: the SFU is not the binding unit; ncu_issue_active_pct is the share of "
                        "issue slots used in the profiled launch",
                "peak_source": "measured on this GPU by the MUFU.EX2 probe kernel (bpq_probe_peak)",
                "fma_peak_tinst_per_s": fma_peak / 1e12, "sms": sms,
                "hbm": {"algorithmic_bytes_per_shot": t.W * 4 + t.N + 2,
                        "achieved_gbs": (t.W * 4 + t.N + 2) * args.shots_per_p / kernel_sec / 1e9,
                        "peak_gbs": hbm_peak, "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth)",
                        "frac": ((t.W * 4 + t.N + 2) * args.shots_per_p / kernel_sec / 1e9 / hbm_peak
                                 if hbm_peak else None)}}

    # end to end through bpq_decode_host with pinned host buffers
    e2e = None
    if not args.no_e2e:
        syn_h = [s.cpu().pin_memory() for s in syns]
        pri_h = [p.cpu().pin_memory() for p in priors]
        out_h = [(torch.empty((B, t.N), dtype=torch.uint8, pin_memory=True), torch.empty(B, dtype=torch.uint8, pin_memory=True),
                  torch.empty(B, dtype=torch.uint8, pin_memory=True)) for _ in P_SWEEP]
        dbuf = torch.empty(bpq.decode_host_bytes(t, B), dtype=torch.uint8, device=dev)
        params = bpq.make_params("ewainit", alpha=0.5)

        def hstep():
            for k in range(len(P_SWEEP)):
                bpq.decode_host(t, syn_h[k], pri_h[k], "ewainit", params=params, max_iter=MAX_ITER, out=out_h[k],
                                dev_buf=dbuf)

        for _ in range(args.warmup):
            hstep()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            hstep()
        el = reduce_max(time.perf_counter() - t0, world)
        shots = reduce_sum(float(B * len(P_SWEEP) * args.steps), world)
        e2e = {"value": shots / el, "unit": "shots/s",
               "h2d_bytes_per_step": len(P_SWEEP) * (B * t.W * 4 + t.N * 12),
               "d2h_bytes_per_step": len(P_SWEEP) * B * (t.N + 2),
               "api": "bpq_decode_host (C ABI, pinned host buffers, copies and a stream sync inside)"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args, args.cpu_seconds)

    if rank == 0:
        line = {"metric": METRIC, "value": head["shots_per_s"], "unit": "shots/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic", "config": workload_config(args),
                "edge_updates_per_s": head["edge_updates_per_s"],
                "variants": results, "vs_plain": (results["ewainit"]["shots_per_s"] / results["plain"]["shots_per_s"]
                                                 if "plain" in results and "ewainit" in results else None),
                "latency_ms": lat, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": len(P_SWEEP) * args.steps, "clocks": clocks,
                "device": torch.cuda.get_device_name(dev)}
        print(json.dumps(line), flush=True)



# ------------------------------------------------------------------ mixed-size batched workload

MIX_CODES = [("planar", d) for d in (5, 9, 13, 17, 21, 25)] + [("toric", d) for d in (8, 12, 16)] + \
    [("xzzx", d) for d in (7, 11, 15)]
MIX_NOISE = [("depolarising p=0.06", (0.02, 0.02, 0.02)), ("Z-biased p=0.06 eta=10", (0.06 / 22, 0.06 / 22, 0.06 * 10 / 11))]
MIX_TOTAL = 1 << 20


def mixed_split(seed):
    """Uneven split of 2^20 shots over the 24 (code, noise) groups: a
    multinomial draw with Dirichlet(1) weights from a seeded generator."""
    rng = np.random.default_rng(seed)
    w = rng.dirichlet(np.ones(len(MIX_CODES) * len(MIX_NOISE)))
    return rng.multinomial(MIX_TOTAL, w)


def run_mixed(args, rank, world):
    import torch

    import paper_2407_11523_gb300 as bpq

    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    counts = mixed_split(SEED)
    tanners = {cd: bpq.Tanner(*cd).upload() for cd in MIX_CODES}
    items, groups = [], []
    k = 0
    for cd in MIX_CODES:
        for noise_name, ch in MIX_NOISE:
            B = int(counts[k])
            t = tanners[cd]
            _, syn = bpq.sample(t, *ch, seed=SEED + 1000 + k, shot0=rank * MIX_TOTAL, B=B)
            items.append((t, syn, bpq.prior_tensor(t, *ch)))
            groups.append((cd, noise_name, B))
            k += 1
    params = bpq.make_params("ewainit", alpha=0.5)
    # autotune each code's launch shape, one-code and batched, on its largest sample
    shapes, batch_shapes = {}, {}
    for cd in MIX_CODES:
        t = tanners[cd]
        best = max((it for it in items if it[0] is t), key=lambda it: it[1].shape[0])
        sample = best[1][: min(8192, best[1].shape[0])].contiguous()
        shapes[f"{cd[0]} d={cd[1]}"] = bpq.autotune(t, sample, best[2], "ewainit", params=params, max_iter=MAX_ITER)
        bpq.autotune_batch(t, sample, best[2], "ewainit", params=params, max_iter=MAX_ITER)
        batch_shapes[f"{cd[0]} d={cd[1]}"] = t.batch_launch("ewainit")
    work = bpq.workspace(dev)
    outs = [(torch.empty((it[1].shape[0], it[0].N), dtype=torch.uint8, device=dev),
             torch.empty(it[1].shape[0], dtype=torch.uint8, device=dev),
             torch.empty(it[1].shape[0], dtype=torch.uint8, device=dev)) for it in items]

    def per_code():
        for (t, syn, prior), o in zip(items, outs):
            if syn.shape[0]:
                bpq.decode(t, syn, prior, "ewainit", params=params, max_iter=MAX_ITER, out=o, work=work)

    plan = bpq.BatchPlan(items, "ewainit", params=params, max_iter=MAX_ITER)
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.graph(graph, stream=side):
        plan.run(stream=side)
    torch.cuda.synchronize()

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        barrier(world)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return reduce_max(e0.elapsed_time(e1) / 1e3 / args.steps, world)

    res = {}
    res["per_code_launches"] = timed(per_code)
    res["batched_launch"] = timed(lambda: plan.run())
    res["batched_graph"] = timed(lambda: graph.replay())
    # equal results, and the edge-updates of one pass
    per_code()
    ref = [tuple(x.clone() for x in o) for o in outs]
    bat = plan.run()
    torch.cuda.synchronize()
    identical = all(torch.equal(a, b) for o, r in zip(bat, ref) for a, b in zip(o, r))
    edge_updates = sum(int(o[2].sum(dtype=torch.int64).item()) * it[0].E for o, it in zip(ref, items))
    errs = []
    for (t, syn, prior), o, (cd, noise_name, B), k in zip(items, ref, groups, range(len(items))):
        if B == 0:
            errs.append(None)
            continue
        ch = MIX_NOISE[k % 2][1]
        err, _ = bpq.sample(t, *ch, seed=SEED + 1000 + k, shot0=rank * MIX_TOTAL, B=B)
        fail = bpq.check_logical(t, err, o[0])
        errs.append(float((fail > 0).float().mean().item()))
    shots = reduce_sum(float(MIX_TOTAL), world)
    if rank == 0:
        sec = res["batched_graph"]
        line = {"metric": "batched mixed-size EWAInit-BP decoded shots/s (one persistent graph-captured launch)",
                "value": shots / sec, "unit": "shots/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "planar d 5..25, toric d 8,12,16, XZZX d 7,11,15 x {depolarising, "
                                       "Z-biased eta=10} at p=0.06; 2^20 shots split by a seeded multinomial; "
                                       "EWAInit-BP alpha=0.5, max_iter 100",
                           "groups": [{"code": f"{cd[0]} d={cd[1]}", "noise": nn, "shots": B, "ler": e}
                                      for (cd, nn, B), e in zip(groups, errs)],
                           "launch_shapes": shapes, "batch_shapes": batch_shapes, "batch_plan": plan.info()},
                "edge_updates_per_s": reduce_sum(float(edge_updates), world) / sec,
                "compare_shots_per_s": {kk: shots / v for kk, v in res.items()},
                "batched_equals_per_code": identical,
                "gpu_launches": 1 * args.steps}
        print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ AEWA-BP workload (Appendix C)

AEWA_L = (3, 7, 11)
AEWA_PER = (0.01, 0.06, 0.1, 0.2)
AEWA_SHOTS = 100_000


def run_aewa(args, rank, world):
    """EWAInit-BP (alpha 0.5) and AEWA-BP on the planar codes L = 3, 7, 11 at
    the error rates of Appendix C's runtime table, max 100 iterations: batch
    throughput, per-decode latency of single shots, and LER."""
    import torch

    import paper_2407_11523_gb300 as bpq

    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    B = AEWA_SHOTS
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    work = bpq.workspace(dev)
    rows, timed_ms, launches = [], {"ewainit": 0.0, "aewa": 0.0}, 0
    for L in AEWA_L:
        t = bpq.Tanner("planar", L).upload()
        for k, p in enumerate(AEWA_PER):
            ch = (p / 3, p / 3, p / 3)
            err, syn = bpq.sample(t, *ch, seed=SEED + 200 + 10 * L + k, shot0=rank * B, B=B)
            prior = bpq.prior_tensor(t, *ch)
            out = (torch.empty((B, t.N), dtype=torch.uint8, device=dev), torch.empty(B, dtype=torch.uint8, device=dev),
                   torch.empty(B, dtype=torch.uint8, device=dev))
            row = {"L": L, "N": t.N, "per": p}
            for v in ("ewainit", "aewa"):
                params = bpq.make_params(v, **({"alpha": 0.5} if v == "ewainit" else {}))
                for _ in range(args.warmup):
                    bpq.decode(t, syn, prior, v, params=params, max_iter=MAX_ITER, out=out, work=work)
                torch.cuda.synchronize()
                barrier(world)
                ms = 0.0
                for s in range(args.steps):
                    flush.fill_(s & 0xFF)  # L2 flush between timed launches (outside the events)
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    bpq.decode(t, syn, prior, v, params=params, max_iter=MAX_ITER, out=out, work=work)
                    b.record(stream)
                    b.synchronize()
                    ms += a.elapsed_time(b)
                    launches += 1
                ms = reduce_max(ms, world)
                timed_ms[v] += ms
                fail = bpq.check_logical(t, err, out[0])
                n_fail = reduce_sum(float((fail > 0).sum().item()), world)
                conv = float(out[1].float().mean().item())
                iters = float(out[2].float().mean().item())
                # per-decode latency: one launch per single shot, 100 different shots
                lat = []
                for i in range(100 if not args.no_latency else 0):
                    o = tuple(x[i:i + 1] for x in out)
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    bpq.decode(t, syn[i:i + 1], prior, v, params=params, max_iter=MAX_ITER, out=o, work=work)
                    b.record(stream)
                    b.synchronize()
                    lat.append(a.elapsed_time(b))
                row[v] = {"shots_per_s": reduce_sum(float(B * args.steps), world) / (ms / 1e3),
                          "ler": n_fail / (B * world), "converged_frac": conv, "avg_iterations": iters,
                          "single_shot_ms_mean": float(np.mean(lat)) if lat else None,
                          "single_shot_ms_p99": float(np.percentile(lat, 99)) if lat else None}
            rows.append(row)
    if rank == 0:
        shots = float(B * args.steps * len(AEWA_L) * len(AEWA_PER) * world)
        line = {"metric": "AEWA-BP decoded shots/s over planar L=3,7,11 x PER {0.01,0.06,0.1,0.2}",
                "value": shots / (timed_ms["aewa"] / 1e3), "unit": "shots/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": timed_ms["aewa"] / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"planar L in {list(AEWA_L)}, depolarising PER in {list(AEWA_PER)}, "
                                       f"{B} shots per point per rank, max_iter {MAX_ITER}; AEWA-BP tries "
                                       "alpha = 1.0, 0.9, ..., 0.0; EWAInit-BP alpha 0.5 alongside",
                           "l2": "a 256 MB buffer is written between timed launches"},
                "ewainit_shots_per_s": shots / (timed_ms["ewainit"] / 1e3),
                "points": rows, "gpu_launches": launches // 2}
        print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ serial schedule workload

SERIAL_CODES = (("planar", 7), ("toric", 15))
SERIAL_P = (0.04, 0.08, 0.12)
SERIAL_SHOTS = 100_000


def run_serial(args, rank, world):
    """Plain BP and EWAInit-BP (alpha 0.5) under the serial schedule of
    Algorithm 1 (bpq_decode_serial) and the parallel schedule, max 100
    iterations: shots/s, LER, convergence and iterations per point."""
    import torch

    import paper_2407_11523_gb300 as bpq

    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    B = min(SERIAL_SHOTS, args.shots_per_p)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    work = bpq.workspace(dev)
    rows, timed_ms, launches = [], 0.0, 0
    for code, d in SERIAL_CODES:
        t = bpq.Tanner(code, d).upload()
        for k, p in enumerate(SERIAL_P):
            ch = (p / 3, p / 3, p / 3)
            err, syn = bpq.sample(t, *ch, seed=SEED + 500 + 10 * d + k, shot0=rank * B, B=B)
            prior = bpq.prior_tensor(t, *ch)
            out = (torch.empty((B, t.N), dtype=torch.uint8, device=dev), torch.empty(B, dtype=torch.uint8, device=dev),
                   torch.empty(B, dtype=torch.uint8, device=dev))
            row = {"code": f"{code} d={d}", "p": p}
            for v in ("plain", "ewainit"):
                params = bpq.make_params(v, **({"alpha": 0.5} if v == "ewainit" else {}))
                for sched in ("serial", "parallel"):
                    for _ in range(args.warmup):
                        bpq.decode(t, syn, prior, v, params=params, max_iter=MAX_ITER, out=out, work=work,
                                   schedule=sched)
                    torch.cuda.synchronize()
                    barrier(world)
                    ms = 0.0
                    for s_ in range(args.steps):
                        flush.fill_(s_ & 0xFF)  # L2 flush between timed launches (outside the events)
                        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        a.record(stream)
                        bpq.decode(t, syn, prior, v, params=params, max_iter=MAX_ITER, out=out, work=work,
                                   schedule=sched)
                        b.record(stream)
                        b.synchronize()
                        ms += a.elapsed_time(b)
                        launches += sched == "serial" and v == "ewainit"
                    ms = reduce_max(ms, world)
                    if sched == "serial" and v == "ewainit":
                        timed_ms += ms
                    fail = bpq.check_logical(t, err, out[0])
                    row[f"{v}_{sched}"] = {
                        "shots_per_s": reduce_sum(float(B * args.steps), world) / (ms / 1e3),
                        "ler": reduce_sum(float((fail > 0).sum().item()), world) / (B * world),
                        "converged_frac": float(out[1].float().mean().item()),
                        "avg_iterations": float(out[2].float().mean().item())}
            rows.append(row)
    if rank == 0:
        shots = float(B * args.steps * len(SERIAL_CODES) * len(SERIAL_P) * world)
        line = {"metric": "serial-schedule EWAInit-BP decoded shots/s (planar d=7, toric d=15; p 0.04, 0.08, 0.12)",
                "value": shots / (timed_ms / 1e3), "unit": "shots/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": timed_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"planar d=7 and toric d=15, depolarising p in {list(SERIAL_P)}, {B} shots "
                                       f"per point per rank, max_iter {MAX_ITER}; plain and EWAInit (alpha 0.5) BP "
                                       "under the serial and the parallel schedule",
                           "l2": "a 256 MB buffer is written between timed launches"},
                "points": rows, "gpu_launches": launches}
        print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ serving workload

SERVE_CODES = [(k, d) for k in ("planar", "xzzx") for d in range(5, 32, 2)]


def run_serve(args, rank, world):
    """Poisson streams of single-shot requests over planar and XZZX codes
    d = 5..31 at p = 0.05 (EWAInit-BP), served by the slot server (a
    persistent kernel whose shot groups take the next request as soon as
    they finish a shot) and by the lane server (micro-batches per stream)
    for comparison; p50/p99 latency and shots/s per offered load."""
    import torch

    import paper_2407_11523_gb300 as bpq

    p = 0.05
    ch = (p / 3, p / 3, p / 3)
    codes = [bpq.Tanner(*cd).upload() for cd in SERVE_CODES]
    priors = [bpq.prior_tensor(t, *ch) for t in codes]
    params = bpq.make_params("ewainit", alpha=0.5)
    servers = {"slots": bpq.Server(codes, priors, "ewainit", params=params, max_iter=MAX_ITER, mode="slots",
                                   slots_per_code=1024),
               "lanes": bpq.Server(codes, priors, "ewainit", params=params, max_iter=MAX_ITER, n_lanes=4,
                                   max_batch=4096)}
    rng = np.random.default_rng(SEED + 7)
    pool = {}
    R_pool = 200000
    code_pool = rng.integers(0, len(codes), size=R_pool)
    for c, t in enumerate(codes):
        n = int((code_pool == c).sum())
        _, syn = bpq.sample(t, *ch, seed=SEED + 2000 + c, shot0=rank * R_pool, B=max(n, 1))
        pool[c] = syn.cpu().numpy().view(np.uint32)
    fill = {c: 0 for c in pool}
    syn_pool = []
    for c in code_pool:
        syn_pool.append(pool[c][fill[c]])
        fill[c] += 1
    out = {}
    launches = 0
    for name, srv in servers.items():
        srv.replay(code_pool[:2000], np.zeros(2000), syn_pool[:2000])  # warm-up
        launches0 = srv.launches()
        results = []
        for load in [float(x) for x in args.loads.split(",")]:
            R = int(min(R_pool, max(2000, load * 0.02)))
            arrival = np.cumsum(rng.exponential(1.0 / load, size=R))
            arrival -= arrival[0]
            ests, conv, iters, done, used = srv.replay(code_pool[:R], arrival, syn_pool[:R])
            lat = done - arrival
            span = done.max() - arrival[0]
            eu = sum(int(iters[r]) * codes[code_pool[r]].E for r in range(R))
            results.append({"offered_per_s": load, "requests": R, "p50_ms": float(np.percentile(lat, 50) * 1e3),
                            "p99_ms": float(np.percentile(lat, 99) * 1e3), "shots_per_s": R / span,
                            "edge_updates_per_s": eu / span,
                            ("ctas" if name == "slots" else "lanes_used"): used,
                            "converged_frac": float(conv.mean())})
        # saturation: every request available at once
        R = R_pool
        ests, conv, iters, done, used = srv.replay(code_pool[:R], np.zeros(R), syn_pool[:R])
        sat = R / done.max()
        out[name] = {"loads": results, "saturation_shots_per_s": sat,
                     "launches": srv.launches() - launches0}
        launches += srv.launches() - launches0
    # the device's own rate on the burst's requests: one batched launch over
    # their syndromes, grouped by code and resident on the device (no host
    # loop, no rings); an L2 flush runs between timed launches
    dev = torch.device("cuda")
    items = []
    for c, t in enumerate(codes):
        n = int((code_pool == c).sum())
        if n:
            items.append((t, torch.from_numpy(np.ascontiguousarray(pool[c][:n]).view(np.int32)).to(dev), priors[c]))
    plan = bpq.BatchPlan(items, "ewainit", params=params, max_iter=MAX_ITER)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(3):
        plan.run()
    torch.cuda.synchronize()
    dev_ms = []
    for s_ in range(5):
        flush.fill_(s_ & 0xFF)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        plan.run()
        e1.record()
        e1.synchronize()
        dev_ms.append(e0.elapsed_time(e1))
    dev_s = reduce_max(statistics.median(dev_ms) / 1e3, world)
    device_rate = R_pool / dev_s
    out["device_batched"] = {"requests": R_pool, "ms": dev_s * 1e3, "shots_per_s": device_rate, "launches": 5}
    for name in ("slots", "lanes"):
        out[name]["saturation_of_device_batched"] = out[name]["saturation_shots_per_s"] / device_rate
    if rank == 0:
        best = out["slots"]["saturation_shots_per_s"]
        line = {"metric": "serving: p50/p99 latency and shots/s under a Poisson request stream (continuous batching)",
                "value": best, "unit": "shots/s", "n_gpus": world, "steps": len(out["slots"]["loads"]), "warmup": 1,
                "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": "single-shot requests, planar and XZZX codes d = 5, 7, ..., 31 (uniform), "
                                       "depolarising p = 0.05, EWAInit-BP alpha = 0.5, max_iter 100; Poisson "
                                       "arrivals; value = the slot server's saturation shots/s (200000 requests "
                                       "available at once)",
                           "slot_server": "1024 request slots per code in mapped host memory, one persistent "
                                          "kernel (bpq_server_create_slots); results written in place to "
                                          "page-locked outputs",
                           "lane_server": "4 lanes x 4096 shots of device budget, one batched launch per dispatch "
                                          "(bpq_server_create)",
                           "device_batched": "the saturation burst's 200000 requests decoded by one batched launch "
                                             "from device-resident syndromes grouped by code (CUDA events, L2 "
                                             "flush between launches): the device's rate with no serving work",
                           "servers": out},
                "gpu_launches": launches}
        print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ training workload

def run_train(args, rank, world):
    import torch

    import paper_2407_11523_gb300 as bpq

    T, K, B, d = 25, 5, 4096, 9
    t = bpq.Tanner("planar", d).upload()
    ps = np.linspace(0.03, 0.10, 8)
    p0 = float(ps.mean())
    prior = bpq.prior_tensor(t, p0 / 3, p0 / 3, p0 / 3)

    def draw(seed, shot0, n_per_p):
        errs, syns = [], []
        for k, p in enumerate(ps):
            e, s_ = bpq.sample(t, p / 3, p / 3, p / 3, seed=seed + k, shot0=shot0, B=n_per_p)
            errs.append(e)
            syns.append(s_)
        return torch.cat(errs), torch.cat(syns)

    # a fresh batch every step (Philox shot offsets advance), drawn before timing
    n_batches = args.warmup + args.steps + 100
    pool = [draw(SEED + 3000, (rank * n_batches + k) * (B // len(ps)), B // len(ps)) for k in range(n_batches)]
    model = args.train_model
    mom = model == "momentum"
    # start at the paper's parameters: EWAInit alpha 0.5; Momentum alpha 0.5, gamma 0
    a = torch.full((T,), 0.5, device="cuda", requires_grad=True)
    b = torch.zeros(T, device="cuda", requires_grad=True)
    w = torch.ones(t.E, device="cuda", requires_grad=True)
    g = torch.zeros(T, device="cuda", requires_grad=True) if mom else None
    opt = torch.optim.Adam([a, b, w] + ([g] if mom else []), lr=0.01)
    it = iter(pool)

    def step():
        err, syn = next(it)
        opt.zero_grad()
        L = bpq.unrolled_loss(t, syn, err, prior, a, b, w, T=T, ckpt_every=K, model=model, gamma=g,
                              loss=args.train_loss)
        L.backward()
        opt.step()
        with torch.no_grad():
            a.clamp_(0.0, 1.0)
            b.clamp_(0.0, 0.95)
            if mom:
                g.clamp_(0.0, 0.95)
        return L.detach()

    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        L = step()
    e1.record(stream)
    e1.synchronize()
    sec = e0.elapsed_time(e1) / 1e3 / args.steps
    losses = [float(step()) for _ in range(100)]  # keep training for the accuracy comparison (not timed)

    # held-out logical error rates: trained vs untrained unrolled decoder vs the early-exit kernel
    err_t, syn_t = draw(SEED + 4000, 10**7 + rank * 65536, 8192)

    def ler_from_Q(Q):
        # hard decision of Sec. II-B1 on the final posterior (evaluation only)
        allpos = (Q > 0).all(-1)
        est = torch.where(allpos, torch.zeros_like(allpos, dtype=torch.long), 1 + Q.argmin(-1))
        fail = bpq.check_logical(t, err_t, est.to(torch.uint8).contiguous())
        return float((fail > 0).float().mean())

    def ler_early_exit(aa, bb, ww, gg):
        # the stopping rule of Algorithms 1 and 2 on the unrolled decoder: each
        # shot takes the decision of the first iteration whose decision
        # satisfies the syndrome (else that of iteration T)
        outcome = torch.full((err_t.shape[0],), 255, dtype=torch.uint8, device=err_t.device)
        for Tp in range(1, T + 1):
            Q, _ = bpq.unrolled_posterior(t, syn_t, err_t, prior, aa[:Tp], bb[:Tp], ww, T=Tp, ckpt_every=Tp,
                                          model=model, gamma=gg[:Tp] if gg is not None else None)
            allpos = (Q > 0).all(-1)
            est = torch.where(allpos, torch.zeros_like(allpos, dtype=torch.long), 1 + Q.argmin(-1))
            f = bpq.check_logical(t, err_t, est.to(torch.uint8).contiguous())
            take = (outcome == 255) & ((f != 1) | (Tp == T))
            outcome[take] = f[take]
        return float((outcome > 0).float().mean())

    with torch.no_grad():
        g0 = torch.zeros_like(a) if mom else None
        gt = g.detach() if mom else None
        Qtr, Ltr = bpq.unrolled_posterior(t, syn_t, err_t, prior, a, b, w, T=T, model=model, gamma=gt,
                                          loss=args.train_loss)
        Q0, L0 = bpq.unrolled_posterior(t, syn_t, err_t, prior, torch.full_like(a, 0.5), torch.zeros_like(b),
                                        torch.ones_like(w), T=T, model=model, gamma=g0, loss=args.train_loss)
        ler_ee = {"trained": ler_early_exit(a.detach(), b.detach(), w.detach(), gt),
                  "untrained": ler_early_exit(torch.full_like(a, 0.5), torch.zeros_like(b), torch.ones_like(w), g0)}
    est_k, conv_k, _ = bpq.decode(t, syn_t, prior, model, max_iter=T, alpha=0.5, **({"gamma": 0.0} if mom else {}))
    ler_kernel = float((bpq.check_logical(t, err_t, est_k) > 0).float().mean())
    if rank == 0:
        name = "Momentum-BP" if mom else "EWAInit-BP"
        line = {"metric": f"differentiable unrolled {name}: training shots/s (forward + hand-written backward)",
                "value": B / sec, "unit": "shots/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"planar d={d} (N={t.N}, E={t.E}), T={T}, checkpoints every {K}, batch {B} "
                                       f"depolarising errors at p in {[round(float(x), 3) for x in ps]}, "
                                       f"prior p={p0:.3f}; "
                                       "trainable alpha_t, beta_t" + (", gamma_t" if mom else "") +
                                       " (T each) and w_e (E); Adam lr 0.01, a fresh Philox batch every step, "
                                       f"{args.warmup + args.steps + 100} steps", "model": model,
                           "loss": args.train_loss},
                "train_loss_first_last": [losses[0], losses[-1]],
                "held_out_loss": {"trained": float(Ltr), "untrained": float(L0)},
                "held_out_ler": {"trained_unrolled": ler_from_Q(Qtr), "untrained_unrolled": ler_from_Q(Q0),
                                 "trained_unrolled_early_exit": ler_ee["trained"],
                                 "untrained_unrolled_early_exit": ler_ee["untrained"],
                                 f"{model}_kernel_early_exit": ler_kernel, "shots": int(err_t.shape[0])},
                "gpu_launches": (7 if mom else 6) * args.steps}
        print(json.dumps(line), flush=True)

def main():
    args = parse()
    rank, world = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "mixed":
        run_mixed(args, rank, world)
    elif args.workload == "serve":
        run_serve(args, rank, world)
    elif args.workload == "aewa":
        run_aewa(args, rank, world)
    elif args.workload == "serial":
        run_serial(args, rank, world)
    elif args.workload == "train":
        run_train(args, rank, world)
    else:
        run_ours(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
