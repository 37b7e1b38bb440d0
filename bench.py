"""Benchmark of the pSRM EM iteration on GB300.

One step = one EM iteration (E-pass, E-step k x k work, M-pass with the fused
Gram, eigen / polar / rho update) over the whole resident workload.

Headline workload: forrest-1024-like - 1024 subjects with uneven voxel counts
v_i ~ U[20000, 60000], T = 500, k = 50 (41 GB of BF16 X^ resident), the
paper's thousand-subject weak-scaling shape (Sec. V-C), on synthetic planted
data (the paper's datasets are not available).  The headline ``value`` is EM
iterations/s of the batched BF16-storage tensor-core form, the median of
several timed regions of K iterations; the plain per-subject FP32 form is
timed beside it on the same workload (``fp32_plain``).  The same run times
the forrest-like high-resolution shape (8 x 600000 voxels, T = 3500,
k = 100) and the greeneyes-like shape (16 subjects, T = 1000, k = 50) under
extra keys, each with its own roofline, clocks, end-to-end job and CPU
baseline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--config 4]
                    [--extra-configs 3,1] [--repeats 5]
                    [--impl ours|reference] [--store bf16|f32|both] [--no-cpu-baseline]

Under torchrun (N > 1) the headline workload's subjects are spread over the
ranks as Algorithm 1 spreads them over processes: each EM iteration is every
rank's share of the E-step, one NCCL all-reduce of the k x T reduction y and
four sums, the rest of the E-step and each rank's M-step (``--sharded``,
strong scaling: value = whole-workload EM iterations/s).  ``--replicas``
runs independent copies of the workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "pSRM EM iterations/s (BF16-batched tensor-core form; FP32 plain form reported beside)"
UNIT = "EM iterations/s"


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.t is not None:
                self.t.join(timeout=2)

    def summary(self):
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = max(smax, float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() in ("active", "1"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def workload(config: int, rank: int, subjects: int = 0, voxels_cap: int = 0, k: int = 0):
    """The config's planted spec and voxel counts; with subjects > 0 only the
    first `subjects` subjects, and with voxels_cap > 0 each subject cut to at
    most that many voxels (smaller cases of the same T and k, for
    profiling); with k > 0 the same shapes with that number of features."""
    import dataclasses

    import synth
    spec = synth.config_spec(config)
    vox = synth.draw_voxel_counts(spec)
    if subjects and subjects < len(vox):
        vox = vox[:subjects]
        spec = dataclasses.replace(spec, n_subjects=subjects,
                                   name=spec.name + " (first %d subjects)" % subjects)
    if voxels_cap and max(vox) > voxels_cap:
        vox = [min(int(v), int(voxels_cap)) for v in vox]
        spec = dataclasses.replace(spec, name=spec.name + " (voxels capped at %d)" % voxels_cap)
    if k and k != spec.k:
        spec = dataclasses.replace(spec, k=int(k), name=spec.name + " (k = %d)" % k)
    return spec, vox


# ncu captures committed under profiles/, by workload: DRAM bytes per launch of
# a kernel, valid while the kernel's source file is unchanged (its SHA-1 is
# recorded beside the number)
PROFILE_TAGS = {1: "greeneyes_like_N16_T1000_k50", 3: "forrest_like_N8_T3500_k100",
                4: "forrest1024_like_N1024_T500_k50"}


def profiled_traffic(kernel: str, config: int, voxels_total: int):
    """DRAM bytes of one launch from the committed ncu summary of this kernel
    on this workload.  A summary of a smaller case of the same shapes (the
    first subjects only: `voxels_captured` below the workload's) is scaled
    by voxel count, since every byte of these passes is per voxel row."""
    import hashlib
    import re
    tag = PROFILE_TAGS.get(config)
    if tag is None:
        return None, None
    path = os.path.join(ROOT, "profiles", f"{kernel}_{tag}.md")
    if not os.path.exists(path):
        return None, None
    text = open(path).read()
    mt = re.search(r"traffic_bytes_per_launch: (\d+)", text)
    ms = re.search(r"source_sha1: ([0-9a-f]{40}) \(([\w.]+) when captured\)", text)
    if not mt or not ms:
        return None, None
    src = os.path.join(ROOT, "paper_1608_04647_gb300", "csrc", ms.group(2))
    if not os.path.exists(src) or hashlib.sha1(open(src, "rb").read()).hexdigest() != ms.group(1):
        return None, os.path.relpath(path, ROOT) + " (stale: kernel source changed since the capture)"
    traffic = int(mt.group(1))
    mv = re.search(r"voxels_captured: (\d+)", text)
    if mv and int(mv.group(1)) != voxels_total:
        traffic = int(round(traffic * voxels_total / int(mv.group(1))))
        return traffic, os.path.relpath(path, ROOT) + " (smaller case, scaled by voxels x%.2f)" % (
            voxels_total / int(mv.group(1)))
    return traffic, os.path.relpath(path, ROOT)


def algorithmic_bytes(vox, T, k, xbytes, abytes):
    """Bytes one EM iteration must move (per pass: read X^ once; A_i read in
    the E-pass and written in the M-pass)."""
    V = float(sum(vox))
    e_pass = V * T * xbytes + V * k * abytes
    m_pass = V * T * xbytes + V * k * abytes
    return e_pass, m_pass


def parse_plan(text: str) -> dict:
    """'single_pass=1,f_l2_hints=7' -> {'single_pass': 1, 'f_l2_hints': 7}"""
    out = {}
    for item in filter(None, (x.strip() for x in text.split(","))):
        key, val = item.split("=")
        out[key.strip()] = int(val)
    return out


def single_pass_bytes(vox, T, k, xbytes, abytes):
    """Bytes one iteration of the single-pass form must move: X^ read once
    and A_i written (the pass's second look at each tile is served by L2)."""
    V = float(sum(vox))
    return V * T * xbytes + V * k * abytes


def paper_flops(vox, T, k):
    """Flop model of Sec. V-A per subject per iteration: two V_i x T x K
    products, one V_i x K x K product and a V_i x K economy SVD counted as
    Householder QR (2 m n^2 - 2/3 n^3)."""
    return float(sum(2 * (2 * v * T * k) + 2 * v * k * k + (2 * v * k * k - 2.0 / 3.0 * k ** 3) for v in vox))


def max_over_ranks(ms: float, world: int, device="cuda") -> float:
    """The slowest rank's time (all ranks receive it)."""
    if world <= 1:
        return ms
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def time_fit(model, stream, steps, warmup, repeats=1):
    """W untimed warm-up iterations, then `repeats` timed regions of exactly
    `steps` EM iterations each (CUDA events on the context's stream,
    synchronised on both sides).  Returns the ms of each region."""
    import torch
    model.fit_async(warmup)
    model.synchronize()
    out = []
    for _ in range(max(1, repeats)):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        model.fit_async(steps)
        e1.record(stream)
        e1.synchronize()
        model.synchronize()
        out.append(e0.elapsed_time(e1))
    return out


def ll_monotonicity(ll):
    """How far the log-likelihood trace ever fell from one iteration to the
    next: the number of decreases, the largest one in nats, and that drop as
    a fraction of the trace's own total increase (EM never decreases the
    likelihood in exact arithmetic; the FP32 and BF16 sums may)."""
    ll = np.asarray(ll, dtype=np.float64)
    d = np.diff(ll)
    drops = d[d < 0]
    rise = float(ll.max() - ll[0]) if len(ll) else 0.0
    worst = float(-drops.min()) if len(drops) else 0.0
    return {"iterations": int(len(ll)), "decreases": int(len(drops)), "max_decrease_nats": worst,
            "max_decrease_of_total_rise": (worst / rise) if rise > 0 else None,
            "total_rise_nats": rise}


def polar_diagnostics(model, n_iter):
    """Per iteration of a fresh fit: how many subjects' Newton-Schulz polar
    factors passed their accuracy certificate and how many fell back to the
    eigen-decomposition path (srm_debug_eig_sweeps after each M-step)."""
    import paper_1608_04647_gb300 as srm
    per_iter = []
    for _ in range(n_iter):
        model.fit(1)
        sw = srm.srm_debug_eig_sweeps(model.ctx, model.N + 1)[: model.N]
        per_iter.append(int(np.sum(sw >= 256)))
    return per_iter


def bench_workload(args, config, rank, world, stores, dev, peaks, e2e=True, cpu=True, label=None):
    """One workload: generate it on the device, tune the batched form, time
    `repeats` regions of K EM iterations (median reported), profile the same
    K iterations kernel by kernel, run one end-to-end job from pinned host
    buffers, and time the FP64 oracle on a bounded sample."""
    import torch

    import paper_1608_04647_gb300 as srm
    from synth.planted_torch import planted_dataset_torch

    spec, vox = workload(config, rank, args.subjects, args.voxels_cap, args.k)
    T, k = spec.T, spec.k
    d = planted_dataset_torch(spec, vox, device="cuda", seed_offset=rank)
    stream = torch.cuda.Stream()
    R = max(1, args.repeats)
    max_iter = args.warmup + R * args.steps + 64
    import tempfile
    cache = args.tune_cache or os.path.join(tempfile.gettempdir(), "srm_plans_bench_c%d_rank%d.txt" % (config, rank))
    if not args.tune_cache and os.path.exists(cache):
        os.remove(cache)
    tune = {"plan": None, "ms": None, "tuning_s": None}

    def make(store, graph=True, profile=False, **kw):
        m = srm.SRM(d["X"], d["W0"], k, store=store, graph=graph, profile=profile,
                    max_iter=kw.pop("max_iter", max_iter), stream=stream, single_pass=args.single_pass, **kw)
        if store == "bf16" and not args.no_autotune and not args.single_pass:
            t0 = time.perf_counter()
            plan, ms, _ = m.autotune(cache, iters=4)
            if tune["plan"] is None:
                tune.update(plan=plan, ms=round(ms, 4), tuning_s=round(time.perf_counter() - t0, 2))
        if store == "bf16" and args.plan:
            m.set_plan(**parse_plan(args.plan))
            if tune.get("override") is None:
                tune.update(plan=m.plan(), override=args.plan)
        return m

    results = {}
    e2e_res = None
    for store in stores:
        if store != stores[0] and e2e and not args.no_e2e and e2e_res is None:
            # the end-to-end job of the head store runs before the other store's
            # contexts come and go (their allocations slow a following setup)
            e2e_res = run_e2e(args, d, spec, vox, stream, world,
                              None if args.no_autotune or args.single_pass else cache, stores[0])
        m = make(store)
        lay = m.layout()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        with ClockSampler(dev) as cs:
            regions = time_fit(m, stream, args.steps, args.warmup, R if store == stores[0] else min(R, 2))
        regions = [max_over_ranks(x, world) for x in regions]
        ms = statistics.median(regions)
        ll = m.ll()
        results[store] = {"ms_total": ms, "ms_per_step": ms / args.steps, "layout": lay, "clocks": cs.summary(),
                          "regions_ms": [round(x, 4) for x in regions], "ll_monotone": ll_monotonicity(ll)}
        m.close()
        del m
        # per-kernel CUDA-event times over a profiled run of the same K steps
        mp = make(store, graph=False, profile=True)
        mp.fit_async(args.warmup)
        mp.kernel_times(reset=True)
        mp.fit_async(args.steps)
        kt = mp.kernel_times()
        mp.close()
        del mp
        results[store]["kernels"] = {n: {"launches": l, "ms": t} for n, (l, t) in kt.items() if l > 0}
        # the workload's own schedule from W^0, one iteration at a time: the
        # log-likelihood trace and the polar factors that needed the fallback
        md = make(store, graph=False, max_iter=spec.n_iter + 8)
        results[store]["polar_fallbacks_per_iteration"] = polar_diagnostics(md, spec.n_iter)
        results[store]["schedule_ll"] = ll_monotonicity(md.ll())
        md.close()
        del md
        torch.cuda.empty_cache()
    head = stores[0]
    xb = 2 if head == "bf16" else 4
    ab = 2 if head == "bf16" else 4
    e_bytes, m_bytes = algorithmic_bytes(vox, T, k, xb, ab)
    f_bytes = single_pass_bytes(vox, T, k, xb, ab)
    ks = results[head]["kernels"]
    single = bool(results[head]["layout"]["single_pass"])
    ms_step = results[head]["ms_per_step"]
    value = world * 1000.0 / ms_step
    # the committed captures are of each workload's own k: none applies to another k
    roofline = roofline_of(ks, head, e_bytes, m_bytes, f_bytes, len(vox), None if args.k else config, int(sum(vox)),
                           peaks)
    iter_bytes = f_bytes if single else e_bytes + m_bytes
    kernels_per_step = sum(v["launches"] for v in ks.values()) / args.steps
    clocks = results[head]["clocks"]
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": head,
        "data": "synthetic planted (Sec. II-A model), generated on device",
        "config": {"workload": label or spec.name, "N": len(vox), "T": T, "k": k, "voxels_total": int(sum(vox)),
                   "store": head, "l2": "inputs larger than L2 (resident X^ %.2f GB > 129 MB)" %
                   (results[head]["layout"]["xhat_bytes"] / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "graph": True, "single_pass": single,
                   "timing": "median of %d timed regions of %d EM iterations each (after %d warm-up iterations); "
                             "CUDA events on the context stream" % (R, args.steps, args.warmup),
                   "regions_ms": results[head]["regions_ms"],
                   "plan": tune["plan"] if head == "bf16" else None,
                   "autotune": None if head != "bf16" or tune["ms"] is None else
                   {"tuned_ms_per_iteration": tune["ms"], "tuning_s": tune["tuning_s"],
                    "plan_override": tune.get("override"),
                    "note": "srm_autotune before the timed region; later contexts replay the cache"}},
        "hbm_gbs_iteration": round(iter_bytes / (ms_step * 1e-3) / 1e9, 1),
        "roofline": roofline,
        "paper_gflops": round(paper_flops(vox, T, k) / (ms_step * 1e-3) / 1e9, 1),
        "gpu_launches": int(round(kernels_per_step * args.steps)),
        "clocks": clocks,
        "ms_x_sm_mhz": round(ms_step * clocks["sm_mhz"], 1) if clocks.get("sm_mhz") else None,
        "kernels_ms_per_step": {n: round(v["ms"] / args.steps, 4) for n, v in ks.items()},
        "kernels_note": "CUDA-event time per step of each kernel kind on the stream it runs on (SRM_PROFILE run "
                        "of the same steps); kinds on the second and third streams (sigma, eig, mtail, refine, rho, "
                        "polar, phi where they run beside a streaming pass) include time spent waiting for SMs",
        "ll_monotone": results[head]["ll_monotone"],
        "schedule": {"n_iter": spec.n_iter, "ll": results[head]["schedule_ll"],
                     "polar_fallbacks_per_iteration": results[head]["polar_fallbacks_per_iteration"],
                     "note": "the workload's fixed schedule from W^0, one iteration at a time: subjects whose "
                             "Newton-Schulz polar factor failed its certificate (eigen-decomposition fallback) "
                             "out of %d" % len(vox)},
    }
    if "f32" in results and head != "f32":
        r = results["f32"]
        ke, km = algorithmic_bytes(vox, T, k, 4, 4)
        out["fp32_plain"] = {"value": round(world * 1000.0 / r["ms_per_step"], 3), "ms_per_step":
                             round(r["ms_per_step"], 4), "regions_ms": r["regions_ms"], "clocks": r["clocks"],
                             "roofline": roofline_of(r["kernels"], "f32", ke, km, ke, len(vox), config,
                                                     int(sum(vox)), peaks),
                             "ll_monotone": r["ll_monotone"],
                             "schedule": {"ll": r["schedule_ll"],
                                          "polar_fallbacks_per_iteration": r["polar_fallbacks_per_iteration"]},
                             "kernels_ms_per_step": {n: round(v["ms"] / args.steps, 4) for n, v in
                                                     r["kernels"].items()}}
    if e2e and not args.no_e2e:
        out["e2e"] = e2e_res if e2e_res is not None else run_e2e(
            args, d, spec, vox, stream, world, None if args.no_autotune or args.single_pass else cache, head)
    if cpu and rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(spec, vox, d, budget_s=args.cpu_budget)
    del d
    torch.cuda.empty_cache()
    return out


def roofline_of(ks, store, e_bytes, m_bytes, f_bytes, n_subjects, config, voxels_total, peaks):
    """The dominant streaming kernel (largest time per step) with its
    algorithmic bytes per launch over its CUDA-event launch duration."""
    streaming = {"estep_tc": e_bytes, "mstep_tc": m_bytes, "fpass_tc": f_bytes} if store == "bf16" else \
        {"estep_simt": e_bytes, "mstep_simt": m_bytes}
    present = [(ks[n]["ms"], n) for n in streaming if n in ks]
    if not present:
        return None
    _, name = max(present)
    t = ks[name]["ms"] / ks[name]["launches"]
    b = streaming[name]
    if store == "f32":
        b = b / n_subjects  # per launch (one launch per subject; the mean subject)
    achieved = b / (t * 1e-3) / 1e9
    traffic, tsrc = profiled_traffic(name, config, voxels_total) if store == "bf16" else (None, None)
    return {"kernel": name, "bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"],
            "unit": "GB/s", "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": traffic,
            "traffic_source": tsrc, "peak_source": peaks["source"] + " (copy bandwidth)",
            "bytes_per_launch": b, "ms_per_launch": t,
            "traffic_over_algorithmic": round(traffic / b, 4) if traffic else None}


def bench_sharded(args, rank, world, dev, peaks):
    """The headline workload's subjects spread over the ranks (Algorithm 1,
    D-SRM): each rank holds a context over its shard, and each EM iteration
    is this rank's share of the E-step, one NCCL all-reduce of y (k x T) and
    four sums, the rest of the E-step and the M-step of its own subjects
    (shard.fit_sharded).  One step = one EM iteration of the whole workload,
    so `value` is whole-workload EM iterations/s ("scaling": "strong")."""
    import torch
    import torch.distributed as dist

    import paper_1608_04647_gb300 as srm
    from paper_1608_04647_gb300.shard import fit_sharded, imbalance, shard_subjects
    from synth.planted_torch import planted_dataset_torch

    spec, vox = workload(args.config, rank, args.subjects, args.voxels_cap, args.k)
    T, k = spec.T, spec.k
    plan = shard_subjects(vox, world)
    mine = plan[rank]
    d = planted_dataset_torch(spec, vox, device="cuda", subjects=mine)
    stream = torch.cuda.Stream()
    R = max(1, args.repeats)
    max_iter = args.warmup + R * args.steps + 64
    import tempfile
    cache = os.path.join(tempfile.gettempdir(), "srm_plans_bench_sharded_c%d_rank%d.txt" % (args.config, rank))
    if os.path.exists(cache):
        os.remove(cache)
    m = srm.SRM(d["X"], d["W0"], k, store="bf16", graph=False, max_iter=max_iter, stream=stream)
    if not args.no_autotune:
        m.autotune(cache, iters=4)
    fit_sharded(m, args.warmup, dist.all_reduce)
    m.synchronize()
    regions = []
    with ClockSampler(dev) as cs:
        for _ in range(R):
            dist.barrier()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fit_sharded(m, args.steps, dist.all_reduce)
            e1.record(stream)
            e1.synchronize()
            m.synchronize()
            regions.append(max_over_ranks(e0.elapsed_time(e1), world))
    ms_step = statistics.median(regions) / args.steps
    ll = m.ll()
    lay = m.layout()
    m.close()
    # per-kernel times of this rank over a profiled run of the same steps
    mp = srm.SRM(d["X"], d["W0"], k, store="bf16", profile=True, max_iter=max_iter, stream=stream)
    if not args.no_autotune:
        mp.autotune(cache, iters=4)
    fit_sharded(mp, args.warmup, dist.all_reduce)
    mp.kernel_times(reset=True)
    fit_sharded(mp, args.steps, dist.all_reduce)
    kt = mp.kernel_times()
    mp.close()
    ks = {n: {"launches": l, "ms": t} for n, (l, t) in kt.items() if l > 0}
    myvox = [vox[i] for i in mine]
    e_bytes, m_bytes = algorithmic_bytes(myvox, T, k, 2, 2)
    f_bytes = single_pass_bytes(myvox, T, k, 2, 2)
    roofline = roofline_of(ks, "bf16", e_bytes, m_bytes, f_bytes, len(myvox), -1, int(sum(myvox)), peaks)
    clocks = cs.summary()
    out = {
        "metric": METRIC, "value": round(1000.0 / ms_step, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "bf16", "data": "synthetic planted (Sec. II-A model), generated on device",
        "config": {"workload": spec.name, "N": len(vox), "T": T, "k": k, "voxels_total": int(sum(vox)),
                   "store": "bf16", "parallelism": "subjects sharded over %d ranks (Algorithm 1), one NCCL "
                   "all-reduce of y and 4 sums per EM iteration" % world,
                   "shard_imbalance": round(imbalance(vox, plan), 4), "subjects_per_rank": [len(p) for p in plan],
                   "l2": "inputs larger than L2 (resident X^ %.2f GB per rank)" % (lay["xhat_bytes"] / 1e9),
                   "timing": "median of %d timed regions of %d EM iterations, max over ranks" % (R, args.steps),
                   "regions_ms": [round(x, 4) for x in regions]},
        "roofline": roofline, "clocks": clocks,
        "gpu_launches": int(round(sum(v["launches"] for v in ks.values()))),
        "kernels_ms_per_step": {n: round(v["ms"] / args.steps, 4) for n, v in ks.items()},
        "ll_monotone": ll_monotonicity(ll),
        "e2e": {"value": None, "unit": UNIT, "skipped": "the sharded run reports device-resident throughput only"},
    }
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(spec, myvox, d, budget_s=args.cpu_budget)
    return out


def run_ours(args, rank, world):
    import torch

    import paper_1608_04647_gb300 as srm
    from paper_1608_04647_gb300 import _build

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    if rank == 0:
        _build.build()
    if world > 1:
        torch.distributed.barrier()
    srm.load_library()
    peaks = load_peaks()
    if args.sharded:
        return bench_sharded(args, rank, world, dev, peaks)
    stores = [args.store] if args.store != "both" else ["bf16", "f32"]
    out = bench_workload(args, args.config, rank, world, stores, dev, peaks)
    extras = [int(x) for x in args.extra_configs.split(",") if x.strip() != ""] \
        if args.subjects == 0 and args.voxels_cap == 0 and args.k == 0 else []
    for c in extras:
        if c == args.config:
            continue
        key = EXTRA_KEYS.get(c, "config_%d" % c)
        out[key] = bench_workload(args, c, rank, world, stores, dev, peaks)
    out["extra_keys"] = sorted(k for k in out if k not in ("metric", "value", "unit", "n_gpus", "steps", "warmup",
                                                           "ms_per_step", "higher_is_better", "scaling",
                                                           "vs_baseline", "dtype", "data", "config", "roofline",
                                                           "cpu_baseline", "clocks", "e2e", "gpu_launches"))
    return out


EXTRA_KEYS = {0: "raider_like", 1: "greeneyes_like", 2: "batched_64", 3: "forrest_like", 4: "forrest1024_like"}


def run_e2e(args, d, spec, vox, stream, world, tune_cache=None, store="bf16"):
    """One whole user job through the public API with host buffers: pinned
    host X (FP32; pageable if the host refuses to pin that much) -> srm_init
    with SRM_HOST_INPUT (the library streams each subject through one staging
    buffer and centres it) -> srm_fit(n_iter) -> parameters, E[S] and the
    log-likelihood back to the host.  Value = EM iterations / job time."""
    import torch

    import paper_1608_04647_gb300 as srm
    try:
        Xh = [x.to("cpu").pin_memory() for x in d["X"]]  # page-locked before the timed region
        memory = "pinned"
    except RuntimeError:
        Xh = [x.to("cpu") for x in d["X"]]
        memory = "pageable"
    n_iter = spec.n_iter
    h2d = sum(x.numel() * x.element_size() for x in Xh)
    times = []
    for rep in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m = srm.SRM(Xh, d["W0"], spec.k, store=store, graph=True, host_input=True, stream=stream,
                    max_iter=n_iter + 8, single_pass=args.single_pass)
        if store == "bf16" and tune_cache:
            m.autotune(tune_cache, iters=4)  # a cached plan: no timing, one file read
        if store == "bf16" and args.plan:
            m.set_plan(**parse_plan(args.plan))
        ll = m.fit(n_iter)
        rho2, sig = m.params()
        S = m.get_s().cpu()
        t1 = time.perf_counter()
        m.close()
        times.append(t1 - t0)
    del Xh
    d2h = S.numel() * 4 + rho2.nbytes + sig.nbytes + ll.nbytes
    best = min(times)
    return {"value": round(world * n_iter / best, 3), "unit": UNIT, "job_s": round(best, 4),
            "jobs_s": [round(t, 4) for t in times],
            "iterations_per_job": n_iter, "h2d_bytes_per_step": int(h2d / n_iter),
            "d2h_bytes_per_step": int(d2h / n_iter),
            "host_memory": memory,
            "note": "step = one EM iteration of a %d-iteration job; host->device copy of X from %s host "
                    "memory (FP32), context setup, centring, fit and result read-back inside the timed region; "
                    "best of 2 jobs" % (n_iter, memory)}


def blas_threads():
    """Threads of the BLAS the oracle's NumPy uses (threadpoolctl if present,
    else the OpenBLAS entry point of the loaded library), or None."""
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        return max((i.get("num_threads", 0) for i in info), default=None)
    except Exception:
        pass
    try:
        import ctypes
        import numpy  # noqa: F401  (loads its BLAS)
        libs = set()
        with open("/proc/self/maps") as f:
            for line in f:
                p = line.split()[-1]
                if "openblas" in os.path.basename(p).lower() and p.endswith(tuple(".so" + s for s in ("", ".0"))) \
                        or ("openblas" in p.lower() and ".so" in p):
                    libs.add(p)
        for p in libs:
            lib = ctypes.CDLL(p)
            for fn in ("scipy_openblas_get_num_threads64_", "openblas_get_num_threads64_",
                       "openblas_get_num_threads"):
                if hasattr(lib, fn):
                    return int(getattr(lib, fn)())
    except Exception:
        pass
    return None


def oracle_seconds_per_voxel(T, k):
    """Estimated time of one FP64 oracle EM iteration per voxel row on this
    kind of host (16 Grace cores: 2.8 ns per voxel x TR at k = 50, linear in
    k), used only to size the bounded samples."""
    return 2.8e-9 * T * max(k, 10) / 50.0


def sample_rows(vox, T, k, target_s):
    """A bounded sample of the workload for the oracle: its first subjects,
    whole, while one EM iteration over them stays within about `target_s`
    seconds; if even the first subject is larger, that subject cut to its
    first rows.  Returns the voxel rows taken from each sampled subject."""
    per = oracle_seconds_per_voxel(T, k)
    rows, tot = [], 0.0
    for v in vox:
        if rows and tot + v * per > target_s:
            break
        rows.append(int(v))
        tot += v * per
    if len(rows) == 1 and rows[0] * per > target_s:
        rows[0] = max(k + 1, int(target_s / per))
    return rows


def describe_sample(rows, vox, T, k):
    cut = len(rows) == 1 and rows[0] < vox[0]
    frac = float(sum(rows)) / float(sum(vox))
    what = ("the first %d voxel rows of subject 0 (of %d)" % (rows[0], vox[0]) if cut else
            "the first %d of %d subjects" % (len(rows), len(vox)))
    return frac, "%s: %d of %d voxels (%.3f%% of the workload), T = %d, k = %d" % (
        what, int(sum(rows)), int(sum(vox)), 100 * frac, T, k)


def cpu_baseline(spec, vox, d, budget_s=20.0):
    """The FP64 oracle as it stands, on this host's cores: consecutive whole
    EM iterations (Algorithm 1: E-step then M-step over every sampled
    subject) on a bounded sample of the workload, with the very data the
    GPU fitted (copied down and up-cast) and the same W^0, until the budget
    is spent or the workload's schedule ends.  The oracle's cost per
    iteration is linear in the voxels, so EM iterations/s of the whole
    workload = sample fraction / seconds per sample iteration."""
    import oracle
    rows = sample_rows(vox, spec.T, spec.k, budget_s / 3.0)
    Xh = [oracle.center(d["X"][i][:r].double().cpu().numpy())[0] for i, r in enumerate(rows)]
    W0 = []
    for i, r in enumerate(rows):
        w = d["W0"][i][:r].double().cpu().numpy()
        if r < vox[i]:
            w = np.linalg.qr(w)[0]  # a cut W^0 is re-orthonormalised (same cost per iteration)
        W0.append(w)
    state = {"W": W0, "rho2": None, "Sigma": None}
    t0 = time.perf_counter()
    iters = 0
    while iters < spec.n_iter:
        r = oracle.fit(Xh, state["W"], 1, rho2_0=state["rho2"], Sigma_0=state["Sigma"], centered=True)
        state = {"W": r["W"], "rho2": r["rho2"], "Sigma": r["Sigma_s"]}
        iters += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = (time.perf_counter() - t0) / iters
    frac, what = describe_sample(rows, vox, spec.T, spec.k)
    return {"value": round(frac / dt, 6), "unit": UNIT, "cores": os.cpu_count(),
            "blas_threads": blas_threads(), "kind": "oracle",
            "seconds_per_sample_iteration": round(dt, 4), "sample_iterations": iters,
            "sample": "%s; %d consecutive EM iterations of the FP64 NumPy oracle from W^0 on the data the GPU "
                      "fitted; value = sample fraction / seconds per sample iteration" % (what, iters)}


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle as it stands, on the host cores, on a
    bounded sample of the same workload.  Each step is one whole EM
    iteration (Algorithm 1) of the oracle over the workload's first subjects
    (all of it where one iteration of the whole workload is short), drawn on
    the host by the same planted generator.  ms_per_step is the measured
    time of one such step; value = EM iterations/s of the whole workload =
    (sample voxels / workload voxels) / seconds per step, the oracle's cost
    being linear in the voxels."""
    import oracle
    import synth
    spec, vox = workload(args.config, rank, args.subjects, args.voxels_cap, args.k)
    rows = sample_rows(vox, spec.T, spec.k, args.ref_step_s)
    dd = synth.planted_dataset(spec, voxel_counts=rows, dtype=np.float64)
    Xh = [oracle.center(x)[0] for x in dd["X"]]
    del dd["X"]
    state = {"W": dd["W0"], "rho2": None, "Sigma": None}

    def step():
        r = oracle.fit(Xh, state["W"], 1, rho2_0=state["rho2"], Sigma_0=state["Sigma"], centered=True)
        state.update(W=r["W"], rho2=r["rho2"], Sigma=r["Sigma_s"])

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    frac, what = describe_sample(rows, vox, spec.T, spec.k)
    value = frac / dt
    sample = ("%s, drawn on the host by the same planted generator; each step one EM iteration of the FP64 NumPy "
              "oracle over it, consecutive from W^0; value = sample fraction / seconds per step" % what)
    return {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic planted (Sec. II-A model), drawn on the host",
            "config": {"workload": spec.name, "N": len(vox), "T": spec.T, "k": spec.k,
                       "voxels_total": int(sum(vox))},
            "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": os.cpu_count(),
                             "blas_threads": blas_threads(), "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_k_sweep(args):
    """Number of features k against throughput on the greeneyes-like shapes
    (N = 16, v ~ U[2e4, 6e4], T = 1000; the paper's E3 runtime-vs-K, whose
    values appear only in a figure): one JSON line per k with EM iterations/s
    of the tuned batched form and each streaming pass's GB/s.  k up to 128
    (the library's limit)."""
    import dataclasses

    import torch

    import paper_1608_04647_gb300 as srm
    import synth
    from paper_1608_04647_gb300 import _build
    from synth.planted_torch import planted_dataset_torch

    _build.build()
    srm.load_library()
    base = synth.config_spec(1)
    vox = synth.draw_voxel_counts(base)
    peaks = load_peaks()
    for k in (10, 30, 60, 100, 128):
        spec = dataclasses.replace(base, k=k, name=f"greeneyes-like N=16 v~U[2e4,6e4] T=1000 k={k}")
        d = planted_dataset_torch(spec, vox, device="cuda")
        stream = torch.cuda.Stream()
        m = srm.SRM(d["X"], d["W0"], k, store="bf16", graph=True,
                    max_iter=args.warmup + max(1, args.repeats) * args.steps + 8, stream=stream)
        plan, _, _ = m.autotune(None, iters=4)
        ms = statistics.median(time_fit(m, stream, args.steps, args.warmup, max(1, args.repeats))) / args.steps
        m.close()
        mp = srm.SRM(d["X"], d["W0"], k, store="bf16", graph=False, profile=True,
                     max_iter=args.warmup + args.steps + 8, stream=stream)
        mp.set_plan(**plan)
        mp.fit_async(args.warmup)
        mp.kernel_times(reset=True)
        mp.fit_async(args.steps)
        kt = mp.kernel_times()
        mp.close()
        e_bytes, m_bytes = algorithmic_bytes(vox, spec.T, k, 2, 2)
        f_bytes = single_pass_bytes(vox, spec.T, k, 2, 2)
        passes = {}
        for name, b in (("estep_tc", e_bytes), ("mstep_tc", m_bytes), ("fpass_tc", f_bytes)):
            if kt.get(name, (0, 0))[0]:
                t = kt[name][1] / kt[name][0]
                passes[name] = {"ms": round(t, 4), "gbs": round(b / (t * 1e-3) / 1e9, 1),
                                "frac": round(b / (t * 1e-3) / 1e9 / peaks["hbm_gbs"], 3)}
        print(json.dumps({"k_sweep": True, "k": k, "metric": METRIC, "value": round(1000.0 / ms, 3), "unit": UNIT,
                          "ms_per_step": round(ms, 4), "single_pass": bool(plan["single_pass"]), "passes": passes,
                          "peak_gbs": peaks["hbm_gbs"],
                          "paper_gflops": round(paper_flops(vox, spec.T, k) / (ms * 1e-3) / 1e9, 1),
                          "kernels_ms_per_step": {n: round(v[1] / args.steps, 4) for n, v in kt.items() if v[0]}}),
              flush=True)
        del d
        torch.cuda.empty_cache()


HTFA_METRIC = "HTFA local cost evaluations/s (F_i of Eq. 14 and ||X_i - W_i F_i||_F^2 for every subject)"
HTFA_UNIT = "evaluations/s"


def fp32_alu_peak_tflops():
    """FP32 FMA peak of the SIMT pipes: 152 SMs x 128 FP32 lanes x 2 flops
    x the maximum SM clock (2070 MHz)."""
    mhz = 2070.0
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    return 152 * 128 * 2 * mhz * 1e6 / 1e12


def htfa_cpu_baseline(spec, d, budget_s=20.0, max_subjects=4):
    """The FP64 oracle (as it stands) on the host cores: one cost evaluation
    (factors, then residual) of the first subjects, time scaled by subject
    count (every subject has the same shape)."""
    import oracle
    n = min(spec.n_subjects, max_subjects)
    Xs = [(d["W"][i].astype(np.float64) @ oracle.rbf_factors(d["positions"][i], d["mu"][i], d["lam"][i])
           + d["E"][i]) for i in range(n)]
    t0 = time.perf_counter()
    reps = 0
    while True:
        for i in range(n):
            F = oracle.rbf_factors(d["positions"][i], d["mu"][i], d["lam"][i])
            oracle.htfa_residual(Xs[i], d["W"][i], F)
        reps += 1
        if time.perf_counter() - t0 > budget_s or reps >= 20:
            break
    dt = (time.perf_counter() - t0) / reps * spec.n_subjects / n
    return {"value": round(1.0 / dt, 6), "unit": HTFA_UNIT, "cores": os.cpu_count(), "blas_threads": blas_threads(),
            "kind": "oracle",
            "sample": "%d subject(s) of %d (T = %d, V = %d, K = %d), %d evaluation(s) of the FP64 NumPy oracle; time "
                      "scaled by subject count (x%.1f)" % (n, spec.n_subjects, spec.T, spec.V, spec.K, reps,
                                                           spec.n_subjects / n)}


def htfa_profiled_traffic(kernel: str, workload: str):
    """DRAM bytes of one launch from the committed ncu summary of this HTFA
    kernel on this workload, if the kernel source is unchanged since."""
    import hashlib
    import re
    tag = {"greeneyes-subsampled-like": "greeneyes_subsampled_like_N40_T174_V6857_K100"}.get(workload)
    if tag is None:
        return None, None
    path = os.path.join(ROOT, "profiles", f"{kernel}_{tag}.md")
    if not os.path.exists(path):
        return None, None
    text = open(path).read()
    mt = re.search(r"traffic_bytes_per_launch: (\d+)", text)
    ms = re.search(r"source_sha1: ([0-9a-f]{40}) \(([\w.]+) when captured\)", text)
    if not mt or not ms:
        return None, None
    src = os.path.join(ROOT, "paper_1608_04647_gb300", "csrc", ms.group(2))
    if not os.path.exists(src) or hashlib.sha1(open(src, "rb").read()).hexdigest() != ms.group(1):
        return None, os.path.relpath(path, ROOT) + " (stale: kernel source changed since the capture)"
    return int(mt.group(1)), os.path.relpath(path, ROOT)


def run_htfa(args):
    """One step = the NLLS solver's cost evaluation for every subject of the
    batch: F_i = srm_htfa_factors (Eq. 14), then r_i = srm_htfa_residual."""
    import torch

    import synth.htfa_inputs as hi
    from paper_1608_04647_gb300 import _build, htfa
    spec = hi.HTFA_CONFIGS[args.htfa_workload]
    d = hi.draw(spec)
    n, T, V, K = spec.n_subjects, spec.T, spec.V, spec.K
    if args.impl == "reference":
        cb = htfa_cpu_baseline(spec, d, budget_s=args.cpu_budget)
        return {"impl": "reference", "metric": HTFA_METRIC, "value": cb["value"], "unit": HTFA_UNIT, "n_gpus": 0,
                "higher_is_better": True, "dtype": "f64", "data": "synthetic (seeded HTFA-shaped inputs)",
                "config": {"workload": spec.name, "n_subjects": n, "T": T, "V": V, "K": K}, "cpu_baseline": cb,
                "e2e": {"value": cb["value"], "unit": HTFA_UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    _build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    X = torch.from_numpy(d["E"]).cuda()        # the data's values do not change the work
    W = torch.from_numpy(d["W"]).cuda()
    mu = torch.from_numpy(d["mu"]).cuda()
    lam = torch.from_numpy(d["lam"]).cuda()
    grid = htfa.GridPositions([torch.from_numpy(a) for a in d["axes"]], torch.from_numpy(d["vox"]).cuda())
    F = torch.empty((n, K, V), device="cuda")
    out = torch.empty((n,), dtype=torch.float64, device="cuda")
    work = torch.empty(max(1, htfa.residual_workspace(n, K, T, V) // 8), dtype=torch.float64, device="cuda")
    fwork = torch.empty(max(1, htfa.factors_workspace(n, K, grid.n_axis) // 8), dtype=torch.float64,
                        device="cuda")
    torch.cuda.synchronize()

    def step():
        htfa.factors(grid, mu, lam, out=F, work=fwork)
        htfa.residual(X, W, F, out=out, work=work)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(0) as cs:
            e0.record(stream)
            for _ in range(args.steps):
                step()
            e1.record(stream)
            torch.cuda.synchronize()
        ms_step = e0.elapsed_time(e1) / args.steps
        # per-call CUDA-event times on the same stream
        n_ev = min(args.steps, 200)
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(n_ev)]
        for i in range(n_ev):
            ev[i][0].record(stream)
            htfa.factors(grid, mu, lam, out=F, work=fwork)
            ev[i][1].record(stream)
            htfa.residual(X, W, F, out=out, work=work)
            ev[i][2].record(stream)
        torch.cuda.synchronize()
        # z-score of the batch (data standardisation; once per dataset, not per evaluation)
        Z = torch.empty_like(X)
        htfa.zscore(X, out=Z)
        z0, z1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        z0.record(stream)
        for _ in range(n_ev):
            htfa.zscore(X, out=Z)
        z1.record(stream)
        torch.cuda.synchronize()
        t_z = z0.elapsed_time(z1) / n_ev
        del Z
    t_f = sum(e[0].elapsed_time(e[1]) for e in ev) / n_ev
    t_r = sum(e[1].elapsed_time(e[2]) for e in ev) / n_ev
    flops = 2.0 * n * T * V * K
    peak = fp32_alu_peak_tflops()
    achieved = flops / (t_r * 1e-3) / 1e12
    f_bytes = n * K * V * 4 + n * V * 12
    r_bytes = n * T * V * 4 + n * K * V * 4 + n * T * K * 4
    hbm = load_peaks()["hbm_gbs"]
    traffic, tsrc = htfa_profiled_traffic("htfa_residual_tc" if K <= 128 else "htfa_residual", spec.name)
    res = {
        "metric": HTFA_METRIC, "value": round(1000.0 / ms_step, 3), "unit": HTFA_UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded HTFA-shaped inputs: grid voxels, centers, widths, weights, noise)",
        "config": {"workload": spec.name, "n_subjects": n, "T": T, "V": V, "K": K,
                   "l2": "inputs larger than L2 (X %.0f MB + F %.0f MB > 129 MB)" % (n * T * V * 4 / 1e6,
                                                                                  n * K * V * 4 / 1e6)},
        "timing_note": "per-call CUDA-event times over the first %d steps of a second run on the same stream" % n_ev,
        "roofline": ({"kernel": "htfa_residual (tensor-core tile + sum launches)", "bound": "hbm",
                      "achieved": round(r_bytes / (t_r * 1e-3) / 1e9, 1), "peak": hbm, "unit": "GB/s",
                      "frac": round(r_bytes / (t_r * 1e-3) / 1e9 / hbm, 4), "traffic": traffic,
                      "traffic_source": tsrc, "algorithmic_bytes_per_launch": r_bytes,
                      "peak_source": load_peaks()["source"] + " (copy bandwidth)",
                      "flops_per_launch": flops, "ms_per_launch": round(t_r, 5),
                      "tflops_effective": round(achieved, 2),
                      "note": "K <= 128: W F from three BF16 pieces per operand on the tensor cores (6 MMAs per "
                              "K step, FP32 accumulate), HBM-bound at K flop per byte x 6"}
                     if K <= 128 else
                     {"kernel": "htfa_residual (tile + sum launches)", "bound": "alu", "achieved": round(achieved, 2),
                      "peak": round(peak, 2), "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                      "traffic": traffic, "traffic_source": tsrc, "algorithmic_bytes_per_launch": r_bytes,
                      "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock",
                      "flops_per_launch": flops, "ms_per_launch": round(t_r, 5),
                      "hbm_gbs": round(r_bytes / (t_r * 1e-3) / 1e9, 1)}),
        "factors": {"ms_per_call": round(t_f, 5), "launches_per_call": 2, "bytes_per_call": f_bytes,
                    "achieved_gbs": round(f_bytes / (t_f * 1e-3) / 1e9, 1), "peak_gbs": hbm,
                    "frac": round(f_bytes / (t_f * 1e-3) / 1e9 / hbm, 4)},
        "zscore": {"ms_per_launch": round(t_z, 5), "bytes_per_launch": 2 * n * T * V * 4,
                   "achieved_gbs": round(2 * n * T * V * 4 / (t_z * 1e-3) / 1e9, 1), "peak_gbs": hbm,
                   "frac": round(2 * n * T * V * 4 / (t_z * 1e-3) / 1e9 / hbm, 4),
                   "note": "timed apart from the step: the data are standardised once, not per evaluation"},
        "gpu_launches": 4 * args.steps, "clocks": cs.summary(),
    }
    if not args.no_e2e:
        Xh = X.cpu().pin_memory()
        Wh, muh, lamh = W.cpu().pin_memory(), mu.cpu().pin_memory(), lam.cpu().pin_memory()
        voxh = grid.vox.cpu().pin_memory()
        outh = torch.empty((n,), dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        e2e_steps = min(args.steps, 50)
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for _ in range(e2e_steps):
                X.copy_(Xh, non_blocking=True)
                W.copy_(Wh, non_blocking=True)
                mu.copy_(muh, non_blocking=True)
                lam.copy_(lamh, non_blocking=True)
                grid.vox.copy_(voxh, non_blocking=True)
                step()
                outh.copy_(out, non_blocking=True)
                stream.synchronize()
        dt = (time.perf_counter() - t0) / e2e_steps
        h2d = sum(t.numel() * t.element_size() for t in (Xh, Wh, muh, lamh, voxh))
        res["e2e"] = {"value": round(1.0 / dt, 3), "unit": HTFA_UNIT, "h2d_bytes_per_step": int(h2d),
                      "d2h_bytes_per_step": int(outh.numel() * 8),
                      "steps": e2e_steps,
                      "note": "pinned host X, W, centers, widths and voxel indices copied in, the residuals copied "
                              "out, every step"}
    if not args.no_cpu_baseline:
        res["cpu_baseline"] = htfa_cpu_baseline(spec, d, budget_s=args.cpu_budget)
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--config", type=int, default=4, help="headline workload (4: forrest-1024-like)")
    ap.add_argument("--extra-configs", default="3,1", help="workloads timed in the same run under extra keys "
                    "(comma list; empty for none)")
    ap.add_argument("--repeats", type=int, default=5, help="timed regions of K steps each; the median is reported")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--store", choices=["bf16", "f32", "both"], default="both")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sharded", action="store_true", help="spread the headline workload's subjects over the "
                    "ranks with one NCCL all-reduce per EM iteration (the default under torchrun with N > 1)")
    ap.add_argument("--replicas", action="store_true", help="under torchrun: independent replicas instead of "
                    "the sharded workload")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0, help="seconds of oracle time for cpu_baseline")
    ap.add_argument("--ref-step-s", type=float, default=1.0, help="reference arm: about this many seconds of "
                    "oracle work per step (the sample size)")
    ap.add_argument("--k-sweep", action="store_true", help="throughput against k (extra lines, not the bench line)")
    ap.add_argument("--single-pass", action="store_true", help="force the single-pass form (SRM_SINGLE_PASS), "
                    "no autotuning")
    ap.add_argument("--no-autotune", action="store_true", help="run the library's default launch plan")
    ap.add_argument("--tune-cache", default=None, help="plan cache file kept across runs (default: a fresh one)")
    ap.add_argument("--plan", default="", help="launch-plan fields set after tuning, e.g. 'single_pass=0' "
                    "(srm_set_plan; for profiling one form)")
    ap.add_argument("--k", type=int, default=0, help="the headline workload's shapes with this number of features "
                    "(a smaller or larger case, for profiling; no extra workloads then)")
    ap.add_argument("--voxels-cap", type=int, default=0, help="cut every subject to at most this many voxels (a "
                    "smaller case of the same T and k, for ncu captures)")
    ap.add_argument("--subjects", type=int, default=0, help="only the first K subjects of the workload (a smaller "
                    "case of the same shapes, for ncu captures)")
    ap.add_argument("--htfa", action="store_true", help="the HTFA cost evaluation instead of the EM iteration "
                    "(its own line)")
    ap.add_argument("--htfa-workload", default="greeneyes-subsampled-like",
                    help="greeneyes-subsampled-like | jacobian-example-like | ragged-small")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.htfa:
        if int(os.environ.get("RANK", "0")) == 0:
            print(json.dumps(run_htfa(args)))
        return
    if args.k_sweep:
        run_k_sweep(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(run_reference(args, rank, world)))
        return
    if world > 1 and not args.replicas:
        args.sharded = True
    if world > 1 or args.sharded:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        os.environ.setdefault("MASTER_PORT", "29511")
        os.environ.setdefault("RANK", str(rank))
        os.environ.setdefault("WORLD_SIZE", str(world))
        torch.distributed.init_process_group("nccl")
    out = run_ours(args, rank, world)
    if world > 1 or args.sharded:
        import torch
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
