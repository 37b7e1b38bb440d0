"""Benchmark of the pSRM EM iteration on GB300.

One step = one EM iteration (E-pass, E-step k x k work, M-pass with the fused
Gram, eigen / polar / rho update) over the whole resident workload.

Default workload: the greeneyes-like case - 16 subjects with uneven voxel
counts v_i ~ U[20000, 60000], T = 1000, k = 50 - on synthetic planted data
(the paper's datasets are not available).  The headline ``value`` is EM
iterations/s of the batched BF16-storage tensor-core form; the plain
per-subject FP32 form is timed beside it on the same workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--config 1]
                    [--impl ours|reference] [--store bf16|f32] [--no-cpu-baseline]

Under torchrun (N > 1) every rank runs an independent replica of the
workload (its own seed) on its own GPU; the path's one exchange step (the
k x T reduction of Algorithm 1) is not distributed here.
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


def workload(config: int, rank: int, subjects: int = 0):
    """The config's planted spec and voxel counts; with subjects > 0 only the
    first `subjects` subjects (a smaller case of the same shapes, for
    profiling)."""
    import dataclasses

    import synth
    spec = synth.config_spec(config)
    vox = synth.draw_voxel_counts(spec)
    if subjects and subjects < len(vox):
        vox = vox[:subjects]
        spec = dataclasses.replace(spec, n_subjects=subjects,
                                   name=spec.name + " (first %d subjects)" % subjects)
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


def time_fit(model, stream, steps, warmup):
    import torch
    model.fit_async(warmup)
    model.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    model.fit_async(steps)
    e1.record(stream)
    e1.synchronize()
    model.synchronize()
    return e0.elapsed_time(e1)  # ms


def run_ours(args, rank, world):
    import torch

    import paper_1608_04647_gb300 as srm
    from paper_1608_04647_gb300 import _build
    from synth.planted_torch import planted_dataset_torch

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    if rank == 0:
        _build.build()
    if world > 1:
        torch.distributed.barrier()
    srm.load_library()
    spec, vox = workload(args.config, rank, args.subjects)
    T, k = spec.T, spec.k
    peaks = load_peaks()
    d = planted_dataset_torch(spec, vox, device="cuda", seed_offset=rank)
    stream = torch.cuda.Stream()
    max_iter = args.warmup + args.steps + 64

    # launch plan of the batched form: tuned once on this device and these
    # shapes (srm_autotune, before any timed region), then replayed from the
    # cache file by every later context of the same shapes
    tune = {"cache": None, "plan": None, "ms": None, "tuning_s": None}
    if args.tune_cache:
        tune["cache"] = args.tune_cache
    else:
        import tempfile
        tune["cache"] = os.path.join(tempfile.gettempdir(), "srm_plans_bench_rank%d.txt" % rank)
        if os.path.exists(tune["cache"]):
            os.remove(tune["cache"])

    def make(store, graph=True, profile=False):
        m = srm.SRM(d["X"], d["W0"], k, store=store, graph=graph, profile=profile, max_iter=max_iter,
                    stream=stream, single_pass=args.single_pass)
        if store == "bf16" and not args.no_autotune and not args.single_pass:
            t0 = time.perf_counter()
            plan, ms, _ = m.autotune(tune["cache"], iters=4)
            if tune["plan"] is None:
                tune.update(plan=plan, ms=round(ms, 4), tuning_s=round(time.perf_counter() - t0, 2))
        if store == "bf16" and args.plan:
            m.set_plan(**parse_plan(args.plan))
            if tune["plan"] is None or tune.get("override") is None:
                tune.update(plan=m.plan(), override=args.plan)
        return m

    results = {}
    stores = [args.store] if args.store != "both" else ["bf16", "f32"]
    clocks = None
    for store in stores:
        m = make(store)
        lay = m.layout()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        with ClockSampler(dev) as cs:
            ms = time_fit(m, stream, args.steps, args.warmup)
        ms = max_over_ranks(ms, world)
        ll = m.ll()
        results[store] = {"ms_total": ms, "ms_per_step": ms / args.steps, "layout": lay,
                          "ll_last": float(ll[-1]), "ll_monotone": bool(np.all(np.diff(ll) >= -1e-6 * np.abs(ll[1:])))}
        if store == stores[0]:
            clocks = cs.summary()
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
    roofline = None
    # dominant kernel = the streaming pass with the largest time per step
    streaming = {"estep_tc": e_bytes, "mstep_tc": m_bytes, "fpass_tc": f_bytes} if head == "bf16" else \
        {"estep_simt": e_bytes, "mstep_simt": m_bytes}
    present = [(ks[n]["ms"], n) for n in streaming if n in ks]
    if present:
        _, name = max(present)
        t = ks[name]["ms"] / ks[name]["launches"]
        b = streaming[name]
        if head == "f32":
            b = b / len(vox)  # per launch (one launch per subject)
        achieved = b / (t * 1e-3) / 1e9
        traffic, tsrc = profiled_traffic(name, args.config, int(sum(vox))) if head == "bf16" else (None, None)
        roofline = {"kernel": name, "bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"],
                    "unit": "GB/s", "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": traffic,
                    "traffic_source": tsrc, "peak_source": peaks["source"] + " (burst copy)",
                    "bytes_per_launch": b, "ms_per_launch": t}
    iter_bytes = f_bytes if single else e_bytes + m_bytes
    kernels_per_step = sum(v["launches"] for v in ks.values()) / args.steps
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": head,
        "data": "synthetic planted (Sec. II-A model), generated on device",
        "config": {"workload": spec.name, "N": len(vox), "T": T, "k": k, "voxels_total": int(sum(vox)),
                   "store": head, "l2": "inputs larger than L2 (resident X^ %.2f GB > 129 MB)" %
                   (results[head]["layout"]["xhat_bytes"] / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "graph": True, "single_pass": single,
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
        "kernels_ms_per_step": {n: round(v["ms"] / args.steps, 4) for n, v in ks.items()},
        "kernels_note": "CUDA-event time per step of each kernel kind on the stream it runs on (SRM_PROFILE run "
                        "of the same steps); kinds on the second and third streams (sigma, eig, mtail, refine, rho, "
                        "polar, phi where they run beside a streaming pass) include time spent waiting for SMs",
        "ll_monotone": results[head]["ll_monotone"],
    }
    if "f32" in results and head != "f32":
        r = results["f32"]
        out["fp32_plain"] = {"value": round(world * 1000.0 / r["ms_per_step"], 3), "ms_per_step":
                             round(r["ms_per_step"], 4),
                             "kernels_ms_per_step": {n: round(v["ms"] / args.steps, 4) for n, v in
                                                     r["kernels"].items()}}
    in_bytes = sum(x.numel() * x.element_size() for x in d["X"])
    if not args.no_e2e and in_bytes <= 16e9:
        out["e2e"] = run_e2e(args, d, spec, vox, stream, world,
                             None if args.no_autotune or args.single_pass else tune["cache"])
    elif not args.no_e2e:
        out["e2e"] = {"value": None, "unit": UNIT, "skipped": "input of %.0f GB too large to pin on the host for "
                      "the end-to-end job" % (in_bytes / 1e9)}
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(spec, vox, budget_s=args.cpu_budget)
    return out


def run_e2e(args, d, spec, vox, stream, world, tune_cache=None):
    """One whole user job through the public API with host buffers: pinned
    host X -> srm_init (host input: H2D copy + centring) -> srm_fit(n_iter)
    -> parameters, E[S] and the log-likelihood back to the host.
    Value = EM iterations / job time."""
    import torch

    import paper_1608_04647_gb300 as srm
    Xh = [x.to("cpu").pin_memory() for x in d["X"]]
    n_iter = spec.n_iter
    h2d = sum(x.numel() * x.element_size() for x in Xh)
    times = []
    for rep in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        store = args.store if args.store != "both" else "bf16"
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
    d2h = S.numel() * 4 + rho2.nbytes + sig.nbytes + ll.nbytes
    best = min(times)
    return {"value": round(world * n_iter / best, 3), "unit": UNIT, "job_s": round(best, 4),
            "iterations_per_job": n_iter, "h2d_bytes_per_step": int(h2d / n_iter),
            "d2h_bytes_per_step": int(d2h / n_iter),
            "note": "step = one EM iteration of a %d-iteration job; host->device copy of X from pinned memory, "
                    "centring, fit and result read-back inside the timed region" % n_iter}


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        return max((i.get("num_threads", 0) for i in info), default=None)
    except Exception:
        return None


def oracle_sample(spec, vox, max_elems=4e7, max_subjects=4):
    """A bounded sample of the workload for the FP64 oracle: the first
    subjects, each cut to at most max_elems / T voxel rows, at most
    max_subjects of them, drawn from the same planted generator."""
    import synth
    rows = max(spec.k + 1, int(max_elems // spec.T))
    sub = [min(int(v), rows) for v in vox[:max_subjects]]
    while len(sub) > 1 and sum(sub) * spec.T > max_elems:
        sub.pop()
    dd = synth.planted_dataset(spec, voxel_counts=sub, dtype=np.float64)
    return sub, dd


def cpu_baseline(spec, vox, budget_s=20.0):
    """The FP64 oracle (as it stands) on the host cores: EM iterations over a
    bounded sample of the workload, time scaled to the whole workload by
    voxel count (the oracle's per-iteration cost is linear in the voxels)."""
    import oracle
    sub, dd = oracle_sample(spec, vox)
    Xh = [oracle.center(x)[0] for x in dd["X"]]
    del dd["X"]
    t0 = time.perf_counter()
    iters = 0
    while True:
        oracle.fit(Xh, dd["W0"], 1, centered=True)
        iters += 1
        if time.perf_counter() - t0 > budget_s or iters >= 5:
            break
    dt = (time.perf_counter() - t0) / iters
    scale = float(sum(vox)) / float(sum(sub))
    per_iter_full = dt * scale
    return {"value": round(1.0 / per_iter_full, 6), "unit": UNIT, "cores": os.cpu_count(),
            "blas_threads": blas_threads(), "kind": "oracle",
            "sample": "%d subject(s) of %d, %d voxels in all (of %d), T = %d, %d EM iteration(s) of the FP64 NumPy "
                      "oracle; time scaled by total voxels (x%.1f)" % (len(sub), len(vox), int(sum(sub)),
                                                                      int(sum(vox)), spec.T, iters, scale)}


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle as it stands, on the host cores, on a
    bounded sample of the same workload; each step one EM iteration over the
    sample, time scaled to the whole workload by voxel count."""
    import oracle
    spec, vox = workload(args.config, rank, args.subjects)
    sub, dd = oracle_sample(spec, vox, max_elems=2e7, max_subjects=2)
    Xh = [oracle.center(x)[0] for x in dd["X"]]
    for _ in range(args.warmup):
        oracle.fit(Xh, dd["W0"], 1, centered=True)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.fit(Xh, dd["W0"], 1, centered=True)
    dt = (time.perf_counter() - t0) / args.steps
    scale = float(sum(vox)) / float(sum(sub))
    per_iter = dt * scale
    value = 1.0 / per_iter
    sample = ("%d subject(s) of %d, %d voxels in all (of %d) per step, one FP64 oracle EM iteration, time scaled by "
              "total voxels (x%.1f)" % (len(sub), len(vox), int(sum(sub)), int(sum(vox)), scale))
    return {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(per_iter * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic planted (Sec. II-A model)",
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
        m = srm.SRM(d["X"], d["W0"], k, store="bf16", graph=True, max_iter=args.warmup + args.steps + 8,
                    stream=stream)
        plan, _, _ = m.autotune(None, iters=4)
        ms = time_fit(m, stream, args.steps, args.warmup) / args.steps
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
    traffic, tsrc = htfa_profiled_traffic("htfa_residual", spec.name)
    res = {
        "metric": HTFA_METRIC, "value": round(1000.0 / ms_step, 3), "unit": HTFA_UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded HTFA-shaped inputs: grid voxels, centers, widths, weights, noise)",
        "config": {"workload": spec.name, "n_subjects": n, "T": T, "V": V, "K": K,
                   "l2": "inputs larger than L2 (X %.0f MB + F %.0f MB > 129 MB)" % (n * T * V * 4 / 1e6,
                                                                                  n * K * V * 4 / 1e6)},
        "timing_note": "per-call CUDA-event times over the first %d steps of a second run on the same stream" % n_ev,
        "roofline": {"kernel": "htfa_residual (tile + sum launches)", "bound": "alu", "achieved": round(achieved, 2),
                     "peak": round(peak, 2), "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                     "traffic": traffic, "traffic_source": tsrc, "algorithmic_bytes_per_launch": r_bytes,
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock",
                     "flops_per_launch": flops, "ms_per_launch": round(t_r, 5),
                     "hbm_gbs": round(r_bytes / (t_r * 1e-3) / 1e9, 1)},
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
    ap.add_argument("--config", type=int, default=1)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--store", choices=["bf16", "f32", "both"], default="both")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--k-sweep", action="store_true", help="throughput against k (extra lines, not the bench line)")
    ap.add_argument("--single-pass", action="store_true", help="force the single-pass form (SRM_SINGLE_PASS), "
                    "no autotuning")
    ap.add_argument("--no-autotune", action="store_true", help="run the library's default launch plan")
    ap.add_argument("--tune-cache", default=None, help="plan cache file kept across runs (default: a fresh one)")
    ap.add_argument("--plan", default="", help="launch-plan fields set after tuning, e.g. 'single_pass=0' "
                    "(srm_set_plan; for profiling one form)")
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
    if world > 1:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        torch.distributed.init_process_group("nccl")
    out = run_ours(args, rank, world)
    if world > 1:
        import torch
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
