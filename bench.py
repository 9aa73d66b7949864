"""Benchmark of quantization-aware interpolation on GB300 (one JSON line).

Workload: a 512^3 float32 Gaussian random field with P(k) ~ k^-11/3 (seeded
FFT synthesis, normalised to [0, 1]), pre-quantized with eb = 1e-3 x range
into int32 indices. One step = one qai_mitigate call over the whole field:
boundary detection, both exact EDTs, sign propagation and the fused IDW
compensation (Algorithm 4), inputs resident in HBM. The fields (512 MiB in,
512 MiB out, 1.5 GiB of intermediates) are far larger than the 129 MB L2, so
no flush is needed between steps.

metric  mitigation GB/s of the fp32 field = 4 N bytes / step time, summed
        over ranks (replicas only: each rank mitigates its own field)
e2e     the same through qai_mitigate_host: pinned host q in, host D'' out,
        both copies inside the timed region
roofline  the dominant kernel's algorithmic bytes / its CUDA-event time vs the
        measured HBM copy bandwidth
cpu_baseline  the FP64 C oracle on the host cores, on a 128 x 512 x 512 slab

``--impl reference`` times the oracle itself on that slab as the reference arm.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SHAPE = (512, 512, 512)
REL_EB = 1e-3
SEED = 2
SAMPLE_Z = 128                      # oracle sample: the first 128 z-planes
METRIC = "mitigation GB/s of fp32 field (detect+EDT+interp) vs HBM roofline; PSNR gain"
WORKLOAD = "grf512_k-11/3_eb1e-3"


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


def hbm_peak():
    p = peaks().get("hbm_gbs")
    return (float(p), "measured") if p else (6800.0, "fallback")


def src_hash(files):
    """Hash of the given repository files (paths relative to the root)."""
    h = hashlib.sha256()
    for f in files:
        h.update(f.encode() + b"\0")
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or
    None when a source file that builds the captured kernels (listed in the
    record) changed since it was captured."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        rec = json.load(open(path))
        if rec.get("src_hash") != src_hash(rec["sources"]):
            return None
    except (OSError, KeyError, ValueError):
        return None
    k = rec.get("kernels", {}).get(kernel)
    return None if k is None else k.get("dram_bytes_per_launch")


class Clocks:
    """nvidia-smi sampler (50 ms period) of SM clock and throttle reasons."""
    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.perf_counter(), [c.strip() for c in line.split(",")]))

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0, t1):
        """Median SM clock and the throttle reasons seen between t0 and t1."""
        import statistics
        sm, mx, reasons = [], [], set()
        for t, r in self.rows:
            if not t0 <= t <= t1:
                continue
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(self.NAMES, r[2:6]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "window": "1 s soak of the same step right before the timed region, and the timed region"}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def synth_quantize(x, eb):
    from paper_2602_20097_gb300 import synth
    return synth.quantize(x, eb)


def make_field(device, seed, shape=SHAPE):
    from paper_2602_20097_gb300 import synth
    x = synth.grf(shape, slope=11.0 / 3.0, seed=seed, device=device)
    eb = REL_EB * synth.value_range(x)
    q = synth.quantize(x, eb)
    return x, q, eb


def quality_gain(x, q, eb, out):
    """PSNR (Eq. 4) and SSIM (Eq. 3, window 7, stride 2) of D' = 2 q eb and of
    D'' against x, from the library's GPU quality kernels (untimed)."""
    from paper_2602_20097_gb300 import qai
    xf = x.float().contiguous()
    dp = qai.dequantize(q, eb)
    a = qai.quality(xf, dp)
    b = qai.quality(xf, out.contiguous())
    return {"psnr_dprime_db": a["psnr"], "psnr_mitigated_db": b["psnr"], "psnr_gain_db": b["psnr"] - a["psnr"],
            "ssim_dprime": a["ssim"], "ssim_mitigated": b["ssim"], "ssim_gain": b["ssim"] - a["ssim"],
            "max_err_over_eps": float((x.double() - out.double()).abs().max()) / eb}


def time_oracle(q_sample, eb, min_s=10.0, max_s=30.0):
    import oracle
    oracle.build()
    runs, t0 = 0, time.perf_counter()
    while True:
        oracle.mitigate(q_sample, eb, debug=False)
        runs += 1
        el = time.perf_counter() - t0
        if el >= min_s or el * (runs + 1) / runs > max_s:
            break
    return runs, el


def run_reference(args):
    """The reference arm: the FP64 oracle timed on the host cores."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    from paper_2602_20097_gb300 import synth
    oracle.build()
    x = synth.grf((SAMPLE_Z,) + SHAPE[1:], slope=11.0 / 3.0, seed=SEED).numpy()
    eb = REL_EB * synth.value_range(x)
    q = synth.quantize(x, eb)
    for _ in range(args.warmup):
        oracle.mitigate(q, eb, debug=False)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.mitigate(q, eb, debug=False)
    el = time.perf_counter() - t0
    gbs = q.size * 4 * args.steps / el / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "shape": list(SHAPE), "rel_eb": REL_EB,
                   "sample": f"{SAMPLE_Z}x512x512 slab of the same synthesis"},
        "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": oracle.threads(), "kind": "oracle",
                         "sample": f"{SAMPLE_Z}x512x512 GRF slab, {args.steps} runs"},
        "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_e2e(q, eb, dev, stream, steps, barrier, world, ws, warmup=3):
    """Same metric through qai_mitigate_host: H2D of q and D2H of D'' timed."""
    import torch
    from paper_2602_20097_gb300 import qai, replicas
    qh = q.cpu().pin_memory()
    oh = torch.empty(tuple(q.shape), dtype=torch.float32).pin_memory()
    del ws
    wsh = qai.alloc_workspace(qai.workspace_size_host(tuple(q.shape)), dev)
    for _ in range(max(3, warmup)):
        qai.mitigate_host(qh, eb, out_host=oh, workspace=wsh)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        qai.mitigate_host(qh, eb, out_host=oh, workspace=wsh)
    e1.record(stream)
    barrier()
    ms_max = replicas.max_over_ranks(e0.elapsed_time(e1) / steps, device=dev)
    return replicas.whole_job_gbs(q.numel() * 4, world, ms_max)


def run_qai(args):
    import torch
    import torch.distributed as dist
    from paper_2602_20097_gb300 import qai, replicas

    world, rank, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    dev = torch.device("cuda", torch.cuda.current_device())

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # replicas: each rank mitigates its own field (seed differs per rank)
    shape = tuple(int(v) for v in args.shape.split(",")) if args.shape else SHAPE
    x, q, eb = make_field(dev, SEED + rank, shape)
    N = q.numel()
    out = torch.empty_like(q, dtype=torch.float32)
    ws = qai.alloc_workspace(qai.workspace_size(tuple(q.shape)), dev)
    stream = torch.cuda.current_stream()
    warm = max(3, args.warmup)
    for _ in range(warm):
        qai.mitigate(q, eb, out=out, workspace=ws)
    # untimed pass with every kernel bracketed by events: the per-kernel
    # breakdown and the dominant kernel; the timed region below brackets only
    # that kernel, so the other launches run back to back as in real use
    qai.profile_read()
    qai.profile_select(None)
    qai.profile_enable(True)
    for _ in range(max(3, min(args.steps, 10))):
        qai.mitigate(q, eb, out=out, workspace=ws)
    torch.cuda.synchronize()
    kstats = qai.profile_read()
    dom_name = max(kstats.items(), key=lambda kv: kv[1][1])[0] if kstats else None
    qai.profile_select(dom_name)
    barrier()
    n0 = qai.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        time.sleep(0.3)                          # let the sampler start
        tc0 = time.perf_counter()
        while time.perf_counter() - tc0 < 1.0:   # soak: same step, untimed
            qai.mitigate(q, eb, out=out, workspace=ws)
            torch.cuda.synchronize()
        qai.profile_read()
        n0 = qai.launch_count()
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            qai.mitigate(q, eb, out=out, workspace=ws)
        ev1.record(stream)
        barrier()
        tc1 = time.perf_counter()
        time.sleep(0.1)
    launches = qai.launch_count() - n0
    dstats = qai.profile_read()
    qai.profile_enable(False)
    qai.profile_select(None)
    ms = ev0.elapsed_time(ev1) / args.steps
    ms_max = replicas.max_over_ranks(ms, device=dev)
    value = replicas.whole_job_gbs(N * 4, world, ms_max)

    route = qai.route_counts(ws, tuple(q.shape))  # how the second EDT went (signed-point route)

    # end to end from pinned host memory through the C ABI (copies timed)
    if args.no_e2e:
        e2e_value = None
    else:
        e2e_value = run_e2e(q, eb, dev, stream, args.steps, barrier, world, ws, args.warmup)
        ws = None

    # quality (untimed): PSNR and SSIM gain and max error / eps of this field
    qual = quality_gain(x, q, eb, out)

    # the same field at the configuration's second bound, eb = 1e-2 x range
    eb2 = 1e-2 * (float(x.max()) - float(x.min()))
    q2 = synth_quantize(x, eb2)
    ws2 = qai.alloc_workspace(qai.workspace_size(tuple(q2.shape)), dev)
    out2 = torch.empty_like(q2, dtype=torch.float32)
    ms2 = _time_steps(lambda: qai.mitigate(q2, eb2, out=out2, workspace=ws2), args.steps)
    second = {"rel_eb": 1e-2, "ms_per_step": ms2, "value": N * 4 / (ms2 * 1e-3) / 1e9,
              "signed_route": qai.route_counts(ws2, tuple(q2.shape)),
              **quality_gain(x, q2, eb2, out2)}
    del q2, ws2, out2
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    peak, peak_src = hbm_peak()
    dom = (dom_name, dstats[dom_name]) if dom_name in dstats else None
    roof = None
    if dom:
        name, (nl, tot_ms, algo_bytes) = dom
        achieved = algo_bytes / (tot_ms * 1e-3) / 1e9
        traffic = ncu_traffic(name)
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": name,
                "peak_source": f"{peak_src} hbm_gbs",
                "algo_bytes_per_launch": algo_bytes / nl,
                "kernel_ms_per_launch": tot_ms / nl}
    kernels = {k: {"launches": v[0], "ms_per_launch": v[1] / v[0],
                   "algo_gbs": v[2] / (v[1] * 1e-3) / 1e9,
                   "share": v[1] / sum(s[1] for s in kstats.values())} for k, v in kstats.items()}
    kernels_note = ("every kernel bracketed by CUDA events in an untimed pass right before the timed "
                    "region; the roofline kernel is timed inside the timed region, alone")

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        qs = q[:min(SAMPLE_Z, q.shape[0])].cpu().numpy()
        import oracle
        runs, el = time_oracle(qs, eb)
        cores = oracle.threads()
        cpu = {"value": qs.size * 4 * runs / el / 1e9, "unit": "GB/s", "cores": cores,
               "kind": "oracle",
               "sample": f"first {SAMPLE_Z} z-planes of the bench field ({SAMPLE_Z}x512x512), {runs} runs, {el:.1f} s"}
        # the same oracle on one thread, on a quarter of that slab
        q1 = qs[:max(1, qs.shape[0] // 4)]
        oracle.set_threads(1)
        try:
            r1, el1 = time_oracle(q1, eb, min_s=2.0, max_s=15.0)
        finally:
            oracle.set_threads(cores)
        cpu["single_thread"] = {"value": q1.size * 4 * r1 / el1 / 1e9, "unit": "GB/s", "cores": 1,
                                "sample": f"first {q1.shape[0]} z-planes of the bench field, {r1} runs, {el1:.1f} s"}

    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": warm, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32+fp32", "data": "synthetic",
        "config": {"workload": WORKLOAD if shape == SHAPE else f"grf{'x'.join(map(str, shape))}_k-11/3_eb1e-3",
                   "shape": list(shape), "rel_eb": REL_EB, "eb": eb,
                   "parallelism": f"replicas x{world}", "l2": "inputs > L2 (1 GiB per step), no flush"},
        "roofline": roof,
        "algo_roofline_frac": (8.0 * N / (ms_max * 1e-3) / 1e9) / peak,
        "e2e": None if e2e_value is None else
        {"value": e2e_value, "unit": "GB/s", "h2d_bytes_per_step": 4 * N, "d2h_bytes_per_step": 4 * N},
        "gpu_launches": launches,
        "clocks": clk.summary(tc0, tc1),
        "cpu_baseline": cpu,
        "quality": qual,
        "signed_route": route,
        "second_bound": second,
        "kernels": kernels,
        "kernels_note": kernels_note,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def _time_steps(fn, steps, warmup=3):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _kernel_shares(fn):
    """Per-kernel device time of one call of ``fn`` (CUDA events around each
    launch, untimed run)."""
    from paper_2602_20097_gb300 import qai
    qai.profile_read()
    qai.profile_enable(True)
    fn()
    stats = qai.profile_read()
    qai.profile_enable(False)
    return {k: round(v[1], 4) for k, v in sorted(stats.items(), key=lambda kv: -kv[1][1]) if v[1] > 0}


def run_aniso(args):
    """The anisotropic shapes with a tanh front, at eb 1e-3 and 1e-2 of the
    value range (one JSON line per shape and bound): throughput, quality gain,
    the routes the EDTs took and the per-kernel times."""
    import torch
    from paper_2602_20097_gb300 import qai, synth
    only = tuple(int(v) for v in args.shape.split(",")) if args.shape else None
    rels = tuple(float(v) for v in args.rel_eb.split(",")) if args.rel_eb else (1e-3, 1e-2)
    for shape, seed in (((1800, 3600), 6), ((256, 384, 384), 4), ((100, 500, 500), 3), ((98, 1200, 1200), 5)):
        if only is not None and shape != only:
            continue
        x = synth.grf_front(shape, seed=seed, device="cuda")
        for rel in rels:
            eb = rel * synth.value_range(x)
            q = synth.quantize(x, eb)
            ws = qai.alloc_workspace(qai.workspace_size(tuple(q.shape)))
            out = torch.empty_like(q, dtype=torch.float32)
            ms = _time_steps(lambda: qai.mitigate(q, eb, out=out, workspace=ws), args.steps)
            routes = qai.route_counts(ws, tuple(q.shape))
            kernels = _kernel_shares(lambda: qai.mitigate(q, eb, out=out, workspace=ws))
            print(json.dumps({"workload": "front_" + "x".join(map(str, shape)) + f"_eb{rel:.0e}".replace("e-0", "e-"),
                              "value": q.numel() * 4 / (ms * 1e-3) / 1e9, "unit": "GB/s", "ms_per_step": ms,
                              **quality_gain(x, q, eb, out), "routes": routes,
                              "kernels_ms": kernels}), flush=True)
            del ws, out, q


def run_batch96(args):
    """96 uneven 2-D/3-D fields: one batched call (persistent grouped launches
    replayed from a cached CUDA graph, autotuned queue order, work-item size
    and column tiles) vs 96 sequential plain calls on one stream."""
    import torch
    from paper_2602_20097_gb300 import qai, synth
    specs = synth.batch_specs()
    qs, ebs = [], []
    for sp in specs:
        x = synth.grf(sp["shape"], slope=sp["slope"], seed=sp["seed"], device="cuda")
        eb = sp["rel_eb"] * synth.value_range(x)
        qs.append(synth.quantize(x, eb))
        ebs.append(eb)
    npts = sum(q.numel() for q in qs)
    batch = qai.Batch(qs, ebs)
    choice = qai.autotune_batched(batch)
    n0 = qai.launch_count()
    ms_b = _time_steps(lambda: qai.mitigate_batched(batch), args.steps)
    launches = (qai.launch_count() - n0) // (args.steps + 3)
    wss = [qai.alloc_workspace(qai.workspace_size(tuple(q.shape))) for q in qs]
    outs = [torch.empty_like(q, dtype=torch.float32) for q in qs]

    def seq():
        for q, eb, o, w in zip(qs, ebs, outs, wss):
            qai.mitigate(q, eb, out=o, workspace=w)
    n1 = qai.launch_count()
    ms_s = _time_steps(seq, args.steps)
    seq_launches = (qai.launch_count() - n1) // (args.steps + 3)
    same = all(torch.equal(a, b) for a, b in zip(batch.outs, outs))
    print(json.dumps({"workload": "batch96_mixed", "fields": len(qs), "points": npts,
                      "value": npts * 4 / (ms_b * 1e-3) / 1e9, "unit": "GB/s", "ms_per_step": ms_b,
                      "sequential": {"value": npts * 4 / (ms_s * 1e-3) / 1e9, "ms_per_step": ms_s,
                                     "launches": seq_launches},
                      "batched_kernels_per_graph": launches, "identical_to_sequential": same,
                      "autotuned": {str(k): v for k, v in choice.items()}}), flush=True)


def run_adjoint1024(args):
    """Forward + adjoint on a 1024^3 k^-11/3 GRF (eb 1e-4): stored vs recompute.
    One workspace serves the forward and, in recompute mode, the backward."""
    import torch
    from paper_2602_20097_gb300 import qai, synth
    shape = (1024, 1024, 1024)
    x = synth.grf(shape, slope=11.0 / 3.0, seed=7, device="cuda")
    eb = 1e-4 * synth.value_range(x)
    q = synth.quantize(x, eb)
    N = q.numel()
    ws = qai.alloc_workspace(max(qai.workspace_size(shape), qai.workspace_size_backward(shape, True)))
    out = torch.empty(shape, dtype=torch.float32, device="cuda")
    ms_fwd = _time_steps(lambda: qai.mitigate(q, eb, out=out, workspace=ws), args.steps)
    qai.profile_read()
    qai.profile_enable(True)
    qai.mitigate(q, eb, out=out, workspace=ws)
    torch.cuda.synchronize()
    fwd_kernels = {k: v[1] / v[0] for k, v in qai.profile_read().items()}
    qai.profile_enable(False)
    g = (out.double() - x.double()).float()  # dL/dD'' of 0.5 * sum (D'' - x)^2
    del x
    res = {}
    for mode in ("stored", "recompute"):
        torch.cuda.synchronize()
        torch.cuda.reset_peak_memory_stats()
        base = torch.cuda.memory_allocated()
        saved = qai.alloc_workspace(qai.saved_size(shape)) if mode == "stored" else None
        bws = ws if mode == "recompute" else qai.alloc_workspace(qai.workspace_size_backward(shape, False))

        def fwd():
            if mode == "stored":
                qai.mitigate_save(q, eb, saved=saved, workspace=ws, out=out)
            else:
                qai.mitigate(q, eb, out=out, workspace=ws)

        def bwd():
            return qai.mitigate_backward(q, eb, g, saved=saved, workspace=bws, want_grad_dprime=False)

        def step():
            fwd()
            return bwd()
        ms = _time_steps(step, args.steps)
        fwd()
        ms_b = _time_steps(bwd, args.steps)
        qai.profile_read()
        qai.profile_enable(True)
        bwd()
        torch.cuda.synchronize()
        kst = qai.profile_read()
        qai.profile_enable(False)
        _, gp = step()
        torch.cuda.synchronize()
        res[mode] = {"ms_fwd_bwd": ms, "ms_bwd": ms_b, "extra_bytes": torch.cuda.max_memory_allocated() - base,
                     "bwd_workspace_bytes": qai.workspace_size_backward(shape, mode == "recompute"),
                     "grad_eta": float(gp[0]), "grad_p": float(gp[1]),
                     "bwd_kernels_ms": {k: v[1] / v[0] for k, v in kst.items()}}
        del saved, bws
    print(json.dumps({"workload": "adjoint_grf1024_eb1e-4", "points": N, "ms_forward": ms_fwd,
                      "value": N * 4 / (ms_fwd * 1e-3) / 1e9, "unit": "GB/s",
                      "fwd_kernels_ms": fwd_kernels, "workspace_bytes": ws.numel(), **res}), flush=True)


def run_quality512(args):
    """SSIM + PSNR kernels on the 512^3 GRF against its mitigated field (eb 1e-3):
    two kernels, each reading both fields once (16 bytes per point)."""
    import torch
    from paper_2602_20097_gb300 import qai, synth
    shape = tuple(int(v) for v in args.shape.split(",")) if args.shape else (512, 512, 512)
    x = synth.grf(shape, slope=11.0 / 3.0, seed=2, device="cuda").float().contiguous()
    eb = REL_EB * synth.value_range(x)
    q = synth.quantize(x, eb)
    y = qai.mitigate(q, eb)
    N = x.numel()
    ws = qai.alloc_workspace(qai.workspace_size_quality(shape))
    res = torch.zeros(6, dtype=torch.float64, device="cuda")
    lib = qai.load()
    dims = qai._dims(shape)

    def step():
        qai._check(lib.qai_quality(x.data_ptr(), y.data_ptr(), len(shape), dims, 7, 2, res.data_ptr(), None,
                                   ws.data_ptr(), ws.numel(), qai._stream()))
    ms = _time_steps(step, args.steps)
    qai.profile_read()
    qai.profile_enable(True)
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    kstats = qai.profile_read()
    qai.profile_enable(False)
    peak, peak_src = hbm_peak()
    kern = {k: {"launches": v[0], "ms": v[1] / v[0], "gbs": v[2] / (v[1] * 1e-3) / 1e9,
                "frac": v[2] / (v[1] * 1e-3) / 1e9 / peak} for k, v in kstats.items()}
    r = qai.quality(x, y)
    print(json.dumps({"workload": "quality_grf" + "x".join(map(str, shape)), "points": N, "ms_per_call": ms,
                      "value": N * 16 / (ms * 1e-3) / 1e9, "unit": "GB/s (16 B/pt read)",
                      "frac_of_hbm": N * 16 / (ms * 1e-3) / 1e9 / peak, "peak_gbs": peak, "peak_src": peak_src,
                      "kernels": kern, "ssim": r["ssim"], "psnr_db": r["psnr"], "windows": r["windows"]}),
          flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["qai", "reference"], default="qai")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--shape", default="", help="Z,Y,X override (profiling of smaller cases); with --workload "
                    "aniso: run only the front of this shape")
    ap.add_argument("--rel-eb", default="", help="with --workload aniso: the bounds (x value range), comma separated")
    ap.add_argument("--workload", default="grf512", choices=["grf512", "aniso", "batch96", "adjoint1024", "quality512"],
                    help="grf512: the headline line; the others print their own lines")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "grf512":
        sys.path.insert(0, ROOT)
        return {"aniso": run_aniso, "batch96": run_batch96, "adjoint1024": run_adjoint1024,
                "quality512": run_quality512}[args.workload](args)
    return run_qai(args)


if __name__ == "__main__":
    sys.exit(main())
