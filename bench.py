"""Benchmark of the coarsened Newton-step solve on GB300.

One step = agipc_aggregate + agipc_assemble_coarse + agipc_pcg +
agipc_prolongate on the 64-box domino workload (145,600 vertices, 663,552
tets, 200k barrier stencils, FP64, PCG to 1e-6 relative residual), inputs
resident in HBM.  Prints one JSON line (see the keys below).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun, one independent replica per GPU (the single-mesh
path does not shard); value = solves of all ranks / max-over-ranks time.
--impl reference times the CPU FP64 oracle (the only reference this method
has) on the same workload and metric.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Newton-step solves/s (coarsen+assemble+PCG+prolong) vs fine PCG; % HBM peak"
UNIT = "solves/s"
TOL = 1e-6
WORKLOAD = "domino_8x8: 64 StVK boxes of 6x12x24 Kuhn-split hexes (145,600 vertices, 663,552 tets), " \
           "200,000 PT/EE barrier stencils, 40-90% collapsible edges per box, FP64, PCG to 1e-6"
KERNELS_PER_STEP = {"aggregate": 9, "assemble_coarse": 13, "pcg": 1, "prolongate": 1}
# FP64 peak of a GB300 from its unit counts and clock: 152 SMs x 2 FP64 FMA per
# clock x 2 flops x 2.07 GHz (a probe of dependent-free FMA streams reaches 1.20).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def _dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(values, ws: int, device):
    """Element-wise maximum of per-rank floats over all ranks (the job's
    time is its slowest replica's); the identity on one rank."""
    if ws == 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t]


def replica_throughput(ws: int, units_per_rank: int, seconds: float) -> float:
    """Whole-job throughput of ws independent replicas that each processed
    units_per_rank units, timed by the slowest one."""
    return ws * units_per_rank / seconds


def shard_instances(counts, ws: int, rank: int):
    """Contiguous instance range [a, b) of rank `rank` when the batched form's
    instances are split over ws GPUs with no exchange (instances are
    independent problems): boundary k is the first instance whose vertex
    prefix sum reaches k / ws of the total, so every rank holds about the
    same number of vertices and the ranges tile 0 .. len(counts)."""
    counts = np.asarray(counts, dtype=np.int64)
    n = counts.size
    if ws <= 1:
        return 0, n
    pre = np.concatenate([[0], np.cumsum(counts)])
    total = pre[-1]
    bounds = [0] + [int(np.searchsorted(pre, k * total / ws, side="left")) for k in range(1, ws)] + [n]
    bounds = np.maximum.accumulate(np.minimum(bounds, n))
    return int(bounds[rank]), int(bounds[rank + 1])


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", "agipc_clocks_%d_%d.csv" % (os.getpid(), gpu_index))

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sms, maxes, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                maxes.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sms)) if sms else None, "sm_max_mhz": max(maxes) if maxes else None,
                "samples": len(sms), "reasons": sorted(reasons)}


TRAFFIC_SOURCES = ("paper_2605_04773_gb300/csrc/pcg.cu", "paper_2605_04773_gb300/csrc/agipc_common.cuh",
                   "paper_2605_04773_gb300/csrc/pcg_slices.cuh")


def kernel_source_hash(files=TRAFFIC_SOURCES) -> str:
    """sha256 of the kernel sources with comments and whitespace removed, so
    that only a change of the code itself invalidates a stored capture."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in files:
        text = open(os.path.join(ROOT, f)).read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()


def _traffic_record():
    """DRAM bytes per launch of pcg_kernel from the committed ncu capture,
    only while the kernel's code is the one that was captured."""
    path = os.path.join(ROOT, "profiles", "pcg_kernel_domino_8x8_coarse.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path))
    if kernel_source_hash() != rec.get("source_sha256"):
        return None
    return rec["dram_bytes_read"] + rec["dram_bytes_write"]


def pcg_flops_per_iter(nnzb: int, n: int) -> int:
    """FP64 flops of one Chronopoulos-Gear PCG iteration: 9 FMAs per 3x3 block
    (18 flops) and, per row, the p, s, x, r updates (4 x 3 FMAs), the 3x3
    preconditioner (15 flops) and the gamma and rho dot products (2 x 3 FMAs)."""
    return 18 * nnzb + (24 + 15 + 12) * n


def pcg_bytes_per_iter(nnzb: int, n: int) -> int:
    """Algorithmic bytes of one FP64 PCG iteration on a 3x3 BSR matrix, the
    byte model the roofline is quoted on: 76 B per block (9 FP64 values and
    a column index) and 200 B per row (the gathered vector, the SpMV output
    and the row-local vectors with fused updates)."""
    return 76 * nnzb + 200 * n


def pcg_mixed_bytes_per_iter(nnzb: int, n: int, refine_every: int = 20) -> float:
    """The same for the precision form: 40 B per block (9 FP32 values and a
    column index) and 240 B per row (FP32 u, w, p, s, FP64 x, r, FP32
    preconditioner), plus the FP64 residual replacement every refine_every
    iterations (76 B per block and 96 B per row)."""
    return 40 * nnzb + 240 * n + (76 * nnzb + 96 * n) / refine_every


def fp64_probe():
    """Build and run fp64_unit_probe.cu (nvcc, sm_103a): the measured FP64
    FMA rate of one SM, returned as parsed JSON."""
    here = os.path.join(ROOT, "paper_2605_04773_gb300")
    exe = os.path.join(here, "_build", "fp64_unit_probe")
    os.makedirs(os.path.dirname(exe), exist_ok=True)
    nvcc = "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                    os.path.join(here, "fp64_unit_probe.cu")], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return json.loads(out.strip().splitlines()[-1])


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2605_04773_gb300 import agipc, build, scenes

    ws, rank, local = _dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    build.build()
    sc = scenes.domino_grid(seed=1002)
    ds = agipc.DeviceScene(sc, dev)
    stream = torch.cuda.current_stream(dev)
    ctx = ds.context()
    step = agipc.CoarsenedStep(ctx, ds, tol=TOL)
    l2 = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def flush():
        l2.fill_(1.0)

    def one(ev=None):
        step.aggregate()
        step.assemble()
        if ev is not None:
            ev[0].record(stream)
        step.solve()
        if ev is not None:
            ev[1].record(stream)
        step.prolongate()

    for _ in range(max(3, args.warmup)):
        one()
    rc = ctx.status()
    if rc != agipc.OK:
        raise RuntimeError("warm-up step failed: %s" % agipc.status_string(rc))

    # ---- device-timed steps (inputs resident; L2 flushed between steps)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    pcg_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(dev.index if dev.index is not None else 0)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    sampler.start()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush()
        starts[k].record(stream)
        one(pcg_ev[k])
        ends[k].record(stream)
    torch.cuda.synchronize(dev)
    t_wall = time.perf_counter() - t_wall
    clocks = sampler.stop()
    rc = ctx.status()
    if rc != agipc.OK:
        raise RuntimeError("timed step failed: %s" % agipc.status_string(rc))
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    pcg_ms = [a.elapsed_time(b) for a, b in pcg_ev]
    total_s = sum(step_ms) / 1e3
    res = step.host()

    # ---- fine PCG arm: same inputs, identity labels, same tolerance
    fine = agipc.FineStep(ctx, ds, tol=TOL)
    fine.run()
    ctx.check()
    fsteps = max(2, min(5, args.steps))
    fs, fe = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fine_ms = []
    for _ in range(fsteps):
        flush()
        fs.record(stream)
        fine.run()
        fe.record(stream)
        fe.synchronize()
        fine_ms.append(fs.elapsed_time(fe))
    ctx.check()
    fres = fine.host()

    # ---- end to end: host buffers, H2D of every input and D2H of dx per step,
    # through the serving pipeline (step k+1's copies overlap step k)
    host_in = {k: getattr(ds, k).cpu().pin_memory() for k in agipc.SCENE_INPUTS}
    h2d = sum(t.numel() * t.element_size() for t in host_in.values())
    dx_host = torch.empty_like(step.dx, device="cpu").pin_memory()
    d2h = dx_host.numel() * dx_host.element_size()
    pipe = agipc.HostPipeline(ctx, (ds, agipc.DeviceScene(sc, dev)), tol=TOL)
    e2e_steps = max(3, min(20, args.steps))
    pipe.run([host_in] * 2, [dx_host] * 2)   # warm-up of the second buffer set
    torch.cuda.synchronize(dev)
    ctx.check()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    pipe.run([host_in] * e2e_steps, [dx_host] * e2e_steps)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_s = e0.elapsed_time(e1) / 1e3
    ctx.check()

    # ---- precision form (FP32 blocks/SpMV/preconditioner, FP64 dots and
    # residual replacement every 20 iterations, small-gap stencils in FP64) on
    # the same workload with 1% of the barrier gaps redrawn below 0.05 dhat
    prec = diff = batched = newton = mid = None
    if not args.skip_forms:
        mid = mid_ratio_point(dev, steps=min(args.steps, 20), fine_ms=float(np.median(fine_ms)))
        prec = precision_form(ctx_factory=lambda d: d.context(), dev=dev, steps=min(args.steps, 20))
        # ---- differentiation form (forward step + adjoint + per-tet VJP)
        diff = differentiation_form(dev, steps=min(args.steps, 10))
        # ---- batched form (256 uneven instances, one graph replay)
        batched = batched_form(dev, steps=min(args.steps, 10), peak_gbs=_peaks()[0], ws=ws, rank=rank)
        # ---- the Newton loop with backtracking (fine assembly to line search)
        newton = newton_form(dev, steps=min(args.steps, 5))

    # ---- max over ranks
    total_s, e2e_s = max_over_ranks([total_s, e2e_s], ws, dev)

    if rank == 0:
        n_c, nnz_c, iters = res["n_c"], res["col"].size, res["iters"]
        peak, peak_kind = _peaks()
        pcg_avg_s = float(np.mean(pcg_ms)) / 1e3
        pcg_bytes = iters * pcg_bytes_per_iter(nnz_c, n_c)
        achieved = pcg_bytes / pcg_avg_s / 1e9
        pcg_flops = iters * pcg_flops_per_iter(nnz_c, n_c)
        achieved_tf = pcg_flops / pcg_avg_s / 1e12
        traffic = _traffic_record()
        fine_iters, fine_nnz = fres["iters"], fres["col"].size
        fine_pcg_bytes = fine_iters * pcg_bytes_per_iter(fine_nnz, sc.n)
        out = {
            "metric": METRIC, "value": replica_throughput(ws, args.steps, total_s), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_fine": sc.n, "n_pairs": sc.n_pairs, "fine_upper_nnzb": sc.nnzb,
                       "tol": TOL, "seed": sc.seed, "l2": "flushed (256 MB write) before every timed step",
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "kernel": "pcg_kernel (persistent, whole coarse solve)",
                         "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_kind": peak_kind,
                         "traffic": traffic, "traffic_unit": "DRAM bytes per launch (ncu)",
                         "algorithmic_bytes_per_launch": pcg_bytes,
                         "byte_model": "76 B per coarse block + 200 B per coarse row per iteration",
                         "launch_ms": 1e3 * pcg_avg_s,
                         "note": "the coarse working set (%.1f MB per iteration) stays in L2 and shared memory; "
                                 "the kernel is bound by FP64 issue (alu_view)" %
                                 (pcg_bytes_per_iter(nnz_c, n_c) / 1e6),
                         "alu_view": {"bound": "alu", "achieved": achieved_tf, "unit": "TFLOP/s",
                                      "peak": FP64_PEAK_TFLOPS, "frac": achieved_tf / FP64_PEAK_TFLOPS,
                                      "peak_kind": "derived (152 SMs x 2 FP64 FMA lanes per clock x 2 flops x "
                                                   "2.07 GHz)",
                                      "algorithmic_flops_per_launch": pcg_flops}},
            "coarse": {"n_c": n_c, "active_ratio": n_c / sc.n, "nnzb_c": nnz_c, "pcg_iters": iters,
                       "relres": res["relres"], "pcg_ms": 1e3 * pcg_avg_s,
                       "step_ms_median": float(np.median(step_ms))},
            "fine_pcg": {"value": 1e3 / float(np.median(fine_ms)), "unit": UNIT, "ms_per_step": float(np.median(fine_ms)),
                         "kernel": "pcg_kernel, 16 warps per SM, matrix streamed from HBM (fine assembly included "
                                   "in ms_per_step)",
                         "pcg_iters": fine_iters, "nnzb": fine_nnz, "relres": fres["relres"],
                         "hbm_gbs_pcg_algorithmic": fine_pcg_bytes / (float(np.median(fine_ms)) / 1e3) / 1e9,
                         "hbm_frac_pcg_algorithmic": fine_pcg_bytes / (float(np.median(fine_ms)) / 1e3) / 1e9 / peak,
                         "fp64_tflops_pcg_algorithmic": fine_iters * pcg_flops_per_iter(fine_nnz, sc.n) /
                                                         (float(np.median(fine_ms)) / 1e3) / 1e12,
                         "speedup_of_coarsened": float(np.median(fine_ms)) / (1e3 * total_s / args.steps)},
            "e2e": {"value": replica_throughput(ws, e2e_steps, e2e_s), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": sum(KERNELS_PER_STEP.values()) * args.steps,
            "clocks": clocks,
            "mid_active_ratio": mid,
            "precision_form": prec,
            "differentiation_form": diff,
            "batched_form": batched,
            "newton_form": newton,
            "wall_s_timed_region": t_wall,
        }
        if ws == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(sc)
        print(json.dumps(out))
    ctx.close()
    if ws > 1:
        dist.destroy_process_group()


def mid_ratio_point(dev, steps: int, fine_ms: float):
    """The coarsened step on the same 64-box scene with per-box collapsible
    fractions U(0.2, 0.6): active ratio about 0.27, inside the range the
    paper observes (0.12-0.68), so the comparison with fine PCG (the same fine
    system, timed by the headline's fine arm) does not rest on one point."""
    import torch
    from paper_2605_04773_gb300 import agipc, scenes
    sc = scenes.domino_grid(seed=1002, frac_range=(0.2, 0.6))
    ds = agipc.DeviceScene(sc, dev)
    ctx = ds.context()
    step = agipc.CoarsenedStep(ctx, ds, tol=TOL)
    stream = torch.cuda.current_stream(dev)
    l2 = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(3):
        step.run()
    ctx.check()
    ms, pcg = [], []
    for _ in range(steps):
        l2.fill_(1.0)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        step.aggregate()
        step.assemble()
        ev[1].record(stream)
        step.solve()
        ev[2].record(stream)
        step.prolongate()
        ev[3].record(stream)
        torch.cuda.synchronize(dev)
        ms.append(ev[0].elapsed_time(ev[3]))
        pcg.append(ev[1].elapsed_time(ev[2]))
    ctx.check()
    res = step.host()
    med, pcg_med = float(np.median(ms)), float(np.median(pcg))
    n_c, nnz_c, iters = res["n_c"], res["col"].size, res["iters"]
    ctx.close()
    return {"value": 1e3 / med, "unit": UNIT, "ms_per_step": med, "pcg_ms": pcg_med, "n_c": n_c,
            "active_ratio": n_c / sc.n, "nnzb_c": nnz_c, "pcg_iters": iters, "relres": res["relres"],
            "pcg_hbm_gbs_algorithmic": iters * pcg_bytes_per_iter(nnz_c, n_c) / (pcg_med / 1e3) / 1e9,
            "speedup_vs_fine_pcg": fine_ms / med,
            "workload": "domino_8x8 as the headline with per-box collapsible fraction U(0.2, 0.6), FP64, tol 1e-6"}


def precision_form(ctx_factory, dev, steps: int):
    """Time the precision form and measure its error against the FP64 path."""
    import scipy.sparse
    import torch
    from paper_2605_04773_gb300 import agipc, scenes
    sc = scenes.domino_grid(seed=1003, small_gap_frac=0.01)
    md = agipc.MixedDeviceScene(sc, dev)
    ctx = ctx_factory(md)
    stream = torch.cuda.current_stream(dev)
    mixed = agipc.MixedStep(ctx, md, tol=TOL)
    full = agipc.CoarsenedStep(ctx, md, tol=TOL)
    for _ in range(3):
        mixed.run()
    ctx.check()
    l2 = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in ev:
        l2.fill_(1.0)
        a.record(stream)
        mixed.run()
        b.record(stream)
    torch.cuda.synchronize(dev)
    ctx.check()
    ms = float(np.median([a.elapsed_time(b) for a, b in ev]))
    m = mixed.host()
    # the FP64 path on the same scene, same timing
    full.run()
    ctx.check()
    for a, b in ev:
        l2.fill_(1.0)
        a.record(stream)
        full.run()
        b.record(stream)
    torch.cuda.synchronize(dev)
    ctx.check()
    ms64 = float(np.median([a.elapsed_time(b) for a, b in ev]))
    f = full.host()
    # errors against the FP64 path on the unrounded inputs
    gc, y32, crp, cci, cval = f["g_c"], m["y"], f["row_ptr"], f["col"], f["val"]
    Hc = scipy.sparse.bsr_matrix((cval, cci, crp), shape=(3 * f["n_c"], 3 * f["n_c"]))
    res32 = np.linalg.norm(Hc @ y32.ravel() + gc.ravel()) / np.linalg.norm(gc)
    fine = agipc.FineStep(ctx, md, tol=TOL)
    fine.inner.assemble()
    ctx.check()
    fh = fine.inner
    nnz = int(fh.nnz.item())
    Hf = scipy.sparse.bsr_matrix((fh.val[:nnz].cpu().numpy().reshape(-1, 3, 3), fh.col[:nnz].cpu().numpy(),
                                  fh.row_ptr.cpu().numpy()), shape=(3 * sc.n, 3 * sc.n))
    g = sc.g.ravel()

    def dE(dx):
        dx = dx.ravel()
        return float(g @ dx + 0.5 * dx @ (Hf @ dx))

    e64, e32 = dE(f["dx"]), dE(m["dx"])
    n64 = int(md.pair_idx64.shape[0])
    # where bytes matter: the fine system (2.3 M blocks, streamed from HBM)
    # solved by the precision form's PCG against the FP64 PCG, same scene
    mfine = agipc.MixedFineStep(ctx, md, tol=TOL)
    mfine.assemble()
    fine.inner.assemble()
    ctx.check()
    fev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(2)]
    f32_ms, f64_ms = [], []
    for _ in range(2):
        for solver, acc in ((mfine, f32_ms), (fine.inner, f64_ms)):
            l2.fill_(1.0)
            fev[0][0].record(stream)
            solver.solve()
            fev[0][1].record(stream)
            torch.cuda.synchronize(dev)
            acc.append(fev[0][0].elapsed_time(fev[0][1]))
    ctx.check()
    mf_it, f64_it = int(mfine.inner.iters.item()), int(fine.inner.iters.item())
    mf_res = float(mfine.inner.relres.item())
    fnnz = int(fine.inner.nnz.item())
    ctx.close()
    return {"value": 1e3 / ms, "unit": UNIT, "ms_per_step": ms, "pcg_iters": m["iters"],
            "fp64_same_scene": {"value": 1e3 / ms64, "ms_per_step": ms64, "pcg_iters": f["iters"]}, "workload":
            "domino_8x8 with 1% of barrier gaps in (0.01, 0.05) dhat (seed 1003), tol 1e-6, refinement every 20",
            "fp64_stencils": n64,
            "dx_rel_err_vs_fp64": float(np.linalg.norm(m["dx"] - f["dx"]) / np.linalg.norm(f["dx"])),
            "coarse_fp64_residual": float(res32), "fp64_path_residual": f["relres"],
            "energy_decrease_fp64": e64, "energy_decrease_mixed": e32,
            "energy_decrease_rel_err": abs(e32 - e64) / abs(e64),
            "fine_system": {"note": "the fine system (contacts merged, %d blocks) streamed from HBM: PCG in the "
                                    "precision form vs the FP64 PCG, same scene, tol 1e-6" % fnnz,
                            "mixed_ms": float(np.median(f32_ms)), "fp64_ms": float(np.median(f64_ms)),
                            "mixed_iters": mf_it, "fp64_iters": f64_it, "mixed_relres": mf_res,
                            "speedup": float(np.median(f64_ms)) / float(np.median(f32_ms)),
                            "mixed_us_per_iter": 1e3 * float(np.median(f32_ms)) / max(mf_it, 1),
                            "fp64_us_per_iter": 1e3 * float(np.median(f64_ms)) / max(f64_it, 1),
                            "kernels": "16 warps per SM, matrix streamed from HBM",
                            "mixed_hbm_frac": pcg_mixed_bytes_per_iter(fnnz, sc.n) * mf_it /
                                              (float(np.median(f32_ms)) / 1e3) / 1e9 / _peaks()[0],
                            "fp64_hbm_frac": pcg_bytes_per_iter(fnnz, sc.n) * f64_it /
                                             (float(np.median(f64_ms)) / 1e3) / 1e9 / _peaks()[0],
                            "byte_models": "FP64: 76 B per block + 200 B per row; precision form: 40 B per block "
                                           "+ 240 B per row + (76 B per block + 96 B per row) / 20"}}


def differentiation_form(dev, steps: int):
    """Time one differentiable coarsened step on the 46^3 StVK grid with a
    log-normal Young's modulus field: forward (fine StVK assembly with PSD
    projection, labels, coarse assembly, PCG, x + U^T y) and backward
    (restriction, adjoint PCG on the same coarse system, prolongation,
    per-tet VJP), both to the headline tolerance."""
    import torch
    from paper_2605_04773_gb300 import agipc, scenes
    sc = scenes.diff_grid()
    pr = scenes.diff_problem(sc)
    dp = agipc.DiffDeviceProblem(pr, dev)
    ctx = dp.context()
    step = agipc.DiffStep(ctx, dp, tol=TOL)
    E = torch.tensor(pr["E"], dtype=torch.float64, device=dev)
    X = torch.tensor(pr["X_rest"], dtype=torch.float64, device=dev)
    xt = torch.tensor(pr["x_target"], dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    v = torch.empty_like(xt)
    for _ in range(3):
        x_next = step.forward(E, X)
        torch.mul(torch.sub(x_next, xt), 2.0, out=v)
        step.backward(v)
    ctx.check()
    l2 = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    names = ("fine_assemble_stvk", "coarse_step", "adjoint", "stvk_vjp")
    rec = {k: [] for k in names + ("forward", "backward")}
    for _ in range(steps):
        l2.fill_(1.0)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        ev[0].record(stream)
        agipc.agipc_fine_assemble_stvk(ctx, dp.n, dp.tets, X, dp.x, dp.xhat_shift, E, dp.nu, dp.mass_h2,
                                       dp.g_extra, dp.row_ptr, dp.col, step.fine_val, step.g, step.workspace)
        ev[1].record(stream)
        agipc.agipc_aggregate(ctx, dp.n, dp.edges, dp.tags, step.labels, step.n_c)
        agipc.agipc_assemble_coarse(ctx, dp.n, step.labels, step.n_c, dp.row_ptr, dp.col, step.fine_val,
                                    dp.pair_idx, dp.pair_blk, step.g, step.row_ptr, step.col, step.val, step.nnz,
                                    step.g_c, step.dinv)
        agipc.agipc_pcg(ctx, dp.n, step.n_c, step.row_ptr, step.col, step.val, step.dinv, step.g_c, step.y,
                        step.tol, step.max_iter, -1, step.iters, step.relres)
        agipc.agipc_prolongate(ctx, dp.n, step.labels, step.y, step.dx)
        agipc.agipc_prolongate_add(ctx, dp.n, step.labels, step.y, dp.x, step.x_next)
        ev[2].record(stream)
        torch.mul(torch.sub(step.x_next, xt), 2.0, out=v)
        ev[3].record(stream)
        agipc.agipc_restrict(ctx, dp.n, step.labels, step.n_c, v, step.v_c)
        agipc.agipc_pcg(ctx, dp.n, step.n_c, step.row_ptr, step.col, step.val, step.dinv, step.v_c, step.lam_c,
                        step.adjoint_tol, step.max_iter, 1, step.adj_iters, step.adj_relres)
        agipc.agipc_prolongate(ctx, dp.n, step.labels, step.lam_c, step.lam)
        ev[4].record(stream)
        agipc.agipc_stvk_vjp(ctx, dp.n, dp.tets, X, dp.x, E, dp.nu, dp.mass_h2, step.lam, step.dx, step.dL_dE,
                             step.dL_dX, step.workspace)
        ev[5].record(stream)
        torch.cuda.synchronize(dev)
        for k, (i, j) in zip(names, ((0, 1), (1, 2), (3, 4), (4, 5))):
            rec[k].append(ev[i].elapsed_time(ev[j]))
        rec["forward"].append(ev[0].elapsed_time(ev[2]))
        rec["backward"].append(ev[3].elapsed_time(ev[5]))
    ctx.check()
    med = {k: float(np.median(v_)) for k, v_ in rec.items()}
    # workspace header: tets per flagged-eigenvalue count in int32 words 1..9
    n_flag = int(step.workspace.view(torch.int32)[1:10].sum().item())
    out = {"value": 1e3 / (med["forward"] + med["backward"]), "unit": "gradient evaluations/s",
           "ms_forward": med["forward"], "ms_backward": med["backward"],
           "ms": {k: med[k] for k in names}, "pcg_iters": int(step.iters.item()),
           "adjoint_iters": int(step.adj_iters.item()), "n_c": int(step.n_c.item()),
           "flagged_tets_last_vjp": n_flag, "n_tets": int(dp.tets.shape[0]),
           "workload": "46^3 Kuhn grid (103,823 vertices, 584,016 tets), log-normal E around 1e5 Pa, "
                       "70% collapsible, FP64, PCG and adjoint PCG to 1e-6"}
    ctx.close()
    return out


def newton_form(dev, steps: int):
    """Time the coarsened Newton loop with backtracking (Algorithm 1's inner
    loop) on the 46^3 StVK grid after an impact: per iteration fine
    assembly, strain-increment tags, labels, coarse assembly, PCG to 1e-3,
    prolongation, 10 post-coarsening PCG iterations, |d|_inf and the line
    search's energy evaluations, until |d|_inf / h <= 1e-3 l (the paper's
    tolerances).  One timed step = one time step's whole Newton loop."""
    import torch
    from paper_2605_04773_gb300 import agipc, scenes
    sc = scenes.diff_grid()
    pr = scenes.newton_problem(sc)
    dp = agipc.DiffDeviceProblem(pr, dev)
    ctx = dp.context()
    E = torch.tensor(pr["E"], dtype=torch.float64, device=dev)
    X = torch.tensor(pr["X_rest"], dtype=torch.float64, device=dev)
    x_last = torch.tensor(pr["x_last"], dtype=torch.float64, device=dev)
    sol = agipc.NewtonSolver(ctx, dp, E, X, x_last)
    for _ in range(2):
        res = sol.run()
    stream = torch.cuda.current_stream(dev)
    l2 = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    ms, its = [], []
    for _ in range(steps):
        l2.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        res = sol.run()
        b.record(stream)
        torch.cuda.synchronize(dev)
        ms.append(a.elapsed_time(b))
        its.append(res["iterations"])
    ctx.check()
    hist = res["history"]
    med = float(np.median(ms))
    out = {"value": float(np.sum(its)) / (float(np.sum(ms)) / 1e3), "unit": "Newton iterations/s",
           "time_steps_per_s": 1e3 / med, "ms_per_time_step": med, "newton_iterations": int(its[-1]),
           "ms_per_newton_iteration": med / its[-1], "converged": bool(res["converged"]),
           "n_c_per_iteration": [h_["n_c"] for h_ in hist], "alpha_per_iteration": [h_["alpha"] for h_ in hist],
           "line_search_trials": int(sum(h_["trials"] for h_ in hist)),
           "coarse_pcg_iters": [h_["coarse_iters"] for h_ in hist],
           "dnorm_over_h": [h_["dnorm"] / dp.h for h_ in hist], "eps_d": sol.eps_d,
           "workload": "46^3 Kuhn grid (103,823 vertices, 584,016 tets), log-normal E around 1e5 Pa, at rest "
                       "shape falling at 1 m/s with a 2 m/s compressive bump at one corner; threshold 5e-5, "
                       "PCG 1e-3, 10 post-coarsening iterations, eps_d = 1e-3 l, FP64"}
    ctx.close()
    return out


def batched_form(dev, steps: int, peak_gbs: float, n_inst: int = 256, ws: int = 1, rank: int = 0):
    """Time the batched form: 256 uneven instances (2k-60k vertices) in one
    CUDA-graph replay of aggregate -> offsets -> mixed assembly -> batched
    PCG -> prolongation, with the autotuned slice width.  With ws > 1 ranks
    each rank runs its contiguous share of the instances (no exchange); the
    job's time is the slowest rank's."""
    import torch
    from paper_2605_04773_gb300 import agipc, scenes
    t0 = time.perf_counter()
    first, last = shard_instances(scenes.instance_vertex_counts(n_inst=n_inst), ws, rank)
    batch = scenes.batch_instances(n_inst=last - first, first=first)
    gen_s = time.perf_counter() - t0
    bd = agipc.BatchDevice(batch, dev)
    ctx = bd.context()
    st = agipc.BatchedStep(ctx, bd, tol=TOL)
    tile, tune_ms = agipc.autotune_batched(st)
    st.run()
    ctx.check()
    st.capture()
    for _ in range(2):
        st.replay()
    ctx.check()
    stream = torch.cuda.current_stream(dev)
    l2 = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    step_ms, pcg_ms = [], []
    for _ in range(steps):
        l2.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st.replay()
        b.record(stream)
        torch.cuda.synchronize(dev)
        step_ms.append(a.elapsed_time(b))
    for _ in range(max(2, steps // 2)):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st.solve()
        b.record(stream)
        torch.cuda.synchronize(dev)
        pcg_ms.append(a.elapsed_time(b))
    ctx.check()
    h = st.host()
    inst_row = h["inst_row"]
    rp = h["row_ptr"]
    n_i = np.diff(inst_row)
    nnz_i = rp[inst_row[1:]] - rp[inst_row[:-1]]
    it = h["iters"].astype(np.int64)
    refines = it // 20 + 1
    # FP32 iteration: 36 B values + 4 B column per block; per row the SpMV's
    # u read and w write (24 B) and the update's vectors (216 B); FP64
    # residual replacement: 72 + 4 B per block and 96 B per row
    alg_bytes = float(np.sum(it * (40 * nnz_i + 240 * n_i) + refines * (76 * nnz_i + 96 * n_i)))
    med_pcg = float(np.median(pcg_ms))
    med_step = float(np.median(step_ms))
    out = {"value": 1e3 / med_step, "unit": "batches/s", "instances_per_s": batch.n_inst * 1e3 / med_step,
           "ms_per_batch": med_step, "pcg_ms": med_pcg, "tile_blocks_per_lane": tile, "autotune_ms": tune_ms,
           "assembly_terms_per_lane": st.assembly_run, "autotune_assembly_ms": st.assembly_ms,
           "n_inst": batch.n_inst, "n_fine": batch.n, "n_tets": int(batch.tets.shape[0]),
           "fine_upper_nnzb": int(batch.col.shape[0]), "n_pairs": int(batch.pair_idx.shape[0]),
           "n_c": h["n_c"], "nnzb_c": int(rp[-1]), "iters_min_median_max": [int(it.min()), int(np.median(it)),
                                                                              int(it.max())],
           "pcg_roofline": {"bound": "hbm", "algorithmic_bytes": alg_bytes, "achieved_gbs": alg_bytes / med_pcg / 1e6,
                            "peak_gbs": peak_gbs, "frac": alg_bytes / med_pcg / 1e6 / peak_gbs},
           "generator_s": gen_s, "graph": "one CUDA graph replay per batch",
           "workload": str(batch.n_inst) + " Kuhn-split hex grids, 2k-60k vertices log-uniform, random aspect, 30-90% collapsible, "
                       "0-5% of vertices in PT barrier stencils; FP32 blocks, FP64 accumulation, tol 1e-6"}
    out["instance_range"] = [first, last]
    if ws > 1:
        # every rank solved its own instances; the job runs as long as its slowest rank
        med_all = max_over_ranks([med_step], ws, dev)[0]
        out["job"] = {"ranks": ws, "instances": n_inst, "ms_per_batch_max_over_ranks": med_all,
                      "instances_per_s": n_inst * 1e3 / med_all, "scaling": "strong (fixed 256-instance batch)"}
    ctx.close()
    return out


def cpu_baseline(sc, reps: int = 1):
    """The CPU FP64 oracle (single thread) on the same workload."""
    import oracle
    oracle.build()
    times = []
    for _ in range(reps):
        t = time.perf_counter()
        oracle.coarsened_step(sc, tol=TOL)
        times.append(time.perf_counter() - t)
    best = min(times)
    return {"value": 1.0 / best, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d full step(s) of the domino_8x8 workload (labels, explicit U H U^T, PCG to 1e-6, "
                      "prolongation), %.2f s each" % (reps, best)}


def run_reference(args):
    ws, rank, _ = _dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2605_04773_gb300 import scenes
    oracle.build()
    sc = scenes.domino_grid(seed=1002)
    warm = min(args.warmup, 1)
    for _ in range(warm):
        oracle.coarsened_step(sc, tol=TOL)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        oracle.coarsened_step(sc, tol=TOL)
        times.append(time.perf_counter() - t)
    total = sum(times)
    value = args.steps / total
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": warm, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "n_fine": sc.n, "n_pairs": sc.n_pairs, "tol": TOL, "seed": sc.seed},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": "%d full oracle steps of the workload (%d warm-up)" % (args.steps, warm)},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_one_form(args):
    """One form on one GPU, its JSON object on stdout: the command the kernel
    profiles under profiles/ are captured with."""
    import torch
    from paper_2605_04773_gb300 import build
    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    steps = max(1, args.steps)
    if args.form == "precision":
        out = precision_form(ctx_factory=lambda d: d.context(), dev=dev, steps=steps)
    elif args.form == "differentiation":
        out = differentiation_form(dev, steps=steps)
    elif args.form == "newton":
        out = newton_form(dev, steps=steps)
    else:
        out = batched_form(dev, steps=steps, peak_gbs=_peaks()[0], n_inst=args.batch_instances)
    print(json.dumps({"form": args.form, **out}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skip-forms", action="store_true", help="only the headline step (profiling runs)")
    ap.add_argument("--form", choices=["precision", "differentiation", "batched", "newton"], default=None,
                    help="run one form alone and print its JSON object (profiling runs)")
    ap.add_argument("--batch-instances", type=int, default=256, help="instances of the batched form with --form")
    ap.add_argument("--fp64-probe", action="store_true", help="measure the FP64 FMA rate of one SM and exit")
    args = ap.parse_args()
    if args.fp64_probe:
        print(json.dumps(fp64_probe()))
    elif args.form is not None:
        run_one_form(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
