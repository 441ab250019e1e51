#!/usr/bin/env python
"""Benchmark: randomized block-Lanczos PCA on the 'precision' workload.

Workload (one step = one whole PCA, Section 3 Steps 1-6, through the C-ABI):
A = U0 diag(exp(-j/40)) V0^T + N(0, 1e-6) noise, m = 1,000,000, n = 4,096,
k = 50, l = 60, i = 2, stored in BF16 (headline) and in FP32 (compared in the
same run).  Metric: A-stream GB/s = (i+2) m n bytes_per_element / t_PCA
(every PCA streams A i+2 times: i+1 fused passes and the T pass), plus
seconds per PCA and the BF16-over-FP32 wall-clock ratio.  A (8.2 / 16.4 GB)
is far larger than the 129 MB L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on a bounded row sample of the same
workload (the paper's algorithm as written, on the host cores).
Multi-GPU: independent replicas (one PCA per rank, weak scaling).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = dict(name="precision", m=1_000_000, n=4096, k=50, l=60, i=2, seed=1007)


def max_over_ranks(ms, world, dist, device=None):
    """Slowest rank's time (the whole job's): all-reduce MAX over the process
    group (a CUDA tensor under NCCL, a CPU tensor under gloo)."""
    if world <= 1:
        return ms
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
CPU_SAMPLE_ROWS = 150_000     # cpu_baseline: one oracle PCA on this many rows (~13 s)
REF_SAMPLE_ROWS = 40_000      # --impl reference: rows per timed step
# DRAM bytes (read + write) per row of A of one launch of the BF16 tensor-core
# fused pass at n = 4,096, L = 64 (ncu capture at m = 100,000; traffic grows
# in proportion to the rows)
FUSED_BF16_N4096_TRAFFIC_PER_ROW = 854.153e6 / 100_000


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--rows", "--m", dest="m", type=int, default=WORKLOAD["m"],
                    help="rows of A (precision workload; the oracle arm's sample is capped by it)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-oracle-accuracy", action="store_true",
                    help="skip the full-size FP64 oracle run that reports each path's error")
    ap.add_argument("--simt", action="store_true", help="force the CUDA-core pass kernels")
    ap.add_argument("--workload", default="precision", choices=["precision", "batched", "out_of_core"],
                    help="precision: the headline (one 1e6 x 4096 PCA); batched: 512 uneven BF16 PCAs; "
                         "out_of_core: FP32 A in pinned host memory (n = 8192), streamed in tiles")
    ap.add_argument("--count", type=int, default=512, help="problems in the batched workload")
    ap.add_argument("--no-batched", action="store_true", help="leave the batched workload out of the default line")
    ap.add_argument("--no-backward", action="store_true", help="batched workload: forward only")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- oracle leg
def oracle_sample(A_host_fp64, k, l, i):
    """Time the oracle on a row sample; returns (seconds, rows, cores)."""
    from oracle import rpca_oracle
    t0 = time.perf_counter()
    rpca_oracle.rpca(A_host_fp64, k, l, i, seed=WORKLOAD["seed"])
    return time.perf_counter() - t0


def sample_rows_fp64(A, rows):
    return A[:rows].float().cpu().double().numpy()


def cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


# ----------------------------------------------------------------- ours
def main():
    args = parse()
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    W = dict(WORKLOAD)
    W["m"] = args.m
    m, n, k, l, i = W["m"], W["n"], W["k"], W["l"], W["i"]
    bytes_bf16, bytes_f32 = 2, 4

    if args.impl == "reference":
        if rank != 0:
            return
        run_reference(args, W)
        return

    torch.cuda.set_device(local)
    if args.workload == "batched":
        run_batched(args, world, rank, local, dist)
        return
    if args.workload == "out_of_core":
        run_out_of_core(args, world, rank, local, dist)
        return
    from paper_1007_5510_gb300 import rpca
    from synth import generators as gen
    rpca.load_library()
    dev = torch.device("cuda", local)
    t0 = time.perf_counter()
    A32 = gen.workload_torch("precision", dev, m=m, n=n, seed=W["seed"] + rank, rank_cap=1024)
    A16 = A32.to(torch.bfloat16)
    A8, s8 = gen.quantize_fp8_torch(A32)          # FP8-e4m3 bytes + per-column FP32 scales
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0

    stream = torch.cuda.current_stream()
    ctx16 = rpca.PCA(m, n, k, l, i, rpca.BF16, seed=W["seed"], timing=True, simt=args.simt)
    ctx32 = rpca.PCA(m, n, k, l, i, rpca.F32, seed=W["seed"], timing=True, simt=args.simt)
    ctx8 = rpca.PCA(m, n, k, l, i, rpca.FP8E4M3, seed=W["seed"], timing=True, simt=args.simt)
    U16 = torch.empty(m, k, device=dev)
    V16 = torch.empty(n, k, device=dev)
    S16 = torch.empty(k, dtype=torch.float64, device=dev)
    U32, V32, S32 = torch.empty_like(U16), torch.empty_like(V16), torch.empty_like(S16)
    U8, V8, S8 = torch.empty_like(U16), torch.empty_like(V16), torch.empty_like(S16)

    def timed(ctx, A, U, S, V, steps, col_scale=None):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(steps):
            ctx.run(A, col_scale=col_scale, U=U, S=S, V=V)
        ev1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ms = ev0.elapsed_time(ev1)
        ms = max_over_ranks(ms, world, dist, dev)
        return ms

    for _ in range(args.warmup):
        ctx16.run(A16, U=U16, S=S16, V=V16)
        ctx32.run(A32, U=U32, S=S32, V=V32)
        ctx8.run(A8, col_scale=s8, U=U8, S=S8, V=V8)
    torch.cuda.synchronize()
    ctx16.phase_times()
    ctx32.phase_times()
    ctx8.phase_times()

    sampler = ClockSampler(local)
    sampler.start()
    launches0 = rpca.kernel_launches()
    ms16 = timed(ctx16, A16, U16, S16, V16, args.steps)
    launches = rpca.kernel_launches() - launches0
    ms32 = timed(ctx32, A32, U32, S32, V32, args.steps)
    ms8 = timed(ctx8, A8, U8, S8, V8, args.steps, col_scale=s8)
    clocks = sampler.stop()
    ph16, runs16 = ctx16.phase_times()
    ph32, runs32 = ctx32.phase_times()
    ph8, runs8 = ctx8.phase_times()
    t8 = ms8 / args.steps / 1e3

    t16 = ms16 / args.steps / 1e3
    t32 = ms32 / args.steps / 1e3
    # passes over A per PCA as the library reports them: i+2, or i+1 when T
    # was formed from the fused passes' F blocks
    np16, np32, np8 = ctx16.passes_last_run(), ctx32.passes_last_run(), ctx8.passes_last_run()
    stream_bytes16 = np16 * m * n * bytes_bf16
    stream_bytes32 = np32 * m * n * bytes_f32
    value = world * stream_bytes16 / t16 / 1e9
    hbm, peak_kind = peaks()

    # dominant kernel: the fused pass (phases 0..i-1 are fused passes)
    def per_launch(ph, runs, idx):
        return sum(ph[j] for j in idx) / max(1, runs * len(idx))
    fused_idx = list(range(i)) if i > 0 else [0]
    fused_ms16 = per_launch(ph16, runs16, fused_idx)
    fused_ms32 = per_launch(ph32, runs32, fused_idx)
    tpass_ms16 = per_launch(ph16, runs16, [i + 2])
    achieved = m * n * bytes_bf16 / (fused_ms16 / 1e3) / 1e9
    names = ["pass%d" % j for j in range(i + 1)] + ["qr_h", "t_pass", "small_svd", "u_v"]
    phases16 = {nm: round(v / max(1, runs16), 4) for nm, v in zip(names, ph16)}
    phases32 = {nm: round(v / max(1, runs32), 4) for nm, v in zip(names, ph32)}

    # accuracy: both outputs against each other and the leading spectrum
    s16 = S16.cpu().numpy()
    s32 = S32.cpu().numpy()
    acc = {"sigma_rel_bf16_vs_f32": float(abs(s16 - s32).max() / s32.max()),
           "sigma_1": float(s32[0]), "sigma_k": float(s32[-1])}
    try:
        acc.update(spectral_errors(A32, [(U32, S32, V32), (U16, S16, V16), (U8, S8, V8)], ["f32", "bf16", "fp8"]))
    except Exception as e:  # measurement only
        acc["spectral_error_failed"] = str(e)[:200]

    e2e = None
    if not args.no_e2e:
        e2e = end_to_end(A16, m, n, k, l, i, bytes_bf16, min(args.steps, 3), dev, world, dist, W["seed"])

    batched = None
    if not args.no_batched:
        # the 512-problem batched workload, forward and backward (sub-object)
        del A8, s8
        ctx8.close()
        torch.cuda.empty_cache()
        tb = time.perf_counter()
        bshapes, bAs = batched_inputs(args.count, rank, dev)
        bgen = time.perf_counter() - tb
        batched = batched_measure(bshapes, bAs, args.steps, args.warmup, world, dist, dev,
                                  backward=not args.no_backward)
        batched["gen_s"] = round(bgen, 2)
        batched["workload"] = ("batched: %d BF16 PCAs, m ~ U[1000, 50000], n ~ U[64, 1024], sigma_j = j^-1.5"
                               % len(bshapes))
        del bAs
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rows = min(CPU_SAMPLE_ROWS, m)
        Ah = sample_rows_fp64(A16, rows)
        secs = oracle_sample(Ah, k, l, i)
        cpu = {"value": round((i + 2) * rows * n * bytes_bf16 / secs / 1e9, 4), "unit": "GB/s",
               "cores": cores(), "kind": "oracle",
               "sample": "first %d of %d rows of the BF16 matrix, upcast to FP64, one PCA "
                         "(%.1f s)" % (rows, m, secs)}
        if not args.no_oracle_accuracy:
            # the same oracle once on the whole FP32 matrix: every path's error
            # against the FP64 result on the unquantised input
            acc.update(oracle_errors(A32, k, l, i, W["seed"],
                                     {"f32": (U32, S32, V32), "bf16": (U16, S16, V16), "fp8": (U8, S8, V8)}))

    if rank == 0:
        line = {
            "metric": "A-stream GB/s (% HBM peak) and s/PCA, BF16 vs FP32 at equal spectral error",
            "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms16 / args.steps, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
            "data": "synthetic", "gpu_launches": int(launches),
            "config": {"workload": "precision: m=%d n=%d k=%d l=%d i=%d, BF16 storage "
                                   "(FP32 measured alongside)" % (m, n, k, l, i),
                       "m": m, "n": n, "k": k, "l": l, "i": i, "streams_per_pca": np16,
                       "l2_flush": "not needed: A (%.1f GB) >> L2" % (m * n * 2 / 1e9),
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "kernels": "cuda-cores" if args.simt else "auto"},
            "s_per_pca": round(t16, 6),
            "pct_hbm_peak": round(100 * stream_bytes16 / t16 / 1e9 / hbm, 2),
            "fp32": {"value": round(world * stream_bytes32 / t32 / 1e9, 2), "unit": "GB/s",
                     "s_per_pca": round(t32, 6), "fused_pass_ms": round(fused_ms32, 4),
                     "streams_per_pca": np32, "phases_ms": phases32},
            "bf16_speedup_vs_fp32": round(t32 / t16, 3),
            "fp8": {"value": round(world * np8 * m * n * 1 / t8 / 1e9, 2), "unit": "GB/s",
                    "s_per_pca": round(t8, 6), "streams_per_pca": np8,
                    "kernels": "tensor cores (FP8 bytes widened to BF16 by converter warps, per-column scales "
                               "folded into X and the result rows)",
                    "phases_ms": {nm: round(v / max(1, runs8), 4) for nm, v in zip(names, ph8)}},
            "phases_ms": phases16,
            "roofline": {"bound": "hbm", "kernel": "fused pass (BF16, l=%d)" % l,
                         "achieved": round(achieved, 2), "peak": hbm, "peak_kind": peak_kind,
                         "unit": "GB/s", "frac": round(achieved / hbm, 4),
                         "traffic": (round(FUSED_BF16_N4096_TRAFFIC_PER_ROW * m)
                                     if (n == 4096 and not args.simt) else None),
                         "algorithmic_bytes_per_launch": m * n * bytes_bf16,
                         "avg_launch_ms": round(fused_ms16, 4),
                         "t_pass_ms": round(tpass_ms16, 4)},
            "accuracy": acc,
            "batched": batched,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "gen_s": round(gen_s, 2),
        }
        print(json.dumps(line))
    ctx16.close()
    ctx32.close()
    if args.no_batched:
        ctx8.close()
    if world > 1:
        dist.destroy_process_group()


def oracle_errors(A32, k, l, i, seed, outs):
    """Relative singular-value error and largest principal angles of U and
    V of each output against the FP64 oracle run on the FP32 matrix (rows
    streamed from a host copy by 8192-row blocks)."""
    from oracle import rpca_oracle, estimator
    m, n = A32.shape
    Ah = A32.cpu()
    t0 = time.perf_counter()
    Uo, So, Vo = rpca_oracle.rpca(lambda r0, r1: Ah[r0:r1].numpy(), k, l, i, seed=seed, normalize=True,
                                  m=m, n=n)
    res = {"oracle_full_s": round(time.perf_counter() - t0, 1)}
    for lab, (U, S, V) in outs.items():
        s = S.cpu().numpy()
        res["vs_fp64_oracle_" + lab] = {
            "sigma_rel": float(np.max(np.abs(s - So) / So)),
            "angle_U": float(estimator.max_principal_angle(U.cpu().double().numpy(), Uo)),
            "angle_V": float(estimator.max_principal_angle(V.cpu().double().numpy(), Vo))}
    return res


def spectral_errors(A, outs, labels, iters=30, nvec=4):
    """||A - U S V^T||_2 by block power iteration on the residual (torch,
    measurement only), same start vectors for every output."""
    import torch
    g = torch.Generator(device=A.device)
    res = {}
    for (U, S, V), lab in zip(outs, labels):
        g.manual_seed(5)
        x = torch.randn(A.shape[1], nvec, generator=g, device=A.device)
        Sf = S.float()
        est = 0.0
        for _ in range(iters):
            y = A @ x - U @ (Sf[:, None] * (V.T @ x))
            z = A.T @ y - V @ (Sf[:, None] * (U.T @ y))
            nz = torch.linalg.norm(z, dim=0)
            est = float(torch.sqrt(nz.max() / torch.linalg.norm(x, dim=0)[nz.argmax()]))
            x = torch.linalg.qr(z.cpu())[0].to(z.device)   # n x nvec: small
        res["spectral_error_" + lab] = est
    for lab in labels[1:]:
        res["spectral_error_ratio_%s_over_f32" % lab] = res["spectral_error_" + lab] / res["spectral_error_f32"]
    return res


def end_to_end(A_dev, m, n, k, l, i, b, steps, dev, world, dist, seed):
    """Same metric through the public API with host buffers: one call per
    step on A in pinned host memory (RPCA_HOST_A | RPCA_HOST_RESIDENT: the
    library copies A in once, the first pass working on each tile as it
    lands), then U S V copied out."""
    import torch
    from paper_1007_5510_gb300 import rpca
    Ah = A_dev.cpu().pin_memory()
    Uh = torch.empty(m, k).pin_memory()
    Vh = torch.empty(n, k).pin_memory()
    Sh = torch.empty(k, dtype=torch.float64).pin_memory()
    U = torch.empty(m, k, device=dev)
    V = torch.empty(n, k, device=dev)
    S = torch.empty(k, dtype=torch.float64, device=dev)
    ctx = rpca.PCA(m, n, k, l, i, rpca.BF16, seed=seed, host_a=True, host_resident=True)
    st = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx.run(Ah, U=U, S=S, V=V)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ev0.record(st)
    for _ in range(steps):
        ctx.run(Ah, U=U, S=S, V=V)
        Uh.copy_(U, non_blocking=True)
        Vh.copy_(V, non_blocking=True)
        Sh.copy_(S, non_blocking=True)
    ev1.record(st)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    ctx.close()
    ms = max_over_ranks(ms, world, dist, dev)
    t = ms / steps / 1e3
    return {"value": round(world * (i + 2) * m * n * b / t / 1e9, 2), "unit": "GB/s",
            "s_per_pca": round(t, 6), "h2d_bytes_per_step": m * n * b,
            "d2h_bytes_per_step": (m + n) * k * 4 + k * 8}


def batched_inputs(count, rank, dev):
    """The batched workload's matrices: `count` BF16 problems (m ~ U[1000,
    50000], n ~ U[64, 1024], sigma_j = j^-1.5), rows padded to a multiple of
    8 elements (16 bytes: the layout the grouped kernels' TMA loads take)."""
    import torch
    from synth import generators as gen
    shapes = gen.batched_shapes(count=count, seed=5510 + rank)
    As = []
    for p, (m, n) in enumerate(shapes):
        buf = torch.zeros(m, (n + 7) // 8 * 8, dtype=torch.bfloat16, device=dev)
        buf[:, :n] = gen.workload_torch("batched", dev, m=m, n=n, seed=1007 + 7919 * rank + p, rank_cap=1024,
                                        dtype=torch.bfloat16)
        As.append(buf[:, :n])
    torch.cuda.synchronize()
    return shapes, As


def batched_measure(shapes, As, steps, warmup, world, dist, dev, backward=True):
    """Forward (grouped kernels) and backward (per-problem adjoint contexts:
    dA_p for dS_p = 1) of the batched workload, device-timed with CUDA events
    on the caller's stream.  Returns a dict of the two measurements."""
    import torch
    from paper_1007_5510_gb300 import rpca
    from synth import generators as gen
    cfg = gen.CONFIGS["batched"]
    k, l, i = cfg["k"], cfg["l"], cfg["i"]
    stream = torch.cuda.current_stream()
    a_bytes = sum(m * n * 2 for m, n in shapes)
    hbm, peak_kind = peaks()

    def timed(fn, nsteps):
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(nsteps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(e0.elapsed_time(e1), world, dist, dev) / nsteps

    b = rpca.Batch(shapes, k, l, i, dtype=rpca.BF16, seeds=range(len(shapes)), nstreams=16)
    holder = {"outs": b.run(As)}
    for _ in range(max(0, warmup - 1)):
        holder["outs"] = b.run(As, holder["outs"])
    torch.cuda.synchronize()
    grouped = b.grouped
    launches0 = rpca.kernel_launches()
    ms = timed(lambda: holder.__setitem__("outs", b.run(As, holder["outs"])), steps)
    launches = (rpca.kernel_launches() - launches0) / steps
    b.close()
    t = ms / 1e3
    fwd = {"ms_per_step": round(ms, 4), "pcas_per_s": round(world * len(shapes) / t, 1),
           "value": round(world * (i + 2) * a_bytes / t / 1e9, 2), "unit": "GB/s",
           "pct_hbm_peak": round(100 * (i + 2) * a_bytes / t / 1e9 / hbm, 2),
           "kernels_per_step": round(launches, 1),
           "form": "grouped kernels (one launch per step of the method over all problems)"
                   if grouped else "per-problem contexts, one graph launch per step"}
    out = {"problems": len(shapes), "a_bytes": a_bytes, "k": k, "l": l, "i": i,
           "lda": "n rounded up to a multiple of 8", "forward": fwd}
    if backward:
        # adjoint contexts (per problem), one forward, then the timed backward
        ba = rpca.Batch(shapes, k, l, i, dtype=rpca.BF16, seeds=range(len(shapes)), nstreams=16, adjoint=True)
        ba.run(As)
        dS = [torch.ones(k, dtype=torch.float64, device=dev) for _ in shapes]
        dA = [torch.empty(m, n, dtype=torch.float32, device=dev) for m, n in shapes]
        ba.backward(As, dS, dA)
        torch.cuda.synchronize()
        bsteps = max(1, min(steps, 2))
        msb = timed(lambda: ba.backward(As, dS, dA), bsteps)
        ba.close()
        del dA
        out["backward"] = {"ms_per_step": round(msb, 4), "steps": bsteps,
                           "grad": "dA_p of sum_j sigma_j for every problem (FP32, m_p x n_p)",
                           "form": "per-problem adjoint contexts over 16 streams"}
    return out


def run_batched(args, world, rank, local, dist):
    """Batched workload: `count` independent BF16 PCAs (m ~ U[1000, 50000],
    n ~ U[64, 1024], sigma_j = j^-1.5, k=16 l=20 i=1) per step, one batch."""
    import torch
    from paper_1007_5510_gb300 import rpca
    from synth import generators as gen
    cfg = gen.CONFIGS["batched"]
    k, l, i = cfg["k"], cfg["l"], cfg["i"]
    dev = torch.device("cuda", local)
    t0 = time.perf_counter()
    shapes, As = batched_inputs(args.count, rank, dev)
    gen_s = time.perf_counter() - t0
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = rpca.kernel_launches()
    res = batched_measure(shapes, As, args.steps, args.warmup, world, dist, dev, backward=not args.no_backward)
    clocks = sampler.stop()
    fwd = res["forward"]
    if rank == 0:
        print(json.dumps({
            "metric": "A-stream GB/s (% HBM peak) and s/PCA, BF16 vs FP32 at equal spectral error",
            "value": fwd["value"], "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": fwd["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "gpu_launches": int(fwd["kernels_per_step"] * args.steps),
            "config": {"workload": "batched: %d BF16 PCAs, m ~ U[1000, 50000], n ~ U[64, 1024], "
                                   "sigma_j = j^-1.5, k=%d l=%d i=%d, %s" % (len(shapes), k, l, i, fwd["form"]),
                       "problems": len(shapes), "a_bytes": res["a_bytes"], "streams_per_pca": i + 2,
                       "lda": res["lda"],
                       "l2_flush": "not needed: A (%.1f GB in total) >> L2" % (res["a_bytes"] / 1e9),
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "pcas_per_s": fwd["pcas_per_s"], "pct_hbm_peak": fwd["pct_hbm_peak"],
            "backward": res.get("backward"),
            "clocks": clocks, "gen_s": round(gen_s, 2),
        }))


def run_out_of_core(args, world, rank, local, dist):
    """Out-of-core form (Section 4.2): A (FP32, n = 8192, rank-64 signal +
    noise, k=40 l=48 i=2) in pinned host memory, every pass streaming it to
    the device in double-buffered 1 GiB tiles.  The roofline is the pinned
    host-to-device bandwidth, measured in the same run."""
    import torch
    from paper_1007_5510_gb300 import rpca
    from synth import generators as gen
    cfg = gen.CONFIGS["out_of_core"]
    n, k, l, i = cfg["n"], cfg["k"], cfg["l"], cfg["i"]
    m = args.m if args.m != WORKLOAD["m"] else 750_000
    dev = torch.device("cuda", local)
    t0 = time.perf_counter()
    Ah = torch.empty(m, n, dtype=torch.float32).pin_memory()
    chunk = 250_000
    for r0 in range(0, m, chunk):
        rows = min(chunk, m - r0)
        Ad = gen.workload_torch("out_of_core", dev, m=rows, n=n, seed=1007 + 7919 * rank + r0)
        Ah[r0:r0 + rows].copy_(Ad)
        del Ad
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    # pinned host -> device bandwidth on 1 GiB copies (the link this form is bound by)
    buf_d = torch.empty(1 << 28, dtype=torch.float32, device=dev)
    src = Ah.view(-1)[: 1 << 28]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(2):
        buf_d.copy_(src, non_blocking=True)
    e0.record(stream)
    for _ in range(5):
        buf_d.copy_(src, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    h2d = 5 * (1 << 30) / (e0.elapsed_time(e1) / 1e3) / 1e9
    del buf_d
    ctx = rpca.PCA(m, n, k, l, i, rpca.F32, seed=1007, host_a=True, timing=True)
    U = torch.empty(m, k, device=dev)
    V = torch.empty(n, k, device=dev)
    S = torch.empty(k, dtype=torch.float64, device=dev)
    for _ in range(args.warmup):
        ctx.run(Ah, U=U, S=S, V=V)
    torch.cuda.synchronize()
    ctx.phase_times()
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = rpca.kernel_launches()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        ctx.run(Ah, U=U, S=S, V=V)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(ev0.elapsed_time(ev1), world, dist, dev)
    launches = rpca.kernel_launches() - launches0
    clocks = sampler.stop()
    ph, runs = ctx.phase_times()
    ctx.close()
    t = ms / args.steps / 1e3
    a_bytes = m * n * 4
    value = world * (i + 2) * a_bytes / t / 1e9
    names = ["pass%d" % j for j in range(i + 1)] + ["qr_h", "t_pass", "small_svd", "u_v"]
    stream_ms = sum(ph[j] for j in range(i + 1)) / max(1, runs) + ph[i + 2] / max(1, runs)
    if rank == 0:
        print(json.dumps({
            "metric": "A-stream GB/s (% HBM peak) and s/PCA, BF16 vs FP32 at equal spectral error",
            "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "gpu_launches": int(launches),
            "config": {"workload": "out_of_core: m=%d n=%d k=%d l=%d i=%d, FP32 A (%.1f GB) in pinned host "
                                   "memory, 1 GiB double-buffered tiles" % (m, n, k, l, i, a_bytes / 1e9),
                       "m": m, "n": n, "k": k, "l": l, "i": i, "streams_per_pca": i + 2,
                       "l2_flush": "not needed: A streams from host memory",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "s_per_pca": round(t, 4),
            "roofline": {"bound": "host-to-device link", "achieved": round((i + 2) * a_bytes / (stream_ms / 1e3) / 1e9, 2),
                         "peak": round(h2d, 2), "peak_kind": "pinned H2D measured in this run (1 GiB copies)",
                         "unit": "GB/s", "frac": round((i + 2) * a_bytes / (stream_ms / 1e3) / 1e9 / h2d, 4)},
            "phases_ms": {nm: round(v / max(1, runs), 3) for nm, v in zip(names, ph)},
            "clocks": clocks, "gen_s": round(gen_s, 2),
        }))


def run_reference(args, W):
    """The oracle arm: FP64 CPU oracle on a bounded row sample per step."""
    import numpy as np
    from synth import generators as gen
    m, n, k, l, i = W["m"], W["n"], W["k"], W["l"], W["i"]
    rows = min(REF_SAMPLE_ROWS, m)
    A = gen.workload_np("precision", m=rows, n=n, seed=W["seed"], rank_cap=1024)
    A = gen.round_bf16_np(A).astype(np.float64)
    for _ in range(args.warmup):
        oracle_sample(A, k, l, i)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_sample(A, k, l, i)
    secs = (time.perf_counter() - t0) / args.steps
    val = (i + 2) * rows * n * 2 / secs / 1e9
    sample = ("%d-row sample of the precision workload (n=%d, BF16 values in FP64), one PCA "
              "per step" % (rows, n))
    print(json.dumps({
        "impl": "reference",
        "metric": "A-stream GB/s (% HBM peak) and s/PCA, BF16 vs FP32 at equal spectral error",
        "value": round(val, 4), "unit": "GB/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(secs * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "precision: m=%d n=%d k=%d l=%d i=%d, BF16 storage" % (m, n, k, l, i),
                   "sample_rows": rows},
        "cpu_baseline": {"value": round(val, 4), "unit": "GB/s", "cores": cores(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(val, 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }))


if __name__ == "__main__":
    main()
