#!/usr/bin/env python
"""Benchmark of the fused forward + zonal + inverse + PSNR path on GB300.

Workload (one step): 64 uint8 images of 512x512 (half AR(1) rho=0.95, half
AR(1) rho=0.80 plus N(0, 8^2)), each compressed at every zonal r in
{1, 6, 16, 36, 64, 100, 150, 256}: 512 image jobs, 134.2 Mpixel, in one
persistent launch of the fused kernel plus the per-image PSNR finalize.
Metric: Gpixel/s over the whole job (all ranks).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank compresses its own shard of images (weak
scaling, no data-path collective); the step time is the max over ranks.
``--impl reference`` times the CPU oracle on a bounded sample instead.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

R_SWEEP = (1, 6, 16, 36, 64, 100, 150, 256)
BOX_EXTENTS = (1, 3, 6, 8)  # the kernels for r <= 36: kept set inside the K x K corner, r <= K (K + 1) / 2


def zonal_launches_per_call(rs):
    """Kernels one atdct16_compress_zonal call launches for jobs with these r:
    one per non-empty class (the smallest box extent K with r <= K (K + 1) / 2
    for 1 <= r <= 36, else the general kernel), then the PSNR finalize."""
    classes = set()
    for r in rs:
        k = next((k for k in BOX_EXTENTS if 1 <= r <= k * (k + 1) // 2), None)
        classes.add(k if k is not None else "general")
    return len(classes) + 1
N_IMAGES = 64
SIDE = 512
METRIC = "Gpixel/s fused fwd+zonal+inv+PSNR"
UNIT = "Gpixel/s"
WORKLOAD = "64x512x512 u8 AR(1) images x zonal r in {1,6,16,36,64,100,150,256}"
N_SETS = 3  # rotating input/output sets: 3 x 268 MB per step-set > 4 x L2
PROF_CALLS = 64  # calls timed one by one (event pair around the fused kernels) for the roofline


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--images", type=int, default=N_IMAGES,
                    help="images per step (default: the 64-image workload; smaller for profiling captures)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="CPU-baseline sample budget")
    ap.add_argument("--e2e-steps", type=int, default=30)
    ap.add_argument("--no-extras", action="store_true", help="skip the quantisation, mixed-batch and serving phases")
    ap.add_argument("--quant-only", action="store_true",
                    help="run only the quantisation phase (--steps/--warmup apply) and print its JSON")
    ap.add_argument("--quant-frames", type=int, default=240)
    ap.add_argument("--quant-chunk", type=int, default=24, help="frames per quantisation call")
    ap.add_argument("--dct-only", action="store_true",
                    help="run only the exact-DCT baseline phase (--steps applies) and print its JSON")
    ap.add_argument("--ssim-only", action="store_true",
                    help="run only the SSIM phase on one compressed step (--steps applies) and print its JSON")
    ap.add_argument("--serve-only", action="store_true",
                    help="run only the serving phase (config 5) and print its JSON")
    ap.add_argument("--coef-only", action="store_true",
                    help="run only the coefficient-pipeline phase (--steps applies) and print its JSON")
    ap.add_argument("--mixed-images", type=int, default=1000)
    ap.add_argument("--serve-rates", default="100,250,500,1000,2000,5000")
    ap.add_argument("--serve-requests", type=int, default=20000, help="serving requests over the whole rate sweep")
    return ap.parse_args()


# --------------------------------------------------------------------------
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.3)

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_source_sha256():
    """Hash of the zonal kernels' source: the headers they include, the
    small-extent kernels with the class split, and the part of
    atdct16_kernels.cu before the quantisation kernel (the general kernel)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1606_05562_gb300", "csrc")
    for f in ("atdct16_butterfly.cuh", "atdct16_ops.cuh", "atdct16_internal.h", "atdct16_device.cuh",
              "atdct16_zonal_box.cu"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    with open(os.path.join(csrc, "atdct16_kernels.cu"), "rb") as fh:
        text = fh.read()
    cut = text.find(b"// Fused quantisation")
    h.update(text if cut < 0 else text[:cut])
    return h.hexdigest()


def recorded_traffic():
    """DRAM bytes per call of the fused zonal kernels from the committed ncu
    summary, if it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "zonal_kernels_64x512x512.md")
    try:
        text = open(p).read()
    except OSError:
        return None
    sha = re.search(r"kernel_source_sha256:\s*([0-9a-f]{64})", text)
    tr = re.search(r"traffic_bytes_per_launch:\s*([0-9.e+]+)", text)
    if not sha or not tr or sha.group(1) != kernel_source_sha256():
        return None
    return float(tr.group(1))


# --------------------------------------------------------------------------
def rank_images(world, rank, n_per_rank=N_IMAGES, side=SIDE):
    """This rank's images of the whole job (n_per_rank x world images of the
    synthetic batch): the LPT image sharding of paper_1606_05562_gb300.shard,
    so every rank compresses n_per_rank whole images and no data-path
    collective is needed (weak scaling)."""
    from paper_1606_05562_gb300 import shard

    shards = shard.balanced_shards([side * side] * (n_per_rank * world), world)
    return shards[rank]


def cpu_baseline(batch, budget_s):
    """The oracle as it stands, on a bounded sample of the workload."""
    import numpy as np

    import oracle as O

    t0 = time.perf_counter()
    px = 0
    done = []
    for i in range(len(batch)):
        for r in R_SWEEP:
            O.compress_zonal_exact(batch[i], r)
            px += batch[i].size
        done.append(i)
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    threads = 1  # numpy int64 einsum runs on one core
    return {"value": px / dt / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{len(done)} of 64 images x 8 r ({px / 1e6:.1f} Mpx) with the exact-integer oracle, {dt:.1f} s"}


def _oracle_image_all_r(img):
    """One image of the workload through the exact-integer oracle at every r
    (a worker of cpu_baseline_all_cores)."""
    import oracle as O

    for r in R_SWEEP:
        O.compress_zonal_exact(img, r)
    return img.size * len(R_SWEEP)


def cpu_baseline_all_cores(batch):
    """The same oracle over the whole step (64 images x 8 r) with one process
    per host core (spawned, each single-threaded), images distributed across
    them: the oracle itself is unchanged."""
    import multiprocessing as mp

    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_image_all_r, [batch[0]] * cores)  # start-up outside the timing
        t0 = time.perf_counter()
        px = sum(pool.imap_unordered(_oracle_image_all_r, list(batch)))
        dt = time.perf_counter() - t0
    return {"value": px / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"all {len(batch)} images x 8 r ({px / 1e6:.1f} Mpx), one spawned process per core, {dt:.1f} s"}


def run_reference(args):
    """The CPU oracle on the same metric: each step compresses a strip of one
    512x512 image at all eight r, the strip height chosen so that the whole
    --steps/--warmup run stays within about two minutes."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1606_05562_gb300 import synth

    import oracle as O

    img = synth.ar1_image(SIDE, SIDE, 0.95, 100)
    t0 = time.perf_counter()
    for r in R_SWEEP:
        O.compress_zonal_exact(img[:16], r)
    per_row_s = (time.perf_counter() - t0) / 16
    budget = 120.0 / max(1, args.steps + max(args.warmup, 0))
    rows = int(min(SIDE, max(16, (budget / max(per_row_s, 1e-9)) // 16 * 16)))
    strip = img[:rows]
    px_step = strip.size * len(R_SWEEP)

    def step():
        for r in R_SWEEP:
            O.compress_zonal_exact(strip, r)

    for _ in range(max(args.warmup, 0)):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = px_step * args.steps / dt / 1e9
    sample = f"{rows}x{SIDE} strip of one AR(1) image x 8 r per step ({px_step / 1e6:.2f} Mpx), exact-integer oracle"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "impl": "reference",
        "config": {"workload": WORKLOAD, "sample_per_step": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
def residual_sequence(synth, n_frames):
    """Frames 0 .. n_frames - 1 of the 4:2:0 int16 residual sequence, drawn in
    spawned processes (one per host core; no GPU work has to be inherited)."""
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    with ctx.Pool(max(1, min(os.cpu_count() or 1, 16))) as pool:
        return pool.map(synth.residual_frame, range(n_frames), chunksize=2)


def transform_matrix(torch, atdct16, dev):
    """T of the library (its 1-D forward of the 16 unit vectors), FP64."""
    plan = atdct16.Plan(atdct16.I16, max_images=1)
    eye = torch.eye(16, dtype=torch.int16, device=dev).contiguous()
    coef = torch.empty(256, dtype=torch.int32, device=dev)
    plan.forward_1d(eye, coef, dtype=atdct16.I16)
    torch.cuda.synchronize()
    plan.close()
    return coef.view(16, 16).t().to(torch.float64).contiguous()  # T[u, k]: column k = T e_k


def quant_phase(torch, atdct16, synth, dev, n_frames, chunk, steps, warmup, peak_gbs, cpu_oracle=False):
    """The video-residual workload: n_frames 4:2:0 int16 frames (1920x1088
    luma + two 960x544 chroma planes, Laplace(0, 6) with 30 % zeros, seed 3),
    every plane quantised at each QP in {22, 27, 32, 37}, streamed through
    the GPU in chunks of `chunk` frames (one call per chunk covers its planes
    at all four QP, one input copy per QP).  Reports the throughput over the
    whole run and the HBM fraction of the quantisation kernel (4 bytes per
    sample: int16 in, int16 out), the level-output variants (+2 bytes per
    sample, row-major and zig-zag) on the first chunk, and per QP the error of
    the FP32 path against the FP64 definition (level flips, PSNR, int16
    planes), computed from the library's exact integer coefficients."""
    import numpy as np

    t_gen = time.perf_counter()
    frames = residual_sequence(synth, n_frames)
    gen_s = time.perf_counter() - t_gen
    qps = synth.QUANT_QP_SWEEP
    nq = len(qps)
    per_chunk = 3 * chunk
    rplan = atdct16.Plan(atdct16.I16, max_images=per_chunk * nq, workspace_bytes=1 << 30)
    zplan = atdct16.Plan(atdct16.I16, max_images=per_chunk * nq, workspace_bytes=1 << 30, zigzag=True)
    tmat = transform_matrix(torch, atdct16, dev)
    nnz = (tmat != 0).sum(dim=1).to(torch.float64)  # non-zeros per row of T
    sq = 1.0 / torch.sqrt(nnz[:, None] * nnz[None, :])   # s_u s_v
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tot_ms = tot_kms = 0.0
    tot_samples = 0
    kms_all = []
    variants = {}
    prec = {qp: {"coefficients": 0, "level_flips_vs_fp64": 0, "max_level_diff": 0, "psnr_rel_err_vs_fp64": 0.0,
                 "max_abs_recon_err_vs_fp64": 0.0, "psnr": [], "snr": []} for qp in qps}
    for c0 in range(0, n_frames, chunk):
        fr = frames[c0:c0 + chunk]
        planes_h = [p for f in fr for p in f]
        planes = [torch.from_numpy(p).to(dev) for p in planes_h]
        ins = [[p.clone() for p in planes] for _ in qps]
        outs = [[torch.empty_like(p) for p in planes] for _ in qps]
        descs = atdct16.descriptors([atdct16.image(p, o, qp) for qp, ii, oo in zip(qps, ins, outs)
                                     for p, o in zip(ii, oo)])
        samples = sum(p.numel() for p in planes) * nq
        psnr = torch.empty(len(descs), dtype=torch.float64, device=dev)
        sse = torch.empty(len(descs), dtype=torch.float64, device=dev)
        levels = torch.empty(samples, dtype=torch.int16, device=dev)
        tags = (("no_levels", None, rplan), ("levels", levels, rplan), ("levels_zigzag", levels, zplan)) \
            if c0 == 0 else (("no_levels", None, rplan),)
        for tag, lv, plan in tags:
            for _ in range(max(warmup, 1 if c0 else 3)):
                plan.compress_quant(descs, psnr, levels=lv)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(steps):
                plan.compress_quant(descs, psnr, levels=lv)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            # the kernel alone: an event pair around each of a few further calls
            plan.set_profiling(True, every=1)
            plan.profile()
            ks = []
            for _ in range(3):
                plan.compress_quant(descs, psnr, levels=lv)
                torch.cuda.synchronize()
                n, kms = plan.profile()
                ks.append(kms / max(n, 1))
            plan.set_profiling(False)
            k = statistics.median(ks)
            if tag == "no_levels":
                tot_ms += ms
                tot_kms += k
                tot_samples += samples
                kms_all.extend(ks)
            if c0 == 0:
                byts = samples * (6 if lv is not None else 4)
                variants[tag] = {"ms_per_call": ms, "kernel_ms": k, "gsamples_s": samples / (ms / 1e3) / 1e9,
                                 "kernel_gbs": byts / (k / 1e3) / 1e9,
                                 "kernel_frac_hbm": byts / (k / 1e3) / 1e9 / peak_gbs}
        # FP32 path against the FP64 definition, from the library's exact coefficients
        rplan.compress_quant(descs, psnr, levels=levels, sse=sse)
        coef = torch.empty(samples // nq, dtype=torch.int32, device=dev)
        off = 0
        for p in planes:
            rplan.forward(p, coef[off:off + p.numel()], dtype=atdct16.I16)
            off += p.numel()
        torch.cuda.synchronize()
        y = coef.to(torch.float64).view(-1, 16, 16)
        energy = [float((p.to(torch.float64) ** 2).sum()) for p in planes]
        for q, qp in enumerate(qps):
            qs = 2.0 ** (qp / 6.0)
            den = torch.sqrt(nnz[:, None] * nnz[None, :] * 2.0 ** (qp / 3.0))
            l64 = torch.sign(y) * torch.floor(y.abs() / den + 0.5)
            lg = levels[q * (samples // nq):(q + 1) * (samples // nq)].to(torch.float64).view(-1, 16, 16)
            d = (lg - l64).abs()
            r = prec[qp]
            r["coefficients"] += int(y.shape[0]) * 256
            r["level_flips_vs_fp64"] += int((d != 0).sum())
            r["max_level_diff"] = max(r["max_level_diff"], int(d.max()))
            rec = torch.einsum("um,buv,vn->bmn", tmat, l64 * sq * qs, tmat)  # T^T (S B' S) T
            err2 = (y * sq - l64 * qs) ** 2  # Parseval: (B - B')^2
            boff = 0
            for i, p in enumerate(planes):
                h, w = p.shape
                nb = (h // 16) * (w // 16)
                s64 = float(err2[boff:boff + nb].sum())
                p64 = 10.0 * math.log10(255.0 ** 2 * h * w / s64) if s64 > 0 else float("inf")
                k = q * len(planes) + i
                pg = float(psnr[k])
                r["psnr_rel_err_vs_fp64"] = max(r["psnr_rel_err_vs_fp64"], abs(pg - p64) / abs(p64))
                r["psnr"].append(pg)
                r["snr"].append(10.0 * math.log10(energy[i] / float(sse[k])))
                og = outs[q][i].to(torch.float64).view(h // 16, 16, w // 16, 16).permute(0, 2, 1, 3).reshape(-1, 16, 16)
                r["max_abs_recon_err_vs_fp64"] = max(r["max_abs_recon_err_vs_fp64"],
                                                     float((og - rec[boff:boff + nb]).abs().max()))
                boff += nb
            del l64, lg, d, rec, err2
        del planes, ins, outs, levels, coef, y
        torch.cuda.empty_cache()
    by_qp = {}
    for qp in qps:
        r = prec[qp]
        by_qp[str(qp)] = {"mean_psnr_db": sum(r["psnr"]) / len(r["psnr"]),
                          "mean_residual_snr_db": sum(r["snr"]) / len(r["snr"]),
                          "coefficients": r["coefficients"],
                          "level_flips_vs_fp64": r["level_flips_vs_fp64"],
                          "level_flip_fraction_vs_fp64": r["level_flips_vs_fp64"] / r["coefficients"],
                          "max_level_diff_vs_fp64": r["max_level_diff"],
                          "psnr_rel_err_vs_fp64": r["psnr_rel_err_vs_fp64"],
                          "max_abs_recon_err_vs_fp64": r["max_abs_recon_err_vs_fp64"]}
    res = {"frames": n_frames, "chunk_frames": chunk, "chunks": (n_frames + chunk - 1) // chunk,
           "qps": list(qps), "samples": tot_samples, "steps_per_chunk": steps, "generate_s": gen_s,
           "ms_total": tot_ms, "gsamples_s": tot_samples / (tot_ms / 1e3) / 1e9,
           "kernel_ms_total": tot_kms, "kernel_gbs": 4.0 * tot_samples / (tot_kms / 1e3) / 1e9,
           "kernel_frac_hbm": 4.0 * tot_samples / (tot_kms / 1e3) / 1e9 / peak_gbs,
           "first_chunk": variants, "by_qp": by_qp,
           "precision_note": "FP64 definition from the library's exact int32 coefficients; all planes of all chunks"}
    if cpu_oracle:
        # the oracle (FP32-decision mode) on one 1920x1088 luma plane at QP 27
        import oracle as O

        t0 = time.perf_counter()
        O.compress_quant(frames[0][0], 27, precision="fp32")
        dt = time.perf_counter() - t0
        res["cpu_oracle"] = {"gsamples_s": frames[0][0].size / dt / 1e9, "cores": 1,
                             "sample": "one 1920x1088 luma plane at QP 27, FP32-decision oracle"}
    rplan.close()
    zplan.close()
    return res


# --------------------------------------------------------------------------
def general_variants_phase(torch, atdct16, batch, dev, reps=100):
    """The general zonal kernel's variants on the r > 36 half of the bench
    workload (the 64 images x r in {64, 100, 150, 256}: 256 jobs, 32768
    tiles, 134 MB moved per launch), each pinned through the batch API:
    integer-pipe forward (int16 SWAR, the default), FP32 column pass, the
    forward as mma.sync f16 products, and as tcgen05 products with TMEM
    accumulators.  Time per launch of the batch (kernel + PSNR finalize),
    and whether every variant stored the same pixels as the default."""
    R = (64, 100, 150, 256)
    base = torch.from_numpy(batch).to(dev)
    src = base.unsqueeze(0).repeat(len(R), 1, 1, 1).contiguous()
    dst = torch.empty_like(src)
    ref = None
    plan = atdct16.Plan(atdct16.U8, max_images=len(R) * base.shape[0])
    psnr = torch.empty(len(R) * base.shape[0], dtype=torch.float64, device=dev)
    descs = [atdct16.image(src[k, i], dst[k, i], r) for k, r in enumerate(R) for i in range(base.shape[0])]
    out = {"r": list(R), "tiles": None, "us_per_launch": {}, "identical_pixels": True}
    for v in (1, 0, 2, 3):
        dst.fill_(7)
        b = atdct16.Batch(plan, descs, psnr, flags=atdct16.batch_variant(v))
        out["tiles"] = b.info()["tiles"]
        for _ in range(5):
            b.launch()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            b.launch()
        e1.record()
        torch.cuda.synchronize()
        out["us_per_launch"][atdct16.ZONAL_VARIANTS[v]] = e0.elapsed_time(e1) / reps * 1e3
        if b.last_device_status() != atdct16.OK:
            raise RuntimeError(f"zonal variant {v}: device status {b.last_device_status()}")
        b.close()
        if ref is None:
            ref = dst.clone()
        elif not torch.equal(dst, ref):
            out["identical_pixels"] = False
    plan.close()
    return out


def coef_phase(torch, atdct16, batch, dev, peak_gbs, reps=50):
    """The standalone coefficient pipeline on one 4096 x 8192 u8 image (the
    64 bench images tiled 8 x 8, beside its mirror image; 33.5 Mpx): 2-D
    forward and exact inverse with row-major and zig-zag block layouts, and
    the 1-D forward / inverse of the same bytes as 16-sample vectors.  Two
    rotating input / coefficient / output sets; every call moves 168 MB
    (> L2).  Algorithmic bytes: 1 per pixel plus 4 per coefficient.  Each
    inverse must reproduce its forward's input exactly (checked)."""
    import numpy as np

    n, side = batch.shape[0], batch.shape[1]
    g = int(round(math.sqrt(n)))
    grid = batch[: g * g].reshape(g, g, side, side).transpose(0, 2, 1, 3).reshape(g * side, g * side)
    img = torch.from_numpy(np.ascontiguousarray(np.concatenate([grid, grid[:, ::-1]], axis=1))).to(dev)
    h, w = img.shape
    px = h * w
    ins = [img, torch.flip(img, dims=[0]).contiguous()]
    coef = [torch.empty(px, dtype=torch.int32, device=dev) for _ in range(2)]
    outs = [torch.empty_like(img) for _ in range(2)]
    byts = 5.0 * px
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for k in range(4):
            fn(k)
        torch.cuda.synchronize()
        e0.record()
        for k in range(reps):
            fn(k)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        gbs = byts / (ms / 1e3) / 1e9
        return {"ms": ms, "gpx_s": px / (ms / 1e3) / 1e9, "gbs": gbs, "frac_hbm": gbs / peak_gbs}

    res = {"image": f"{h}x{w} u8", "pixels": px, "bytes_per_call": byts, "reps": reps}
    exact = True
    for zig in (False, True):
        plan = atdct16.Plan(atdct16.U8, max_images=1, zigzag=zig)
        tag = "zigzag" if zig else "rowmajor"
        res["forward_2d_" + tag] = timed(lambda k: plan.forward(ins[k % 2], coef[k % 2]))
        res["inverse_2d_" + tag] = timed(lambda k: plan.inverse(coef[k % 2], outs[k % 2]))
        torch.cuda.synchronize()
        exact = exact and all(torch.equal(o, i) for o, i in zip(outs, ins))
        if not zig:
            res["forward_1d"] = timed(lambda k: plan.forward_1d(ins[k % 2], coef[k % 2]))
            res["inverse_1d"] = timed(lambda k: plan.inverse_1d(coef[k % 2], outs[k % 2]))
            torch.cuda.synchronize()
            exact = exact and all(torch.equal(o, i) for o, i in zip(outs, ins))
        if plan.last_device_status() != atdct16.OK:
            raise RuntimeError("device-side status error in the coefficient phase")
        plan.close()
    res["round_trips_exact"] = bool(exact)
    return res


# --------------------------------------------------------------------------
def _percentiles(v):
    v = sorted(v)
    q = lambda f: v[min(len(v) - 1, int(round(f * (len(v) - 1))))]
    return {"p10": q(0.1), "p50": q(0.5), "p90": q(0.9)}


def config1_phase(torch, atdct16, synth, dev, reps=200):
    """One 256 x 256 u8 image (256 blocks): per-call latency of the forward to
    int32 coefficients, the exact inverse and the fused zonal path (r = 36),
    from CUDA events around each call; the round trip must be exact."""
    img = synth.single_image_256()
    x = torch.from_numpy(img).to(dev)
    coef = torch.empty(img.size, dtype=torch.int32, device=dev)
    out = torch.empty_like(x)
    rec = torch.empty_like(x)
    psnr = torch.empty(1, dtype=torch.float64, device=dev)
    plan = atdct16.Plan(atdct16.U8, max_images=1)
    desc = atdct16.descriptors([atdct16.image(x, rec, 36)])
    calls = {"forward_us": lambda: plan.forward(x, coef), "inverse_us": lambda: plan.inverse(coef, out),
             "zonal_r36_us": lambda: plan.compress_zonal(desc, psnr)}
    res = {"image": "256x256 u8", "reps": reps}
    for name, fn in calls.items():
        for _ in range(5):
            fn()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for a, b in ev:
            a.record()
            fn()
            b.record()
        torch.cuda.synchronize()
        res[name] = _percentiles([a.elapsed_time(b) * 1e3 for a, b in ev])
    res["round_trip_exact"] = bool(torch.equal(out, x))
    plan.close()
    return res


def psnr_u8_by_r(torch, atdct16, src, dst):
    """PSNR of the stored u8 reconstructions (atdct16_psnr per image), mean per r."""
    nr, n = src.shape[0], src.shape[1]
    out = torch.empty(nr * n, dtype=torch.float64, device=src.device)
    for k in range(nr):
        for i in range(n):
            atdct16.psnr(src[k, i], dst[k, i], out[k * n + i:k * n + i + 1])
    torch.cuda.synchronize()
    per = out.view(nr, n)
    return {str(r): (float(per[k][~per[k].isinf()].mean()) if bool((~per[k].isinf()).any()) else float("inf"))
            for k, r in enumerate(R_SWEEP)}


# --------------------------------------------------------------------------
def ssim_phase(torch, atdct16, plan, descs, n_jobs, px, reps=5):
    """SSIM (Sec. 4) of every reconstruction of one bench step against its
    original, through atdct16_ssim_batch: time per batch and the mean MSSIM
    per zonal r."""
    out = torch.empty(n_jobs, dtype=torch.float64, device="cuda")
    plan.ssim(descs, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        plan.ssim(descs, out)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    per_r = out.view(len(R_SWEEP), -1).mean(dim=1).tolist()
    return {"images": n_jobs, "ms_per_batch": ms, "gpx_s": px / (ms / 1e3) / 1e9,
            "mean_mssim_by_r": {str(r): v for r, v in zip(R_SWEEP, per_r)}}


# --------------------------------------------------------------------------
def dct_baseline_phase(torch, atdct16, plan, sets, n_jobs, px, psnr_approx, steps=200):
    """The exact-DCT baseline (dense FP32 DCT-II through the same zonal
    procedure) on the bench workload: throughput against the multiplierless
    kernel, and the APE (Sec. 4) of the approximation's mean PSNR and MSSIM
    per r with respect to the exact DCT's."""
    psnr = torch.empty(n_jobs, dtype=torch.float64, device="cuda")
    for w in range(3):
        plan.compress_zonal_dct(sets[w % len(sets)][2], psnr)
    torch.cuda.synchronize()
    plan.set_profiling(True)
    plan.profile()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for k in range(steps):
        plan.compress_zonal_dct(sets[k % len(sets)][2], psnr)
    e1.record()
    torch.cuda.synchronize()
    n, kms = plan.profile()
    plan.set_profiling(False)
    ms = e0.elapsed_time(e1) / steps
    # quality: the last call wrote set (steps - 1) % 3; compare on that set
    last = sets[(steps - 1) % len(sets)][2]
    dct_psnr = psnr.clone()
    ssim_dct = torch.empty(n_jobs, dtype=torch.float64, device="cuda")
    plan.ssim(last, ssim_dct)
    approx_psnr = torch.empty(n_jobs, dtype=torch.float64, device="cuda")
    plan.compress_zonal(last, approx_psnr)
    ssim_approx = torch.empty(n_jobs, dtype=torch.float64, device="cuda")
    plan.ssim(last, ssim_approx)
    torch.cuda.synchronize()
    nr = len(R_SWEEP)
    ape = {}
    for k, r in enumerate(R_SWEEP):
        sl = slice(k * n_jobs // nr, (k + 1) * n_jobs // nr)
        pa, pd = approx_psnr[sl], dct_psnr[sl]
        fin = ~(pa.isinf() | pd.isinf())
        mp_a = float(pa[fin].mean()) if bool(fin.any()) else float("inf")
        mp_d = float(pd[fin].mean()) if bool(fin.any()) else float("inf")
        ms_a, ms_d = float(ssim_approx[sl].mean()), float(ssim_dct[sl].mean())
        ape[str(r)] = {"mean_psnr_approx": mp_a, "mean_psnr_dct": mp_d,
                       "ape_psnr_pct": 100.0 * abs(mp_a - mp_d) / mp_d if math.isfinite(mp_d) else 0.0,
                       "mean_mssim_approx": ms_a, "mean_mssim_dct": ms_d,
                       "ape_mssim_pct": 100.0 * abs(ms_a - ms_d) / ms_d}
    return {"ms_per_step": ms, "kernel_ms": kms / max(n, 1), "gpx_s": px / (ms / 1e3) / 1e9,
            "kernel_gbs": 2 * px / (kms / max(n, 1) / 1e3) / 1e9, "ape_by_r": ape}


# --------------------------------------------------------------------------
def mixed_batch_phase(torch, atdct16, synth, dev, n_images, seed=4, cpu_oracle=False):
    """1000 mixed-size u8 AR(1) images (sides log-uniform in [128, 4096],
    multiples of 16, rho in [0.8, 0.97]), zonal r = 36: per-image launches of
    the plain entry point against one autotuned CUDA-graph launch of the
    whole batch.  Images are crops of four seeded 4096x4096 AR(1) fields
    (one rho each), copied into distinct device buffers."""
    import numpy as np

    rhos = (0.8, 0.85, 0.9, 0.97)
    fields = [torch.from_numpy(synth.ar1_image(4096, 4096, rho, seed * 1000 + k)).to(dev) for k, rho in enumerate(rhos)]
    sizes = synth.mixed_sizes(n_images, 128, 4096, seed + 7)
    rng = np.random.default_rng(seed)
    total = sum(h * w for h, w in sizes)
    src_all = torch.empty(total, dtype=torch.uint8, device=dev)
    dst_a = torch.empty_like(src_all)
    dst_b = torch.empty_like(src_all)
    srcs, da, db = [], [], []
    off = 0
    for i, (h, w) in enumerate(sizes):
        f = fields[i % 4]
        y0 = int(rng.integers(0, 4096 - h + 1)) // 16 * 16
        x0 = int(rng.integers(0, 4096 - w + 1)) // 16 * 16
        s = src_all[off:off + h * w].view(h, w)
        s.copy_(f[y0:y0 + h, x0:x0 + w])
        srcs.append(s)
        da.append(dst_a[off:off + h * w].view(h, w))
        db.append(dst_b[off:off + h * w].view(h, w))
        off += h * w
    r = 36
    plan1 = atdct16.Plan(atdct16.U8, max_images=1)
    p1 = torch.empty(n_images, dtype=torch.float64, device=dev)
    descs_a = [atdct16.image(s, d, r) for s, d in zip(srcs, da)]

    def per_image():
        for i, d in enumerate(descs_a):
            plan1.compress_zonal([d], p1[i:i + 1])

    per_image()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    per_image()
    e1.record()
    torch.cuda.synchronize()
    ms_a = e0.elapsed_time(e1)
    planb = atdct16.Plan(atdct16.U8, max_images=n_images, workspace_bytes=1 << 30)
    p2 = torch.empty(n_images, dtype=torch.float64, device=dev)
    t0 = time.perf_counter()
    batch = atdct16.Batch(planb, [atdct16.image(s, d, r) for s, d in zip(srcs, db)], p2,
                          flags=atdct16.BATCH_AUTOTUNE | atdct16.BATCH_GRAPH)
    tune_s = time.perf_counter() - t0
    batch.launch()
    torch.cuda.synchronize()
    reps = 10
    e0.record()
    for _ in range(reps):
        batch.launch()
    e1.record()
    torch.cuda.synchronize()
    ms_b = e0.elapsed_time(e1) / reps
    same = bool(torch.equal(dst_a, dst_b)) and bool(torch.equal(p1.isinf(), p2.isinf()))
    fin = ~p1.isinf()
    same = same and bool(torch.equal(p1[fin], p2[fin]))
    info = batch.info()
    tuning = batch.tuning()
    batch.close()
    out = {"images": n_images, "pixels": int(total), "r": r,
           "per_image_launches_gpx_s": total / (ms_a / 1e3) / 1e9,
           "graph_batch_gpx_s": total / (ms_b / 1e3) / 1e9,
           "graph_batch_gbs": 2.0 * total / (ms_b / 1e3) / 1e9,
           "speedup": ms_a / ms_b, "identical_results": same, "autotune_s": tune_s, "tuned": info,
           "tuning": {"chosen": tuning["chosen"], "candidates": len(tuning["candidates"]),
                      "candidate_ms": {"min": min(c["ms"] for c in tuning["candidates"]),
                                       "median": statistics.median(c["ms"] for c in tuning["candidates"]),
                                       "max": max(c["ms"] for c in tuning["candidates"])},
                      # tiles per CTA, staging depth, vector bytes, CTAs per SM (0: max), phase, variant: ms
                      "table": [[c["tiles_per_cta"], c["staging_depth"], c["vector_bytes"], c["box_ctas"],
                                 c["phase"], c["variant"], c["general_ctas"], round(c["ms"], 4)]
                                for c in tuning["candidates"]]}}
    if cpu_oracle:
        # the exact-integer oracle on the first images of the set, up to about 8 Mpx
        import oracle as O

        t0, px = time.perf_counter(), 0
        for s_img in srcs:
            if px > 8_000_000:
                break
            O.compress_zonal_exact(s_img.cpu().numpy(), r)
            px += s_img.numel()
        dt = time.perf_counter() - t0
        out["cpu_oracle"] = {"gpx_s": px / dt / 1e9, "cores": 1, "sample": f"first images of the set, {px / 1e6:.1f} Mpx"}
    del fields, src_all, dst_a, dst_b
    return out


SERVE_STAGES = ("queue", "h2d", "slot_wait", "compute", "d2h", "notice")


def serve_counts(rates, total):
    """Requests per rate: `total` split in proportion to sqrt(rate), so that
    the low rates keep enough samples for a p99 without running for minutes."""
    w = [math.sqrt(r) for r in rates]
    n = [int(round(total * x / sum(w))) for x in w]
    n[-1] += total - sum(n)
    return n


def serving_phase(torch, atdct16, synth, rates, total, seed=5):
    """Config 5: `total` requests in all, Poisson arrivals at each rate of the
    sweep (requests split across the rates by serve_counts); uint8 requests
    with sides log-uniform in [64, 8192] (multiples of 16) cut from a seeded
    8192 x 8192 AR(1) field in pinned host memory, r uniform in {6, 16, 36,
    64}; 40 GB device arena.  Latency runs from each request's scheduled
    arrival to its completion.  Per request the stages on the server's clock
    give where the time went: queue (arrival to the start of its upload:
    admission under the memory budget and the copy engine's backlog), h2d (its
    upload), slot_wait (upload end to the start of its launch), compute (the
    fused launch it rode in), d2h (to the end of its download) and notice
    (until the scheduler saw it complete)."""
    import threading

    import numpy as np

    field = torch.from_numpy(synth.ar1_image(8192, 8192, 0.95, seed * 1000)).pin_memory()
    ring_bytes = 1 << 31
    ring = torch.empty(ring_bytes, dtype=torch.uint8).pin_memory()
    srv = atdct16.Server(memory_budget_bytes=40 << 30, max_batch=64, compute_slots=3)
    results = []
    for rate, n in zip(rates, serve_counts(rates, total)):
        rng = np.random.default_rng(seed + int(rate))
        sizes = synth.mixed_sizes(n, 64, 8192, seed * 31 + int(rate))
        rs = rng.choice((6, 16, 36, 64), size=n)
        arrivals = synth.poisson_arrivals(n, rate, seed * 17 + int(rate))
        tim = [None] * n
        tickets = [None] * n
        done_upto = [0]
        cv = threading.Condition()

        def collector():
            for i in range(n):
                with cv:
                    while tickets[i] is None:
                        cv.wait()
                _, t = srv.wait_timing(tickets[i])
                tim[i] = t
                with cv:
                    done_upto[0] = i + 1
                    cv.notify_all()

        th = threading.Thread(target=collector)
        th.start()
        ring_pos, slices = 0, []
        t0 = atdct16.server_clock() + 0.05
        for i in range(n):
            h, w = sizes[i]
            y0 = int(rng.integers(0, 8192 - h + 1)) // 16 * 16
            x0 = int(rng.integers(0, 8192 - w + 1)) // 16 * 16
            if ring_pos + h * w > ring_bytes:
                ring_pos = 0
            # do not overwrite an output slice still in flight
            while slices and any(s0 < ring_pos + h * w and ring_pos < s1 and k >= done_upto[0]
                                 for (s0, s1, k) in slices[-64:]):
                with cv:
                    cv.wait(timeout=0.01)
            dst = ring[ring_pos:ring_pos + h * w].view(h, w)
            slices.append((ring_pos, ring_pos + h * w, i))
            ring_pos += h * w
            src = field[y0:y0 + h, x0:x0 + w]
            t_arr = t0 + float(arrivals[i])
            delay = t_arr - atdct16.server_clock()
            if delay > 0:
                time.sleep(delay)
            t = srv.submit(src, dst, int(rs[i]), arrival=t_arr)
            with cv:
                tickets[i] = t
                cv.notify_all()
        th.join()
        t_end = max(x["done"] for x in tim)
        lat = np.array([x["done"] - x["arrival"] for x in tim]) * 1e3
        stages = {
            "queue": [x["h2d_start"] - x["arrival"] for x in tim],
            "h2d": [x["h2d_end"] - x["h2d_start"] for x in tim],
            "slot_wait": [x["compute_start"] - x["h2d_end"] for x in tim],
            "compute": [x["compute_end"] - x["compute_start"] for x in tim],
            "d2h": [x["d2h_end"] - x["compute_end"] for x in tim],
            "notice": [x["done"] - x["d2h_end"] for x in tim],
        }
        st_ms = {k: np.array(v) * 1e3 for k, v in stages.items()}
        tail = lat >= np.percentile(lat, 99)
        px = sum(h * w for h, w in sizes)
        results.append({
            "rate": rate, "requests": n, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "achieved_req_s": n / (t_end - t0), "gpx_s": px / (t_end - t0) / 1e9, "pixels": int(px),
            "stages_p50_ms": {k: float(np.percentile(v, 50)) for k, v in st_ms.items()},
            "stages_p99_ms": {k: float(np.percentile(v, 99)) for k, v in st_ms.items()},
            # where the slowest 1 % of requests spent their time (mean per stage)
            "p99_tail_breakdown_ms": {k: float(v[tail].mean()) for k, v in st_ms.items()},
            "p99_tail_mean_mpx": float(np.mean([sizes[i][0] * sizes[i][1] for i in np.nonzero(tail)[0]]) / 1e6)})
    st = srv.stats()
    srv.close()
    return {"rates": results, "requests": sum(r["requests"] for r in results), "launches": st["launches"],
            "arena_gb": 40, "stages": list(SERVE_STAGES),
            "note": "latency = scheduled Poisson arrival to completion; H2D and D2H of the request included"}


def serving_in_own_process(args):
    """The serving phase in a fresh process (`--serve-only`), as a server runs:
    its pinned buffers and device arena are allocated in a process that has not
    run the other phases."""
    cmd = [sys.executable, os.path.abspath(__file__), "--serve-only", "--serve-rates", args.serve_rates,
           "--serve-requests", str(args.serve_requests)]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=900)
    if r.returncode != 0:
        raise RuntimeError("serving phase failed: " + r.stderr[-2000:])
    res = json.loads(r.stdout.strip().splitlines()[-1])["serving"]
    res["process"] = "own process (bench.py --serve-only)"
    return res


# --------------------------------------------------------------------------
def run_ours(args):
    import torch

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_1606_05562_gb300 import atdct16, synth
    from paper_1606_05562_gb300 import build as b

    b.build()
    # Config 5 first, in its own process, before this process holds any device
    # or pinned host buffers (a server process starts on a quiet GPU: after the
    # other phases, with their buffers still held by this process, the serving
    # loop's large downloads ran several times slower).
    serving = {"skipped": "measured at N = 1"}
    if world == 1 and not args.no_extras:
        try:
            serving = serving_in_own_process(args)
        except Exception as e:  # noqa: BLE001 - reported in the line
            serving = {"error": f"{type(e).__name__}: {e}"[:500]}
    n_img = args.images
    batch = synth.image_batch_512(n_img * world, SIDE, first_seed=100, indices=rank_images(world, rank, n_per_rank=n_img))
    nr = len(R_SWEEP)
    jobs = nr * n_img
    px_step = jobs * SIDE * SIDE

    # rotating sets of inputs (one copy per r) and outputs, > 4 x L2 in total
    base = torch.from_numpy(batch).to(dev)
    sets = []
    for _ in range(N_SETS):
        src = base.unsqueeze(0).repeat(nr, 1, 1, 1).contiguous()
        dst = torch.empty_like(src)
        descs = atdct16.descriptors(
            [atdct16.image(src[k, i], dst[k, i], r) for k, r in enumerate(R_SWEEP) for i in range(n_img)])
        sets.append((src, dst, descs))
    plan = atdct16.Plan(atdct16.U8, max_images=jobs)
    psnr = torch.empty(jobs, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    def barrier():
        if dist:
            dist.barrier()

    for w in range(max(args.warmup, 3)):
        plan.compress_zonal(sets[w % N_SETS][2], psnr)
    torch.cuda.synchronize()
    gpu_id = "0"
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = ClockSampler(gpu_id)
    barrier()
    clocks.start()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        plan.compress_zonal(sets[k % N_SETS][2], psnr)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    # the fused kernels' duration per call: PROF_CALLS further calls, each
    # with a CUDA-event pair around the fused kernel launches only (the plan's
    # profiling hook; an event between them and the PSNR finalize keeps the
    # finalize from overlapping their last CTAs), on the launching stream
    plan.set_profiling(True, every=1)
    plan.profile()
    kern = []
    for k in range(PROF_CALLS):
        plan.compress_zonal(sets[k % N_SETS][2], psnr)
        torch.cuda.synchronize()
        n_l, k_ms = plan.profile()
        kern.append(k_ms / max(n_l, 1))
    plan.set_profiling(False)
    kernel_pct = _percentiles(kern)
    # spread of the step time: 200 more steps with an event pair around each
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(200)]
    for k, (a, b) in enumerate(evs):
        a.record(stream)
        plan.compress_zonal(sets[k % N_SETS][2], psnr)
        b.record(stream)
    torch.cuda.synchronize()
    step_pct = _percentiles([a.elapsed_time(b) for a, b in evs])
    if dist:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * px_step / (ms / 1e3) / 1e9
    if plan.last_device_status() != atdct16.OK:
        raise RuntimeError("device-side status error during the bench")

    # roofline of the fused kernel: algorithmic bytes = 1 B in + 1 B out per
    # pixel, the per-tile FP32 partials and the job descriptors
    tiles = jobs * (SIDE // 16) * ((SIDE + 127) // 128)
    algo_bytes = 2.0 * px_step + 4.0 * tiles + 64.0 * jobs
    k_s = kernel_pct["p50"] / 1e3
    if kernel_pct["p50"] > ms:
        raise RuntimeError(f"fused kernel time {kernel_pct['p50']:.4f} ms exceeds the step time {ms:.4f} ms")
    peak, peak_src = measured_peak_hbm()
    achieved = algo_bytes / k_s / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": recorded_traffic(), "peak_source": peak_src, "kernel": "zonal fused kernels",
            "kernel_ms": kernel_pct["p50"], "kernel_ms_percentiles": kernel_pct,
            "kernel_launches_timed": len(kern), "algorithmic_bytes_per_launch": algo_bytes}

    # end to end through the public API with host buffers.  Every step: the H2D
    # copy of its 64 source images from pinned memory, the 512-job call, and the
    # D2H copy of all its reconstructions and PSNRs into pinned memory.  Two steps
    # are in flight: step k's results go back over the host link while step k+1
    # uploads and computes (separate copy streams, double-buffered device and host
    # buffers, ordered by events).  The serial figure (one step at a time on one
    # stream) and a PSNR-only readback are reported beside it.
    h_src = torch.from_numpy(batch).pin_memory()
    d_src2 = [torch.empty_like(base) for _ in range(2)]
    d_dst2 = [torch.empty((nr, n_img, SIDE, SIDE), dtype=torch.uint8, device=dev) for _ in range(2)]
    h_dst2 = [torch.empty(d_dst2[0].shape, dtype=torch.uint8).pin_memory() for _ in range(2)]
    psnr2 = [torch.empty(jobs, dtype=torch.float64, device=dev) for _ in range(2)]
    h_psnr2 = [torch.empty(jobs, dtype=torch.float64).pin_memory() for _ in range(2)]
    descs2 = [atdct16.descriptors([atdct16.image(d_src2[b][i], d_dst2[b][k, i], r)
                                   for k, r in enumerate(R_SWEEP) for i in range(n_img)]) for b in range(2)]
    s_in, s_cmp, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_cmp = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]

    def e2e_step(k, pipelined=True, images_back=True):
        b = k & 1 if pipelined else 0
        si, sc, so = (s_in, s_cmp, s_out) if pipelined else (stream, stream, stream)
        si.wait_event(ev_cmp[b])  # step k - 2's kernel has read d_src2[b]
        with torch.cuda.stream(si):
            d_src2[b].copy_(h_src, non_blocking=True)
        ev_in[b].record(si)
        sc.wait_event(ev_in[b])
        sc.wait_event(ev_out[b])  # step k - 2's results have left d_dst2[b] / psnr2[b]
        plan.compress_zonal(descs2[b], psnr2[b], stream=sc)
        ev_cmp[b].record(sc)
        so.wait_event(ev_cmp[b])
        with torch.cuda.stream(so):
            if images_back:
                h_dst2[b].copy_(d_dst2[b], non_blocking=True)
            h_psnr2[b].copy_(psnr2[b], non_blocking=True)
        ev_out[b].record(so)

    def e2e_run(pipelined, images_back=True):
        for k in range(3):
            e2e_step(k, pipelined, images_back)
        torch.cuda.synchronize()
        barrier()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(s_in if pipelined else stream)
        for k in range(args.e2e_steps):
            e2e_step(k, pipelined, images_back)
        t1.record(s_out if pipelined else stream)
        torch.cuda.synchronize()
        e_ms = t0.elapsed_time(t1) / args.e2e_steps
        if dist:
            t = torch.tensor([e_ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e_ms = float(t.item())
        return e_ms

    e2e = None
    if args.e2e_steps > 0:
        serial_ms = e2e_run(False)
        metric_ms = e2e_run(True, images_back=False)
        e2e_ms = e2e_run(True)
        ok = torch.equal(h_dst2[0], h_dst2[1]) and bool((h_psnr2[0] == h_psnr2[1]).all())
        e2e = {"value": world * px_step / (e2e_ms / 1e3) / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": int(h_src.numel()), "d2h_bytes_per_step": int(h_dst2[0].numel() + 8 * jobs),
               "ms_per_step": e2e_ms, "steps_in_flight": 2, "serial_ms_per_step": serial_ms,
               "serial_value": world * px_step / (serial_ms / 1e3) / 1e9,
               "link_gbs": (h_src.numel() + h_dst2[0].numel() + 8 * jobs) / (e2e_ms / 1e3) / 1e9,
               "results_consistent": ok,
               # the same pipeline reading back only the per-image PSNR (the reconstructions stay
               # in device memory, e.g. for a following device-side consumer)
               "psnr_only": {"value": world * px_step / (metric_ms / 1e3) / 1e9, "ms_per_step": metric_ms,
                             "h2d_bytes_per_step": int(h_src.numel()), "d2h_bytes_per_step": int(8 * jobs)}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD.replace("64x", f"{n_img}x", 1), "images": n_img, "side": SIDE, "r_sweep": list(R_SWEEP),
                       "jobs_per_step": jobs, "pixels_per_step": px_step, "parallelism": f"dp{world} (image shards)",
                       "l2": f"{N_SETS} rotating input/output sets of {2 * px_step / 1e6:.0f} MB (> 4 x L2)"},
            "roofline": roof,
            "e2e": e2e,
            "gpu_launches": world * zonal_launches_per_call(R_SWEEP) * args.steps,  # all ranks
            "clocks": clk,
            "step_ms_percentiles": step_pct,
        }
        line["cpu_baseline"] = cpu_baseline(batch, args.cpu_seconds) if args.cpu_seconds > 0 else None
        if args.cpu_seconds > 0:
            line["cpu_baseline_all_cores"] = cpu_baseline_all_cores(batch)
        if not args.no_extras:
            # the extra phases never take the headline with them: a phase that
            # fails records its error in its own key
            def phase(key, fn):
                try:
                    line[key] = fn()
                except Exception as e:  # noqa: BLE001 - reported in the line
                    line[key] = {"error": f"{type(e).__name__}: {e}"[:500]}
                torch.cuda.empty_cache()

            phase("config1", lambda: config1_phase(torch, atdct16, synth, dev))
            phase("psnr_u8_by_r", lambda: psnr_u8_by_r(torch, atdct16, sets[0][0], sets[0][1]))
            phase("coefficients", lambda: coef_phase(torch, atdct16, batch, dev, peak))
            phase("general_variants", lambda: general_variants_phase(torch, atdct16, batch, dev))
            phase("ssim", lambda: ssim_phase(torch, atdct16, plan, sets[0][2], jobs, px_step))
            phase("dct_baseline", lambda: dct_baseline_phase(torch, atdct16, plan, sets, jobs, px_step, None))
            del sets
            torch.cuda.empty_cache()
            phase("quant", lambda: quant_phase(torch, atdct16, synth, dev, args.quant_frames, args.quant_chunk, 5, 1,
                                               peak, cpu_oracle=args.cpu_seconds > 0))
            phase("mixed_batch", lambda: mixed_batch_phase(torch, atdct16, synth, dev, args.mixed_images,
                                                           cpu_oracle=args.cpu_seconds > 0))
            line["serving"] = serving  # measured first (above)
        print(json.dumps(line), flush=True)
    plan.close()
    if dist:
        dist.destroy_process_group()
    return 0


def run_quant_only(args):
    """The quantisation phase alone, on one GPU (profiling entry)."""
    import torch

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    from paper_1606_05562_gb300 import atdct16, synth
    from paper_1606_05562_gb300 import build as b

    b.build()
    peak, _ = measured_peak_hbm()
    res = quant_phase(torch, atdct16, synth, dev, args.quant_frames, args.quant_chunk, args.steps, args.warmup, peak)
    print(json.dumps({"quant": res}), flush=True)
    return 0


def run_coef_only(args):
    """The coefficient-pipeline phase alone, on one GPU (profiling entry)."""
    import torch

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    from paper_1606_05562_gb300 import atdct16, synth
    from paper_1606_05562_gb300 import build as b

    b.build()
    peak, _ = measured_peak_hbm()
    batch = synth.image_batch_512(N_IMAGES, SIDE, first_seed=100)
    print(json.dumps({"coefficients": coef_phase(torch, atdct16, batch, torch.device("cuda", 0), peak,
                                                 reps=max(args.steps, 1))}), flush=True)
    return 0


def run_dct_only(args):
    """The exact-DCT baseline phase alone, on one GPU (profiling entry)."""
    import torch

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    from paper_1606_05562_gb300 import atdct16, synth
    from paper_1606_05562_gb300 import build as b

    b.build()
    batch = synth.image_batch_512(N_IMAGES, SIDE, first_seed=100)
    nr = len(R_SWEEP)
    jobs = nr * N_IMAGES
    base = torch.from_numpy(batch).to(dev)
    sets = []
    for _ in range(N_SETS):
        src = base.unsqueeze(0).repeat(nr, 1, 1, 1).contiguous()
        dst = torch.empty_like(src)
        sets.append((src, dst, atdct16.descriptors(
            [atdct16.image(src[k, i], dst[k, i], r) for k, r in enumerate(R_SWEEP) for i in range(N_IMAGES)])))
    plan = atdct16.Plan(atdct16.U8, max_images=jobs)
    res = dct_baseline_phase(torch, atdct16, plan, sets, jobs, jobs * SIDE * SIDE, None, steps=max(args.steps, 1))
    plan.close()
    print(json.dumps({"dct_baseline": res}), flush=True)
    return 0


def run_ssim_only(args):
    """The SSIM phase alone, on one GPU (profiling entry): one zonal step of
    the bench workload, then SSIM of its 512 reconstructions."""
    import torch

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    from paper_1606_05562_gb300 import atdct16, synth
    from paper_1606_05562_gb300 import build as b

    b.build()
    batch = synth.image_batch_512(N_IMAGES, SIDE, first_seed=100)
    nr = len(R_SWEEP)
    jobs = nr * N_IMAGES
    src = torch.from_numpy(batch).to(dev).unsqueeze(0).repeat(nr, 1, 1, 1).contiguous()
    dst = torch.empty_like(src)
    descs = atdct16.descriptors(
        [atdct16.image(src[k, i], dst[k, i], r) for k, r in enumerate(R_SWEEP) for i in range(N_IMAGES)])
    plan = atdct16.Plan(atdct16.U8, max_images=jobs)
    psnr = torch.empty(jobs, dtype=torch.float64, device=dev)
    plan.compress_zonal(descs, psnr)
    res = ssim_phase(torch, atdct16, plan, descs, jobs, jobs * SIDE * SIDE, reps=max(args.steps, 1))
    plan.close()
    print(json.dumps({"ssim": res}), flush=True)
    return 0


def run_serve_only(args):
    """The serving phase alone, on one GPU."""
    import torch

    torch.cuda.set_device(0)
    from paper_1606_05562_gb300 import atdct16, synth
    from paper_1606_05562_gb300 import build as b

    b.build()
    rates = [float(v) for v in args.serve_rates.split(",") if v]
    print(json.dumps({"serving": serving_phase(torch, atdct16, synth, rates, args.serve_requests)}), flush=True)
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.quant_only:
        return run_quant_only(args)
    if args.coef_only:
        return run_coef_only(args)
    if args.serve_only:
        return run_serve_only(args)
    if args.ssim_only:
        return run_ssim_only(args)
    if args.dct_only:
        return run_dct_only(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
