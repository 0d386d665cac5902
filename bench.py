#!/usr/bin/env python
"""Benchmark of the batched render path on a 4M-leaf multi-room floor.

One step renders a batch of 256 cameras of mixed resolution (64 x 320x240,
128 x 640x480, 64 x 1280x720; fx = 0.9375 W; per-camera tau ~ U[2, 8] px)
from a 25 x 12 x 3 m floor of 4M leaf Gaussians (~4.6M hierarchy nodes) with
float16 SH / scale / opacity storage, through one captured CUDA graph. The same
cameras are also rendered by the plain per-view float32 path (one camera per
call, host-synchronised stage sizes, no graph) for the comparison the metric
names, and end to end through the host-buffer entry point.

`--impl reference` times the float64 CPU oracle on the same workload instead.
Prints one JSON line (rank 0)."""
import argparse
import dataclasses
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpix/s batched render vs plain per-view FP32 on same GB300 at <=2e-3 err; p99 ms"
WORKLOAD = "batch256_floor4m_f16"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cams", type=int, default=256)
    ap.add_argument("--leaves", default="floor4m")
    ap.add_argument("--tile", default="32x32", help="binning tile (the autotuner's pick by default)")
    ap.add_argument("--cta", default="16x16", help="compositing block (0x0: the tile)")
    ap.add_argument("--batch", type=int, default=128)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-stage-timing", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-blend", action="store_true",
                    help="skip the level-of-detail blending leg")
    ap.add_argument("--no-slice", action="store_true",
                    help="skip the GS-slice occupancy leg")
    ap.add_argument("--no-cut-variants", action="store_true",
                    help="skip the frustum-culled / shared cut leg")
    ap.add_argument("--no-order-leg", action="store_true",
                    help="skip the compositing work-order comparison")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the per-config legs (1M-leaf 640x480 and 4M-leaf 720p plain "
                         "paths, the FP16/BF16 error table, the oracle timings)")
    ap.add_argument("--c1-poses", type=int, default=200)
    ap.add_argument("--c2-poses", type=int, default=100)
    ap.add_argument("--serving-seconds", type=float, default=5.0,
                    help="seconds of simulated agent load for the serving leg (0: skip)")
    ap.add_argument("--serving-scene", default="floor8m")
    ap.add_argument("--cpu-cams", type=int, default=3)
    ap.add_argument("--pairs-per-pixel", type=int, default=0,
                    help="planner estimate of pairs per pixel (0: the library's default)")
    ap.add_argument("--record-capacity", type=int, default=1 << 29,
                    help="record slots of the work buffers (smaller for profiling runs)")
    ap.add_argument("--pair-capacity", type=int, default=(1 << 31) - (1 << 24),
                    help="(tile, Gaussian) pair slots of the work buffers")
    return ap.parse_args()


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def max_over_ranks(x, pg):
    """The largest value of a per-rank float over all ranks (x itself without a
    process group): the timed region of a multi-GPU run lasts as long as its
    slowest rank."""
    if not pg:
        return float(x)
    import torch
    dev = "cuda" if pg.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def whole_job_mpix_per_s(pixels_per_rank, steps, world, total_ms):
    """Mpix/s of the whole job: every rank renders its own batch of
    pixels_per_rank pixels per step (weak scaling)."""
    return world * pixels_per_rank * steps / (total_ms * 1e3)


def make_workload(args, rank):
    from scenegen import make_scene, mixed_batch_cameras
    scene = make_scene(args.leaves)
    cams = mixed_batch_cameras(scene, args.cams, seed=1002 + rank)
    return scene, cams


def config_dict(args, scene, cams, world):
    pix = sum(c.width * c.height for c in cams)
    return {"workload": WORKLOAD, "scene": args.leaves, "leaves": int(scene.n_leaves),
            "nodes": int(scene.n_nodes), "cameras_per_step": len(cams),
            "resolutions": "320x240:640x480:1280x720 = 1:2:1", "tau_px": "U[2,8]",
            "mpix_per_step": round(pix / 1e6, 4), "attr_storage": "f16 sh/scale/opacity",
            "tile": args.tile, "composite_block": args.cta, "smem_batch": args.batch,
            "cuda_graph": True,
            "l2": "inputs exceed L2 (scene ~0.6 GB, pair buffers GBs)",
            "parallelism": f"replicas{world}"}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
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
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows]
        mx = max(float(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum, mean
# over the launches of one render of this workload at 32x32 tiles in 16x16
# compositing blocks, batch 128; for "onesweep" over all 18 radix passes) from
# the one-pass ncu capture summarised in profiles/traffic_batch256_floor4m_f16.md.
# Each figure is tied to the sources of the kernel it was taken on (sha256 of
# the files, concatenated, first 16 hex digits) and reads null once they change.
MEASURED_TRAFFIC = {
    "onesweep": (1_257_100_000, ("k_sort.cu", "ngs_internal.cuh"), "4db60b1584962499"),
    "composite": (712_500_000, ("k_composite.cu", "ngs_internal.cuh"), "76ceb844a89ff03c"),
    "cut_preprocess": (3_596_900_000, ("k_preprocess.cu", "ngs_internal.cuh"), "6d567f9e49be4b20"),
    "duplicate": (2_100_600_000, ("k_binning.cu", "ngs_internal.cuh"), "b3d4843c4c7845b0"),
    "pair_offsets": (1_220_500_000, ("k_binning.cu", "ngs_internal.cuh"), "b3d4843c4c7845b0"),
}


def measured_traffic(kernel):
    import hashlib
    e = MEASURED_TRAFFIC.get(kernel)
    if not e:
        return None
    nbytes, files, digest = e
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2603_15186_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return nbytes if h.hexdigest()[:16] == digest else None


# ---------------------------------------------------------------------------
# parity of a rendered image against the oracle's render of the same view
# ---------------------------------------------------------------------------

def parity_report(got, ref):
    """Max error of the pixels with no near-threshold decision, the fraction
    of pixels with one (flagged), and the flagged pixels' error against the
    nearest outcome of their near-threshold decisions (the oracle lists every
    way they can go); pixels with more outcomes than listed count as
    unchecked."""
    import oracle as O
    got = np.asarray(got, dtype=np.float64)
    flagged = ref.flags != 0
    err = np.abs(got - ref.image)
    out = {"max_abs_err": float(err[:, ~flagged].max()) if (~flagged).any() else 0.0,
           "flagged_frac": float(flagged.mean()), "flagged_max_err_vs_nearest_outcome": 0.0,
           "unchecked_frac": 0.0}
    ys, xs = np.nonzero(flagged)
    if len(ys):
        pix = np.stack([xs, ys], 1)
        best, over = np.empty(len(pix)), np.empty(len(pix), dtype=bool)
        for s0 in range(0, len(pix), 16384):
            pc = pix[s0:s0 + 16384]
            alts, cnt = O.alternatives(ref.pre, ref.vals, ref.ranges, ref.cam, pc, tile=ref.tile,
                                       max_out=256)
            d = np.abs(alts - got[:, pc[:, 1], pc[:, 0]].T[:, None, :]).max(axis=2)
            m = np.arange(256)[None, :] < np.minimum(np.abs(cnt), 256)[:, None]
            best[s0:s0 + 16384] = np.where(m, d, np.inf).min(axis=1)
            over[s0:s0 + 16384] = (cnt > 256) | (cnt < 0)
        over &= best > 2e-3
        out["flagged_max_err_vs_nearest_outcome"] = float(best[~over].max()) if (~over).any() else 0.0
        out["unchecked_frac"] = float(over.sum() / flagged.size)
    return out


# ---------------------------------------------------------------------------
# algorithmic bytes per stage (what each kernel must move at minimum)
# ---------------------------------------------------------------------------

def stage_bytes(st, n_nodes, n_cams, pixels, tiles, attr="f16"):
    """Minimum HBM bytes per stage for one step. The fused cut + preprocess
    must read every node's box once per sub-batch (the cameras of a sub-batch
    share it through L2) and write one record, key and rect per visible
    Gaussian (the attributes of the visible ones are not counted: which nodes
    are visible in several cameras of a sub-batch is not known here)."""
    rec = 48 if attr == "f32" else 32
    V, P = st["visible_total"], st["pair_total"]
    return {
        "cut_preprocess": st["sub_batches"] * n_nodes * 32 + V * (rec + 4 + 8),
        "gather_keys": 12 * V,
        "depth_hist": 4 * V,
        # the last depth pass writes values only; the last tile pass writes
        # values and each tile's range (8 B per tile) instead of keys
        "depth_pass0": 16 * V, "depth_pass1": 16 * V, "depth_pass2": 16 * V, "depth_pass3": 12 * V,
        # pair offsets: index, gathered 8-byte rect and offset per Gaussian,
        # plus the rect written in depth order for the pair emission, which
        # reads it, the offset and the index back sequentially
        "pair_offsets": 24 * V,
        "duplicate": 16 * V + 8 * P,
        "tile_hist": 4 * P,
        "tile_pass0": 16 * P, "tile_pass1": 12 * P + 8 * tiles, "tile_pass2": 0,
        "ranges": 8 * tiles,
        "composite": 12 * pixels + st["records_staged"] * (4 + rec),
    }


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(args, world, rank, local, pg):
    import torch
    import oracle as O
    from paper_2603_15186_gb300 import Renderer
    from scenegen import quantize_attributes

    torch.cuda.set_device(local)
    t0 = time.time()
    scene, cams = make_workload(args, rank)
    gen_s = time.time() - t0
    stored, deq = quantize_attributes(scene, "f16")
    tw, th = (int(x) for x in args.tile.split("x"))
    pixels = sum(c.width * c.height for c in cams)
    tiles = sum(-(-c.width // tw) * -(-c.height // th) for c in cams)

    R = Renderer(device=local, tile=(tw, th), batch=args.batch, cut_capacity=1 << 27,
                 record_capacity=args.record_capacity, pair_capacity=args.pair_capacity)
    R.load_scene(scene, attr_dtype="f16", stored=stored)
    R.set_cta(*(int(x) for x in args.cta.split("x")))
    if args.pairs_per_pixel:
        R.set_pairs_per_pixel(args.pairs_per_pixel)
    R.set_mode("batched")
    R.set_stage_timing(not args.no_stage_timing)
    imgs = R.new_images(cams)
    tune = None
    if not args.no_autotune:
        # tile shape x compositing batch, picked on this very camera batch
        tune = R.autotune(cams, imgs, reps=2)
        tw, th = tune["tile"]
        args.tile, args.batch = f"{tw}x{th}", tune["batch"]
        args.cta = "{}x{}".format(*tune["cta"])
        tiles = sum(-(-c.width // tw) * -(-c.height // th) for c in cams)
    for _ in range(max(args.warmup, 3)):
        R.render(cams, imgs)
    stats = R.stats()

    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stage_acc = {}
    g0.record(stream)
    for k in range(args.steps):
        ev[k][0].record(stream)
        R.render(cams, imgs, stream=stream, sync=False)
        ev[k][1].record(stream)
        if not args.no_stage_timing:
            for name, ms in R.stage_times().items():
                stage_acc[name] = stage_acc.get(name, 0.0) + ms
    g1.record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clk = clocks.stop()
    R.synchronize()
    total_ms = g0.elapsed_time(g1)
    step_ms = np.array([a.elapsed_time(b) for a, b in ev])
    total_ms = max_over_ranks(total_ms, pg)
    ms_per_step = total_ms / args.steps
    value = whole_job_mpix_per_s(pixels, args.steps, world, total_ms)
    stats = R.stats()
    kernels_per_step = stats["kernels"]
    tail_ms = stats["composite_tail_ms"]   # of the last timed step

    # roofline of the dominant kernel, from this run's events and counters
    roof = None
    if stage_acc:
        per_step = {k: v / args.steps for k, v in stage_acc.items()}
        byts = stage_bytes(stats, scene.n_nodes, len(cams), pixels, tiles, "f16")
        peak, peak_kind = measured_peaks()
        # kernels as the launch list names them: every digit pass of both sorts
        # is one k_onesweep launch
        groups = {"onesweep": ["depth_pass0", "depth_pass1", "depth_pass2", "depth_pass3",
                               "tile_pass0", "tile_pass1", "tile_pass2"],
                  "composite": ["composite"], "cut_preprocess": ["cut_preprocess"],
                  "gather_keys": ["gather_keys"],
                  "duplicate": ["duplicate"], "pair_offsets": ["pair_offsets"],
                  "ranges": ["ranges"], "histograms": ["depth_hist", "tile_hist"]}
        gt = {g: sum(per_step.get(s, 0.0) for s in ss) for g, ss in groups.items()}
        # a digit pass that did not run (tile ids of fewer bits) has no time
        ran = {g: [s for s in ss if per_step.get(s, 0.0) > 0.05 or len(ss) == 1]
               for g, ss in groups.items()}

        def launches_of(g):
            if g == "onesweep":
                return len(ran[g]) * stats["sub_batches"]
            return stats["sub_batches"]

        def hbm_entry(g):
            n_launch = max(launches_of(g), 1)
            b = sum(byts[s] for s in ran[g]) / n_launch
            dur_ms = gt[g] / n_launch
            achieved = b / (dur_ms * 1e-3) / 1e9
            return {"kernel": g, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                    "unit": "GB/s", "frac": round(achieved / peak, 4),
                    "traffic": measured_traffic(g), "peak_kind": f"{peak_kind} copy bandwidth",
                    "launches_per_step": n_launch, "avg_launch_ms": round(dur_ms, 4),
                    "algorithmic_bytes_per_launch": int(b)}

        def alu_entry():
            # the compositing kernel is bound by FP32 issue: per pixel-Gaussian
            # evaluation its inner loop issues 10.5 FP32-pipe lane operations in
            # the common path (exponent from per-row coefficients 2, threshold
            # compare 1, threshold factor 1, clamp 1, weight alpha T 1, colour 3,
            # T - alpha T 1, and the stop test's two compares once per group of
            # four records: 0.5) and one exp2 (a group in which a pixel stops is
            # redone with the stop factor: extra work on top of this bound)
            sms = torch.cuda.get_device_properties(local).multi_processor_count
            mhz = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["sm_max_mhz"]) \
                if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 2070.0
            peak_e = sms * 128 * mhz * 1e6 / 10.5 / 1e12
            n_launch = max(launches_of("composite"), 1)
            dur_ms = gt["composite"] / n_launch
            ach = stats["evaluations"] / n_launch / (dur_ms * 1e-3) / 1e12
            hb = byts["composite"] / n_launch / (dur_ms * 1e-3) / 1e9
            return {"kernel": "composite", "bound": "alu", "achieved": round(ach, 3),
                    "peak": round(peak_e, 3), "unit": "Teval/s", "frac": round(ach / peak_e, 4),
                    "traffic": measured_traffic("composite"),
                    "peak_kind": f"{sms} SMs x 128 FP32 lanes x {mhz:.0f} MHz / 10.5 FP32 lane ops "
                                 "per evaluation (the inner loop's common path)",
                    "launches_per_step": n_launch, "avg_launch_ms": round(dur_ms, 4),
                    "hbm_achieved_gbs": round(hb, 1)}

        dom = max(gt, key=gt.get)
        roof = alu_entry() if dom == "composite" else hbm_entry(dom)
        roof["others"] = [alu_entry() if g == "composite" else hbm_entry(g)
                          for g in sorted(gt, key=gt.get, reverse=True)[1:3]]
        roof["stage_ms_per_step"] = {k: round(v, 4) for k, v in per_step.items()}

    out = {"metric": METRIC, "value": round(value, 2), "unit": "Mpix/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic", "config": config_dict(args, scene, cams, world),
           "p50_ms": round(float(np.percentile(step_ms, 50)), 3),
           "p99_ms": round(float(np.percentile(step_ms, 99)), 3),
           "frames_per_s": round(world * len(cams) * args.steps / (total_ms * 1e-3), 1),
           "gpu_launches": int(kernels_per_step * args.steps),
           "clocks": clk, "roofline": roof,
           "work": {k: stats[k] for k in ("cut_total", "candidate_total", "visible_total",
                                          "pair_total", "records_staged", "evaluations",
                                          "sub_batches")},
           "scene_gen_s": round(gen_s, 1), "autotune": tune}
    # longest-first compositing order against tile order: step time and the
    # compositing launches' tails (first CTA out of work -> last CTA done)
    if not args.no_order_leg:
        R.set_stage_timing(False)
        order = {}
        for name, on in (("tile_order", False), ("longest_first", True)):
            R.set_composite_order(on)
            for _ in range(3):
                R.render(cams, imgs)
            torch.cuda.synchronize()
            tails, ms = [], []
            for _ in range(max(3, min(args.steps, 5))):
                a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a_.record(stream)
                R.render(cams, imgs, stream=stream, sync=False)
                b_.record(stream)
                torch.cuda.synchronize()
                ms.append(a_.elapsed_time(b_))
                tails.append(R.stats()["composite_tail_ms"])
            order[name] = {"ms_per_step_median": round(float(np.median(ms)), 3),
                           "composite_tail_ms_median": round(float(np.median(tails)), 3)}
        out["composite_order"] = order
        out["composite_tail_ms"] = round(tail_ms, 3)
        R.set_stage_timing(not args.no_stage_timing)

    # plain per-view float32 path on the same cameras
    plain_imgs = None
    if not args.no_plain:
        P = Renderer(device=local, tile=(tw, th), batch=args.batch, cut_capacity=1 << 23,
                     record_capacity=1 << 23, pair_capacity=1 << 27)
        P.load_scene(scene, attr_dtype="f32")
        P.set_cta(*(int(x) for x in args.cta.split("x")))
        P.set_mode("plain")
        plain_imgs = P.new_images(cams)
        # the same warm-up and timed step count as the batched arm
        for _ in range(max(args.warmup, 3)):
            P.render(cams, plain_imgs, stream=stream)
        torch.cuda.synchronize()
        pev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        for k in range(args.steps):
            pev[k][0].record(stream)
            P.render(cams, plain_imgs, stream=stream)
            pev[k][1].record(stream)
        torch.cuda.synchronize()
        pstep = np.array([a_.elapsed_time(b_) for a_, b_ in pev])
        pms = float(pstep.mean())
        diff = max(float((x - y).abs().max().item()) for x, y in zip(imgs, plain_imgs))
        out["plain_fp32"] = {"value": round(pixels / (pms * 1e3), 2), "unit": "Mpix/s",
                             "ms_per_step": round(pms, 3),
                             "p50_ms": round(float(np.percentile(pstep, 50)), 3),
                             "p99_ms": round(float(np.percentile(pstep, 99)), 3),
                             "steps": args.steps, "warmup": max(args.warmup, 3),
                             "speedup_batched_over_plain": round(value / world / (pixels / (pms * 1e3)), 3),
                             "max_abs_diff_vs_batched_f16": diff}
        P.close()

    # end to end through the host-buffer entry point (pinned host images)
    if not args.no_e2e:
        import ctypes as C
        from paper_2603_15186_gb300.renderer import camera_array
        host = torch.empty(3 * pixels, dtype=torch.float32, pin_memory=True)
        hp = host.data_ptr()
        ptrs, off = [], 0
        for c in cams:
            ptrs.append(C.c_void_p(hp + 4 * off))
            off += 3 * c.width * c.height
        parr = (C.c_void_p * len(cams))(*ptrs)
        carr = camera_array(cams)
        R.set_stage_timing(False)
        R.render_host_ptrs(carr, len(cams), parr)
        ke = max(2, min(args.steps, 5))
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(ke):
            carr = camera_array(cams)           # cameras come from the host every step
            R.render_host_ptrs(carr, len(cams), parr)
        e2e_s = (time.perf_counter() - t) / ke
        from paper_2603_15186_gb300 import _lib
        out["e2e"] = {"value": round(world * pixels / (e2e_s * 1e6), 2), "unit": "Mpix/s",
                      "h2d_bytes_per_step": len(cams) * C.sizeof(_lib.Camera),
                      "d2h_bytes_per_step": 12 * pixels, "ms_per_step": round(e2e_s * 1e3, 3),
                      "path": "ngs_render_host: camera table H2D, render; the compositing kernels write the images into pinned host memory (device-mapped), synchronised"}

    # CPU oracle baseline on a bounded sample, and parity of the batched images
    if rank == 0 and not args.no_cpu:
        sa = O.SceneArrays(scene, overrides=deq)
        order = np.argsort([c.width * c.height for c in cams], kind="stable")[:args.cpu_cams]
        t = time.time()
        refs = [O.render(sa, cams[i], tile=(tw, th)) for i in order]
        cpu_s = time.time() - t
        cpu_pix = sum(cams[i].width * cams[i].height for i in order)
        reps = [parity_report(imgs[i].cpu().numpy(), ref) for i, ref in zip(order, refs)]
        out["cpu_baseline"] = {"value": round(cpu_pix / (cpu_s * 1e6), 4), "unit": "Mpix/s",
                               "cores": O.num_threads(), "kind": "oracle",
                               "sample": f"{len(order)} full views ({cpu_pix} px) of the batch, "
                                         f"float64 oracle incl. cut/preprocess/binning, {cpu_s:.1f} s"}
        out["parity_vs_oracle"] = {
            "max_abs_err": max(r["max_abs_err"] for r in reps), "tolerance": 2e-3,
            "flagged_pixel_frac": max(r["flagged_frac"] for r in reps),
            "flagged_max_err_vs_nearest_outcome": max(r["flagged_max_err_vs_nearest_outcome"]
                                                      for r in reps),
            "unchecked_frac": max(r["unchecked_frac"] for r in reps),
            "views": [int(i) for i in order],
            "flag_rule": "a decision (alpha vs 1/255, T(1-alpha) vs 1e-4) within the oracle's "
                         "float32 error bound of its threshold"}
    # level-of-detail blending (each cut node moved toward its parent), same
    # batch, same launch configuration
    if not args.no_blend:
        R.set_stage_timing(False)
        R.set_lod_blend(True)
        for _ in range(max(args.warmup, 3)):
            R.render(cams, imgs)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            R.render(cams, imgs, stream=stream, sync=False)
        b.record(stream)
        torch.cuda.synchronize()
        R.synchronize()
        bms = a.elapsed_time(b) / args.steps
        bst = R.stats()
        blend = {"value": round(world * pixels / (bms * 1e3), 2), "unit": "Mpix/s",
                 "ms_per_step": round(bms, 3), "visible_total": bst["visible_total"],
                 "pair_total": bst["pair_total"],
                 "note": "pre-culls bound the node-parent segment while blending"}
        if rank == 0 and not args.no_cpu:
            reps = [parity_report(imgs[i].cpu().numpy(),
                                  O.render(sa, cams[i], tile=(tw, th), blend=True)) for i in order]
            blend["max_abs_err_vs_oracle"] = max(r["max_abs_err"] for r in reps)
            blend["flagged_max_err_vs_nearest_outcome"] = max(
                r["flagged_max_err_vs_nearest_outcome"] for r in reps)
        out["lod_blend"] = blend
        R.set_lod_blend(False)
    if not args.no_cut_variants:
        out["cut_variants"] = run_cut_variants(args, R, scene, cams, rank, stream)
    if not args.no_slice:
        out["gs_slice"] = run_slice(args, R, scene, stored, deq, rank, stream)
    R.close()
    if not args.no_configs:
        out["configs"] = run_config_legs(args, local, rank, scene, stream)
    if args.serving_seconds > 0:
        out["serving"] = run_serving(args, local)
    if rank == 0:
        print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# level-of-detail cut variants on the batch's cameras
# ---------------------------------------------------------------------------

def run_cut_variants(args, R, scene, cams, rank, stream):
    """The batch's cameras are walker-major (consecutive cameras are nearby
    poses of one walk). Times one cut per camera (the camera-blocked two-pass
    kernel), the same with the frustum cull (groups of one), and one
    frustum-culled cut per group of 8 consecutive cameras; reports the cut
    sizes, node-camera tests per second and, for the first group, agreement
    with the oracle away from float32-reachable decisions."""
    import torch
    import oracle as O
    n = len(cams)
    M = int(scene.n_nodes)
    # a cut is an antichain of the tree: at most one leaf count per camera
    cap = min(n * int(scene.n_leaves), (1 << 31) - 1)
    hbm, kind = measured_peaks()
    groups8 = list(range(0, n, 8)) + [n]
    variants = [
        ("per_camera", n, lambda: R.select_cut(cams, cap=cap, stream=stream)),
        ("per_camera_frustum", n, lambda: R.select_cut_shared(
            cams, list(range(n + 1)), frustum=True, cap=cap, stream=stream)),
        ("shared_8_frustum", len(groups8) - 1, lambda: R.select_cut_shared(
            cams, groups8, frustum=True, cap=cap, stream=stream)),
    ]
    out = {"cameras": n, "nodes": M}
    res = {}
    for name, units, fn in variants:
        fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ids, off = fn()
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        t = min(ms)
        total = int(off[-1].item())
        # algorithmic bytes: every node's box read once, the selected ids
        # written (the kernels are bound by the per-camera granularity and
        # plane arithmetic, so this fraction stays small)
        nbytes = M * 32 + 4 * total
        if name == "shared_8_frustum":
            res[name] = (ids, off)
        del ids
        out[name] = {"ms": round(t, 3), "units": units, "cut_nodes_total": total,
                     "node_camera_tests_per_s": round(M * n / (t * 1e-3) / 1e9, 2),
                     "unit_tests": "G/s", "algorithmic_GBps": round(nbytes / (t * 1e-3) / 1e9, 1),
                     "frac_of_hbm": round(nbytes / (t * 1e-3) / 1e9 / hbm, 3),
                     "hbm_peak": f"{hbm:.0f} GB/s ({kind})"}
    out["frustum_cut_fraction"] = round(
        out["per_camera_frustum"]["cut_nodes_total"] / max(out["per_camera"]["cut_nodes_total"], 1), 4)
    if rank == 0 and not args.no_cpu:
        gb = groups8[:2]
        sa = O.SceneArrays(scene)
        t0 = time.time()
        want, woff, near = O.select_cut_shared(sa, cams[:gb[1]], gb, frustum=True)
        ids, off = res["shared_8_frustum"]
        got = ids[: int(off[1].item())].cpu().numpy()
        a, b_ = np.zeros(M, bool), np.zeros(M, bool)
        a[got] = True
        b_[want[woff[0]:woff[1]]] = True
        out["oracle_group0_s"] = round(time.time() - t0, 2)
        out["group0_mismatch_away_from_threshold"] = int(((a != b_) & (near[0] == 0)).sum())
        out["group0_near_frac"] = float(near[0].mean())
    return out


# ---------------------------------------------------------------------------
# GS-slice occupancy leg: the floor's leaves cut by planes every 10 cm
# ---------------------------------------------------------------------------

def slice_grid(scene, cell=0.05, z0=0.05, dz=0.1, nz=13, threshold=0.5):
    """Cells of `cell` metres over the scene's box, planes every 10 cm from
    5 cm to 1.25 m (the robot's height range)."""
    from types import SimpleNamespace
    lo, hi = scene.aabb_min[0], scene.aabb_max[0]
    return SimpleNamespace(x0=float(lo[0]), y0=float(lo[1]), cell=cell,
                           nx=int(np.ceil((hi[0] - lo[0]) / cell)),
                           ny=int(np.ceil((hi[1] - lo[1]) / cell)), z0=z0, dz=dz, nz=nz,
                           threshold=threshold)


def run_slice(args, R, scene, stored, deq, rank, stream):
    import torch
    import oracle as O
    g = slice_grid(scene)
    val, occ = R.slice_occupancy(g, stream=stream)
    for _ in range(2):
        R.slice_occupancy(g, val, occ, stream=stream)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(args.steps, 3)
    a.record(stream)
    for _ in range(reps):
        R.slice_occupancy(g, val, occ, stream=stream)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    evals = R.stats()["evaluations"]
    leaves = int(scene.n_leaves)
    outd = {"grid": f"{g.nx}x{g.ny} cells of {g.cell} m, {g.nz} planes {g.z0}..{g.z0 + (g.nz - 1) * g.dz:.2f} m",
            "leaves": leaves, "ms": round(ms, 3),
            "leaf_planes_per_s": round(leaves * g.nz / (ms * 1e-3) / 1e9, 3), "unit": "G/s",
            "cell_evaluations_per_s": round(evals / (ms * 1e-3) / 1e9, 2),
            "cell_evaluations": int(evals), "occupied_frac": float(occ.float().mean().item())}
    if rank == 0 and not args.no_cpu:
        t = time.time()
        want, wocc = O.slice_occupancy(O.SceneArrays(scene, overrides=deq), g)
        outd["oracle_s"] = round(time.time() - t, 2)
        outd["oracle_cores"] = O.num_threads()
        got = val.cpu().numpy().astype(np.float64)
        exempt = (np.minimum(got, want) <= 1.0 / 255.0 + 1e-3) & (np.abs(got - want) > 1e-3)
        outd["max_abs_err_vs_oracle"] = float(np.abs(got - want)[~exempt].max())
        outd["cutoff_exempt_frac"] = float(exempt.mean())
        near = np.abs(want - g.threshold) <= 1e-3
        outd["mask_mismatch_away_from_threshold"] = int(
            (occ.cpu().numpy()[~near] != wocc[~near]).sum())
    outd["navigation"] = run_nav(args, R, g, occ, rank, stream)
    return outd


def run_nav(args, R, g, occ, rank, stream):
    """Navigable map for a robot between planes 1 and 9 (0.15..0.85 m) with a
    10 cm footprint (2 cells), breadth-first distance fields of 9 goals (the
    paper's 9 annotated landmarks) and shortest paths for 64 agents."""
    import torch
    import oracle as O
    rng = np.random.default_rng(77)
    blocked, _ = R.nav_fields(occ, [(0, 0)], 1, 9, 2, stream=stream)
    free = np.argwhere(blocked.cpu().numpy() == 0)
    goals = [tuple(int(v) for v in free[k][::-1]) for k in rng.choice(len(free), 9, replace=False)]
    times = []
    for _ in range(3):
        torch.cuda.synchronize()
        t = time.perf_counter()
        blocked, dist = R.nav_fields(occ, goals, 1, 9, 2, stream=stream)
        times.append(time.perf_counter() - t)
    starts = [(int(free[k][1]), int(free[k][0]), int(rng.integers(9)))
              for k in rng.choice(len(free), 64, replace=False)]
    R.nav_paths(dist, starts, 4096, stream=stream)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    paths, lens = R.nav_paths(dist, starts, 4096, stream=stream)
    b.record(stream)
    torch.cuda.synchronize()
    dist_h = dist.cpu().numpy().view(np.uint32)
    out = {"grid": f"{g.nx}x{g.ny}", "goals": len(goals), "agents": len(starts),
           "fields_ms": round(1e3 * min(times), 3), "paths_ms": round(a.elapsed_time(b), 3),
           "reachable_frac": float((dist_h[0] < 0xFFFFFFFF).mean()),
           "mean_path_cells": float(lens.float().mean().item())}
    if rank == 0 and not args.no_cpu:
        occ_h = occ.cpu().numpy()
        t = time.time()
        b_ref = O.nav_blocked(occ_h, 1, 9, 2)
        refs = [O.nav_field(b_ref, q) for q in goals]
        out["oracle_fields_s"] = round(time.time() - t, 3)
        ph, lh = paths.cpu().numpy(), lens.cpu().numpy()
        same_paths = all(np.array_equal(ph[k, :lh[k]], O.nav_path(refs[s_[2]], s_[:2], 4096))
                         for k, s_ in enumerate(starts))
        out["bit_exact_vs_oracle"] = bool(
            np.array_equal(blocked.cpu().numpy(), b_ref) and
            all(np.array_equal(dist_h[q], refs[q]) for q in range(len(goals))) and same_paths)
    return out


# ---------------------------------------------------------------------------
# per-config legs: the plain FP32 path at floor scale, the precision form's
# error against the oracle, the oracle timed single-threaded and on all cores
# ---------------------------------------------------------------------------

def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def _time_views(R, cams, stream):
    """Renders each camera alone (one ngs_render call per view) after a few
    warm-up views; per-view milliseconds from CUDA events on `stream`."""
    import torch
    imgs = R.new_images(cams)
    for c, im in zip(cams[:5], imgs[:5]):
        R.render([c], [im], stream=stream)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in cams]
    for (a, b), c, im in zip(ev, cams, imgs):
        a.record(stream)
        R.render([c], [im], stream=stream)
        b.record(stream)
    torch.cuda.synchronize()
    ms = np.array([a.elapsed_time(b) for a, b in ev])
    pix = sum(c.width * c.height for c in cams)
    return imgs, {"mpix_per_s": round(pix / (ms.sum() * 1e3), 2),
                  "frames_per_s": round(len(cams) / (ms.sum() * 1e-3), 1),
                  "p50_ms": round(float(np.percentile(ms, 50)), 3),
                  "p99_ms": round(float(np.percentile(ms, 99)), 3), "views": len(cams)}


def _error_vs(got, ref):
    """Max-abs error (all pixels and the pixels with no near-threshold
    decision) and PSNR (peak 1) of a GPU image against an oracle render."""
    got = np.asarray(got, dtype=np.float64)
    err = np.abs(got - ref.image)
    ok = ref.flags == 0
    mse = float(np.mean(err ** 2))
    return {"max_abs": float(err.max()), "max_abs_unflagged": float(err[:, ok].max()),
            "psnr_db": round(10 * np.log10(1.0 / mse), 2) if mse > 0 else None,
            "flagged_frac": round(float(1 - ok.mean()), 5)}


def _oracle_mpix(O, sa, cams, tile, threads):
    O.set_threads(threads)
    t = time.time()
    for c in cams:
        O.render(sa, c, tile=tile)
    s = time.time() - t
    pix = sum(c.width * c.height for c in cams)
    return {"mpix_per_s": round(pix / (s * 1e6), 4), "s_per_view": round(s / len(cams), 3),
            "views": len(cams), "threads": threads}


def run_config_legs(args, local, rank, floor4m, stream):
    """1M-leaf floor (640x480, fx 600, tau 0 / 3 / 6 on a 200-pose walk) and
    4M-leaf floor (1280x720, fx 1200, tau 3, 100 poses): per-view plain FP32
    Mpix/s and p50/p99; the 4M floor also with FP16 and BF16 attributes (plain
    per view, and FP16 batched), and their error against the oracle on the
    FP32 attributes at poses 0, 33, 66 and 99 (the oracle renders the cut the
    GPU selected, checked against its own away from the tau threshold). The
    oracle is timed on all cores and single-threaded on these configs and on
    the 10k-leaf box (its two views)."""
    import torch
    import oracle as O
    from paper_2603_15186_gb300 import Renderer
    from scenegen import camera_c0, make_scene, quantize_attributes, walk_cameras
    tw, th = (int(x) for x in args.tile.split("x"))
    cw, ch = (int(x) for x in args.cta.split("x"))
    tile = (tw, th)
    out = {"tile": args.tile, "composite_block": args.cta}
    ncores = O.num_threads()
    host = {"nproc": os.cpu_count(), "cpu_model": cpu_model(), "oracle_threads_all": ncores}

    def new_ctx(records=1 << 24, pairs=1 << 27):
        R = Renderer(device=local, tile=tile, batch=args.batch, cut_capacity=1 << 24,
                     record_capacity=records, pair_capacity=pairs)
        R.set_cta(cw, ch)
        return R

    # C1: plain FP32 at floor scale
    t0 = time.time()
    s1 = make_scene("floor1m")
    gen1 = time.time() - t0
    walk = walk_cameras(s1, args.c1_poses, 41, 640, 480, fx=600.0, tau=0.0)
    R = new_ctx()
    R.load_scene(s1, attr_dtype="f32")
    R.set_mode("plain")
    c1 = {"scene": "floor1m", "leaves": int(s1.n_leaves), "nodes": int(s1.n_nodes),
          "resolution": "640x480", "poses": len(walk), "scene_gen_s": round(gen1, 1)}
    sa1 = O.SceneArrays(s1) if rank == 0 and not args.no_cpu else None
    for tau in (0.0, 3.0, 6.0):
        cams = [dataclasses.replace(c, tau=tau) for c in walk]
        imgs, tm = _time_views(R, cams, stream)
        if sa1 is not None:
            k = len(cams) // 2
            ids, off = R.select_cut([cams[k]])
            gpu = ids[: int(off[1].item())].cpu().numpy()
            own, near = O.select_cut(sa1, cams[k])
            a_, b_ = np.zeros(s1.n_nodes, bool), np.zeros(s1.n_nodes, bool)
            a_[gpu] = True
            b_[own] = True
            tm["cut_mismatch_away_from_tau"] = int(((a_ != b_) & (near == 0)).sum())
            ref = O.render(sa1, cams[k], tile=tile, ids=gpu.astype(np.int32))
            tm["error_vs_oracle"] = _error_vs(imgs[k].cpu().numpy(), ref)
        c1[f"tau{tau:g}"] = tm
        del imgs
    R.close()
    out["c1_floor1m_640x480_plain_fp32"] = c1

    # C2: the 4M floor at 720p, FP32 / FP16 / BF16 attributes
    cams2 = walk_cameras(floor4m, args.c2_poses, 51, 1280, 720, fx=1200.0, tau=3.0)
    probe = [k for k in (0, 33, 66, 99) if k < len(cams2)]
    c2 = {"scene": "floor4m", "leaves": int(floor4m.n_leaves), "resolution": "1280x720",
          "tau": 3.0, "poses": len(cams2), "error_poses": probe}
    imgs_by = {}
    for dt in ("f32", "f16", "bf16"):
        # the FP16 context also renders the 100 poses as one batched call
        R = new_ctx(1 << 27, 1 << 29) if dt == "f16" else new_ctx()
        if dt == "f32":
            R.load_scene(floor4m, attr_dtype="f32")
        else:
            R.load_scene(floor4m, attr_dtype=dt, stored=quantize_attributes(floor4m, dt)[0])
        R.set_mode("plain")
        imgs, tm = _time_views(R, cams2, stream)
        imgs_by[dt] = [imgs[k].cpu().numpy() for k in probe]
        del imgs
        if dt == "f16":
            R.set_mode("batched")
            bimgs = R.new_images(cams2)
            for _ in range(3):
                R.render(cams2, bimgs, stream=stream)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 5
            a.record(stream)
            for _ in range(reps):
                R.render(cams2, bimgs, stream=stream, sync=False)
            b.record(stream)
            torch.cuda.synchronize()
            bms = a.elapsed_time(b) / reps
            pix2 = sum(c.width * c.height for c in cams2)
            tm["batched_mpix_per_s"] = round(pix2 / (bms * 1e3), 2)
            tm["batched_ms_per_call"] = round(bms, 3)
            del bimgs
        if dt == "f32":
            gpu_cuts = []
            for k in probe:
                ids, off = R.select_cut([cams2[k]])
                gpu_cuts.append(ids[: int(off[1].item())].cpu().numpy().astype(np.int32))
        c2[f"plain_{dt}"] = tm
        R.close()
    if rank == 0 and not args.no_cpu:
        sa2 = O.SceneArrays(floor4m)
        O.set_threads(ncores)
        t = time.time()
        refs = []
        mism = 0
        for k, gcut in zip(probe, gpu_cuts):
            own, near = O.select_cut(sa2, cams2[k])
            a_, b_ = np.zeros(floor4m.n_nodes, bool), np.zeros(floor4m.n_nodes, bool)
            a_[gcut] = True
            b_[own] = True
            mism += int(((a_ != b_) & (near == 0)).sum())
            refs.append(O.render(sa2, cams2[k], tile=tile, ids=gcut))
        c2_oracle_s = time.time() - t
        c2["cut_mismatch_away_from_tau"] = mism
        table = {}
        for dt in ("f32", "f16", "bf16"):
            errs = [_error_vs(g, r) for g, r in zip(imgs_by[dt], refs)]
            table[dt] = {"max_abs": max(e["max_abs"] for e in errs),
                         "max_abs_unflagged": max(e["max_abs_unflagged"] for e in errs),
                         "psnr_db_min": min(e["psnr_db"] for e in errs if e["psnr_db"]),
                         "per_pose": errs}
        c2["error_vs_oracle_fp32_attributes"] = table
        c2["oracle_all_cores_s_for_error_poses"] = round(c2_oracle_s, 2)
        # oracle timings: all cores and single-threaded
        box = make_scene("box10k")
        sab = O.SceneArrays(box)
        c0cams = [camera_c0(0.0), camera_c0(4.0)]
        c1s = [dataclasses.replace(walk[k], tau=tau) for tau in (0.0, 3.0, 6.0)
               for k in range(0, len(walk), max(1, len(walk) // 5))[:5]]
        sa1 = O.SceneArrays(s1)
        timing = {"host": host}
        timing["c0_box10k_128x128"] = {"all_cores": _oracle_mpix(O, sab, c0cams, tile, ncores),
                                        "single_thread": _oracle_mpix(O, sab, c0cams, tile, 1)}
        timing["c1_floor1m_640x480"] = {
            "all_cores": _oracle_mpix(O, sa1, c1s, tile, ncores),
            "single_thread": _oracle_mpix(O, sa1, c1s[5:6], tile, 1),
            "sample": "all cores: tau 0/3/6 x 5 poses; one thread: one tau 3 pose"}
        timing["c2_floor4m_1280x720"] = {
            "all_cores": {"mpix_per_s": round(len(probe) * 0.9216 / c2_oracle_s, 4),
                          "s_per_view": round(c2_oracle_s / len(probe), 3), "views": len(probe),
                          "threads": ncores},
            "single_thread": _oracle_mpix(O, sa2, cams2[:1], tile, 1),
            "sample": "all cores: poses 0/33/66/99 (the error table's renders, on the GPU's "
                      "cut); one thread: pose 0"}
        O.set_threads(ncores)
        out["oracle_timing"] = timing
    out["c2_floor4m_1280x720"] = c2
    return out


# ---------------------------------------------------------------------------
# serving leg: many agents, Poisson arrivals, continuous batching
# ---------------------------------------------------------------------------

def run_serving(args, local):
    """64 agents on independent collision-free walks through the two-wing
    8M-leaf floor, Poisson arrivals at 31.25 requests/s each (2000/s in all),
    resolutions 320x240 : 640x480 : 1280x720 = 1 : 2 : 1 per agent, tau ~ U[2, 8].
    Requests are submitted at their arrival times to the serving loop; latency
    is submission to completion."""
    import torch
    from paper_2603_15186_gb300 import Renderer, Server, camera_struct
    from scenegen import make_scene, quantize_attributes, walk_cameras
    t0 = time.time()
    scene = make_scene(args.serving_scene)
    stored, _ = quantize_attributes(scene, "f16")
    gen_s = time.time() - t0
    rng = np.random.default_rng(4004)
    n_agents, rate = 64, 2000.0 / 64
    res = [(320, 240)] * 16 + [(640, 480)] * 32 + [(1280, 720)] * 16
    rng.shuffle(res)
    steps = int(args.serving_seconds * rate * 2) + 8
    walks = []
    for a in range(n_agents):
        w, h = res[a]
        taus = rng.uniform(2.0, 8.0, size=steps)
        walks.append([camera_struct(c) for c in
                      walk_cameras(scene, steps, 5000 + a, w, h, tau=0.0, taus=taus)])
    events = []
    for a in range(n_agents):
        t, k = rng.exponential(1.0 / rate), 0
        while t < args.serving_seconds:
            events.append((t, a, k))
            k += 1
            t += rng.exponential(1.0 / rate)
    events.sort()
    R = Renderer(device=local, cut_capacity=1 << 20, record_capacity=1 << 27,
                 pair_capacity=1 << 29)
    R.load_scene(scene, attr_dtype="f16", stored=stored)
    ring = 4
    bufs = [[torch.empty((3, res[a][1], res[a][0]), device="cuda") for _ in range(ring)]
            for a in range(n_agents)]
    S = Server(R, lanes=2, max_cams=64, lane_record_capacity=1 << 27,
               lane_pair_capacity=(1 << 29) + (1 << 28))
    # warm-up burst, not counted
    for a in range(n_agents):
        S.submit_struct(walks[a][0], bufs[a][0].data_ptr())
    S.wait_all()
    S.stop()
    S = Server(R, lanes=2, max_cams=64, lane_record_capacity=1 << 27,
               lane_pair_capacity=(1 << 29) + (1 << 28))
    offered = sum(res[a][0] * res[a][1] for _, a, _ in events) / 1e6 / args.serving_seconds
    start = time.perf_counter()
    for t, a, k in events:
        delay = start + t - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        S.submit_struct(walks[a][k % len(walks[a])], bufs[a][k % ring].data_ptr())
    S.wait_all()
    st = S.stats()
    S.stop()
    R.close()
    return {"scene": args.serving_scene, "leaves": int(scene.n_leaves), "agents": n_agents,
            "offered_req_per_s": round(len(events) / args.serving_seconds, 1),
            "offered_mpix_per_s": round(offered, 1), "load_seconds": args.serving_seconds,
            "requests": st["submitted"], "completed": st["completed"], "failed": st["failed"],
            "launches": st["launches"], "p50_ms": round(st["p50_ms"], 3),
            "p99_ms": round(st["p99_ms"], 3), "mean_ms": round(st["mean_ms"], 3),
            "mpix_per_s": round(st["mpix"] / max(st["span_s"], 1e-9), 1),
            "span_s": round(st["span_s"], 3), "lanes": 2, "max_cams_per_launch": 64,
            "attr_storage": "f16", "scene_gen_s": round(gen_s, 1)}


# ---------------------------------------------------------------------------
# reference arm: the float64 oracle on the host cores
# ---------------------------------------------------------------------------

def run_reference(args, world, rank):
    if rank != 0:
        return
    import oracle as O
    from scenegen import quantize_attributes
    scene, cams = make_workload(args, 0)
    _, deq = quantize_attributes(scene, "f16")
    sa = O.SceneArrays(scene, overrides=deq)
    tw, th = (int(x) for x in args.tile.split("x"))
    # each step: one view of the batch (cycling through it), full oracle pipeline
    order = list(range(len(cams)))
    for k in range(args.warmup):
        O.render(sa, cams[order[k % len(order)]], tile=(tw, th))
    t = time.time()
    pix = 0
    for k in range(args.steps):
        c = cams[order[(args.warmup + k) % len(order)]]
        O.render(sa, c, tile=(tw, th))
        pix += c.width * c.height
    s = time.time() - t
    val = pix / (s * 1e6)
    out = {"impl": "reference", "metric": METRIC, "value": round(val, 4), "unit": "Mpix/s",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(1e3 * s / args.steps, 2), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": config_dict(args, scene, cams, world),
           "cpu_baseline": {"value": round(val, 4), "unit": "Mpix/s", "cores": O.num_threads(),
                            "kind": "oracle",
                            "sample": "one view of the 256-camera batch per step (cycling)"},
           "e2e": {"value": round(val, 4), "unit": "Mpix/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    world, rank, local, pg = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local, pg)
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
