#!/usr/bin/env python
"""Throughput of the coherent-dedispersion pulse search on GB300.

Workload (one "step"): the Chimageator search of a 12-antenna array (positions
seeded within 6 km), 32 MHz of complex baseband at 1.4 GHz, 2^22 samples per
antenna, 64 trial DMs in 0-300 pc cm^-3 (FFT length >= 2^18, grown per DM so
that each overlap-save block keeps >= half its samples), 32x32 beams over
1 deg, dumps of 4096 samples, 3 injected bursts.  A step runs every stage of
the path: forward FFTs, chirp multiply + inverse FFT for every DM, and the
phased-sum beam detector with its integrate-and-dump.

Output: one JSON line (rank 0).  ``value`` is dedispersed antenna*DM*samples
per second over all ranks with inputs resident in HBM; ``e2e`` is the same
metric through the same call with pinned host input and host output (copies
inside the timed region).  ``--impl reference`` times the FP64 CPU oracle on
a bounded sample of the same workload instead.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "dedispersed antenna*DM*samples/s"
UNIT = "antenna*DM*samples/s"
WORKLOAD = ("chimageator: 12 ant within 6 km, 32 MHz @ 1.4 GHz, 2^22 samples/antenna, "
            "64 DMs 0-300, FFT >= 2^18, 32x32 beams over 1 deg, dump 4096")
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                  "sm_max_mhz": 2070.0}
N_SM = 152
DTYPE_LABEL = {1: "f32", 2: "f32 (beams: split-bf16 x3 on tensor cores, f32 acc)",
               3: "f32 (beams: visibility quadratic form)",
               4: "f32 dedispersion, bf16 beams (tensor cores, f32 acc)",
               5: "f32 dedispersion, bf16 voltages, f32 visibilities and beams"}
MODE_NAME = {1: "fp32_simt", 2: "tc_3xbf16", 3: "vis", 4: "tc_bf16", 5: "vis_bf16"}
FP32_LANES_PER_SM = 128


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--beam-mode", type=int, default=0,
                    help="0 auto (the faster exact form: 3 on this workload), 1 FP32 CUDA "
                         "cores, 2 tcgen05 split-BF16, "
                         "3 visibility quadratic form, 4 tcgen05 BF16 (reduced precision)")
    ap.add_argument("--no-alt", action="store_true",
                    help="skip the extra timings of the other beam modes and of detection")
    ap.add_argument("--chirpolator-only", action="store_true",
                    help="time only the Chirpolator search on the same workload (for profiling "
                         "its kernels); prints one line with its per-step and per-stage times")
    ap.add_argument("--cpi-only", action="store_true",
                    help="time only the paper's Chirpolator pre-integrator on the same workload "
                         "(for profiling its kernels); prints one line")
    ap.add_argument("--chimg-only", action="store_true",
                    help="time only the paper's Chimageator pre-integrator on a uniform linear "
                         "array shaped like the workload; prints one line")
    ap.add_argument("--truedelay-only", action="store_true",
                    help="time only the true-delay beams (8 x 8 pixels) on the same workload (for "
                         "profiling their kernels); prints one line")
    ap.add_argument("--precision-only", action="store_true",
                    help="time only the 36-antenna int8 channel leg; with --n-samp and --dms "
                         "(profiling: the lowest DMs of its 256, which stay valid on a shorter "
                         "series) only the library's choice of form; prints one line")
    ap.add_argument("--cpu-dumps", type=int, default=640,
                    help="dumps per selected DM in the oracle's bounded CPU sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the 36-antenna int8 channel leg (~100 GB of device memory)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--dms", type=int, default=0,
                    help="profiling only: keep this many evenly spaced DMs of the 64")
    ap.add_argument("--n-samp", type=int, default=0,
                    help="profiling only: shorter series (samples per antenna)")
    return ap.parse_args()


def committed_traffic(kernel_files, key):
    """Per-unit DRAM traffic of a kernel from its committed ncu summary, or None
    when the kernel's source changed since that capture (hash mismatch)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in kernel_files:
        with open(os.path.join(ROOT, "paper_1109_3186_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    cur = h.hexdigest()[:16]
    for fn in sorted(os.listdir(os.path.join(ROOT, "profiles"))):
        if not fn.endswith(".md"):
            continue
        txt = open(os.path.join(ROOT, "profiles", fn)).read()
        m = re.search(r"^(traffic_per_\w+): " + re.escape(key) + r": ([0-9.]+)", txt, re.M)
        if not m:
            continue
        sha = re.search(r"Source hash[^`]*`([0-9a-f]+)`", txt)
        if sha and sha.group(1) == cur:
            return float(m.group(2))
        return None
    return None


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return pk, "measured"
    except (OSError, ValueError):
        return dict(FALLBACK_PEAKS), "fallback"


def scenario(rank: int, args=None):
    from paper_1109_3186_gb300 import skymodel
    kw = {}
    if args is not None and args.n_samp:
        kw["n_samp"] = args.n_samp
    # each rank searches its own observation (weak scaling, no exchange)
    sc = skymodel.chimageator_medium(seed=1002 + 1000 * rank, **kw)
    if args is not None and args.dms:
        keep = np.unique(np.linspace(0, len(sc.dms) - 1, args.dms).round().astype(int))
        sc.dms = sc.dms[keep]
    return sc


def config_block(sc, n_gpus):
    full = sc.n_samp == 1 << 22 and len(sc.dms) == 64
    return {"workload": WORKLOAD if full else "REDUCED (profiling): " + WORKLOAD, "n_ant": sc.n_ant, "n_samp": sc.n_samp, "n_dm": len(sc.dms),
            "dm_max": float(sc.dms.max()), "bw_hz": sc.bw, "f0_hz": sc.f0,
            "nfft_min": sc.nfft_min, "n_pix": int(sc.pix_lm.shape[0]), "dump_len": sc.dump_len,
            "l2": "inputs larger than L2 (voltages 403 MB, forward spectra 2.7 GB)",
            "parallelism": "replicas%d" % n_gpus}


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_uuid: str | None):
        self.uuid = device_uuid
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
               "-lms", "200"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        loaded = [s for s in sm if s > 0.5 * (max(mx) if mx else 1)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows)}


def device_uuid(torch, dev):
    try:
        u = torch.cuda.get_device_properties(dev).uuid
        s = str(u)
        return s if s.startswith("GPU-") else "GPU-" + s
    except Exception:
        return None


# ---------------------------------------------------------------- oracle leg
def cpu_sample(sc, x, n_dumps: int):
    """Bounded oracle run: one middle DM of each FFT-length group, n_dumps dumps
    in the middle of the valid range.  Returns (units, seconds, cores, text)."""
    import oracle
    groups = {}
    for d, dm in enumerate(sc.dms):
        nf = oracle.nfft_for_dm(sc.f0, sc.bw, sc.k_dm, dm, sc.n_samp, sc.nfft_min)
        groups.setdefault(nf, []).append(d)
    sel = [g[len(g) // 2] for _, g in sorted(groups.items())]
    lay = oracle.layout(sc.dms, max(sel), sc.f0, sc.bw, sc.k_dm, sc.n_samp, sc.nfft_min)
    first, last = oracle.dump_range(sc.n_samp, lay["n_hi"], lay["n_lo"], sc.dump_len)
    mid = (first + last) // 2
    m0 = max(first, mid - n_dumps // 2)
    m1 = min(last + 1, m0 + n_dumps)
    t = time.perf_counter()
    oracle.chimageator(x, sc.f0, sc.bw, sc.k_dm, sc.dms, sc.nfft_min, sc.dump_len, sc.xyz,
                       sc.pix_lm, d_sel=sel, m0=m0, m1=m1)
    dt = time.perf_counter() - t
    units = sc.n_ant * len(sel) * (m1 - m0) * sc.dump_len
    text = ("FP64 oracle, DMs %s (one per FFT-length group), dumps %d..%d (%d x %d samples), "
            "all %d antennas and %d beams" % ([float(round(sc.dms[d], 2)) for d in sel], m0, m1 - 1,
                                              m1 - m0, sc.dump_len, sc.n_ant, sc.pix_lm.shape[0]))
    return units, dt, oracle.num_threads(), text


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return 0
    sc = scenario(0, args)
    x = sc.voltages()
    n_d = max(4, args.cpu_dumps // 2)
    for _ in range(args.warmup):
        cpu_sample(sc, x, 2)
    tot_u, tot_t = 0, 0.0
    cores, text = 1, ""
    for _ in range(args.steps):
        u, dt, cores, text = cpu_sample(sc, x, n_d)
        tot_u += u
        tot_t += dt
    value = tot_u / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot_t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_block(sc, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": text},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- our leg
def stage_roofline(sc, plan, stage_ms, peaks, peak_kind, beam_mode, steps):
    """Algorithmic bytes / flops per stage for one step, and achieved rates."""
    M, N, L = sc.n_ant, sc.n_samp, sc.dump_len
    n_pix = 0 if sc.pix_lm is None else sc.pix_lm.shape[0]
    first, last = plan.dump_range()
    groups = {}
    n_searched = {}
    fwd_pts = inv_pts = g_bytes = y_bytes = 0
    for d in range(len(sc.dms)):
        lay = plan.dm_layout(d)
        pts = M * lay["n_blk"] * lay["nfft"]
        groups[lay["nfft"]] = pts
        inv_pts += pts
        g_bytes += 8 * lay["nfft"]
        y_bytes += 8 * M * max(0, N - lay["n_hi"] - lay["n_lo"])
        if last[d] >= first[d]:
            n_searched[lay["nfft"]] = n_searched.get(lay["nfft"], 0) + 1
    fwd_pts = sum(groups.values())
    # row pass: a group's spectra are read once per chunk of dm_chunk DMs; each
    # DM reads its chirp table and writes its transformed rows
    chunk = max(1, plan.info.get("dm_chunk", 1))
    spec_reads = sum(8.0 * groups[g] * -(-n // chunk) for g, n in n_searched.items())
    # chirp tables: the group's FP64 phase table read once per chunk, each DM's table written
    g_reads = sum(8.0 * g * -(-n // chunk) for g, n in n_searched.items())
    hbm = peaks.get("hbm_gbs", FALLBACK_PEAKS["hbm_gbs"])
    sm_max = peaks.get("sm_max_mhz", FALLBACK_PEAKS["sm_max_mhz"])
    fp32_tflops = N_SM * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    n_dump_valid = int(np.sum(np.maximum(0, last - first + 1)))
    if beam_mode in (2, 4):
        # the inverse column pass writes the BF16 image of the valid dumps
        # (head + tail, or head only: 8 or 4 B per antenna-sample) instead of y
        y_bytes = float(n_dump_valid) * L * M * (8 if beam_mode == 2 else 4)
    y_elem = 4 if beam_mode == 5 else 8  # BF16 or FP32 complex voltages
    if beam_mode == 5:
        y_bytes = y_bytes / 2
    stages = {
        # read x (8 B complex64 or 2 B complex int8), write, read, write the spectrum
        "forward": ("hbm", (24.0 + (2.0 if plan.in_type == 1 else 8.0)) * fwd_pts, hbm, "GB/s"),
        "chirp": ("hbm", g_reads + g_bytes, hbm, "GB/s"),
        "inv_rows": ("hbm", spec_reads + 8.0 * inv_pts + g_bytes, hbm, "GB/s"),
        "inv_cols": ("hbm", 8.0 * inv_pts + y_bytes, hbm, "GB/s"),
    }
    beam_flops = float(n_dump_valid) * L * n_pix * (8 * M + 3)
    n_pair = M * (M + 1) // 2
    # correlate: read the dedispersed voltages of every valid dump, write V
    stages["correlate"] = ("hbm", float(n_dump_valid) * (L * y_elem * M + 8 * n_pair), hbm, "GB/s")
    if beam_mode == 4:
        beam_flops = float(n_dump_valid) * L * n_pix * (8 * M + 3)
    if beam_mode in (3, 5):
        # beams from visibilities: 2 FMA per (pair, pixel, dump)
        stages["beamform"] = ("alu", 4.0 * n_pair * n_pix * n_dump_valid, fp32_tflops, "TFLOP/s")
    elif beam_mode == 1:
        stages["beamform"] = ("alu", beam_flops, fp32_tflops, "TFLOP/s")
    else:
        stages["beamform"] = ("tensor", beam_flops,
                              peaks.get("bf16_tflops_sustained", FALLBACK_PEAKS["bf16_tflops_sustained"]),
                              "TFLOP/s")
        # what the tensor pipe executes: 128-row tiles x K steps of 16
        G = (M + 3) // 4
        ksteps = (3 * G + 1) // 2 if beam_mode == 2 else (G + 1) // 2
        n_rowtiles = (2 * n_pix + 127) // 128
        executed = float(n_dump_valid) * L * n_rowtiles * 128 * 2 * 16 * ksteps
    out = {}
    if beam_mode in (2, 4):
        ms, n = stage_ms.get("beamform", (0.0, 0))
        if ms > 0:
            out["_tensor_executed_tflops"] = executed / (ms / steps * 1e-3) / 1e12
    for name, (bound, work, peak, unit) in stages.items():
        ms, n = stage_ms.get(name, (0.0, 0))
        if ms <= 0 or n == 0:
            continue
        per_launch_work = work / (n / steps)
        avg_ms = ms / n
        rate = per_launch_work / (avg_ms * 1e-3)
        achieved = rate / 1e9 if unit == "GB/s" else rate / 1e12
        out[name] = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                     "frac": achieved / peak, "ms_per_step": ms / steps,
                     "launches_per_step": n / steps, "peak_source": peak_kind}
    return out


def max_over_ranks(x: float, dist, device: str) -> float:
    """The largest value of x over all ranks (the job's time is its slowest
    rank's); x itself without a process group."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank: int, world: int, seconds: float) -> float:
    """Whole-job throughput: every rank searches its own observation of the
    same size (weak scaling), so the job covers world x units in the slowest
    rank's time."""
    return world * units_per_rank / seconds


def extra_forms(sc, plan, xd, stream, args):
    """Timings of the forms beside the headline search (rank 0): the
    incoherent filterbank search, the learned proposer's inference, the
    selective coherent search over a proposal-like cell mask, and a batch of
    uneven observations under CUDA graphs."""
    import torch
    import paper_1109_3186_gb300 as chirp
    from paper_1109_3186_gb300 import skymodel
    out = {}

    def timed(fn, k):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    n_dm = len(sc.dms)
    # incoherent search (filterbank of 32 channels, 16 spectra per sample, the same DM grid)
    pfb = chirp.Plan.from_scenario(sc, beam_mode=chirp.BEAM_VIS, stream=stream, fb_chan=32,
                                   fb_int=16, fb_dm=sc.dms)
    T_fb = pfb.info["fb_samples"]
    D = torch.empty((n_dm, T_fb), dtype=torch.float32, device="cuda")
    ms = timed(lambda: pfb.incoherent(xd, D), 5)
    out["incoherent"] = {"ms": ms, "input_antenna_samples_per_s": sc.n_ant * sc.n_samp / (ms * 1e-3),
                         "fb_chan": 32, "fb_int": 16, "n_dm": n_dm}
    # learned proposer inference (z-score, conv net, window mask); weights seeded
    net = chirp.PropNet(n_dm, 64, 9, 5, 1, T_fb, stream=stream)
    rng = np.random.default_rng(7)
    net.set_params((0.05 * rng.standard_normal(net.n_params)).astype(np.float32))
    xz = torch.empty_like(D)
    z = torch.empty((1, n_dm, T_fb), dtype=torch.float32, device="cuda")
    win = 8
    mask = torch.empty((n_dm, (T_fb + win - 1) // win), dtype=torch.int32, device="cuda")

    def infer():
        net.normalize(D, xz)
        net.forward(xz[None], z)
        net.propose(z[0], win, 0.0, mask)
    ms = timed(infer, 5)
    out["proposer_inference"] = {"ms": ms, "params": int(net.n_params), "precision": "f32"}
    pfb.close()
    # selective coherent search: per DM, seeded runs of dumps covering ~1/3 of the cells
    first, last = plan.dump_range()
    cells = np.zeros((n_dm, plan.n_dump), np.uint8)
    for d in range(n_dm):
        n_valid = max(0, last[d] - first[d] + 1)
        for _ in range(6):
            if n_valid <= 0:
                break
            run = max(1, n_valid // 18)
            m0 = first[d] + int(rng.integers(0, max(1, n_valid - run)))
            cells[d, m0:m0 + run] = 1
    frac = float(cells[:, :].sum()) / max(1, int(np.sum(np.maximum(0, last - first + 1))))
    P = torch.empty((n_dm, plan.n_dump, plan.n_pix), dtype=torch.float32, device="cuda")
    ms_sel = timed(lambda: plan.chimageator_selective(xd, cells, P), 3)
    ms_full = timed(lambda: plan.chimageator(xd, P), 3)
    # the same selection in the reduced-precision form (BF16-rounded voltages,
    # FP32 visibilities and beams)
    p16 = chirp.Plan.from_scenario(sc, beam_mode=chirp.BEAM_VIS_BF16, stream=stream)
    ms_sel16 = timed(lambda: p16.chimageator_selective(xd, cells, P), 3)
    ms_full16 = timed(lambda: p16.chimageator(xd, P), 3)
    p16.close()
    pipeline = out["incoherent"]["ms"] + out["proposer_inference"]["ms"] + ms_sel16
    out["selective"] = {"ms": ms_sel, "full_grid_ms": ms_full, "cell_fraction": frac,
                        "speedup": ms_full / ms_sel, "reduced_precision_ms": ms_sel16,
                        "reduced_precision_full_grid_ms": ms_full16,
                        "reduced_precision_form": "vis_bf16",
                        "incoherent_proposer_selective_reduced_ms": pipeline,
                        "pipeline_speedup_vs_full_grid": ms_full / pipeline,
                        "mask": "seeded runs of dumps per DM (6 runs of 1/18 of the valid dumps), "
                                "not a trained proposer's output"}
    del P
    try:
        out["learned_99pct_recall"] = learned_leg(sc, plan, xd, stream, ms_full, timed)
    except Exception as exc:  # an auxiliary leg: record, do not lose the line
        out["learned_99pct_recall"] = {"error": str(exc)}
    torch.cuda.empty_cache()
    try:
        out["batch"] = batch_leg(args)
    except Exception as exc:  # an auxiliary leg: record, do not lose the line
        out["batch"] = {"error": str(exc)}
    return out


def learned_leg(sc, plan, xd, stream, full_ms, timed):
    """The learned form on this workload's array class, with the trained
    network's own proposals.  The proposer (61.6k parameters, FP32, the
    library's training kernels) is trained on 768 seeded 2^21-sample segments
    of the same array size, band, DM grid and dump length (0-4 bursts: DM
    uniform over the grid, width 20 us-1 ms, S/N 6-30, random beam
    direction; a narrowband tone in 10 %; drawn on the device).  Its
    threshold is the highest of a sweep that keeps >= 99 % of the bursts the
    full-grid search detects (candidates >= 7 sigma within one trial DM and
    two dumps) on 128 calibration segments; recall and cell fraction are then
    measured on 128 held-out segments.  On this step's voltages the trained
    network proposes the cells, the reduced-precision selective search runs
    them, and the pipeline (incoherent search + proposer + selective search)
    is timed against the full FP32 grid; its recall there is of the bursts
    the full grid detects in this observation."""
    import torch
    import paper_1109_3186_gb300 as chirp
    from paper_1109_3186_gb300 import propose as pp
    n_dm = len(sc.dms)
    setup = pp.ProposalSetup(n_ant=sc.n_ant, max_baseline_m=6000.0, f0=sc.f0, bw=sc.bw,
                             n_samp=1 << 21, dm_max=float(sc.dms.max()), n_dm=n_dm,
                             nfft_min=sc.nfft_min, dump_len=sc.dump_len, n_side=4,
                             fb_chan=32, fb_int=16)
    n_train, n_cal, n_test = 768, 128, 128
    t0 = time.perf_counter()
    prop = pp.Proposer(setup, stream=stream)
    feats, ys = [], []
    for seed in range(30000, 30000 + n_train):
        x, pulses = pp.segment_device(setup, seed)
        feats.append(prop.features(x))
        ys.append(pp.labels(setup, pulses))
    del x
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    losses = prop.train(feats, ys, steps=1500, batch=16, lr=1e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del feats, ys
    # calibration and held-out segments: features and full-grid detections
    P = torch.empty((n_dm, prop.plan.n_dump, prop.plan.n_pix), dtype=torch.float32, device="cuda")
    ev_feats, ev_truth = [], []
    for seed in range(40000, 40000 + n_cal + n_test):
        x, pulses = pp.segment_device(setup, seed)
        ev_feats.append(prop.features(x))
        prop.plan.chimageator(x, P)
        c = prop.plan.detect(P, 7.0)
        ev_truth.append((pulses, set(zip(c["dm"].tolist(), c["dump"].tolist()))))
    del x, P
    ddm = float(setup.dms[1] - setup.dms[0])
    span = setup.win * setup.t_fb

    def sweep(lo, hi, thr):
        cl = [pp.cells_of(prop.propose(ev_feats[i], thr), setup.n_samp, setup.dump_len, span)
              for i in range(lo, hi)]
        f, n = pp.recall(ev_truth[lo:hi], cl, ddm, setup.dump_len)
        return f, n, float(np.mean([c.mean() for c in cl]))

    curve, thr99 = [], None
    for thr in (2.0, 1.0, 0.0, -1.0, -2.0, -3.0, -4.0, -5.0, -6.0, -8.0, -10.0, -14.0):
        fc, nc, _ = sweep(0, n_cal, thr)
        fh, nh, frh = sweep(n_cal, n_cal + n_test, thr)
        curve.append({"threshold": thr, "calibration": "%d/%d" % (fc, nc),
                      "held_out": "%d/%d" % (fh, nh), "held_out_cell_fraction": frh})
        if thr99 is None and nc and fc >= 0.99 * nc:
            thr99 = thr
    if thr99 is None:
        thr99 = curve[-1]["threshold"]
    fh, nh, frh = sweep(n_cal, n_cal + n_test, thr99)
    # this step's voltages: the trained network's own proposals
    pfb = chirp.Plan.from_scenario(sc, beam_mode=chirp.BEAM_VIS, stream=stream, fb_chan=32,
                                   fb_int=16, fb_dm=sc.dms)
    T_fb = pfb.info["fb_samples"]
    net = chirp.PropNet(n_dm, 64, 9, 5, 1, T_fb, stream=stream)
    net.set_params(prop.net.params())
    D = torch.empty((n_dm, T_fb), dtype=torch.float32, device="cuda")
    xz = torch.empty_like(D)
    z = torch.empty((1, n_dm, T_fb), dtype=torch.float32, device="cuda")
    mask = torch.empty((n_dm, (T_fb + setup.win - 1) // setup.win), dtype=torch.int32,
                       device="cuda")

    def propose_step():
        pfb.incoherent(xd, D)
        net.normalize(D, xz)
        net.forward(xz[None], z)
        net.propose(z[0], setup.win, thr99, mask)
    ms_prop = timed(propose_step, 5)
    cells = pp.cells_of(mask.cpu().numpy().astype(np.uint8), sc.n_samp, sc.dump_len, span)
    first, last = plan.dump_range()
    valid = np.zeros_like(cells, dtype=bool)
    for d in range(n_dm):
        valid[d, first[d]:last[d] + 1] = True
    frac_obs = float(cells[valid].sum()) / max(1, int(valid.sum()))
    Pf = torch.empty((n_dm, plan.n_dump, plan.n_pix), dtype=torch.float32, device="cuda")
    plan.chimageator(xd, Pf)
    c = plan.detect(Pf, 7.0)
    f_obs, n_obs = pp.recall([(sc.pulses, set(zip(c["dm"].tolist(), c["dump"].tolist())))],
                             [cells], float(sc.dms[1] - sc.dms[0]), sc.dump_len)
    p16 = chirp.Plan.from_scenario(sc, beam_mode=chirp.BEAM_VIS_BF16, stream=stream)
    ms_sel16 = timed(lambda: p16.chimageator_selective(xd, cells, Pf), 3)
    ms_full16 = timed(lambda: p16.chimageator(xd, Pf), 3)
    p16.close()
    pfb.close()
    del Pf
    pipe = ms_prop + ms_sel16
    return {"trained_on": "%d seeded 2^21-sample segments of this array class (12 antennas within "
                          "6 km, 32 MHz, 64 DMs 0-300, dumps 4096), drawn on the device" % n_train,
            "params": int(net.n_params), "precision": "f32", "train_steps": 1500,
            "final_loss": float(np.mean(losses[-50:])), "first_loss": float(losses[0]),
            "data_s": t_data, "train_s": t_train, "threshold": thr99,
            "held_out_recall": "%d/%d" % (fh, nh), "held_out_cell_fraction": frh,
            "curve": curve,
            "observation_cell_fraction": frac_obs,
            "observation_recall": "%d/%d" % (f_obs, n_obs),
            "incoherent_proposer_ms": ms_prop, "selective_reduced_ms": ms_sel16,
            "incoherent_proposer_selective_reduced_ms": pipe,
            "full_grid_fp32_ms": full_ms, "full_grid_reduced_ms": ms_full16,
            "speedup_vs_full_fp32": full_ms / pipe, "speedup_vs_full_reduced": ms_full16 / pipe,
            "reduced_precision_form": "vis_bf16"}


def batch_leg(args):
    """The batched form at its stated scale: 24 observations drawn with a
    fixed seed -- 2^U{20..24} samples, U{32..512} trial DMs over 0..U(50, 300)
    pc cm^-3, U{8..64} antennas within 6 km, U(16, 64) MHz at 1.4 GHz, dumps
    of 2^U{9..13} samples, 8 x 8 beams over 1 deg -- each a lean plan (one
    FFT-length group's spectra at a time) on its own stream under CUDA
    graphs (complex64 noise drawn on the device).  The observations go in
    waves: plans are created in order until their workspaces, outputs and
    inputs would pass 200 GB or the free device memory, one chirp_batch_run
    queues the whole wave (run once untimed, then timed: the second call
    captures and launches the graphs), the wave's plans are destroyed and the
    next wave starts.  value = all 24 observations' antenna*DM*samples over
    the sum of the waves' timed calls."""
    import torch
    import paper_1109_3186_gb300 as chirp
    from paper_1109_3186_gb300 import skymodel
    g = np.random.default_rng(1004)
    shapes = []
    for i in range(24):
        M = int(g.integers(8, 65))
        N = int(2 ** g.integers(20, 25))
        nd = int(g.integers(32, 513))
        dm_max = float(g.uniform(50.0, 300.0))
        bw = float(g.uniform(16e6, 64e6))
        L = int(2 ** g.integers(9, 14))
        shapes.append((i, M, N, nd, dm_max, bw, L))
    units, total_s, waves, budget, peak_used = 0, 0.0, [], 200e9, 0
    pending = list(shapes)
    while pending:
        plans, xs, outs, used, wave = [], [], [], 0, []
        try:
            while pending:
                i, M, N, nd, dm_max, bw, L = pending[0]
                scb = skymodel.chimageator_medium(n_samp=N, n_dm=nd, n_ant=M, dm_max=dm_max,
                                                  nfft_min=1 << 16, dump_len=L, n_side=8,
                                                  n_pulse=0, seed=3000 + i, bw=bw)
                st = torch.cuda.Stream()
                try:
                    pl = chirp.Plan.from_scenario(scb, stream=st,
                                                  flags=chirp.FLAG_GRAPHS | chirp.FLAG_LEAN)
                except chirp.ChirpError:  # does not fit beside this wave's plans
                    if not plans:
                        raise
                    break
                # workspace (one group's spectra), the voltage buffer the
                # visibility form allocates on its first run, output, input
                need = pl.info["workspace_bytes"] + 4 * nd * pl.n_dump * pl.n_pix + 8 * M * N + \
                    (8 * M * N if pl.info["beam_mode"] in (1, 3, 5) else 0)
                free, _ = torch.cuda.mem_get_info()
                if plans and (used + need > budget or need > free - 8e9):
                    pl.close()
                    break
                pending.pop(0)
                used += need
                plans.append(pl)
                xs.append(torch.complex(torch.randn(M, N, device="cuda"),
                                        torch.randn(M, N, device="cuda")) * (0.5 ** 0.5))
                outs.append(torch.empty((nd, pl.n_dump, pl.n_pix), dtype=torch.float32,
                                        device="cuda"))
                units += pl.info["valid_samples"]
                wave.append([M, N, nd, round(dm_max, 1), round(bw / 1e6, 1), L])
            bes = [1] * len(plans)
            torch.cuda.synchronize()
            chirp.chirp_batch_run(plans, xs, outs, bes)  # eager (lazy allocations)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            chirp.chirp_batch_run(plans, xs, outs, bes)  # captured and launched
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            for pl in plans:
                pl.status()
            total_s += dt
            peak_used = max(peak_used, used)
            waves.append({"observations": len(plans), "s": dt, "shapes_M_N_ndm_dmmax_MHz_L": wave})
        finally:
            for pl in plans:
                pl.close()
            del xs, outs
            torch.cuda.empty_cache()
    return {"value": units / total_s, "unit": UNIT, "ms_per_batch": total_s * 1e3,
            "observations": sum(w["observations"] for w in waves), "waves": waves,
            "peak_device_bytes": peak_used,
            "recipe": "seeded: 2^20-2^24 samples, 32-512 DMs over 0-U(50,300), 8-64 antennas, "
                      "16-64 MHz, dumps 2^9-2^13, 8x8 beams; lean plans, one stream each, CUDA "
                      "graphs, waves of at most 200 GB, host-timed"}


def cpi_search(sc, xd, stream, args, peaks):
    """The paper's own Chirpolator pre-integrator (pair mixing, block-based
    sliding DFTs, moving sums, matched-filter image; chirp_cpi_run) on the
    same observation: the trial DMs above 0 (the linear-chirp model needs a
    sweep), blocks of 2048 samples, F = 2.  Device buffers, CUDA events on the
    plan's stream; per-pass times from a separate loop of single runs."""
    import torch
    from paper_1109_3186_gb300.cpi import CPI_STAGES, CpiPlan
    dms = sc.dms[sc.dms > 0]
    L, F = 2048, 2
    plan = CpiPlan(sc.xyz, sc.f0, sc.bw, sc.n_samp, dms, L, sc.pix_lm, F, k_dm=sc.k_dm,
                   stream=stream)
    E = torch.empty((len(dms), plan.n_blk, plan.n_pix), dtype=torch.float32, device="cuda")
    for _ in range(max(3, args.warmup)):
        plan.run(xd, E)
    torch.cuda.synchronize()
    k = max(3, args.steps)
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(k):
        plan.run(xd, E)
    a1.record(stream)
    torch.cuda.synchronize()
    ms = a0.elapsed_time(a1) / k
    st = dict.fromkeys(CPI_STAGES, 0.0)
    for _ in range(3):
        plan.run(xd, E)
        for name, v in plan.timing().items():
            st[name] += v / 3
    nws = [plan.layout(d)["n_win"] for d in range(len(dms))]
    plan_cc = CpiPlan(sc.xyz, sc.f0, sc.bw, sc.n_samp, dms, L, sc.pix_lm, F, k_dm=sc.k_dm,
                      stream=stream, image_mode=1)
    for _ in range(2):
        plan_cc.run(xd, E)
    a0.record(stream)
    for _ in range(k):
        plan_cc.run(xd, E)
    a1.record(stream)
    torch.cuda.synchronize()
    ms_cc = a0.elapsed_time(a1) / k
    plan_cc.close()
    windows = sum(max(0, plan.n_blk - nw + 1) for nw in nws)
    units = sc.n_ant * len(dms) * plan.n_blk * L
    sm_max = peaks.get("sm_max_mhz", FALLBACK_PEAKS["sm_max_mhz"])
    alu = N_SM * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    hbm = peaks.get("hbm_gbs", FALLBACK_PEAKS["hbm_gbs"])
    nk = 2 * plan.max_bin + 1
    # image: one complex multiply-add (8 flops) per (window, pixel, pair, filter bin), + |P|^2
    img_flops = 8.0 * windows * plan.n_pix * plan.n_pair * (2 * F + 1) + 3.0 * windows * plan.n_pix
    # moving sums: each (DM, block, bin, pair) reads V twice and writes X (8 B each)
    cic_bytes = 24.0 * len(dms) * plan.n_blk * nk * plan.n_pair
    # moments: read the voltages once, write J moments per (sub-block, pair)
    mom_bytes = 8.0 * sc.n_ant * plan.n_blk * L + 8.0 * plan.n_blk * (L // plan.info["sub_len"]) \
        * plan.info["n_terms"] * plan.n_pair
    # image on the tensor cores: the dense-in-bins contraction, 2 x (2 n_pix
    # rows) x (2 nk n_pair real K) x (complete-window tiles of 256) per DM, one
    # term; the split-BF16 form executes three such products (K and rows
    # padded to the 32 / 128 tiles)
    rows = -(-2 * plan.n_pix // 128) * 128
    kpad = -(-2 * nk * plan.n_pair // 32) * 32
    tiles = sum(max(0, -(-plan.n_blk // 256) - (nw - 1) // 256) for nw in nws)
    dense = 2.0 * (2 * plan.n_pix) * (2 * nk * plan.n_pair) * windows
    executed = 3 * 2.0 * rows * kpad * 256 * tiles
    bf16 = peaks.get("bf16_tflops_sustained", FALLBACK_PEAKS["bf16_tflops_sustained"])
    roof = {
        "moments": ("hbm", mom_bytes / (st["moments"] * 1e-3) / 1e9, hbm, "GB/s"),
        "cic": ("hbm", cic_bytes / (st["cic"] * 1e-3) / 1e9, hbm, "GB/s"),
        "image": ("tensor", dense / (st["image"] * 1e-3) / 1e12, bf16, "TFLOP/s"),
    }
    out = {"value": units / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": k,
           "beam_dm_windows_per_s": windows * plan.n_pix / (ms * 1e-3),
           "n_dm": len(dms), "blk_len": L, "half_width": F, "max_bin": plan.max_bin,
           "n_freq": plan.info["n_freq"], "sub_len": plan.info["sub_len"],
           "n_terms": plan.info["n_terms"], "gpu_launches_per_step": 5,
           "stages_ms": st,
           "roofline": {n: {"bound": b, "achieved": a, "peak": pk, "unit": u, "frac": a / pk}
                        for n, (b, a, pk, u) in roof.items()},
           "image_tensor_executed_tflops": executed / (st["image"] * 1e-3) / 1e12,
           "image_useful_sparse_tflops": img_flops / (st["image"] * 1e-3) / 1e12,
           "cuda_core_image_ms_per_step": ms_cc,
           "dtype": "f32 (moving sums compensated, two floats; image: split-bf16 x3 on tensor "
                    "cores, f32 acc)",
           "note": "paper's own pre-integrator on the raw voltages: DMs > 0 of the 64"}
    plan.close()
    return out


def chimg_ula_search(stream, args):
    """The paper's Chimageator pre-integrator (chirp_chimg_run) on a uniform
    linear array shaped like the benchmark's observation: 12 antennas spaced
    6000/11 m along u, 32 MHz at 1.4 GHz, 2^22 samples (seeded noise and one
    linear chirp), the 63 trial DMs above 0 of 64 in 0-300, 64 directions over
    +-0.5 deg, dumps of 4096, Ns = 32, F = 2.  Device buffers, CUDA events on
    the plan's stream."""
    import torch
    from paper_1109_3186_gb300.chimg import ChimgPlan
    M, D, f0, bw, n, L = 12, 6000.0 / 11, 1.4e9, 32e6, 1 << 22, 4096
    if args.n_samp:
        n = args.n_samp
    dms = np.linspace(0.0, 300.0, 64)[1:]
    l_dirs = np.sin(np.radians(np.linspace(-0.5, 0.5, 64)))
    g = torch.Generator(device="cuda").manual_seed(1003)
    x = torch.randn((M, n), dtype=torch.complex64, device="cuda", generator=g)
    plan = ChimgPlan(M, D, f0, bw, n, dms, L, l_dirs, 32, 2, stream=stream)
    E = torch.empty((len(dms), plan.n_dump, len(l_dirs)), dtype=torch.float32, device="cuda")
    for _ in range(max(3, args.warmup)):
        plan.run(x, E)
    torch.cuda.synchronize()
    k = max(3, args.steps)
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(k):
        plan.run(x, E)
    a1.record(stream)
    torch.cuda.synchronize()
    ms = a0.elapsed_time(a1) / k
    windows = int(sum(max(0, plan.n_dump - w + 1) for w in plan.n_win))
    out = {"value": M * len(dms) * plan.n_dump * L / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
           "steps": k, "beam_dm_windows_per_s": windows * len(l_dirs) / (ms * 1e-3),
           "n_ant": M, "spacing_m": D, "n_dm": len(dms), "n_dir": len(l_dirs), "dump_len": L,
           "n_spatial": 32, "half_width": 2, "gpu_launches_per_step": 2,
           "dtype": "f32 (filter taps built in f64)",
           "note": "paper's own Chimageator pre-integrator, uniform linear array, seeded noise"}
    plan.close()
    return out


def chirpolator_only(sc, x, stream, args):
    """The Chirpolator search alone on the benchmark's observation: W warm-up
    and K timed steps, CUDA events on the plan's stream; one JSON line."""
    import torch
    import paper_1109_3186_gb300 as chirp
    plan = chirp.Plan.from_scenario(sc, stream=stream)
    xd = torch.from_numpy(x).cuda()
    V = torch.empty((len(sc.dms), plan.n_dump, plan.n_pair), dtype=torch.complex64, device="cuda")
    for _ in range(args.warmup):
        plan.chirpolator(xd, V)
    torch.cuda.synchronize()
    plan.stage_timing(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plan.chirpolator(xd, V)
    e1.record(stream)
    torch.cuda.synchronize()
    stage = plan.stage_timing(False)
    plan.status()
    ms = e0.elapsed_time(e1) / args.steps
    line = {"mode": "chirpolator", "ms_per_step": ms, "steps": args.steps,
            "value": plan.info["valid_samples"] / (ms * 1e-3), "unit": UNIT,
            "corr_mode": {1: "fp32_simt", 2: "tc_3xbf16", 3: "tc_bf16"}[plan.info["corr_mode"]],
            "stages_ms": {k: v[0] / args.steps for k, v in stage.items() if v[1]},
            "config": config_block(sc, 1)}
    print(json.dumps(line), flush=True)
    plan.close()
    return 0


def _roof_entry(r):
    return {k: r[k] for k in ("bound", "achieved", "peak", "unit", "frac", "peak_source")}


def timed_steps(plan, fn, k, stream):
    """Mean ms of k calls of fn on the plan's stream (CUDA events), with the
    plan's per-stage event timing on; returns (ms, per-stage totals)."""
    import torch
    fn()
    torch.cuda.synchronize()
    plan.stage_timing(True)
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(k):
        fn()
    a1.record(stream)
    torch.cuda.synchronize()
    stage = plan.stage_timing(False)
    plan.status()
    return a0.elapsed_time(a1) / k, stage


def beam_mode_leg(sc, xd, Pd, stream, mode, k, peaks, peak_kind, units):
    """One other Chimageator form on the headline workload: throughput, every
    stage's time and roofline, and (tensor-core forms) the beam GEMM's rate
    of algorithmic and of executed tensor flops."""
    import paper_1109_3186_gb300 as chirp
    pl = chirp.Plan.from_scenario(sc, beam_mode=mode, stream=stream)
    ms, stage = timed_steps(pl, lambda: pl.chimageator(xd, Pd), k, stream)
    roof = stage_roofline(sc, pl, stage, peaks, peak_kind, mode, k)
    tex = roof.pop("_tensor_executed_tflops", None)
    out = {"value": units / (ms * 1e-3), "ms_per_step": ms, "steps": k,
           "dtype": DTYPE_LABEL[mode],
           "stages_ms": {n: r["ms_per_step"] for n, r in roof.items()}}
    if "beamform" in roof:
        out["roofline"] = dict(_roof_entry(roof["beamform"]), kernel="beamform")
        if tex is not None:
            out["roofline"]["tensor_executed_tflops"] = tex
            out["roofline"]["tensor_executed_frac"] = tex / roof["beamform"]["peak"]
    pl.close()
    return out


def truedelay_leg(sc, xd, stream, peaks, peak_kind, args):
    """True-delay (wideband) beams on the headline observation for 8 x 8
    pixels over 1 deg (chirp_truedelay_run: n_pix / n_ant times the inverse
    FFT work of the phased beams), beside the phased beams of the same
    pixels; device buffers, per-stage CUDA events."""
    import torch
    import paper_1109_3186_gb300 as chirp
    from paper_1109_3186_gb300 import skymodel
    pix = skymodel.pixel_grid(8, 1.0)
    plan = chirp.Plan(sc.xyz, sc.f0, sc.bw, sc.n_samp, sc.dms, sc.dump_len, sc.nfft_min,
                      pix_lm=pix, k_dm=sc.k_dm, stream=stream)
    P = torch.empty((len(sc.dms), plan.n_dump, plan.n_pix), dtype=torch.float32, device="cuda")
    k = 2
    ms, stage = timed_steps(plan, lambda: plan.truedelay(xd, P), k, stream)
    ms_pb, _ = timed_steps(plan, lambda: plan.chimageator(xd, P), k, stream)
    first, last = plan.dump_range()
    n_valid = int(np.sum(np.maximum(0, last - first + 1)))
    # beam sequences: every (DM, block, pixel) is one inverse FFT of its group's length
    pts = sum(plan.n_pix * plan.dm_layout(d)["n_blk"] * plan.dm_layout(d)["nfft"]
              for d in range(len(sc.dms)) if last[d] >= first[d])
    hbm = peaks.get("hbm_gbs", FALLBACK_PEAKS["hbm_gbs"])
    st = {n: stage[n][0] / k for n in ("td_spectra", "inv_rows", "inv_cols", "forward", "chirp")
          if stage[n][1]}
    out = {"value": plan.info["valid_samples"] / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
           "steps": k, "n_pix": plan.n_pix,
           "beam_dm_dumps_per_s": n_valid * plan.n_pix / (ms * 1e-3),
           "phased_beams_same_pixels_ms": ms_pb, "stages_ms": st,
           "beam_ifft_points_per_step": pts,
           "dtype": "f32 (weight phases in 64-bit fixed point from f64)",
           "note": "8x8 pixels over 1 deg on the headline observation"}
    # the beam inverse passes: per point 8 B written and 8 B / (DMs per launch)
    # read (the row pass reads a group's beam spectra once for up to dm_chunk
    # DMs; the chirp tables are negligible), 8 B read (column pass; powers by
    # one atomic add per row and dump)
    if "inv_rows" in st and "inv_cols" in st:
        chunk = max(1, plan.info.get("dm_chunk", 1))
        byts = (8.0 + 8.0 / chunk) * pts + 8.0 * pts
        rate = byts / ((st["inv_rows"] + st["inv_cols"]) * 1e-3) / 1e9
        out["roofline"] = {"kernel": "beam inverse passes", "bound": "hbm", "achieved": rate,
                           "peak": hbm, "unit": "GB/s", "frac": rate / hbm,
                           "peak_source": peak_kind}
    plan.close()
    return out


def chirpolator_6ant_leg(stream, peaks, peak_kind, args):
    """The plain-FP32 Chirpolator workload at its stated shape: 6 antennas
    within 2 km, 8 MHz at 1.4 GHz, 2^20 samples, 16 DMs in 0-150, FFT 2^16,
    dumps of 1024, one burst (seed 1001); device buffers."""
    import torch
    import paper_1109_3186_gb300 as chirp
    from paper_1109_3186_gb300 import skymodel
    sc = skymodel.chirpolator_small()
    xd = torch.from_numpy(sc.voltages()).cuda()
    plan = chirp.Plan.from_scenario(sc, stream=stream)
    V = torch.empty((len(sc.dms), plan.n_dump, plan.n_pair), dtype=torch.complex64, device="cuda")
    k = max(20, 4 * args.steps)
    ms, stage = timed_steps(plan, lambda: plan.chirpolator(xd, V), k, stream)
    roof = stage_roofline(sc, plan, stage, peaks, peak_kind, None, k)
    roof.pop("_tensor_executed_tflops", None)
    first, last = plan.dump_range()
    n_valid = int(np.sum(np.maximum(0, last - first + 1)))
    dom = max(roof, key=lambda n: roof[n]["ms_per_step"])
    out = {"value": plan.info["valid_samples"] / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
           "steps": k, "baseline_dm_dumps_per_s": n_valid * plan.n_pair / (ms * 1e-3),
           "corr_mode": {1: "fp32_simt", 2: "tc_3xbf16", 3: "tc_bf16"}[plan.info["corr_mode"]],
           "dtype": "f32",
           "workload": "chirpolator: 6 ant within 2 km, 8 MHz @ 1.4 GHz, 2^20 samples/antenna, "
                       "16 DMs 0-150, FFT 2^16, dump 1024",
           "l2": "voltages 50 MB, spectra 86 MB: may stay resident in L2 (129 MB)",
           "roofline": dict(_roof_entry(roof[dom]), kernel=dom),
           "stages_ms": {n: r["ms_per_step"] for n, r in roof.items()}}
    plan.close()
    return out


def precision_channel_leg(stream, peaks, peak_kind, args):
    """One coarse channel of the precision form at its stated shape: 36
    antennas within 6 km, 42 MHz at 1.253 GHz (channel 0 of 8 x 42 MHz about
    1.4 GHz), complex int8 voltages (noise drawn on the device, 16 counts
    rms per component), 2^24 samples, 256 DMs (0, then log-spaced 1-2000),
    64 x 64 beams over 1 deg, dumps of 4096.  Three forms: the library's
    choice (exact visibility identity), the visibility identity with a BF16
    tensor-core correlator, and the one-term BF16 beam GEMM on the tensor
    cores.  About 100 GB of device memory per plan."""
    import torch
    import paper_1109_3186_gb300 as chirp
    from paper_1109_3186_gb300 import skymodel
    sc = skymodel.precision_form(channel=0, n_pulse=0)
    reduced = args.precision_only and (args.n_samp or args.dms)
    if reduced:  # profiling: a shorter series and the lowest DMs
        if args.n_samp:
            sc.n_samp = args.n_samp
        if args.dms:
            sc.dms = sc.dms[:args.dms]
    M, N = sc.n_ant, sc.n_samp
    g = torch.Generator(device="cuda").manual_seed(1003)
    q = torch.randn((M, N, 2), generator=g, device="cuda").mul_(16.0).round_().clamp_(-127, 127)
    q = q.to(torch.int8)
    scale = np.full(M, (0.5 ** 0.5) / 16.0, np.float32)
    out = {"workload": "precision form, one channel: 36 ant within 6 km, 42 MHz @ 1.253 GHz, "
                       "int8, 2^24 samples/antenna, 256 DMs (0 + log 1-2000), 64x64 beams, "
                       "dump 4096 (noise drawn on the device)"}
    forms = (("auto", dict()),
             ("vis_corr_tc_bf16", dict(beam_mode=chirp.BEAM_VIS, corr_mode=chirp.CORR_TC_BF16)),
             ("tc_bf16", dict(beam_mode=chirp.BEAM_TC_BF16)))
    if reduced:
        forms = forms[:1]
        out["workload"] = "REDUCED (profiling): " + out["workload"] + \
            ", here %d samples, %d DMs" % (N, len(sc.dms))
    P = None
    for name, kw in forms:
        plan = chirp.Plan.from_scenario(sc, stream=stream, in_type=chirp.IN_CI8, in_scale=scale,
                                        **kw)
        if P is None:
            P = torch.empty((len(sc.dms), plan.n_dump, plan.n_pix), dtype=torch.float32,
                            device="cuda")
        ms, stage = timed_steps(plan, lambda: plan.chimageator(q, P), 2, stream)
        mode = plan.info["beam_mode"]
        roof = stage_roofline(sc, plan, stage, peaks, peak_kind, mode, 2)
        tex = roof.pop("_tensor_executed_tflops", None)
        dom = max(roof, key=lambda n: roof[n]["ms_per_step"])
        first, last = plan.dump_range()
        beam_dumps = int(np.sum(np.maximum(0, last - first + 1))) * plan.n_pix
        ent = {"value": plan.info["valid_samples"] / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
               "steps": 2, "beam_mode": MODE_NAME[mode],
               "corr_mode": {1: "fp32_simt", 2: "tc_3xbf16", 3: "tc_bf16"}[plan.info["corr_mode"]],
               "beam_dm_dumps_per_s": beam_dumps / (ms * 1e-3),
               "workspace_gb": plan.info["workspace_bytes"] / 1e9,
               "roofline": dict(_roof_entry(roof[dom]), kernel=dom),
               "stages_ms": {n: r["ms_per_step"] for n, r in roof.items()}}
        if "beamform" in roof and roof["beamform"]["bound"] == "tensor":
            ent["beamform_roofline"] = _roof_entry(roof["beamform"])
            if tex is not None:
                ent["beamform_roofline"]["tensor_executed_tflops"] = tex
        out[name] = ent
        plan.close()
        torch.cuda.empty_cache()
    del P, q
    return out


def run_ours(args):
    import torch
    import paper_1109_3186_gb300 as chirp

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    stream = torch.cuda.current_stream()
    if args.precision_only:
        line = precision_channel_leg(stream, *load_peaks(), args)
        line["mode"] = "precision_36ant_channel"
        print(json.dumps(line), flush=True)
        return 0
    sc = scenario(rank, args)
    x = sc.voltages()
    if args.chirpolator_only:
        return chirpolator_only(sc, x, stream, args)
    if args.chimg_only:
        line = chimg_ula_search(stream, args)
        line["mode"] = "chimg_ula"
        print(json.dumps(line), flush=True)
        return 0
    if args.truedelay_only:
        line = truedelay_leg(sc, torch.from_numpy(x).cuda(), stream, *load_peaks(), args)
        line["mode"] = "truedelay"
        line["config"] = config_block(sc, 1)
        print(json.dumps(line), flush=True)
        return 0
    if args.cpi_only:
        import torch as _t
        line = cpi_search(sc, _t.from_numpy(x).cuda(), stream, args, load_peaks()[0])
        line["mode"] = "cpi"
        line["config"] = config_block(sc, 1)
        print(json.dumps(line), flush=True)
        return 0
    plan = chirp.Plan.from_scenario(sc, beam_mode=args.beam_mode, stream=stream)
    n_dm, n_dump, n_pix = len(sc.dms), plan.n_dump, plan.n_pix
    xd = torch.from_numpy(x).cuda()
    Pd = torch.empty((n_dm, n_dump, n_pix), dtype=torch.float32, device="cuda")
    units = plan.info["valid_samples"]
    first, last = plan.dump_range()
    beam_dumps = int(np.sum(np.maximum(0, last - first + 1))) * n_pix

    for _ in range(args.warmup):
        plan.chimageator(xd, Pd)
    torch.cuda.synchronize()
    # Stage breakdown: the same number of steps with an event pair around
    # every launch (a few microseconds each), before the timed region.
    plan.stage_timing(True)
    for _ in range(args.steps):
        plan.chimageator(xd, Pd)
    torch.cuda.synchronize()
    stage = plan.stage_timing(False)
    dom_stage = max(stage, key=lambda k: stage[k][0])
    barrier()
    torch.cuda.synchronize()

    # Timed region: only the dominant stage's launches carry event pairs (its
    # per-launch duration for the roofline comes from these very steps).
    peaks, peak_kind = load_peaks()
    clocks = ClockSampler(device_uuid(torch, local))
    clocks.start()
    plan.stage_timing(True, stages=[dom_stage])
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plan.chimageator(xd, Pd)
    e1.record(stream)
    torch.cuda.synchronize()
    stage[dom_stage] = plan.stage_timing(False)[dom_stage]
    plan.status()
    clk = clocks.stop()
    barrier()
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ms, dist, "cuda")
    value = job_value(units, world, ms * 1e-3)

    # end to end through the same call: pinned host input, host output
    e2e = None
    if not args.no_e2e:
        xh = torch.from_numpy(x).pin_memory()
        Ph = torch.empty((n_dm, n_dump, n_pix), dtype=torch.float32).pin_memory()
        plan.chimageator(xh, Ph)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            plan.chimageator(xh, Ph)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / args.steps
        dt = max_over_ranks(dt, dist, "cuda")
        e2e = {"value": job_value(units, world, dt), "unit": UNIT, "ms_per_step": dt * 1e3,
               "h2d_bytes_per_step": int(x.nbytes), "d2h_bytes_per_step": int(Ph.numel() * 4)}

    roof = stage_roofline(sc, plan, stage, peaks, peak_kind, plan.info["beam_mode"], args.steps)
    tensor_exec = roof.pop("_tensor_executed_tflops", None)
    dom = max(roof, key=lambda k: roof[k]["ms_per_step"]) if roof else None
    # kernels launched in the timed steps: one per timed stage launch, plus the
    # second kernel (row pass) of every forward launch
    launches = int(sum(n for _, n in stage.values())) + int(stage.get("forward", (0, 0))[1])

    # the other beam modes and candidate detection, timed the same way (rank 0)
    alt = {}
    if not args.no_alt and rank == 0:
        for mode in (2, 4, 5, 3, 1):
            if mode == plan.info["beam_mode"]:
                continue
            k = 2 if mode == 1 else max(2, args.steps // 2)
            alt[MODE_NAME[mode]] = beam_mode_leg(sc, xd, Pd, stream, mode, k, peaks, peak_kind,
                                                 units)
        # the Chirpolator back-end on the same voltages and DMs
        Vd = torch.empty((n_dm, n_dump, plan.n_pair), dtype=torch.complex64, device="cuda")
        plan.chirpolator(xd, Vd)
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        k = max(2, args.steps // 2)
        a0.record(stream)
        for _ in range(k):
            plan.chirpolator(xd, Vd)
        a1.record(stream)
        torch.cuda.synchronize()
        ms2 = a0.elapsed_time(a1) / k
        n_valid_dumps = int(np.sum(np.maximum(0, last - first + 1)))
        alt["chirpolator"] = {"value": units / (ms2 * 1e-3), "ms_per_step": ms2, "steps": k,
                              "baseline_dm_dumps_per_s": n_valid_dumps * plan.n_pair / (ms2 * 1e-3),
                              "corr_mode": {1: "fp32_simt", 2: "tc_3xbf16", 3: "tc_bf16"}[
                                  plan.info["corr_mode"]]}
        del Vd
        alt["cpi"] = cpi_search(sc, xd, stream, args, peaks)
        try:
            alt["chimg_ula"] = chimg_ula_search(stream, args)
        except Exception as exc:  # an auxiliary leg: record, do not lose the line
            alt["chimg_ula"] = {"error": str(exc)}
        alt.update(extra_forms(sc, plan, xd, stream, args))
        alt["chirpolator_6ant"] = chirpolator_6ant_leg(stream, peaks, peak_kind, args)
        try:
            alt["truedelay_64pix"] = truedelay_leg(sc, xd, stream, peaks, peak_kind, args)
        except Exception as exc:  # an auxiliary leg: record, do not lose the line
            alt["truedelay_64pix"] = {"error": str(exc)}
        if not args.no_precision:
            try:
                alt["precision_36ant_channel"] = precision_channel_leg(stream, peaks, peak_kind,
                                                                       args)
            except Exception as exc:  # an auxiliary leg: record, do not lose the line
                alt["precision_36ant_channel"] = {"error": str(exc)}
            torch.cuda.empty_cache()
        plan.chimageator(xd, Pd)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cands = plan.detect(Pd, 6.0, max_cand=1 << 20)
        alt["detect"] = {"ms": 1e3 * (time.perf_counter() - t0), "candidates": int(len(cands)),
                         "snr_min": 6.0, "note": "chirp_detect on one step's powers, host-timed"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": DTYPE_LABEL[plan.info["beam_mode"]],
                "data": "synthetic (seeded sky model: noise + dispersed bursts)",
                "config": config_block(sc, world),
                "beam_dm_dumps_per_s": world * beam_dumps / (ms * 1e-3),
                "gpu_launches": launches, "clocks": clk,
                "stage_timing": "CUDA events per launch on the plan's stream: the roofline "
                                "stage inside the timed steps, the other stages in an "
                                "instrumented pass of as many steps just before them"}
        if e2e:
            line["e2e"] = e2e
        if alt:
            line["other_modes"] = alt
        if dom:
            r = roof[dom]
            traffic = None
            if dom == "beamform" and plan.info["beam_mode"] == 2:
                per = committed_traffic(["beamform_tc.cu", "tc.cuh"], "k_beam_tc<256>")
                if per is not None:  # bytes per valid-dump DM*sample x samples per launch
                    traffic = per * beam_dumps / n_pix * sc.dump_len / n_dm
            elif dom == "inv_rows":
                per = committed_traffic(["dedisperse.cu", "fft.cuh"], "k_inv_rows_multi<4096>")
                if per is not None:
                    traffic = per * plan.info["ifft_points"] / n_dm
            line["roofline"] = {"kernel": dom, "bound": r["bound"], "achieved": r["achieved"],
                                "peak": r["peak"], "unit": r["unit"], "frac": r["frac"],
                                "traffic": traffic, "peak_source": r["peak_source"]}
            if dom == "beamform" and tensor_exec is not None:
                # algorithmic flops above; the split-BF16 contraction executes more
                line["roofline"]["tensor_executed_tflops"] = tensor_exec
                line["roofline"]["tensor_executed_frac"] = tensor_exec / r["peak"]
            line["stages"] = roof
        if not args.no_cpu_baseline:
            u, dt, cores, text = cpu_sample(sc, x, args.cpu_dumps)
            line["cpu_baseline"] = {"value": u / dt, "unit": UNIT, "cores": cores,
                                    "kind": "oracle", "sample": text, "seconds": dt}
        print(json.dumps(line), flush=True)
    plan.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
