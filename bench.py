"""Throughput of the Gibbs TOD step (decode -> project -> gain -> n_corr ->
bin -> solve) on synthetic Planck-LFI-shaped data.

The headline workload is the batched 70 GHz-like band: 12 detectors x 2000
scans of U[150k, 300k] samples at 78.8 Hz, Nside 1024 (5.3e9 samples per
step).  The same step on the 30 GHz-like band and the added rows (noise
PSD step, compressed TOD and flags, smooth gain prior) are measured in a
secondary section.

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle on a
bounded sample of the same workload instead.  Launched by torchrun for
N > 1 GPUs, the band is split into contiguous scan ranges of nearly equal
sample counts, one per rank; every rank runs its scans' step and the
per-pixel normal equations are reduced over the ranks by pixel range (the
one exchange of the step), solved per range and gathered; the max time
over ranks is reported.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TOD samples/s per Gibbs TOD step"
WORKLOAD = "lfi70"
SECONDARY = "lfi30"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return rank, ws


def max_over_ranks(x: float, device="cuda") -> float:
    """The largest x over the ranks of the default process group (x itself
    when there is no group or one rank)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.th = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.th:
            self.th.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# DRAM bytes (read + write) of a kernel per byte of its algorithmic traffic,
# from an ncu capture of that kernel on a smaller case of the same band (the
# summary under profiles/ gives the command and the figures); a full launch's
# traffic is that ratio times its algorithmic bytes (every pass moves each
# sample's values in proportion).  Valid only while the kernel's sources
# hash to the digest taken with it; otherwise the traffic is reported as null.
TX_SOURCES = ["csrc/k_tx.cu", "csrc/fft_reg.cuh", "csrc/common.cuh", "csrc/internal.cuh"]
KERNEL_TRAFFIC = {
    # profiles/k_tx_passes_lfi70_40scans.md: the first CG filter launch of the
    # 480-detscan case (every detscan iterating: 8 x 104,686,200 algorithmic
    # bytes) read 0.419479 GB and wrote 0.362901 GB of DRAM
    "k_nc_filter": {"dram_per_algorithmic_byte": (0.419479e9 + 0.362901e9) / (8.0 * 104686200),
                    "sources": TX_SOURCES,
                    "sha256": "ece2d38fbdda3dc570e0a2892d3cf1950c6666566aa940065793cfe39f668a1e"},
}


def sources_digest(sources) -> str | None:
    h = hashlib.sha256()
    for rel in sources:
        try:
            with open(os.path.join(ROOT, "paper_2201_03509_gb300", rel), "rb") as f:
                h.update(f.read())
        except OSError:
            return None
    return h.hexdigest()


def build_band(cfg, scans=None):
    """The band (or the listed scans of it) generated straight into
    concatenated arrays and ingested by the library; the uncompressed
    pointing is dropped once it is encoded."""
    import synth
    import paper_2201_03509_gb300 as tg
    arr = synth.make_band_arrays(cfg, tg.kept_lengths(cfg), scans=scans)
    ing = tg.ingest_arrays(arr)
    arr.pix = arr.psi = None
    return arr, ing


# ---------------------------------------------------------------------------
# algorithmic work per stage (compulsory HBM bytes of this design)
# ---------------------------------------------------------------------------
def stage_bytes(N, npix, npairs, comp_bytes, ncorr_bytes):
    """Compulsory HBM bytes of each stage for one step.  The gain and n_corr
    transforms go through one complex intermediate of 4 bytes per sample
    between their column and row passes (the two-pass transform of the
    measurement plan)."""
    return {
        "decode": comp_bytes + 6.0 * N,                 # streams in, pix int32 + psi uint16 out
        "project": 6.0 * N + 4.0 * N,                   # pix, psi in, s out (map gathers hit L2)
        # columns: s, flags in, Y out; rows: Y in and out; inverse columns: Y, d, flags in
        "gain": ((4.0 + 0.125 + 4.0) + 8.0 + (4.0 + 4.0 + 0.125)) * N,
        "ncorr": ncorr_bytes,
        "bin": 10.0 * N + N / 8.0 + 6.0 * N + 80.0 * npairs,   # d, n_corr, psi, flags, load order + slot, runs out
        "solve": 76.0 * npix + 61.0 * npix,
    }


def ncorr_algorithmic_bytes(lens, iters, flagged):
    """HBM bytes of one n_corr draw: right-hand side (columns: d, s, flags
    in, Y out; rows: Y in and out; inverse columns: Y, flags in, x0 out),
    then per CG iteration of a flagged detscan (scatter: Y out; rows: Y in
    and out; gather: Y in, flags) and its correction (scatter; rows;
    inverse columns: Y, x0 in, x out)."""
    lens = np.asarray(lens, np.float64)
    b = lens * ((8.0 + 0.125 + 4.0) + 8.0 + (4.0 + 0.125 + 4.0))
    b += np.where(flagged, lens * ((4.0 + 8.0 + 4.0 + 0.125) * np.asarray(iters) + (4.0 + 8.0 + 12.0)), 0.0)
    return float(b.sum())


def kernel_bytes(N, npix, npairs, comp_bytes, lens, iters, flagged, launched=8):
    """Algorithmic HBM bytes of one step per kernel class (the names of
    tod_kernel_name).  Transforms: the column pass moves its inputs and the
    complex intermediate Y (4 B per sample), the row pass reads and writes
    Y, the inverse column pass reads Y and moves its outputs.  A CG pass
    touches only the detscans still iterating: iteration i of detscan q
    runs when q took more than i iterations; the cooperative tail runs the
    iterations past the `launched` ones (the CG iterations launched one by
    one); the correction passes run over every detscan that ran the CG.
    Small per-detscan kernels are left out."""
    lens = np.asarray(lens, np.float64)
    it = np.asarray(iters, np.float64)
    fl = np.asarray(flagged, bool)
    act = [float(lens[fl & (it > i)].sum()) for i in range(launched)]
    tail = float((lens * np.maximum(it - launched, 0) * fl).sum())
    ran = float(lens[fl & (it > 0)].sum())
    return {
        "k_decode": comp_bytes + 6.0 * N,
        "k_project": 10.0 * N,
        "k_gain_cols": 8.125 * N, "k_gain_rows": 8.0 * N, "k_gain_colsinv": 8.125 * N,
        "k_nc_flag_count": N / 8.0, "k_nc_flag_write": N / 8.0 + N / 4.0,
        "k_nc_rhs_cols": 12.125 * N, "k_nc_rhs_rows": 8.0 * N, "k_nc_x0_cols": 8.125 * N,
        "k_nc_scatter": 4.0 * sum(act), "k_nc_filter": 8.0 * sum(act), "k_nc_gather": 4.125 * sum(act),
        "k_nc_tail": 16.125 * tail,
        "k_nc_scatter_final": 4.0 * ran, "k_nc_filter_final": 8.0 * ran, "k_nc_gather_final": 12.125 * ran,
        "k_bin": 16.125 * N + 80.0 * npairs,
        "k_reduce": 80.0 * npairs + 84.0 * npix,
        "k_solve": 137.0 * npix,
    }


def _event():
    import torch
    return torch.cuda.Event(enable_timing=True)


def measure_step(args, cfg, arr, ing, local, rank, ws, label="main"):
    """Build the plan and step of one band (this rank's scan range under
    torchrun) and time it."""
    import torch
    import paper_2201_03509_gb300 as tg
    from paper_2201_03509_gb300.step import GibbsTODStep
    nscan_local = (len(ing["offsets"]) - 1) // cfg.ndet
    m4 = np.zeros((arr.npix, 4), np.float32)
    m4[:, :3] = arr.map_tqu.T
    map_in = torch.from_numpy(m4).cuda()
    tuned = None
    tp, rmax = 0, 0
    if args.autotune and label == "main":
        # measured tile shape (column pairs, largest radix) on the band's first scans
        from paper_2201_03509_gb300.autotune import autotune
        tp, rmax, tms = autotune(cfg.nside, cfg.ndet, nscan_local, cfg.fsamp, ing["offsets"], ing["pix_streams"],
                                 ing["psi_streams"], ing["tod"], ing["flag_words"], arr.psd, map_in,
                                 nscan_sample=args.tune_scans, device=local)
        tuned = {"tile_pairs": tp, "max_radix": rmax,
                 "candidates_ms": {"T%d_R%d" % k: round(v, 3) for k, v in sorted(tms.items())}}
    plan = tg.Plan(cfg.nside, cfg.ndet, nscan_local, cfg.fsamp, ing["offsets"], ing["pix_streams"],
                   ing["psi_streams"], tile_pairs=tp, device=local, max_radix=rmax)
    shard = None
    if ws > 1:
        from paper_2201_03509_gb300.shard import ShardedMaps
        shard = ShardedMaps(plan, ws, rank)
    step = GibbsTODStep(plan, arr.psd, ing["flag_words"], cg_tol=args.cg_tol, shard=shard)
    step.set_tod(ing["tod"])
    N, nq, npix = plan.N, plan.nq, plan.npix
    stream = torch.cuda.current_stream()

    def one(it):
        step.run(map_in, tg.Rng(args.seed, 0, it), tg.MODE_DRAW)

    for w in range(args.warmup):
        one(10_000 + w)
    torch.cuda.synchronize()
    plan.status()
    sampler = ClockSampler(local)
    sampler.start()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    t0, t1 = _event(), _event()
    t0.record(stream)
    for k in range(args.steps):
        one(k)                     # the step as a user runs it (GibbsTODStep.run)
    t1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    clocks = sampler.stop()
    elapsed = max_over_ranks(t0.elapsed_time(t1) / 1e3)
    iters = step.cg_iters.cpu().numpy()

    # the same step captured in CUDA graphs (iteration read on the device),
    # timed right after the eager steps
    graph_ms = None
    if not args.no_graph and ws == 1:
        try:
            step.capture(map_in, args.seed, 0, tg.MODE_DRAW)
            for k in range(2):
                step.replay(30_000 + k)
            torch.cuda.synchronize()
            g0, g1 = _event(), _event()
            g0.record(stream)
            for k in range(args.steps):
                step.replay(40_000 + k)
            g1.record(stream)
            torch.cuda.synchronize()
            graph_ms = g0.elapsed_time(g1) / args.steps
            step.graph = None
            step.graphs = []
        except Exception as ex:          # report, do not hide
            graph_ms = "capture failed: %s" % ex

    # per-stage times: the step's calls one by one on one stream with events
    # between them (the n_corr preparation, which the step overlaps with
    # decode, projection and gain, as its own stage), after the timed region
    names = ["decode", "project", "gain", "ncorr_prepare", "ncorr", "bin", "solve"]

    def calls(rng, ev=None):
        p = step.plan
        mark = (lambda i: ev[i].record(stream)) if ev else (lambda i: None)
        mark(0)
        p.decode(step.pix, step.psi)
        mark(1)
        p.project(map_in, step.pix, step.psi, None, step.s)
        mark(2)
        p.sample_gain(step.d, step.s, step.flags, step.psd, rng, tg.MODE_DRAW, step.gain, step.mu, step.sigma)
        mark(3)
        p.ncorr_prepare(step.psd)
        mark(4)
        p.sample_ncorr_prepared(step.d, step.s, step.gain, step.flags, step.psd, rng, tg.MODE_DRAW, step.ncorr,
                                step.cg_iters, step.cg_tol, step.cg_maxiter)
        mark(5)
        p.bin(step.psi, step.d, step.ncorr, step.gain, step.flags, step.psd, step.A, step.b, step.hits)
        mark(6)
        p.solve_maps(step.A, step.b, step.hits, step.rcond_min, step.map, step.map32, step.rcond, step.valid)
        mark(7)

    evs = [[_event() for _ in range(8)] for _ in range(args.steps)]
    for k in range(args.steps):
        calls(tg.Rng(args.seed, 0, 20_000 + k), evs[k])
    torch.cuda.synchronize()
    st = plan.status(raise_on_error=False)
    stage_ms = {nm: float(np.mean([evs[k][i].elapsed_time(evs[k][i + 1]) for k in range(args.steps)]))
                for i, nm in enumerate(names)}
    iters_stage = step.cg_iters.cpu().numpy()
    # per-kernel times: the same calls with the library's kernel timing on
    # (two events around every launch, on the launching stream)
    kt_steps = 2
    plan.set_kernel_timing(True)
    its_kt = []
    for k in range(kt_steps):
        calls(tg.Rng(args.seed, 0, 25_000 + k))
        its_kt.append(step.cg_iters.clone())
    plan.set_kernel_timing(False)
    kt = plan.kernel_times()
    kernel_ms = {nm: (ms / kt_steps, n / kt_steps) for nm, (ms, n) in kt.items()}
    iters_kt = [t.cpu().numpy() for t in its_kt]
    plan.status(raise_on_error=False)

    # the eager step with the pointing decoded in-step (no next-step decode
    # under the n_corr draw)
    inline_ms = None
    if not args.no_graph and ws == 1:
        step.lookahead = False
        for k in range(2):
            one(45_000 + k)
        torch.cuda.synchronize()
        h0, h1 = _event(), _event()
        h0.record(stream)
        for k in range(args.steps):
            one(46_000 + k)
        h1.record(stream)
        torch.cuda.synchronize()
        inline_ms = h0.elapsed_time(h1) / args.steps
        step.lookahead = True
    # the plain per-scan path: every pass launched once per detscan
    plain_ms = None
    if not args.no_plain and label == "main":
        plan.set_schedule(plan.SCHED_PER_SCAN)
        torch.cuda.synchronize()
        p0, p1 = _event(), _event()
        p0.record(stream)
        step.run(map_in, tg.Rng(args.seed, 0, 50_000), tg.MODE_DRAW)
        p1.record(stream)
        torch.cuda.synchronize()
        plain_ms = p0.elapsed_time(p1)
        plan.set_schedule(plan.SCHED_PERSISTENT)

    # end to end through the public API with host buffers: every step's d
    # copied in from page-locked host memory (double-buffered, the copy for
    # step k+1 under step k) and the map and gains copied out
    d_host = torch.from_numpy(ing["tod"])
    registered = False
    try:
        rc = torch.cuda.cudart().cudaHostRegister(d_host.data_ptr(), d_host.numel() * 4, 0)
        registered = int(rc) == 0
    except Exception:
        registered = False
    if not registered:
        d_host = d_host.pin_memory()
    map_host = torch.empty((3, npix), dtype=torch.float64).pin_memory()
    gain_host = torch.empty(nq, dtype=torch.float64).pin_memory()
    step.prefetch_tod(d_host)
    step.run(map_in, tg.Rng(args.seed, 0, 19_999), tg.MODE_DRAW)
    torch.cuda.synchronize()
    e0, e1 = _event(), _event()
    e0.record(stream)
    step.prefetch_tod(d_host)
    for k in range(args.steps):
        step.run(map_in, tg.Rng(args.seed, 0, 20_000 + k), tg.MODE_DRAW)
        if k + 1 < args.steps:
            step.prefetch_tod(d_host)
        map_host.copy_(step.map, non_blocking=True)
        gain_host.copy_(step.gain, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(e0.elapsed_time(e1) / 1e3)
    if registered:
        torch.cuda.cudart().cudaHostUnregister(d_host.data_ptr())

    off = ing["offsets"]
    lens = np.diff(off)
    fl = ing["flags"]
    flagged = np.array([bool(fl[int(off[q]):int(off[q + 1])].any()) for q in range(nq)])
    return dict(plan=plan, step=step, map_in=map_in, N=N, nq=nq, npix=npix, elapsed=elapsed, e2e_s=e2e_s,
                stage_ms=stage_ms, iters=iters, iters_stage=iters_stage, clocks=clocks, graph_ms=graph_ms,
                inline_ms=inline_ms,
                kernel_ms=kernel_ms, iters_kt=iters_kt,
                plain_ms=plain_ms, tuned=tuned, status_errors=int(np.count_nonzero(st)), lens=lens,
                flagged=flagged,
                comp_bytes=int(ing["pix_streams"]["words"].nbytes + ing["psi_streams"]["words"].nbytes),
                npairs=int(plan.info()["nruns"]))


def roofline_and_stages(res, peaks, peak_src):
    """Per-stage GB/s over the stages' algorithmic bytes, the per-kernel
    table (CUDA-event time per step, launches, share of the step's kernel
    time, algorithmic bytes and GB/s), and the roofline of the dominant
    kernel: its algorithmic bytes per launch over its mean launch time."""
    N, npix = res["N"], res["npix"]
    ncorr_b = ncorr_algorithmic_bytes(res["lens"], res["iters_stage"], res["flagged"])
    byts = stage_bytes(N, npix, res["npairs"], res["comp_bytes"], ncorr_b)
    stage_ms = res["stage_ms"]
    stage_gbs = {k: (byts[k] / (stage_ms[k] / 1e3) / 1e9 if k in byts else None) for k in stage_ms}
    # kernel bytes averaged over the timed calls' own CG iteration counts
    kb = {}
    kms = res["kernel_ms"]
    launched = int(round(kms["k_nc_filter"][1])) if "k_nc_filter" in kms else 8
    for it in res["iters_kt"]:
        for nm, v in kernel_bytes(N, npix, res["npairs"], res["comp_bytes"], res["lens"], it,
                                  res["flagged"], launched).items():
            kb[nm] = kb.get(nm, 0.0) + v / len(res["iters_kt"])
    total = sum(ms for ms, _ in kms.values())
    table = {}
    for nm, (ms, n) in sorted(kms.items(), key=lambda x: -x[1][0]):
        b = kb.get(nm)
        table[nm] = {"ms_per_step": ms, "launches_per_step": n, "share": ms / total if total else None,
                     "algorithmic_bytes": b, "gbs": (b / (ms / 1e3) / 1e9) if (b and ms > 0) else None}
    dom = max((nm for nm in kms if nm in kb), key=lambda nm: kms[nm][0])
    ms, n = kms[dom]
    pk = float(peaks["hbm_gbs"])
    per_launch = kb[dom] / n
    ms_launch = ms / n
    ach = per_launch / (ms_launch / 1e3) / 1e9
    traffic = None
    tr = KERNEL_TRAFFIC.get(dom)
    if tr and tr.get("sha256") and sources_digest(tr["sources"]) == tr["sha256"]:
        traffic = tr["dram_per_algorithmic_byte"] * per_launch
    roof = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": pk, "unit": "GB/s", "frac": ach / pk,
            "traffic": traffic, "traffic_unit": "bytes per launch", "launches_per_step": n,
            "ms_per_launch": ms_launch, "algorithmic_bytes_per_launch": per_launch,
            "share_of_kernel_time": ms / total if total else None,
            "timing": "CUDA events around each launch on its stream (library kernel timing), after the "
                      "timed region",
            "peak_source": "%s hbm_gbs (MEASURED_PEAKS.json)" % peak_src}
    return roof, stage_gbs, table


def oracle_errors(args, cfg, arr, ing, res, nsample=3):
    """Error of each output against the FP64 oracle on sampled detscans of
    the band (the first, the longest, the most flagged), from the inputs of
    the last per-stage step: decoded pointing (mismatching values),
    projection, gain mean and draw, n_corr (relative l2)."""
    import oracle
    step = res["step"]
    off = ing["offsets"]
    nq = len(off) - 1
    lens = np.diff(off)
    nfl = np.array([int(ing["flags"][int(off[q]):int(off[q + 1])].sum()) for q in range(nq)])
    qs = sorted({0, int(np.argmax(lens)), int(np.argmax(nfl))})[:nsample]
    it = 20_000 + args.steps - 1
    pix = step.pix.cpu().numpy()
    psi = step.psi.cpu().numpy().view(np.uint16)
    s32 = step.s.cpu().numpy()
    gains = step.gain.cpu().numpy()
    mus = step.mu.cpu().numpy()
    ncorr = step.ncorr.cpu().numpy()
    m_in = res["map_in"].cpu().numpy()[:, :3].T.astype(np.float64)
    errs = {"decode_mismatches": 0, "project": 0.0, "gain_mean": 0.0, "gain": 0.0, "ncorr": 0.0}
    for q in qs:
        a, b = int(off[q]), int(off[q + 1])
        n = b - a
        det = q % cfg.ndet
        pr = oracle.decode_detscan(ing["pix_streams"], q, n, cfg.ndet)
        qr = oracle.decode_detscan(ing["psi_streams"], q, n, cfg.ndet)
        errs["decode_mismatches"] += int(np.count_nonzero(pr != pix[a:b]) + np.count_nonzero(qr != psi[a:b]))
        sref = oracle.project(m_in, pr, qr)
        errs["project"] = max(errs["project"], float(np.abs(s32[a:b] - sref).max() / np.abs(sref).max()))
        s0, fk, al = arr.psd[det]
        d = ing["tod"][a:b].astype(np.float64)
        M = (~ing["flags"][a:b]).astype(np.float64)
        P = oracle.noise_psd(n, cfg.fsamp, s0, fk, al)
        g, mu, _ = oracle.sample_gain(s32[a:b].astype(np.float64), d, M, P,
                                      oracle.gain_normal(args.seed, 0, q, it))
        errs["gain_mean"] = max(errs["gain_mean"], abs(mus[q] - mu) / abs(mu))
        errs["gain"] = max(errs["gain"], abs(gains[q] - g) / abs(g))
        w1 = oracle.omega1(args.seed, 0, q, it, n)
        w2 = oracle.omega2(args.seed, 0, q, it, n)
        x, _ = oracle.sample_ncorr(d, s32[a:b].astype(np.float64), gains[q], M, s0, fk, al, cfg.fsamp, w1, w2)
        errs["ncorr"] = max(errs["ncorr"], float(np.linalg.norm(ncorr[a:b] - x) / np.linalg.norm(x)))
    errs["detscans"] = [int(q) for q in qs]
    errs["norms"] = ("max over the detscans; decode: mismatching values; project: max |err| / max |ref|; "
                     "gain: relative; ncorr: relative l2")
    return errs


# ---------------------------------------------------------------------------
# the oracle on the host cores
# ---------------------------------------------------------------------------
_W = {}


def _worker_init(cfg_dict, nscan, seed):
    import synth
    import oracle
    from oracle import _huff
    _huff.build()
    cfg = synth.scaled(synth.BandConfig(**cfg_dict), nscan=nscan)
    band = synth.make_band(cfg, threads=1)
    _W.update(cfg=cfg, band=band, ing=oracle.ingest(band), seed=seed)


def _worker_detscan(q):
    import oracle
    cfg, band, ing = _W["cfg"], _W["band"], _W["ing"]
    oracle.gibbs_tod_step(ing, cfg, band.npix, band.map_tqu, band.psd, _W["seed"], 0, 0, detscans=[q])
    return int(ing["offsets"][q + 1] - ing["offsets"][q])


def cpu_baseline(args, cfg, budget_s=20.0):
    """The FP64 oracle, as it stands, on the first detscans of the workload,
    one detscan per task over a process pool of every host core."""
    import dataclasses
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    cores = os.cpu_count() or 1
    nq = min(args.cpu_detscans, cfg.ndet * cfg.nscan)
    nscan = -(-nq // cfg.ndet)
    ctx = mp.get_context("spawn")
    with ProcessPoolExecutor(cores, mp_context=ctx, initializer=_worker_init,
                             initargs=(dataclasses.asdict(cfg), nscan, args.seed)) as ex:
        # one untimed task per worker: the workers build the sample first
        list(ex.map(_worker_detscan, [0] * cores))
        t = time.time()
        done = samples = 0
        q = 0
        while q < nq and time.time() - t < budget_s:
            batch = list(range(q, min(nq, q + cores)))
            samples += sum(ex.map(_worker_detscan, batch))
            done += len(batch)
            q += len(batch)
        el = time.time() - t
    return {"value": samples / el, "unit": "samples/s", "cores": cores, "kind": "oracle",
            "sample": "%d of %d detscans (%d samples) of the %s workload, one detscan per task on %d "
                      "processes; FP64 numpy/scipy + C Huffman" % (done, cfg.ndet * cfg.nscan, samples,
                                                                  cfg.name, cores),
            "seconds": el, "nproc": cores}


def secondary_section(args, local):
    """The 30 GHz band's step and the added rows measured on it."""
    import torch
    import synth
    import paper_2201_03509_gb300 as tg
    from paper_2201_03509_gb300.step import GibbsTODStep
    cfg = synth.CONFIGS[SECONDARY]
    if args.secondary_nscan:
        cfg = synth.scaled(cfg, nscan=args.secondary_nscan)
    t_set = time.time()
    arr, ing = build_band(cfg)
    res = measure_step(args, cfg, arr, ing, local, 0, 1, label="secondary")
    plan, step, map_in = res["plan"], res["step"], res["map_in"]
    N, stream = res["N"], torch.cuda.current_stream()
    peaks, peak_src = _peaks()
    roof, stage_gbs, ktab = roofline_and_stages(res, peaks, peak_src)
    out = {"workload": cfg.name, "samples_per_step": N, "ms_per_step": 1e3 * res["elapsed"] / args.steps,
           "value": N * args.steps / res["elapsed"], "e2e_value": N * args.steps / res["e2e_s"],
           "stage_ms": res["stage_ms"], "stage_gbs": stage_gbs, "kernels": ktab, "roofline": roof,
           "cg_iters_mean": float(res["iters"].mean()), "graph_ms_per_step": res["graph_ms"],
           "setup_s": time.time() - t_set}
    # row A10: the n_corr draw writing its spectra, then Metropolis steps
    if not args.no_psd:
        spec = torch.empty(N, dtype=torch.float32, device=step.d.device)
        psd_out = torch.empty_like(step.psd)
        acc = torch.zeros(plan.ndet, dtype=torch.int32, device=step.d.device)
        rng = tg.Rng(args.seed, 0, 60_000)
        plan.set_ncorr_spectrum(spec)
        plan.ncorr_prepare(step.psd)
        ts = []
        for k in range(2):
            a0, a1 = _event(), _event()
            a0.record(stream)
            plan.sample_ncorr_prepared(step.d, step.s, step.gain, step.flags, step.psd, rng, tg.MODE_DRAW,
                                       step.ncorr, step.cg_iters, step.cg_tol, step.cg_maxiter)
            a1.record(stream)
            torch.cuda.synchronize()
            ts.append(a0.elapsed_time(a1))
        plan.set_ncorr_spectrum(None)
        nst = 10
        plan.sample_noise_psd(spec, step.psd, rng, nst, 2e-4, 2e-4, psd_out, acc)      # warm-up
        b0, b1 = _event(), _event()
        b0.record(stream)
        plan.sample_noise_psd(spec, step.psd, rng, nst, 2e-4, 2e-4, psd_out, acc)
        b1.record(stream)
        torch.cuda.synchronize()
        plan.status()
        per_eval = b0.elapsed_time(b1) / (nst + 1)
        out["noise_psd"] = {"ncorr_with_spectrum_ms": min(ts), "metropolis_steps": nst,
                            "ms": b0.elapsed_time(b1), "ms_per_evaluation": per_eval,
                            "gbs_per_evaluation": 4.0 * N / (per_eval / 1e3) / 1e9,
                            "accepted": acc.cpu().tolist()}
    # row A11: the step decoding d and the flag mask every step
    if not args.no_data_streams:
        band = synth.make_band(cfg)
        t_enc = time.time()
        ingd = tg.ingest_data(band, ing["offsets"])
        del band
        plan.attach_data(ingd["tod_streams"], ingd["tod_scale"], ingd["flag_streams"], ingd["flag_select"])
        enc_s = time.time() - t_enc
        dstep = GibbsTODStep(plan, arr.psd, None, cg_tol=args.cg_tol, data_streams=True)
        for k in range(args.warmup):
            dstep.run(map_in, tg.Rng(args.seed, 0, 70_000 + k), tg.MODE_DRAW)
        torch.cuda.synchronize()
        c0, c1 = _event(), _event()
        c0.record(stream)
        for k in range(args.steps):
            dstep.run(map_in, tg.Rng(args.seed, 0, 70_100 + k), tg.MODE_DRAW)
        c1.record(stream)
        torch.cuda.synchronize()
        ds_ms = c0.elapsed_time(c1) / args.steps
        dec = {}
        for name, dd, ff in (("tod", dstep.d, None), ("flags", None, dstep.flags)):
            tt = []
            for _ in range(3):
                a0, a1 = _event(), _event()
                a0.record(stream)
                plan.decode_data(dd, ff)
                a1.record(stream)
                torch.cuda.synchronize()
                tt.append(a0.elapsed_time(a1))
            dec[name] = min(tt)
        plan.status()
        tod_bytes = int(ingd["tod_streams"]["words"].nbytes)
        flag_bytes = int(ingd["flag_streams"]["words"].nbytes)
        out["data_streams"] = {"ms_per_step": ds_ms, "value": N / (ds_ms / 1e3), "decode_tod_ms": dec["tod"],
                               "decode_flags_ms": dec["flags"], "tod_bits_per_sample": 8.0 * tod_bytes / N,
                               "flag_bits_per_sample": 8.0 * flag_bytes / N,
                               "resident_bytes_per_sample": {"fp32_d_and_bitmask": 4.125,
                                                             "compressed": (tod_bytes + flag_bytes) / N},
                               "launches_per_step": dstep.launches_per_step, "ingest_s": enc_s}
        del dstep
    # row A12: the joint gain draw under the smooth prior across scans
    if not args.no_gain_smooth:
        prior = torch.tensor([[1e-3, -2.0]] * plan.ndet, dtype=torch.float64, device=step.d.device)
        gsm = torch.empty_like(step.gain)
        gits = torch.zeros(plan.ndet, dtype=torch.int32, device=step.d.device)
        ts = []
        for k in range(4):
            a0, a1 = _event(), _event()
            a0.record(stream)
            plan.sample_gain_smooth(step.mu, step.sigma, prior, tg.Rng(args.seed, 0, 80_000 + k), tg.MODE_DRAW,
                                    gsm, gits, cg_tol=1e-6)
            a1.record(stream)
            torch.cuda.synchronize()
            ts.append(a0.elapsed_time(a1))
        plan.status()
        out["gain_smooth"] = {"ms": min(ts[1:]), "cg_iters": gits.cpu().tolist(), "nscan": plan.nscan,
                              "ndet": plan.ndet, "prior": {"sigma_g": 1e-3, "alpha_g": -2.0}, "cg_tol": 1e-6}
    plan.close()
    return out


def sweep_section(args, local):
    """The multi-band Gibbs sweep: the 30, 44 and 70 GHz-like bands of 1500
    scans (7.2e9 samples per iteration) on one GPU, each band's step on its
    own stream, `--sweep-iters` iterations carrying maps and noise
    parameters (one Metropolis step of the noise PSD per iteration); the
    first iteration is checked against the oracle on sampled detscans of
    every band and is not timed."""
    import torch
    import synth
    import oracle
    import paper_2201_03509_gb300 as tg
    from paper_2201_03509_gb300.sweep import BandChain, MultiBandSweep
    t_set = time.time()
    chains, keep = [], []
    for b, name in enumerate(synth.SWEEP_BANDS):
        cfg = synth.CONFIGS[name]
        arr, ing = build_band(cfg)
        plan = tg.Plan(cfg.nside, cfg.ndet, cfg.nscan, cfg.fsamp, ing["offsets"], ing["pix_streams"],
                       ing["psi_streams"], device=local)
        chains.append(BandChain(plan, arr.psd, ing["flag_words"], ing["tod"], arr.map_tqu, b,
                                cg_tol=args.cg_tol, psd_steps=1))
        keep.append((cfg, arr, ing))
        torch.cuda.synchronize()
    sw = MultiBandSweep(chains)
    setup_s = time.time() - t_set
    # iteration 0 (untimed): the truth map and noise parameters in, checked
    sw.run(1, args.seed, it0=0)
    errs = []
    for (cfg, arr, ing), c in zip(keep, chains):
        c.plan.status()
        off = ing["offsets"]
        lens = np.diff(off)
        qs = sorted({0, int(np.argmax(lens)), len(lens) - 1})
        g = c.step.gain.cpu().numpy()
        e = {"band": cfg.name, "gain": 0.0, "ncorr": 0.0, "detscans": qs}
        for q in qs:
            a, bq = int(off[q]), int(off[q + 1])
            n = bq - a
            det = q % cfg.ndet
            pr = oracle.decode_detscan(ing["pix_streams"], q, n, cfg.ndet)
            qr = oracle.decode_detscan(ing["psi_streams"], q, n, cfg.ndet)
            sref = oracle.project(arr.map_tqu, pr, qr)
            s0, fk, al = arr.psd[det]
            d = ing["tod"][a:bq].astype(np.float64)
            M = (~ing["flags"][a:bq]).astype(np.float64)
            P = oracle.noise_psd(n, cfg.fsamp, s0, fk, al)
            rg, _, _ = oracle.sample_gain(sref, d, M, P, oracle.gain_normal(args.seed, c.band_id, q, 0))
            x, _ = oracle.sample_ncorr(d, sref, rg, M, s0, fk, al, cfg.fsamp,
                                       oracle.omega1(args.seed, c.band_id, q, 0, n),
                                       oracle.omega2(args.seed, c.band_id, q, 0, n))
            xg = c.step.ncorr[a:bq].cpu().numpy().astype(np.float64)
            e["gain"] = max(e["gain"], abs(g[q] - rg) / abs(rg))
            e["ncorr"] = max(e["ncorr"], float(np.linalg.norm(xg - x) / np.linalg.norm(x)))
        errs.append(e)
    del keep
    sampler = ClockSampler(local)
    sampler.start()
    res = sw.run(args.sweep_iters, args.seed, it0=1)
    clocks = sampler.stop()
    # the same iterations with the bands taking turns (for comparison)
    seq = sw.run(min(3, args.sweep_iters), args.seed, it0=1 + args.sweep_iters, concurrent=False)
    for c in chains:
        c.plan.status()
    out = {"bands": [c.plan.info()["nsamples"] for c in chains], "band_names": list(synth.SWEEP_BANDS),
           "iterations": args.sweep_iters, "samples_per_iteration": res["samples_per_iteration"],
           "ms_per_iteration": res["ms"] / args.sweep_iters,
           "value": res["samples_per_iteration"] * args.sweep_iters / (res["ms"] / 1e3), "unit": "samples/s",
           "band_ms_to_last_iteration": res["band_ms"], "clocks": clocks, "setup_s": setup_s,
           "bands_in_turn_ms_per_iteration": seq["ms"] / min(3, args.sweep_iters),
           "psd_steps_per_iteration": 1, "oracle_error_first_iteration": errs,
           "timing": "CUDA events on the caller's stream around all iterations; bands on their own streams"}
    for c in chains:
        c.plan.close()
    return out


def run_ours(args):
    import torch
    import synth
    import paper_2201_03509_gb300 as tg

    rank, ws = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    tg.build() if rank == 0 or ws == 1 else None
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    t_setup = time.time()
    cfg = synth.CONFIGS[args.workload]
    if args.nscan:
        cfg = synth.scaled(cfg, nscan=args.nscan)
    scans = None
    if ws > 1:
        # contiguous scan ranges of nearly equal sample counts
        from paper_2201_03509_gb300.shard import partition_scans
        kept = tg.kept_lengths(cfg)
        bounds = partition_scans(kept * cfg.ndet, ws)
        scans = range(int(bounds[rank]), int(bounds[rank + 1]))
    arr, ing = build_band(cfg, scans)
    setup_s = time.time() - t_setup
    res = measure_step(args, cfg, arr, ing, local, rank, ws)
    peaks, peak_src = _peaks()
    roof, stage_gbs, ktab = roofline_and_stages(res, peaks, peak_src)
    N, nq, npix = res["N"], res["nq"], res["npix"]
    Ntot = N
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([float(N)], dtype=torch.float64, device="cuda")
        dist.all_reduce(t)
        Ntot = int(t.item())
    elapsed = res["elapsed"]
    graph_ms, plain_ms = res["graph_ms"], res["plain_ms"]
    out = {
        "metric": METRIC, "value": Ntot * args.steps / elapsed, "unit": "samples/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
        "higher_is_better": True, "scaling": "strong" if ws > 1 else "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": cfg.name, "ndetscan": cfg.ndet * cfg.nscan, "samples_per_step": Ntot,
                   "nside": cfg.nside, "flag_frac": cfg.flag_frac,
                   "tile_pairs": res["plan"].info()["tile_pairs"], "autotune": res["tuned"],
                   "l2": "inputs larger than L2 (%.1f GB of d per step)" % (4.0 * Ntot / 1e9),
                   "parallelism": "single GPU" if ws == 1 else
                   "%d scan ranges (one per rank), normal equations reduced by pixel range" % ws},
        "e2e": {"value": Ntot * args.steps / res["e2e_s"], "unit": "samples/s", "h2d_bytes_per_step": 4 * N,
                "d2h_bytes_per_step": 8 * (3 * npix + nq)},
        "gpu_launches": res["step"].launches_per_step * args.steps,
        "stage_ms": res["stage_ms"], "stage_gbs": stage_gbs, "kernels": ktab,
        "cg_iters": {"mean": float(res["iters"].mean()), "max": int(res["iters"].max()),
                     "min": int(res["iters"].min())},
        "graph": ({"ms_per_step": graph_ms, "value": Ntot / (graph_ms / 1e3),
                   "eager_in_step_decode_ms_per_step": res["inline_ms"]}
                  if isinstance(graph_ms, float) else graph_ms),
        "plain_per_scan": ({"ms_per_step": plain_ms, "value": N / (plain_ms / 1e3),
                            "speedup_batched": plain_ms / (1e3 * elapsed / args.steps)}
                           if plain_ms else None),
        "device_status_errors": res["status_errors"],
        "roofline": roof, "clocks": res["clocks"], "setup_s": setup_s,
    }
    if rank == 0 and ws == 1 and not args.no_oracle_error:
        out["oracle_error"] = oracle_errors(args, cfg, arr, ing, res)
    res["plan"].close()
    del res
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    if rank == 0 and ws == 1 and not args.no_secondary and args.workload != SECONDARY:
        out["secondary"] = secondary_section(args, local)
    if rank == 0 and ws == 1 and args.sweep:
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        out["sweep"] = sweep_section(args, local)
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args, cfg, budget_s=args.cpu_seconds)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_reference(args):
    """The FP64 oracle, as it stands, timed on the host cores: a spawn-start
    process pool of every core, each step one batch of detscans of the
    workload (one per task), after one untimed task per worker in which the
    workers build their copy of the sample."""
    rank, ws = _dist()
    if rank != 0:
        return
    import dataclasses
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    import synth
    from oracle import _huff
    _huff.build()                 # once, before the workers load it
    cfg = synth.CONFIGS[args.workload]
    cores = os.cpu_count() or 1
    per_step = args.ref_detscans_per_step if args.ref_detscans_per_step > 0 else cores
    # only the scans the timed sample touches are generated
    nq = max(per_step, min(args.cpu_detscans, cfg.ndet * cfg.nscan))
    nscan = -(-nq // cfg.ndet)
    nq = min(nq, cfg.ndet * nscan)
    procs = min(cores, per_step)
    ctx = mp.get_context("spawn")
    with ProcessPoolExecutor(procs, mp_context=ctx, initializer=_worker_init,
                             initargs=(dataclasses.asdict(cfg), nscan, args.seed)) as ex:
        list(ex.map(_worker_detscan, [0] * procs))
        q = 0

        def step():
            nonlocal q
            batch = [(q + i) % nq for i in range(per_step)]
            q = (q + per_step) % nq
            return sum(ex.map(_worker_detscan, batch))

        for w in range(args.warmup):
            step()
        t = time.time()
        samples = 0
        for k in range(args.steps):
            samples += step()
        el = time.time() - t
    v = samples / el
    out = {"metric": METRIC, "value": v, "unit": "samples/s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference",
           "config": {"workload": cfg.name, "sample": "%d detscans per step" % per_step},
           "cpu_baseline": {"value": v, "unit": "samples/s", "cores": procs, "kind": "oracle",
                            "sample": "%d detscans (%d samples) per step of the %s workload, one detscan per "
                                      "task on %d processes" % (per_step, samples // max(1, args.steps), cfg.name,
                                                                procs)},
           "e2e": {"value": v, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=["lfi70", "lfi30"])
    ap.add_argument("--nscan", type=int, default=0, help="fewer scans (testing only)")
    ap.add_argument("--secondary-nscan", type=int, default=0,
                    help="fewer scans of the 30 GHz band in the secondary section (testing only)")
    ap.add_argument("--seed", type=int, default=2022)
    ap.add_argument("--cg-tol", type=float, default=1e-6)
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--cpu-detscans", type=int, default=64)
    ap.add_argument("--ref-detscans-per-step", type=int, default=0,
                    help="detscans per step of the reference arm (0: one per host core)")
    ap.add_argument("--tune-scans", type=int, default=12)
    ap.add_argument("--sweep", action="store_true",
                    help="also run the 3-band (30/44/70 GHz-like, 7.2e9 samples) Gibbs sweep section")
    ap.add_argument("--sweep-iters", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the per-scan comparison step")
    ap.add_argument("--no-graph", action="store_true", help="skip the CUDA-graph replay")
    ap.add_argument("--autotune", action="store_true",
                    help="time the tile shapes on the first scans and step with the fastest (default: the "
                         "plan's own shape, the one the full-size parity tests run)")
    ap.add_argument("--no-oracle-error", action="store_true", help="skip the oracle comparison")
    ap.add_argument("--no-secondary", action="store_true", help="skip the 30 GHz section and the added rows")
    ap.add_argument("--no-psd", action="store_true", help="skip the noise-PSD step measurement")
    ap.add_argument("--no-data-streams", action="store_true",
                    help="skip the step with compressed TOD and flags")
    ap.add_argument("--no-gain-smooth", action="store_true",
                    help="skip the joint gain draw under the smooth prior")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
