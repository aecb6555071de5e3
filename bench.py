"""Throughput of the Gibbs TOD step (decode -> project -> gain -> n_corr ->
bin -> solve) on synthetic LFI-30-GHz-shaped data.

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle on a
bounded sample of the same workload instead.  Launched by torchrun for
N > 1 GPUs: every rank runs an independent replica of the band (the step
shards by detscan with no exchange but the final map reduction, which this
single-band benchmark replicates), and the max time over ranks is
reported.
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
CONFIG_NAME = "lfi30"


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


# DRAM bytes of one n_corr call per TOD sample, from the ncu capture of
# k_ncorr summarised in profiles/k_ncorr_lfi30_400detscans.md (400 detscans
# of the 30 GHz band; scaled to a full launch by samples, since the kernel
# moves each sample's d, s and n_corr once and its scratch in proportion),
# valid only while the kernel's sources hash to the digest taken with it.
NCORR_TRAFFIC = {"bytes_per_sample": 15.82,
                 "sources": ["csrc/k_dct.cu", "csrc/common.cuh", "csrc/internal.cuh", "csrc/api.cu"],
                 "sha256": "a01eb296836fd5ea94b8c3d7cc90763b7bf552c1645ee3220d546fcab52d24f1"}


def ncorr_sources_digest() -> str | None:
    h = hashlib.sha256()
    for rel in NCORR_TRAFFIC["sources"]:
        try:
            with open(os.path.join(ROOT, "paper_2201_03509_gb300", rel), "rb") as f:
                h.update(f.read())
        except OSError:
            return None
    return h.hexdigest()


def make_workload(nscan: int | None):
    import synth
    import paper_2201_03509_gb300 as tg
    cfg = synth.CONFIGS[CONFIG_NAME]
    if nscan:
        cfg = synth.scaled(cfg, nscan=nscan)
    band = synth.make_band(cfg)
    ing = tg.ingest(band)
    return cfg, band, ing


# ---------------------------------------------------------------------------
# per-stage algorithmic work (compulsory bytes per stage)
# ---------------------------------------------------------------------------
def stage_bytes(N, nq, npix, npairs, comp_bytes):
    """Compulsory HBM bytes of each stage for one step."""
    return {
        "decode": comp_bytes + 6.0 * N,                 # streams in, pix int32 + psi uint16 out
        "project": 6.0 * N + 4.0 * N,                   # pix, psi in, s out (map gathers hit L2)
        "gain": 8.0 * N + N / 8.0,                      # s, d, flags
        "ncorr": 12.0 * N + N / 8.0,                    # s, d in, n_corr out, flags
        "bin": 10.0 * N + N / 8.0 + 6.0 * N + 80.0 * npairs,   # d, n_corr, psi, flags, load order + slot, runs out
        "reduce": 80.0 * npairs + 76.0 * npix,
        "solve": 76.0 * npix + 61.0 * npix,
    }


def run_ours(args):
    import torch
    import paper_2201_03509_gb300 as tg
    from paper_2201_03509_gb300.step import GibbsTODStep

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
    cfg, band, ing = make_workload(args.nscan)
    m4 = np.zeros((band.npix, 4), np.float32)
    m4[:, :3] = band.map_tqu.T
    map_in = torch.from_numpy(m4).cuda()
    tuned = None
    cs, rmax = 0, 0
    if not args.no_autotune:
        # measured launch shape (cluster size, largest radix) on the band's first scans
        from paper_2201_03509_gb300.autotune import autotune
        cs, rmax, tms = autotune(cfg.nside, cfg.ndet, cfg.nscan, cfg.fsamp, ing["offsets"], ing["pix_streams"],
                                 ing["psi_streams"], ing["tod"], ing["flag_words"], band.psd, map_in,
                                 device=local)
        tuned = {"tile_pairs": cs, "max_radix": rmax,
                 "candidates_ms": {"C%d_R%d" % k: round(v, 3) for k, v in sorted(tms.items())}}
    plan = tg.Plan(cfg.nside, cfg.ndet, cfg.nscan, cfg.fsamp, ing["offsets"], ing["pix_streams"],
                   ing["psi_streams"], tile_pairs=cs, device=local, max_radix=rmax)
    info = plan.info()
    step = GibbsTODStep(plan, band.psd, ing["flag_words"], cg_tol=args.cg_tol)
    step.set_tod(ing["tod"])
    N, nq, npix = plan.N, plan.nq, plan.npix
    setup_s = time.time() - t_setup
    stream = torch.cuda.current_stream()

    def one(it, timed_events=None):
        rng = tg.Rng(args.seed, 0, it)
        if timed_events is None:
            step.run(map_in, rng, tg.MODE_DRAW)
            return
        ev = timed_events
        p = step.plan
        ev[0].record(stream)
        p.decode(step.pix, step.psi)
        ev[1].record(stream)
        p.project(map_in, step.pix, step.psi, None, step.s)
        ev[2].record(stream)
        p.sample_gain(step.d, step.s, step.flags, step.psd, rng, tg.MODE_DRAW, step.gain, step.mu, step.sigma)
        ev[3].record(stream)
        p.ncorr_prepare(step.psd)
        ev[4].record(stream)
        p.sample_ncorr_prepared(step.d, step.s, step.gain, step.flags, step.psd, rng, tg.MODE_DRAW, step.ncorr,
                                step.cg_iters, step.cg_tol, step.cg_maxiter)
        ev[5].record(stream)
        p.bin(step.psi, step.d, step.ncorr, step.gain, step.flags, step.psd, step.A, step.b, step.hits)
        ev[6].record(stream)
        p.solve_maps(step.A, step.b, step.hits, step.rcond_min, step.map, step.map32, step.rcond, step.valid)
        ev[7].record(stream)

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
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for k in range(args.steps):
        one(k)                     # the step as a user runs it (GibbsTODStep.run)
    t1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    clocks = sampler.stop()
    elapsed = t0.elapsed_time(t1) / 1e3
    # per-stage times: the same calls in sequence on one stream with events
    # between them (the n_corr preparation, which the step overlaps with
    # decode, projection and gain, as its own stage), after the timed region
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(8)] for _ in range(args.steps)]
    for k in range(args.steps):
        one(args.steps + k, evs[k])
    torch.cuda.synchronize()
    st = plan.status(raise_on_error=False)
    names = ["decode", "project", "gain", "ncorr_prepare", "ncorr", "bin", "solve"]
    stage_ms = {nm: float(np.mean([evs[k][i].elapsed_time(evs[k][i + 1]) for k in range(args.steps)]))
                for i, nm in enumerate(names)}
    iters = step.cg_iters.cpu().numpy()
    elapsed = max_over_ranks(elapsed)

    # the same step captured in a CUDA graph (iteration read on the device)
    graph_ms = None
    try:
        step.capture(map_in, args.seed, 0, tg.MODE_DRAW)
        for k in range(2):
            step.replay(30_000 + k)
        torch.cuda.synchronize()
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for k in range(args.steps):
            step.replay(40_000 + k)
        g1.record(stream)
        torch.cuda.synchronize()
        graph_ms = g0.elapsed_time(g1) / args.steps
    except Exception as ex:          # report, do not hide
        graph_ms = "capture failed: %s" % ex
    # the plain per-scan path: one cluster launch per detscan per stage
    plain_ms = None
    if not args.no_plain:
        plan.set_schedule(plan.SCHED_PER_SCAN)
        torch.cuda.synchronize()
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        step.run(map_in, tg.Rng(args.seed, 0, 50_000), tg.MODE_DRAW)
        p1.record(stream)
        torch.cuda.synchronize()
        plain_ms = p0.elapsed_time(p1)
        plan.set_schedule(plan.SCHED_PERSISTENT)

    # end to end through the public API with host buffers
    d_host = torch.from_numpy(ing["tod"]).pin_memory()
    map_host = torch.empty((3, npix), dtype=torch.float64).pin_memory()
    gain_host = torch.empty(nq, dtype=torch.float64).pin_memory()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    # every step's d is copied from pinned host memory; the copy for step k+1
    # runs on a second stream while step k computes (double-buffered d); one
    # untimed step first sets up the second buffer and the copy stream
    step.prefetch_tod(d_host)
    step.run(map_in, tg.Rng(args.seed, 0, 19_999), tg.MODE_DRAW)
    torch.cuda.synchronize()
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

    # row A10 (outside the step's value): the n_corr draw writing its
    # spectra, then the noise-PSD Metropolis step on them
    psd_info = None
    if not args.no_psd:
        spec = torch.empty(N, dtype=torch.float32, device=step.d.device)
        psd_out = torch.empty_like(step.psd)
        acc = torch.zeros(plan.ndet, dtype=torch.int32, device=step.d.device)
        rng = tg.Rng(args.seed, 0, 60_000)
        plan.set_ncorr_spectrum(spec)
        plan.ncorr_prepare(step.psd)
        ts = []
        for k in range(2):
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            plan.sample_ncorr_prepared(step.d, step.s, step.gain, step.flags, step.psd, rng, tg.MODE_DRAW,
                                       step.ncorr, step.cg_iters, step.cg_tol, step.cg_maxiter)
            a1.record(stream)
            torch.cuda.synchronize()
            ts.append(a0.elapsed_time(a1))
        plan.set_ncorr_spectrum(None)
        nst = 10
        plan.sample_noise_psd(spec, step.psd, rng, nst, 2e-4, 2e-4, psd_out, acc)      # warm-up
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        plan.sample_noise_psd(spec, step.psd, rng, nst, 2e-4, 2e-4, psd_out, acc)
        b1.record(stream)
        torch.cuda.synchronize()
        plan.status()
        psd_ms = b0.elapsed_time(b1)
        per_eval = psd_ms / (nst + 1)
        psd_info = {"ncorr_with_spectrum_ms": min(ts), "metropolis_steps": nst, "ms": psd_ms,
                    "ms_per_evaluation": per_eval, "gbs_per_evaluation": 4.0 * N / (per_eval / 1e3) / 1e9,
                    "accepted": acc.cpu().tolist()}

    # compressed TOD and flags (outside the step's value): the same step
    # decoding d and the flag mask on the device every step
    ds_info = None
    if not args.no_data_streams:
        t_enc = time.time()
        ingd = tg.ingest_data(band, ing["offsets"])
        plan.attach_data(ingd["tod_streams"], ingd["tod_scale"], ingd["flag_streams"], ingd["flag_select"])
        enc_s = time.time() - t_enc
        dstep = GibbsTODStep(plan, band.psd, None, cg_tol=args.cg_tol, data_streams=True)
        for k in range(args.warmup):
            dstep.run(map_in, tg.Rng(args.seed, 0, 70_000 + k), tg.MODE_DRAW)
        torch.cuda.synchronize()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
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
                a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a0.record(stream)
                plan.decode_data(dd, ff)
                a1.record(stream)
                torch.cuda.synchronize()
                tt.append(a0.elapsed_time(a1))
            dec[name] = min(tt)
        plan.status()
        tod_bytes = int(ingd["tod_streams"]["words"].nbytes)
        flag_bytes = int(ingd["flag_streams"]["words"].nbytes)
        ds_info = {"ms_per_step": ds_ms, "value": ws * N / (ds_ms / 1e3),
                   "decode_tod_ms": dec["tod"], "decode_flags_ms": dec["flags"],
                   "tod_bits_per_sample": 8.0 * tod_bytes / N, "flag_bits_per_sample": 8.0 * flag_bytes / N,
                   "resident_bytes_per_sample": {"fp32_d_and_bitmask": 4.125,
                                                 "compressed": (tod_bytes + flag_bytes) / N},
                   "launches_per_step": dstep.launches_per_step, "ingest_s": enc_s}
        del dstep

    # joint gain draw under the smooth prior across scans (outside the step's
    # value), from the last step's per-detscan conditionals
    gs_info = None
    if not args.no_gain_smooth:
        prior = torch.tensor([[1e-3, -2.0]] * plan.ndet, dtype=torch.float64, device=step.d.device)
        gsm = torch.empty_like(step.gain)
        gits = torch.zeros(plan.ndet, dtype=torch.int32, device=step.d.device)
        ts = []
        for k in range(4):
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            plan.sample_gain_smooth(step.mu, step.sigma, prior, tg.Rng(args.seed, 0, 80_000 + k), tg.MODE_DRAW,
                                    gsm, gits, cg_tol=1e-6)
            a1.record(stream)
            torch.cuda.synchronize()
            ts.append(a0.elapsed_time(a1))
        plan.status()
        gs_info = {"ms": min(ts[1:]), "cg_iters": gits.cpu().tolist(), "nscan": plan.nscan, "ndet": plan.ndet,
                   "prior": {"sigma_g": 1e-3, "alpha_g": -2.0}, "cg_tol": 1e-6}

    # roofline of the dominant stage
    peaks, peak_src = _peaks()
    comp = int(ing["pix_streams"]["words"].nbytes + ing["psi_streams"]["words"].nbytes)
    npairs = int(getattr(plan, "npairs", 0) or 0)
    byts = stage_bytes(N, nq, npix, npairs, comp)
    dom = max(stage_ms, key=stage_ms.get)
    lens = np.diff(ing["offsets"])
    sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    if dom in ("gain", "ncorr"):
        # FP32 FFT work: 5 (n/2) log2(n/2) flops per complex transform of a
        # length-n real DCT, plus the split (~10 n); transforms per detscan:
        # gain 2, n_corr 2 + 2 per CG iteration + 1 (the correction's inverse).
        per = 2.5 * lens * np.log2(lens / 2.0) + 10.0 * lens
        if dom == "gain":
            flops = float(np.sum(2 * per))
        else:
            flops = float(np.sum(per * (2 + np.where(iters > 0, 2 * iters + 1, 0))))
        peak_tf = 152 * 128 * 2 * (peaks.get("sm_max_mhz", 2070.0) * 1e6) / 1e12
        ach = flops / (stage_ms[dom] / 1e3) / 1e12
        traffic = None
        if dom == "ncorr" and ncorr_sources_digest() == NCORR_TRAFFIC["sha256"]:
            traffic = NCORR_TRAFFIC["bytes_per_sample"] * N
        roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": peak_tf, "unit": "TFLOP/s",
                "frac": ach / peak_tf, "traffic": traffic, "traffic_unit": "bytes per launch",
                "peak_source": "FP32 FMA issue: 152 SMs x 128 lanes x 2 flop x sm_max_mhz"}
    else:
        ach = byts.get(dom, 0.0) / (stage_ms[dom] / 1e3) / 1e9
        pk = float(peaks["hbm_gbs"])
        roof = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": pk, "unit": "GB/s",
                "frac": ach / pk, "traffic": None, "peak_source": peak_src}
    stage_gbs = {k: (byts[k] / (stage_ms[k] / 1e3) / 1e9 if k in byts else None) for k in stage_ms}

    value = ws * N * args.steps / elapsed
    out = {
        "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": cfg.name, "ndetscan": nq, "samples_per_step": N, "nside": cfg.nside,
                   "flag_frac": cfg.flag_frac, "tile_pairs": info["tile_pairs"], "autotune": tuned,
                   "l2": "inputs larger than L2 (%.2f GB per step)" % (4.0 * N / 1e9),
                   "parallelism": "replica x%d" % ws},
        "e2e": {"value": ws * N * args.steps / e2e_s, "unit": "samples/s", "h2d_bytes_per_step": 4 * N,
                "d2h_bytes_per_step": 8 * (3 * npix + nq)},
        "gpu_launches": GibbsTODStep.LAUNCHES_PER_STEP * args.steps,
        "stage_ms": stage_ms, "stage_gbs": stage_gbs,
        "cg_iters": {"mean": float(iters.mean()), "max": int(iters.max()), "min": int(iters.min())},
        "graph": ({"ms_per_step": graph_ms, "value": ws * N / (graph_ms / 1e3)}
                  if isinstance(graph_ms, float) else graph_ms),
        "plain_per_scan": ({"ms_per_step": plain_ms, "value": N / (plain_ms / 1e3),
                            "speedup_batched": plain_ms / (1e3 * elapsed / args.steps)}
                           if plain_ms else None),
        "noise_psd": psd_info,
        "data_streams": ds_info,
        "gain_smooth": gs_info,
        "device_status_errors": int(np.count_nonzero(st)),
        "roofline": roof, "clocks": clocks, "setup_s": setup_s,
    }
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args, cfg, band, budget_s=args.cpu_seconds)
    plan.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def cpu_baseline(args, cfg, band, budget_s=20.0, steps=1):
    """The FP64 oracle, as it stands, on the first detscans of the workload."""
    import oracle
    ing = oracle_ingest_subset(band, cfg, max_detscans=args.cpu_detscans)
    off = ing["offsets"]
    nq = len(off) - 1
    t = time.time()
    done = 0
    samples = 0
    while done < nq and time.time() - t < budget_s:
        oracle.gibbs_tod_step(ing, cfg, band.npix, band.map_tqu, band.psd, args.seed, 0, 0,
                              detscans=[done])
        samples += int(off[done + 1] - off[done])
        done += 1
    el = time.time() - t
    return {"value": samples / el, "unit": "samples/s", "cores": 1, "kind": "oracle",
            "sample": "%d of %d detscans (%d samples), FP64 numpy/scipy + C Huffman, one thread"
                      % (done, cfg.ndet * cfg.nscan, samples), "seconds": el}


def oracle_ingest_subset(band, cfg, max_detscans):
    """The oracle's own ingest of the first scans (enough for the sample)."""
    import oracle
    import synth
    nscan = max(1, -(-max_detscans // cfg.ndet))
    sub = synth.Band(cfg=synth.scaled(cfg, nscan=nscan), npix=band.npix, map_tqu=band.map_tqu,
                     scan_len=band.scan_len[:nscan], gain=band.gain[:nscan * cfg.ndet], psd=band.psd,
                     pix=band.pix[:nscan * cfg.ndet], psi=band.psi[:nscan * cfg.ndet],
                     flags=band.flags[:nscan * cfg.ndet], tod=band.tod[:nscan * cfg.ndet])
    return oracle.ingest(sub)


def run_reference(args):
    rank, ws = _dist()
    if rank != 0:
        return
    import oracle  # noqa: F401
    from oracle import _huff
    _huff.build()
    import synth
    cfg = synth.CONFIGS[CONFIG_NAME]
    # only the scans the timed sample touches are generated
    nsc = max(1, -(-args.cpu_detscans // cfg.ndet))
    sub_cfg = synth.scaled(cfg, nscan=nsc)
    band = synth.make_band(sub_cfg)
    ing = oracle.ingest(band)
    off = ing["offsets"]
    per_step = max(1, min(len(off) - 1, args.ref_detscans_per_step))
    import oracle as orc
    for w in range(args.warmup):
        orc.gibbs_tod_step(ing, sub_cfg, band.npix, band.map_tqu, band.psd, args.seed, 0, w,
                           detscans=list(range(min(1, per_step))))
    t = time.time()
    samples = 0
    for k in range(args.steps):
        qs = list(range(per_step))
        orc.gibbs_tod_step(ing, sub_cfg, band.npix, band.map_tqu, band.psd, args.seed, 0, k, detscans=qs)
        samples += int(sum(off[q + 1] - off[q] for q in qs))
    el = time.time() - t
    v = samples / el
    out = {"metric": METRIC, "value": v, "unit": "samples/s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference",
           "config": {"workload": cfg.name, "sample": "%d detscans per step" % per_step},
           "cpu_baseline": {"value": v, "unit": "samples/s", "cores": 1, "kind": "oracle",
                            "sample": "%d detscans (%d samples) per step of the %s workload"
                                      % (per_step, samples // max(1, args.steps), cfg.name)},
           "e2e": {"value": v, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nscan", type=int, default=0, help="fewer scans (testing only)")
    ap.add_argument("--seed", type=int, default=2022)
    ap.add_argument("--cg-tol", type=float, default=1e-6)
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--cpu-detscans", type=int, default=24)
    ap.add_argument("--ref-detscans-per-step", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the per-scan comparison step")
    ap.add_argument("--no-autotune", action="store_true", help="use the plan's default launch shape")
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
