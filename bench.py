"""Benchmark: lensed T/Q/U map sets per second at Nside 2048, lmax 4096, order 4.

One step = one full lensing pass through the C ABI (deflection synthesis, Legendre
stage of T and Q/U with all derivative orders, ring FFTs into the derivative maps,
gather + Taylor sum + rotation) for the step's synthetic skies, whose coefficients
are already resident in HBM. The headline form is the BF16x3 tensor-core
contraction (tcgen05; each operand split into BF16 hi + lo, FP32 accumulation) with
sixteen realisations per Legendre launch (--form, --batch); the plain FP64 GPU form is
timed on the same GPU beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--form fp32|tf32|tf32x3|bf16x3]

Other workloads: batched64_n4_TQU (64 uneven realisations in one batch) and
adjoint_nside1024_lmax2048_n4_TQU (one gradient evaluation of a quadratic map loss
per step: forward lens plus tl_lens_adjoint).

Multi-GPU: one process per GPU (torchrun); every rank lenses its own independent
realisations (weak scaling, no data-path collective); the time is the max over
ranks. --impl reference times the FP64 CPU oracle on a bounded sample of the
same workload on the host cores (rank 0 only).
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

import skygen  # noqa: E402

WORKLOAD = "nside2048_lmax4096_n4_TQU"
METRIC = "lensed TQU maps/sec @Nside2048 lmax4096 order4 (mixed vs FP64 GPU, err vs oracle)"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP32 SIMT peak from unit counts: SMs (read from the device) x 128 FP32 lanes x
# 2 flop/FMA x the maximum SM clock of MEASURED_PEAKS.json
FP32_LANES_PER_SM = 128


def fp32_peak_tflops(dev, peaks):
    """(peak TFLOP/s, description) of the FP32 SIMT pipe of device `dev`."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = peaks.get("sm_max_mhz", 2070.0)
    return (sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12,
            f"derived: {sms} SMs (device) x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x {mhz:.0f} MHz (sm_max_mhz)")

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) from one-kernel ncu
# captures of `bench.py --workload nside512_lmax1024_n4_TQU --steps 1 --warmup 1
# --form F` (16 realisations per launch; the command and counters are kept with the
# profile summaries): bytes per realisation (ring FFTs, gather: the same in every
# tensor-core form) or per Legendre launch of form F, with the sha256 prefix of the
# kernel sources it was taken at. The full-size workload scales them by its pixel
# count (rings x m grows the same way); a changed source, another order or form
# gives null.
TRAFFIC_NSIDE512 = {
    ("fft_total", None): (858.2e6, ['ringfft.cu', 'fft.cuh', 'regfft.cuh', 'common.cuh'], "331f595a91f2531e"),
    ("gather_total", None): (627.4e6, ['gather.cu', 'geometry.cuh'], "bcdaeea7440cc516"),
    ("legendre_QU", "bf16x3"): (3.1023e9, ['legendre_umma.cu', 'legendre.cuh', 'common.cuh'], "1b171c4fa0306540"),
    ("legendre_T", "bf16x3"): (2.4593e9, ['legendre_umma.cu', 'legendre.cuh', 'common.cuh'], "1b171c4fa0306540"),
}


def captured_traffic(stage, w, per_step_units, form):
    """Scaled DRAM bytes of a stage for workload w and contraction form, or None
    (see TRAFFIC_NSIDE512)."""
    key = (stage, None) if (stage, None) in TRAFFIC_NSIDE512 else (stage, form)
    if key not in TRAFFIC_NSIDE512 or w.order != 4:
        return None
    byt, files, sha = TRAFFIC_NSIDE512[key]
    m = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1307_0719_gb300", "csrc", f), "rb") as fh:
            m.update(fh.read())
    if m.hexdigest()[:16] != sha:
        return None
    return byt * (w.nside / 512) ** 2 * per_step_units


def legendre_flops_per_launch(nside: int, lmax: int, order: int, spin: int, phi: bool = True,
                              part: str = "all", nreal: int = 1) -> float:
    """Algorithmic flops of one Legendre-stage launch, per (ring pair, l, m) triple:
    the derivative recurrence costs sum_{j<=n} (2j + 3) flops per ring (one multiply,
    j Leibniz multiply-adds and the closing multiply-add of each order), the
    contraction 2 flops per real coefficient and order: spin 0 has re/im (and the
    potential's re/im for j <= 1 when it shares the launch), spin 2 has the four
    reals of S1 and S2 plus one add for cos(theta) + m s/(l(l+1)). Spin 0 runs
    its recurrence once per ring pair (north/south parity), spin 2 on both rings."""
    n = order
    rec = sum(2 * j + 3 for j in range(n + 1))
    if spin == 0:
        r_part, c_part = rec, 4 * (n + 1) + (8 if phi else 0)
    else:
        r_part, c_part = 2 * (rec + 1), 2 * 8 * (n + 1)
    per = {"all": r_part + nreal * c_part, "recurrence": r_part, "contraction": nreal * c_part}[part]
    pairs = 2 * nside  # north rings incl. the equator
    lm = (lmax + 1) * (lmax + 2) // 2
    return float(per) * pairs * lm


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except (OSError, FileNotFoundError):
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

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def shard(n_units: int, rank: int, world: int):
    """Independent realisations owned by a rank (contiguous split)."""
    base, extra = divmod(n_units, world)
    start = rank * base + min(rank, extra)
    return list(range(start, start + base + (1 if rank < extra else 0)))


def max_over_ranks(x: float, device=None) -> float:
    """The largest value of x over all ranks of the default process group (the step
    time of the slowest rank); x itself without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def oracle_sample(w, sky, npix_sample: int, seed: int = 0, nthreads=None):
    """Time the FP64 CPU oracle on a bounded sample of the workload: the pixel-relative
    Taylor lensing of `npix_sample` output pixels (each needs the deflection at its
    own ring and the derivative coefficients at its expansion pixel's ring, i.e.
    two of the map's 2 x (4 Nside - 1) ring syntheses). Returns (seconds, pix, values)."""
    import oracle.healpix as hp
    import oracle.lens as OL
    rng = np.random.default_rng(seed)
    pix = np.sort(rng.choice(hp.npix(w.nside), npix_sample, replace=False))
    t0 = time.perf_counter()
    out = OL.lens_at_pixels(w.nside, w.lmax, w.order, pix, sky["T"], sky.get("E"), sky.get("B"),
                            sky["phi"], nthreads=nthreads)
    dt = time.perf_counter() - t0
    return dt, pix, out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = skygen.WORKLOADS[args.workload]
    sky = skygen.workload_sky(args.workload)
    cores = os.cpu_count() or 1
    nrings_total = 2 * (4 * w.nside - 1)
    times = []
    for i in range(args.warmup + args.steps):
        dt, pix, _ = oracle_sample(w, sky, args.sample_pixels, seed=i, nthreads=cores)
        if i >= args.warmup:
            times.append(dt)
    t = float(np.mean(times))
    # full-map time extrapolated by the number of ring syntheses
    est_map_s = t * nrings_total / (2 * args.sample_pixels)
    value = 1.0 / est_map_s
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "maps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "nside": w.nside, "lmax": w.lmax, "order": w.order,
                   "fields": "TQU", "form": "FP64 CPU oracle"},
        "cpu_baseline": {"value": value, "unit": "maps/s", "cores": cores, "kind": "oracle",
                         "sample": f"{args.sample_pixels} output pixels per step "
                                   f"({2 * args.sample_pixels} of {nrings_total} ring syntheses); "
                                   "full-map time extrapolated by ring count"},
        "e2e": {"value": value, "unit": "maps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    os.environ["TAYLENS_TIMING"] = "1"
    from paper_1307_0719_gb300 import api

    w = skygen.WORKLOADS[args.workload]
    forms = {"fp32": api.MIXED_FP32, "tf32": api.MIXED_TF32, "tf32x3": api.MIXED_TF32x3, "bf16x3": api.MIXED_BF16x3}
    prec = forms[args.form]
    plan = api.Plan(w.nside, w.lmax, w.order, pol=w.pol, precision=prec)
    # one Legendre launch's worth of realisations per step (16 on the tensor cores)
    nb = args.batch if args.batch else plan.batch
    # each rank lenses its own realisations (seeds offset by rank and index): weak scaling
    skies = [skygen.make_sky(w.nside, w.lmax, w.pol, w.seed_t + 1000 * rank + 100 * i,
                             w.seed_e + 1000 * rank + 100 * i, w.seed_phi + 1000 * rank + 100 * i,
                             w.damp_t, w.damp_e) for i in range(nb)]
    sky = skies[0]
    dl = [{k: torch.from_numpy(v).to(dev) for k, v in sk.items()} for sk in skies]
    d = dl[0]
    outs = [torch.empty((3, plan.npix), dtype=torch.float32, device=dev) for _ in range(nb)]
    out = outs[0]
    stream = torch.cuda.current_stream()

    def step():
        plan.lens_batch(dl, outs=outs)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    stage_sum = None
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            step()
            st = np.array(plan.last_stage_ms())  # events on the launch stream
            stage_sum = st if stage_sum is None else stage_sum + st
        ev1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ms = max_over_ranks(ev0.elapsed_time(ev1), dev)
    ms_per_step = ms / args.steps
    value = world * nb * args.steps / (ms / 1e3)
    stages = stage_sum / args.steps
    names = ["prep_T", "legendre_T", "deflection_fft", "prep_QU", "legendre_QU", "ringfft", "gather",
             "fft_total", "gather_total"]
    stage_ms = {n: float(v) for n, v in zip(names, stages)}

    # rooflines per stage: the Legendre kernels against the FP32 pipe (tensor-core forms
    # count the recurrence, the contraction runs on the tensor cores), the ring FFTs and
    # the gather against HBM (algorithmic bytes: every input read once, every output
    # written once). The dominant stage (largest time per step) is `roofline`.
    tc = args.form != "fp32"
    part = "recurrence" if tc else "all"
    nr_launch = min(nb, plan.batch) if tc else 1
    peaks = {}
    if os.path.exists(PEAKS_FILE):
        with open(PEAKS_FILE) as f:
            peaks = json.load(f)
    clocks = clk.summary()
    fp32_peak, fp32_src = fp32_peak_tflops(dev, peaks)
    hbm = peaks.get("hbm_gbs")
    # stage times are those of the step's last tl_lens_batch chunk: one Legendre launch of
    # up to 16 realisations on tensor cores, one realisation otherwise
    launches = 1
    nchunk = min(nb, plan.batch) if tc else 1
    rl = {}
    nf = 3 if w.pol else 1  # fields: T, Q, U (or T alone)
    for st, spin in (("legendre_QU", 2), ("legendre_T", 0)):
        if not stage_ms.get(st):
            continue  # a temperature-only workload has no spin-2 stage
        fl = legendre_flops_per_launch(w.nside, w.lmax, w.order, spin, part=part) * launches
        ach = fl / (stage_ms[st] / 1e3) / 1e12
        e = {"kernel": f"legendre_spin{spin}_{'umma' if tc else 'kernel'}<{w.order}>", "bound": "alu",
             "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s", "frac": ach / fp32_peak,
             "traffic": captured_traffic(st, w, 1, args.form) if (tc and nb == 16) else None,
             "peak_source": fp32_src,
             "counts": "recurrence only (contraction on the tensor cores)" if tc else "recurrence + contraction"}
        if tc:
            cf = legendre_flops_per_launch(w.nside, w.lmax, w.order, spin, part="contraction", nreal=nr_launch)
            e["tensor_tflops_contraction"] = cf / (stage_ms[st] / 1e3) / 1e12
        rl[st] = e
    nplanes = nf * (w.order + 1) + 2  # D7 planes read once: T, Q, U (j <= n) and phi (j <= 1)
    nmaps = nf * (w.order + 1) * (w.order + 2) // 2 + 2  # derivative maps and the deflection
    nrings = 4 * w.nside - 1
    npix = 12 * w.nside * w.nside
    fft_bytes = nchunk * (nplanes * nrings * (w.lmax + 1) * 8 + nmaps * npix * 4)
    gat_bytes = nchunk * npix * (nf * (w.order + 1) * (w.order + 2) // 2 * 4 + 2 * 4 + nf * 4)
    for st, byt, kname in (("fft_total", fft_bytes, "ringfft_kernel<float> (all ring groups)"),
                           ("gather_total", gat_bytes, f"gather_kernel<float, {w.order}, 1>")):
        ach = byt / (stage_ms[st] / 1e3) / 1e9 if stage_ms.get(st) else None
        rl[st] = {"kernel": kname, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                  "frac": (ach / hbm) if (ach and hbm) else None,
                  "traffic": captured_traffic(st, w, nchunk, args.form) if tc else None,
                  "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy)",
                  "algorithmic_bytes": byt}
    dom = max(rl, key=lambda k: stage_ms.get(k, 0.0))
    roof = dict(rl[dom], stage=dom)

    # end to end through the C ABI with host buffers (tl_lens_batch_host): every step
    # passes the coefficients in pinned host memory; the call copies them in, lenses
    # them and copies the maps back, all inside the timed region
    e2e = None
    if not args.no_e2e:
        hin = [{k: torch.from_numpy(v).pin_memory() for k, v in sk.items()} for sk in skies]
        hout = [torch.empty((3, plan.npix), dtype=torch.float32).pin_memory() for _ in range(nb)]

        def e2e_step():
            plan.lens_batch_host(hin, outs=hout)  # synchronises before returning

        e2e_step()
        k2 = max(1, min(args.steps, 3))
        t0 = time.perf_counter()
        for _ in range(k2):
            e2e_step()
        e2e_s = max_over_ranks((time.perf_counter() - t0) / k2, dev)
        e2e = {"value": world * nb / e2e_s, "unit": "maps/s", "h2d_bytes_per_step": nb * 4 * plan.nalm * 16,
               "d2h_bytes_per_step": nb * 3 * plan.npix * 4, "realisations_per_step": nb,
               "api": "tl_lens_batch_host (C ABI, host buffers, copies inside the call)"}
        del hin, hout

    lensed = out.cpu().numpy()
    launches_per_step = plan.batch_launches(nb)
    plan.close()
    del plan
    torch.cuda.empty_cache()

    # plain FP64 GPU form on the same GPU
    fp64 = None
    if not args.no_fp64:
        p64 = api.Plan(w.nside, w.lmax, w.order, pol=w.pol, precision=api.FP64)
        o64 = torch.empty((3, p64.npix), dtype=torch.float64, device=dev)
        p64.lens(d["T"], d["E"], d["B"], d["phi"], out=o64)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k64 = max(1, args.fp64_steps)
        e0.record(stream)
        for _ in range(k64):
            p64.lens(d["T"], d["E"], d["B"], d["phi"], out=o64)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1) / k64
        st64 = dict(zip(names, [float(x) for x in p64.last_stage_ms()]))
        lensed64 = o64.cpu().numpy()
        p64.close()
        fp64 = {"maps_per_s": world * 1e3 / ms64, "ms_per_step": ms64, "steps": k64, "stage_ms": st64,
                "mixed_over_fp64": value / (world * 1e3 / ms64)}
    else:
        lensed64 = None

    # rank 0: CPU baseline (oracle) on a bounded sample + error of both forms there
    cpu = None
    err = None
    if rank == 0 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        dt, pix, ref = oracle_sample(w, sky, args.sample_pixels, nthreads=cores)
        nrings_total = 2 * (4 * w.nside - 1)
        est = dt * nrings_total / (2 * args.sample_pixels)
        cpu = {"value": 1.0 / est, "unit": "maps/s", "cores": cores, "kind": "oracle",
               "sample": f"{args.sample_pixels} output pixels ({2 * args.sample_pixels} of "
                         f"{nrings_total} ring syntheses) in {dt:.1f} s; full-map time "
                         "extrapolated by ring count"}

        # error of both forms on a sample that includes the polar caps: every pixel of
        # the first and last two rings, 8 pixels on each cap edge, belt edge and the
        # equator, 16 random pixels (the oracle evaluates each pixel on its own)
        import oracle.healpix as hp
        import oracle.lens as OL
        epix = hp.check_pixels(w.nside, seed=0, n_random=16, per_ring=8, cap_rings=2)
        ref = OL.lens_at_pixels(w.nside, w.lmax, w.order, epix, sky["T"], sky.get("E"), sky.get("B"),
                                sky["phi"], nthreads=cores)

        def errs(maps):
            o = {}
            for i, f in enumerate("TQU"):
                r = ref[f]
                dlt = maps[i][epix] - r
                o[f] = {"rel_rms": float(np.sqrt(np.mean(dlt ** 2) / np.mean(r ** 2))),
                        "max_rel": float(np.max(np.abs(dlt)) / np.sqrt(np.mean(r ** 2)))}
            return o
        err = {args.form: errs(lensed), "npix": int(len(epix)),
               "sample": "every pixel of the first and last 2 rings; 8 on the cap edges, belt edges and "
                         "equator; 16 random"}
        if lensed64 is not None:
            err["fp64"] = errs(lensed64)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "maps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {"fp32": "f32", "tf32": "tf32", "tf32x3": "tf32x3", "bf16x3": "bf16x3"}[args.form],
            "data": "synthetic (seeded Gaussian alm, analytic spectra)",
            "config": {"workload": args.workload, "nside": w.nside, "lmax": w.lmax, "order": w.order,
                       "fields": "TQU", "form": {"fp32": "mixed FP32 (SIMT contraction)",
                                                 "tf32": "mixed, TF32 tensor-core contraction",
                                                 "tf32x3": "mixed, 3xTF32 tensor-core contraction",
                                                 "bf16x3": "mixed, BF16x3 tensor-core contraction"}[args.form]
                       + "; FP64 seeds and rescaling; float pixel lookup with double fallback", "realisations_per_step": nb,
                       "parallelism": f"replicas{world}", "l2": "inputs larger than L2 (alm 537 MB, "
                       "derivative maps 9 GB per step)"},
            "stage_ms": stage_ms, "roofline": roof, "roofline_stages": rl, "clocks": clocks,
            "gpu_launches": args.steps * launches_per_step, "e2e": e2e, "fp64": fp64, "err_vs_oracle": err,
            "cpu_baseline": cpu,
        }
        if world == 1 and not args.no_extra and args.workload == WORKLOAD:
            # the batched (64 uneven realisations) and gradient workloads as sub-records,
            # each with its own warm-up and timed steps, after this line's timed region
            sub = argparse.Namespace(**vars(args))
            sub.steps, sub.warmup, sub.no_e2e, sub.no_cpu_baseline = 3, 3, False, True
            for key, fn in (("batched64", run_batched), ("adjoint", lambda a: run_adjoint(a, standalone=False))):
                try:
                    torch.cuda.empty_cache()
                    rec = fn(sub)
                    if rec is not None:
                        rec.pop("metric", None)
                    line[key] = rec
                except Exception as exc:  # a failed extra never hides the headline
                    line[key] = {"error": f"{type(exc).__name__}: {exc}"}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_batched(args):
    """64 realisations (seeds 100..163) with lmax drawn from {512, 1024, 2048, 3000} and
    Nside the next power of two >= lmax/2, order 4, in one tl_batch: the persistent
    Legendre launch per wave replayed from a CUDA graph, against a per-realisation loop."""
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1307_0719_gb300 import api
    forms = {"fp32": api.MIXED_FP32, "tf32": api.MIXED_TF32, "tf32x3": api.MIXED_TF32x3, "bf16x3": api.MIXED_BF16x3}
    lst = skygen.batched_lmax_list(64)
    mine = [lst[i] for i in shard(len(lst), rank, world)]
    nsides = [x[1] for x in mine]
    lmaxs = [x[2] for x in mine]
    skies = []
    for seed, ns, lm in mine:
        sk = skygen.make_sky(ns, lm, True, seed, seed, seed, 400.0, 3200.0)
        skies.append({k: torch.from_numpy(v).to(dev) for k, v in sk.items()})
    b = api.Batch(nsides, lmaxs, 4, pol=True, precision=forms[args.form])
    outs = b.outputs(dev)
    b.autotune(skies, outs)
    mode = "graph" if args.form != "fp32" else "loop"
    for _ in range(args.warmup):
        b.lens(skies, outs, mode)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record()
        for _ in range(args.steps):
            b.lens(skies, outs, mode)
        e1.record()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    # comparison: one tl_lens per realisation, no graph
    b.lens(skies, outs, "loop")
    torch.cuda.synchronize()
    e0.record()
    b.lens(skies, outs, "loop")
    e1.record()
    torch.cuda.synchronize()
    ms_loop = e0.elapsed_time(e1)
    line = {
        "metric": "lensed TQU maps/sec, 64 uneven realisations (batched)", "value": len(mine) * 1e3 / ms,
        "unit": "maps/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.form,
        "data": "synthetic (seeded Gaussian alm, analytic spectra)",
        "config": {"workload": "batched64_n4_TQU", "realisations": len(mine), "order": 4,
                   "lmax_counts": {str(l): lmaxs.count(l) for l in sorted(set(lmaxs))},
                   "groups": b.groups, "waves": b.waves, "persistent_grid": b.grid, "mode": mode},
        "loop": {"maps_per_s": len(mine) * 1e3 / ms_loop, "ms_per_step": ms_loop},
        "graph_over_loop": ms_loop / ms, "clocks": clk.summary(),
    }
    b.close()
    return line if rank == 0 else None


ADJ_WORKLOAD = "adjoint_nside1024_lmax2048_n4_TQU"
ADJ_METRIC = "gradient evaluations/sec of L = sum (s' - s_target)^2 wrt alm_T,E,B,phi @Nside1024 lmax2048 order4"


def run_adjoint(args, standalone=True):
    """One step = forward lens, loss gradient g = 2 (maps - targets), tl_lens_adjoint
    (which recomputes the derivative maps) for dL/dalm of T, E, B and phi. Targets are
    the lensed maps of an independent sky (seeds 9000..9002)."""
    import torch
    rank, world, local = dist_env()
    if world > 1 and standalone:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    os.environ["TAYLENS_TIMING"] = "1"
    from paper_1307_0719_gb300 import api
    w = skygen.WORKLOADS["nside1024_lmax2048_n4_TQU"]
    forms = {"fp32": api.MIXED_FP32, "tf32": api.MIXED_TF32, "tf32x3": api.MIXED_TF32x3, "bf16x3": api.MIXED_BF16x3}
    form = args.form if args.form_given else "fp32"
    sky = skygen.make_sky(w.nside, w.lmax, True, w.seed_t + 1000 * rank, w.seed_e + 1000 * rank,
                          w.seed_phi + 1000 * rank, w.damp_t, w.damp_e)
    tsky = skygen.make_sky(w.nside, w.lmax, True, 9000, 9001, 9002, w.damp_t, w.damp_e)
    d = {k: torch.from_numpy(v).to(dev) for k, v in sky.items()}
    dt = {k: torch.from_numpy(v).to(dev) for k, v in tsky.items()}
    plan = api.Plan(w.nside, w.lmax, w.order, pol=True, precision=forms[form])
    target = plan.lens(dt["T"], dt["E"], dt["B"], dt["phi"]).clone()
    del dt
    out = torch.empty((3, plan.npix), dtype=torch.float32, device=dev)
    g = torch.empty_like(out)
    stream = torch.cuda.current_stream()

    def step(alm):
        plan.lens(alm["T"], alm["E"], alm["B"], alm["phi"], out=out)
        torch.sub(out, target, out=g)
        g.mul_(2.0)
        return plan.lens_adjoint(alm["T"], alm["E"], alm["B"], alm["phi"], g[0], g[1], g[2])

    for _ in range(args.warmup):
        step(d)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    names = ["forward", "gather_adj", "ringfft_adj", "legendre_T_adj", "legendre_QU_adj", "finish"]
    stage_sum = np.zeros(len(names))
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            step(d)
            stage_sum += np.array(plan.last_stage_ms())
        ev1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ms = max_over_ranks(ev0.elapsed_time(ev1), dev)
    value = world * args.steps / (ms / 1e3)
    stage_ms = {n: float(v) for n, v in zip(names, stage_sum / args.steps)}
    peaks = {}
    if os.path.exists(PEAKS_FILE):
        with open(PEAKS_FILE) as f:
            peaks = json.load(f)
    fp32_peak, fp32_src = fp32_peak_tflops(dev, peaks)
    dom = max(("gather_adj", "ringfft_adj", "legendre_T_adj", "legendre_QU_adj"), key=lambda k: stage_ms[k])
    if dom.startswith("legendre"):
        spin = 2 if dom == "legendre_QU_adj" else 0
        fl = legendre_flops_per_launch(w.nside, w.lmax, w.order, spin)
        ach = fl / (stage_ms[dom] / 1e3) / 1e12
        roof = {"kernel": f"legendre_adj{spin}_kernel<float, {w.order}>", "bound": "alu", "achieved": ach,
                "peak": fp32_peak, "unit": "TFLOP/s", "frac": ach / fp32_peak, "traffic": None,
                "peak_source": fp32_src,
                "counts": "recurrence + transposed contraction (same per-triple count as the forward)"}
    else:
        roof = {"kernel": dom, "bound": "hbm", "achieved": None, "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                "frac": None, "traffic": None}
    # end to end: coefficients and targets from pinned host memory, gradients back
    e2e = None
    if not args.no_e2e:
        hin = {k: torch.from_numpy(v).pin_memory() for k, v in sky.items()}
        hout = {k: torch.empty(plan.nalm, dtype=torch.complex128).pin_memory() for k in ("T", "E", "B", "phi")}
        k2 = max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(k2):
            dd = {k: v.to(dev, non_blocking=True) for k, v in hin.items()}
            gr = step(dd)
            for k in hout:
                hout[k].copy_(gr[k], non_blocking=True)
            torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / k2
        e2e = {"value": world / e2e_s, "unit": "gradient evaluations/s", "h2d_bytes_per_step": 4 * plan.nalm * 16,
               "d2h_bytes_per_step": 4 * plan.nalm * 16}
    gr = step(d)
    torch.cuda.synchronize()
    gnorm = {k: float(v.abs().pow(2).sum().sqrt()) for k, v in gr.items()}
    plan.close()
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        # oracle adjoint on a reduced geometry of the same order; time extrapolated by the
        # Legendre work (rings x coefficients), which dominates it
        import oracle.adjoint as OA
        ns, lm = 32, 64
        ssk = skygen.make_sky(ns, lm, True, 2, 3, 4, w.damp_t, w.damp_e)
        rng = np.random.default_rng(0)
        gg = {f: rng.normal(size=12 * ns * ns) for f in "TQU"}
        cores = os.cpu_count() or 1
        t0 = time.perf_counter()
        OA.lens_adjoint(ns, lm, w.order, ssk["T"], ssk["E"], ssk["B"], ssk["phi"], gg["T"], gg["Q"], gg["U"],
                        nthreads=cores)
        dt_s = time.perf_counter() - t0
        scale = ((4 * w.nside - 1) * (w.lmax + 1) * (w.lmax + 2)) / ((4 * ns - 1) * (lm + 1) * (lm + 2))
        cpu = {"value": 1.0 / (dt_s * scale), "unit": "gradient evaluations/s", "cores": cores, "kind": "oracle",
               "sample": f"oracle adjoint at Nside {ns}, lmax {lm}, order {w.order} in {dt_s:.1f} s, "
                         f"extrapolated x{scale:.0f} by rings x coefficients"}
    if rank == 0:
        line = {
            "metric": ADJ_METRIC, "value": value, "unit": "gradient evaluations/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {"fp32": "f32", "tf32": "tf32", "tf32x3": "tf32x3", "bf16x3": "bf16x3"}[form],
            "data": "synthetic (seeded Gaussian alm, analytic spectra; targets from seeds 9000-9002)",
            "config": {"workload": ADJ_WORKLOAD, "nside": w.nside, "lmax": w.lmax, "order": w.order,
                       "fields": "TQU", "form": form + "; FP64 geometry and Jacobian",
                       "parallelism": f"replicas{world}",
                       "l2": "inputs larger than L2 (derivative maps 2.3 GB, their gradients 2.3 GB)"},
            "stage_ms": stage_ms, "roofline": roof, "clocks": clk.summary(),
            "gpu_launches": args.steps * 20, "e2e": e2e, "grad_norms": gnorm, "cpu_baseline": cpu,
        }
    if world > 1 and standalone:
        dist.destroy_process_group()
    return line if rank == 0 else None


def run_sweep(args):
    """Error table of the full-size workload (Nside 2048, lmax 4096, T+Q/U) at orders
    2..6 for every precision form against the FP64 oracle, on a pixel sample that
    holds every pixel of the first and last two rings, 8 pixels on the cap and belt
    edges and the equator and 16 random ones: per map (T, Q, U) the relative RMS
    over the sample and the largest error relative to the sample's RMS. Prints one
    JSON line (not a throughput record)."""
    import torch
    import oracle.healpix as hp
    import oracle.lens as OL
    from paper_1307_0719_gb300 import api
    w = skygen.WORKLOADS[WORKLOAD]
    dev = torch.device("cuda", 0)
    sky = skygen.workload_sky(WORKLOAD)
    d = {k: torch.from_numpy(v).to(dev) for k, v in sky.items()}
    pix = hp.check_pixels(w.nside, seed=0, n_random=16, per_ring=8, cap_rings=2)
    forms = [("fp64", api.FP64), ("fp32", api.MIXED_FP32), ("tf32", api.MIXED_TF32), ("tf32x3", api.MIXED_TF32x3),
             ("bf16x3", api.MIXED_BF16x3)]
    orders = [int(x) for x in args.sweep_orders.split(",")]
    table = {}
    cores = os.cpu_count() or 1
    for n in orders:
        ref = OL.lens_at_pixels(w.nside, w.lmax, n, pix, sky["T"], sky["E"], sky["B"], sky["phi"], nthreads=cores)
        row = {}
        for name, prec in forms:
            plan = api.Plan(w.nside, w.lmax, n, pol=True, precision=prec)
            try:
                out = plan.lens(d["T"], d["E"], d["B"], d["phi"]).double().cpu().numpy()
            finally:
                torch.cuda.synchronize()
                plan.close()
            torch.cuda.empty_cache()
            e = {}
            for i, f in enumerate("TQU"):
                r = ref[f]
                dlt = out[i][pix] - r
                rms = np.sqrt(np.mean(r ** 2))
                e[f] = {"rel_rms": float(np.sqrt(np.mean(dlt ** 2)) / rms), "max_rel": float(np.max(np.abs(dlt)) / rms)}
            row[name] = e
            print(json.dumps({"order": n, "form": name, "err": e}), file=sys.stderr, flush=True)
        table[str(n)] = row
    print(json.dumps({"sweep": "error vs FP64 oracle", "workload": WORKLOAD, "npix_sample": int(len(pix)),
                      "sample": "every pixel of the first and last 2 rings; 8 on the cap edges, belt edges and "
                                "equator; 16 random",
                      "errors": table}), flush=True)


def _ring_latitude_deg(nside):
    """Latitude (degrees) of each HEALPix ring 1 .. 4 Nside - 1 and its pixel count,
    for binning the output maps by latitude."""
    i = np.arange(1, 4 * nside, dtype=np.float64)
    ii = np.minimum(i, 4 * nside - i)
    z = np.where(ii < nside, 1.0 - ii * ii / (3.0 * nside * nside), 4.0 / 3.0 - 2.0 * ii / (3.0 * nside))
    z = np.where(i > 2 * nside, -z, z)
    n = np.where(ii < nside, 4 * ii, 4 * nside).astype(np.int64)
    return np.degrees(np.arcsin(z)), n


def _lensed_spectra(plan, lmax, maps):
    """TT, EE, BB, TE, TB, EB of lensed maps through tl_map2alm and tl_anafast."""
    from paper_1307_0719_gb300 import api
    a = plan.map2alm(maps[0].contiguous(), maps[1].contiguous(), maps[2].contiguous())
    return api.anafast(lmax, a["T"], a["E"], a["B"]).cpu().numpy()


def run_experiment(args):
    """The paper's accuracy experiments (Sec. III.A) on synthetic skies, one JSON line
    each. No CAMB spectra exist here, so the convergence study measures each order
    against the highest one on the same realisations (self-convergence).
      convergence (Fig. 3 analogue): for each Nside of 512, 1024, 2048 (lmax = 2 Nside,
        the workloads' spectra) the lensed TT, EE, BB spectra (tl_map2alm + tl_anafast
        of the lensed maps, two realisations summed) at orders 0 .. 5 against order 6.
        Per Delta l = 50 bin the deviation is (sum_bin C_l(n)) / (sum_bin C_l(6)) - 1;
        l_star is the centre of the last bin before the first one whose |deviation|
        reaches 0.5% (the paper's definition of the highest accurate multipole).
      rotation (Fig. 7 analogue): Nside 2048, lmax 4096, order 4, one realisation. The
        maps with the geodesic displacement and the rotation R against (a) the same
        without R and (b) the naive displacement (coordinates added) without R: per
        latitude bin the error's standard deviation over the signal's, for T and for
        P = Q + iU, and the error's TT, EE, BB spectra over the signal's per Delta l =
        50 bin (maximum over l <= 2 Nside)."""
    import torch
    from paper_1307_0719_gb300 import api
    dev = torch.device("cuda", 0)
    prec = api.MIXED_FP32
    if args.experiment == "convergence":
        out = {"experiment": "self-convergence of the lensed spectra against order 6 (Fig. 3 analogue)",
               "form": "mixed FP32", "realisations": 2, "bins": "Delta l = 50 from l = 2",
               "criterion": "|sum_bin C_l(n) / sum_bin C_l(6) - 1| < 0.5%", "nside": {}}
        for name in ("nside512_lmax1024_n4_TQU", "nside1024_lmax2048_n4_TQU", "nside2048_lmax4096_n4_TQU"):
            w = skygen.WORKLOADS[name]
            skies = [skygen.make_sky(w.nside, w.lmax, True, w.seed_t + 100 * i, w.seed_e + 100 * i,
                                     w.seed_phi + 100 * i, w.damp_t, w.damp_e) for i in range(2)]
            cls = {}
            for n in range(0, 7):
                plan = api.Plan(w.nside, w.lmax, n, pol=True, precision=prec)
                try:
                    acc = 0.0
                    for sk in skies:
                        d = {k: torch.from_numpy(v).to(dev) for k, v in sk.items()}
                        acc = acc + _lensed_spectra(plan, w.lmax, plan.lens(d["T"], d["E"], d["B"], d["phi"]))
                        del d
                    cls[n] = acc
                finally:
                    torch.cuda.synchronize()
                    plan.close()
            bins = [(lo, min(lo + 50, w.lmax + 1)) for lo in range(2, w.lmax + 1, 50)]
            row = {}
            for n in range(0, 6):
                per = {}
                for q, spec in ((0, "TT"), (1, "EE"), (2, "BB")):
                    devs = [float(cls[n][q][lo:hi].sum() / cls[6][q][lo:hi].sum() - 1.0) for lo, hi in bins]
                    ls = None
                    for (lo, hi), e in zip(bins, devs):
                        if abs(e) >= 5e-3:
                            break
                        ls = 0.5 * (lo + hi - 1)
                    lim = lambda lm: float(max(abs(e) for (lo, hi), e in zip(bins, devs) if hi - 1 <= lm))
                    per[spec] = {"l_star": ls, "l_star_over_nside": None if ls is None else ls / w.nside,
                                 "max_dev_l_le_nside": lim(w.nside), "max_dev_l_le_1p5nside": lim(1.5 * w.nside)}
                row[str(n)] = per
            out["nside"][str(w.nside)] = {"lmax": w.lmax, "orders": row}
            print(json.dumps({"progress": name, "orders": row}), file=sys.stderr, flush=True)
        print(json.dumps(out), flush=True)
        return
    # rotation
    w = skygen.WORKLOADS["nside2048_lmax4096_n4_TQU"]
    sky = skygen.workload_sky(w.name)
    d = {k: torch.from_numpy(v).to(dev) for k, v in sky.items()}
    variants = {"full": dict(rotate=True), "no_R": dict(rotate=False), "naive": dict(rotate=False, naive=True)}
    maps = {}
    for key, kw in variants.items():
        plan = api.Plan(w.nside, w.lmax, w.order, pol=True, precision=prec, **kw)
        try:
            maps[key] = plan.lens(d["T"], d["E"], d["B"], d["phi"])
        finally:
            torch.cuda.synchronize()
            plan.close()
    lat, nring = _ring_latitude_deg(w.nside)
    edges = np.array([0, 10, 20, 30, 40, 50, 60, 70, 80, 85, 88, 89, 90.0])
    rbin = np.clip(np.searchsorted(edges, np.abs(lat), side="right") - 1, 0, len(edges) - 2)
    pbin = torch.from_numpy(np.repeat(rbin, nring)).to(dev)
    nb = len(edges) - 1

    def per_bin(x):  # mean of x per latitude bin
        x = x.double()
        s = torch.zeros(nb, dtype=torch.float64, device=dev).index_add_(0, pbin, x)
        c = torch.zeros(nb, dtype=torch.float64, device=dev).index_add_(0, pbin, torch.ones_like(x))
        return (s / c).cpu().numpy()

    def std_bin(x):
        x = x.double()
        m = per_bin(x)
        return np.sqrt(np.maximum(per_bin(x * x) - m * m, 0.0))

    F = maps["full"]
    sT, sP = std_bin(F[0]), np.sqrt(std_bin(F[1]) ** 2 + std_bin(F[2]) ** 2)
    plan = api.Plan(w.nside, w.lmax, 0, pol=True, precision=prec)
    try:
        c_sig = _lensed_spectra(plan, w.lmax, F)
        res = {}
        for key in ("no_R", "naive"):
            E = maps[key] - F  # rounded relative to the difference itself
            eT, eP = std_bin(E[0]), np.sqrt(std_bin(E[1]) ** 2 + std_bin(E[2]) ** 2)
            c_err = _lensed_spectra(plan, w.lmax, E)
            spec = {}
            for q, nm in ((0, "TT"), (1, "EE"), (2, "BB")):
                r = [float(c_err[q][lo:lo + 50].sum() / c_sig[q][lo:lo + 50].sum())
                     for lo in range(2, 2 * w.nside + 1, 50)]
                spec[nm] = {"max_err_over_signal_l_le_2nside": max(r)}
            res[key] = {"by_latitude": [{"abs_lat_deg": [float(edges[b]), float(edges[b + 1])],
                                         "T": float(eT[b] / sT[b]), "P": float(eP[b] / sP[b])} for b in range(nb)],
                        "spectra": spec}
    finally:
        torch.cuda.synchronize()
        plan.close()
    print(json.dumps({"experiment": "error of leaving out R, and of the naive displacement (Fig. 7 analogue)",
                      "workload": w.name, "form": "mixed FP32, order 4",
                      "measure": "std of error / std of signal per |latitude| bin; error C_l / signal C_l",
                      "variants": res}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=sorted(skygen.WORKLOADS) + ["batched64_n4_TQU", ADJ_WORKLOAD])
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--form", default=None, choices=["fp32", "tf32", "tf32x3", "bf16x3"])
    ap.add_argument("--batch", type=int, default=0,
                    help="realisations per step (default: the plan's Legendre batch, 16 on tensor cores)")
    ap.add_argument("--sample-pixels", type=int, default=16)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweep-errors", action="store_true",
                    help="print the error table of the full-size workload per order and form, then exit")
    ap.add_argument("--sweep-orders", default="2,3,4,5,6")
    ap.add_argument("--experiment", default=None, choices=["convergence", "rotation"],
                    help="print one of the paper's accuracy experiments on synthetic skies, then exit")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the batched and gradient sub-records of the default line")
    args = ap.parse_args()
    args.form_given = args.form is not None
    if args.form is None:
        args.form = "bf16x3"
    if args.sweep_errors:
        run_sweep(args)
    elif args.experiment:
        run_experiment(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched64_n4_TQU":
        line = run_batched(args)
        if line:
            print(json.dumps(line), flush=True)
    elif args.workload == ADJ_WORKLOAD:
        line = run_adjoint(args)
        if line:
            print(json.dumps(line), flush=True)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
