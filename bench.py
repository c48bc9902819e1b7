"""Throughput benchmark of the lattice-Boltzmann Maxwell hot path on one GB300.

Workload (default): 4096 x 4096 periodic 2D heterogeneous medium (n = 1 + 2 s,
s seeded smoothed random field, sigma = 20 cells, seed 2), Ricker point
current at the centre (~20 cells per local wavelength), 64 receivers, 5000
time steps, FP32 storage.  One benchmark step is one full pass of the hot
path over that input: medium upload, initial state, 5000 fused
stream-collide steps with the source and receivers (2500 launches of the
two-step kernel, the library's default for this case), field extraction,
receiver traces and the FP64 diagnostics.  The distributions (2 x 336 MB)
are larger than L2, so no flush is needed between steps.

Metric: Mlups (10^6 lattice-site updates per second) = sites x 5000 / time.
The stream-collide kernels are bound by HBM bandwidth: 44 algorithmic bytes
per site per launch (5 populations read + 5 written in FP32, plus c_L^2),
whether a launch advances one step or two.

--impl reference times the FP64 CPU oracle (test infrastructure) on a
bounded sample of the same workload.  With torchrun (N > 1) the path shards:
the 4096^2 recipe is weak-scaled into a (4096 N) x 4096 grid, rank r holding
the slab of rows [4096 r, 4096 (r+1)) (medium seed 2 + r, its own Ricker
source and receivers), periodic across the ranks; each slab steps two steps
per launch and exchanges a two-row halo with its neighbours over NCCL
(send / receive of device buffers) after every launch.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1108_2651_gb300 import workloads as W  # noqa: E402

BYTES_PER_SITE = {"f32": 44, "f16": 24, "bf16": 24, "i16b": 26.5}
# DRAM bytes (read + write) per launch from one ncu capture of the kernel as it is now built, keyed by
# (workload, storage, variant); the capture and its command are summarised in profiles/.  Only reported for
# the kernel that was captured.
NCU_TRAFFIC = {("het2d_4096", "f32", "tb2-0"): 433.764864e6 + 300.201472e6,
               ("het2d_4096", "f32", "tb2-10"): 412.030720e6 + 284.538624e6,
               ("het2d_4096", "f16", "tb2-0"): 238.282240e6 + 128.542464e6,
               ("het2d_4096", "i16b", "tb2-0"): 264.385536e6 + 150.971648e6,
               # dram__bytes.sum.per_second x gpu__time_duration.sum (6.657849 TB/s x 174.752 us), step2d_gen
               ("het2d_drude_4096", "f32", "disp"): 6.657849e12 * 174.752e-6,
               ("het2d_aniso_4096", "f32", "tb2an"): 431.234560e6 + 297.513216e6,
               ("het2d_drude_4096", "f32", "tb2pole"): 801.680128e6 + 435.911168e6}
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")


def BATCH_SPL(variant):
    """Steps per launch of a batch launch shape (lbem_batch_set_variant: 9, 10, 11 advance two steps)."""
    return 2 if variant >= 9 else 1


def measured_peak_gbs():
    try:
        with open(PEAKS) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi SM clock and throttle reasons, sampled every 200 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                vals = [v.strip() for v in out.stdout.strip().split(",")]
                if len(vals) == 6:
                    self.samples.append(vals)
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if s[2 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def workload(name):
    if name == "het2d_4096":
        return W.heterogeneous_2d(4096, seed=2, nsteps=5000)
    if name == "het2d_1024":
        return W.heterogeneous_2d(1024, seed=1, nsteps=5000)
    if name == "het2d_walls_4096":
        return W.heterogeneous_2d_walls(4096, seed=2, nsteps=5000)
    if name == "het2d_drude_4096":
        return W.heterogeneous_2d_drude(4096, seed=2, nsteps=5000)
    if name == "het2d_aniso_4096":
        return W.heterogeneous_2d_aniso(4096, seed=2, nsteps=5000)
    if name == "het3d_192":
        return W.heterogeneous_3d(192, seed=4, nsteps=1000)
    if name == "het3d_box_192":  # the same in a PEC box with a 16-site absorbing layer
        q = W.heterogeneous_3d(192, seed=4, nsteps=1000)
        q.bc, q.layer, q.gamma_max = (1, 1, 1), 16, 0.2
        return q
    raise ValueError(name)


def run_batch_main(args, lbem, torch, stream, peak, peak_kind):
    """The 256-media batch as the timed workload (used to profile the batched kernel on its own)."""
    probs = W.batch_2d(256, nsteps=args.lb_steps or 2000)
    nsteps = probs[0].nsteps
    ss = []
    for q in probs:
        s = lbem.Solver(q.shape, stream=stream.cuda_stream)
        s.set_problem(q)
        ss.append(s)
    b = lbem.lbem_batch_create([s.h for s in ss], stream.cuda_stream)
    v = lbem.lbem_batch_autotune(b, 200) if args.autotune else lbem.lbem_batch_get_variant(b)[0]
    if args.variant is not None:
        lbem.lbem_batch_set_variant(b, args.variant)
        v = args.variant
    for _ in range(args.warmup):
        for s in ss:
            lbem.lbem_set_fields(s.h)
        lbem.lbem_batch_step(b, nsteps)
    torch.cuda.synchronize()
    evs = []
    with ClockSampler(0) as clk:
        for _ in range(args.steps):
            for s in ss:
                lbem.lbem_set_fields(s.h)
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            lbem.lbem_batch_step(b, nsteps)
            e.record(stream)
            evs.append((a, e))
        torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(e) for a, e in evs]))
    sites = sum(int(np.prod(q.shape)) for q in probs)
    lbem.lbem_batch_destroy(b)
    for s in ss:
        s.close()
    spl = BATCH_SPL(v)
    launches = nsteps // spl + nsteps % spl
    per = ms / launches
    gbs = 44 * sites / (per * 1e-3) / 1e9
    value = sites * nsteps / (ms * 1e-3) / 1e6
    print(json.dumps({"metric": "Mlups", "value": value, "unit": "Mlups", "n_gpus": 1, "steps": args.steps,
                      "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                      "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": "batch256", "media": len(probs), "sites": sites, "lb_steps": nsteps},
                      "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                                   "traffic": None, "kernel": ("step2d_batch_ss2" if v >= 14 else "step2d_batch_tb2" if spl == 2
                                                                 else "step2d_batch") + f" (variant {v})", "steps_per_launch": spl,
                                   "ms_per_launch": per, "peak_kind": peak_kind},
                      "gpu_launches": args.steps * launches, "clocks": clk.summary()}), flush=True)


def run_adjoint_main(args, lbem, torch, stream, peak, peak_kind):
    """The 3D adjoint on a 96^3 heterogeneous medium as the timed workload (small enough to profile): one
    benchmark step = forward record (lb_steps steps, checkpoint every 10) + the backward pass."""
    nsteps = args.lb_steps or 40
    q = W.heterogeneous_3d(96, seed=4, nsteps=nsteps)
    s = lbem.Solver(q.shape, stream=stream.cuda_stream)
    s.set_problem(q)
    lbem.lbem_set_variant(s.h, 1)
    n3 = 96 ** 3
    cot = torch.empty(q.rec_site.size * nsteps, dtype=torch.float32, device="cuda")
    grad = torch.empty(n3, dtype=torch.float32, device="cuda")

    def one(ev=None):
        lbem.lbem_set_fields(s.h)
        lbem.lbem_forward_record(s.h, nsteps, 10)
        lbem.lbem_traces(s.h, cot)
        if ev is not None:
            ev[0].record(stream)
        lbem.lbem_adjoint(s.h, cot, grad)
        if ev is not None:
            ev[1].record(stream)

    for _ in range(args.warmup):
        one()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        start.record(stream)
        for k in range(args.steps):
            one(evs[k])
        stop.record(stream)
        torch.cuda.synchronize()
    ms = start.elapsed_time(stop) / args.steps
    bwd = float(np.mean([a.elapsed_time(b) for a, b in evs]))
    s.close()
    # backward bytes: recompute of nsteps - every forward steps (172 B/site) + nsteps adjoint steps (272 B/site)
    bb = ((nsteps - 10) * 172 + nsteps * 272) * n3
    gbs = bb / (bwd * 1e-3) / 1e9
    print(json.dumps({"metric": "Mlups", "value": n3 * nsteps / (ms * 1e-3) / 1e6, "unit": "Mlups", "n_gpus": 1,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": "adjoint3d_96", "grid": [96, 96, 96], "lb_steps": nsteps,
                                 "checkpoint_every": 10, "note": "value counts forward site-steps per second of "
                                 "forward record + backward pass"},
                      "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                                   "traffic": None, "kernel": "backward pass (recompute + adjoint3d_site)",
                                   "ms_backward": bwd, "peak_kind": peak_kind},
                      "gpu_launches": None, "clocks": clk.summary()}), flush=True)


def _time_run(lbem, torch, s, p, nsteps, stream, passes=1):
    """Device time (ms) of `passes` full runs of nsteps steps on solver s (launch shape autotuned), after one
    untimed run; returns (ms, variant, steps per launch)."""
    s.set_problem(p)
    v = lbem.lbem_autotune(s.h, 50)
    spp = lbem.lbem_get_temporal_blocking(s.h)[0]
    lbem.lbem_step(s.h, nsteps)
    ev = []
    for _ in range(passes):
        lbem.lbem_set_fields(s.h)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        lbem.lbem_step(s.h, nsteps)
        b.record(stream)
        ev.append((a, b))
    torch.cuda.synchronize()
    return float(np.mean([a.elapsed_time(b) for a, b in ev])), v, spp


def other_forms(lbem, torch, p, peak, stream):
    """Mlups and HBM roofline of the other forms on this GPU: 16-bit storage and single-step launches of the
    same workload, the 256-media batch (2000 steps, one graph-captured launch per step), the 192^3 3D forward
    (1000 steps) and the 3D adjoint."""
    out = {}
    n = int(np.prod(p.shape))
    for st in ("f16", "bf16", "i16b"):
        s = lbem.Solver(p.shape, storage=st, stream=stream.cuda_stream)
        ms, v, spp = _time_run(lbem, torch, s, p, p.nsteps, stream)
        s.close()
        per = ms / (p.nsteps // spp + p.nsteps % spp)  # per launch of `spp` steps
        gbs = BYTES_PER_SITE[st] * n / (per * 1e-3) / 1e9
        out[st] = {"mlups": n * p.nsteps / (ms * 1e-3) / 1e6, "ms_per_launch": per, "achieved_gbs": gbs,
                   "frac": gbs / peak, "bytes_per_site_per_launch": BYTES_PER_SITE[st], "steps_per_launch": spp,
                   "variant": v}
    # single-step launches (same workload, FP32): the fastest single-step kernel, 44 B/site per step
    s = lbem.Solver(p.shape, stream=stream.cuda_stream)
    lbem.lbem_set_temporal_blocking(s.h, 1, -1)
    ms, v, _ = _time_run(lbem, torch, s, p, p.nsteps, stream)
    s.close()
    per = ms / p.nsteps
    gbs = 44 * n / (per * 1e-3) / 1e9
    out["f32_single_step"] = {"mlups": n * p.nsteps / (ms * 1e-3) / 1e6, "ms_per_launch": per, "achieved_gbs": gbs,
                              "frac": gbs / peak, "bytes_per_site": 44, "steps_per_launch": 1, "variant": v}
    # config 1: the 1024^2 medium (seed 1), 5000 steps, FP32; its 2 x 21 MB distributions and 4 MB medium stay in
    # the 129 MB L2, so the bytes per launch over the launch time are an effective rate, above the HBM copy rate
    # the launches are short here, so both stepping modes are timed with CUDA-graph replay and the faster is kept
    p1 = W.heterogeneous_2d(1024, seed=1, nsteps=5000)
    n1 = int(np.prod(p1.shape))
    best1 = None
    for spl_set in (1, 2):
        s = lbem.Solver(p1.shape, stream=stream.cuda_stream)
        s.set_problem(p1)
        lbem.lbem_set_temporal_blocking(s.h, spl_set, -1)
        lbem.lbem_set_graphs(s.h, True)
        lbem.lbem_step(s.h, p1.nsteps)
        evs1 = []
        for _ in range(3):
            lbem.lbem_set_fields(s.h)
            a1, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a1.record(stream)
            lbem.lbem_step(s.h, p1.nsteps)
            b1.record(stream)
            evs1.append((a1, b1))
        torch.cuda.synchronize()
        ms1 = float(np.mean([a1.elapsed_time(b1) for a1, b1 in evs1]))
        spp1, v1 = lbem.lbem_get_temporal_blocking(s.h)[0], lbem.lbem_get_variant(s.h)[0]
        s.close()
        if best1 is None or ms1 < best1[0]:
            best1 = (ms1, v1, spp1)
    ms, v, spp = best1
    per = ms / (p1.nsteps // spp + p1.nsteps % spp)
    gbs = 44 * n1 / (per * 1e-3) / 1e9
    out["f32_1024"] = {"mlups": n1 * p1.nsteps / (ms * 1e-3) / 1e6, "ms_per_launch": per, "effective_gbs": gbs,
                       "frac": gbs / peak, "bytes_per_site_per_launch": 44, "steps_per_launch": spp, "variant": v,
                       "l2_resident": True, "graphs": True, "lb_steps": p1.nsteps}
    probs = W.batch_2d(256, nsteps=2000)
    ss = []
    for q in probs:
        s = lbem.Solver(q.shape, stream=stream.cuda_stream)
        s.set_problem(q)
        ss.append(s)
    b = lbem.lbem_batch_create([s.h for s in ss], stream.cuda_stream)
    # trials of 200 steps: a two-step variant packs and unpacks the members once per call, which a short trial
    # would not amortise
    v = lbem.lbem_batch_autotune(b, 200)
    lbem.lbem_batch_step(b, 2000)
    for s in ss:
        lbem.lbem_set_fields(s.h)
    torch.cuda.synchronize()
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    lbem.lbem_batch_step(b, 2000)
    e.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(e)
    sites = sum(int(np.prod(q.shape)) for q in probs)
    lbem.lbem_batch_destroy(b)
    for s in ss:
        s.close()
    spl = BATCH_SPL(v)
    per = ms / (2000 // spl)
    gbs = 44 * sites / (per * 1e-3) / 1e9
    out["batch256"] = {"mlups": sites * 2000 / (ms * 1e-3) / 1e6, "ms_per_launch": per, "achieved_gbs": gbs,
                       "frac": gbs / peak, "sites": sites, "media": len(probs), "lb_steps": 2000, "variant": v,
                       "graph": True, "steps_per_launch": spl,
                       "kernel": "step2d_batch_ss2" if v >= 14 else "step2d_batch_tb2" if spl == 2 else "step2d_batch"}
    # heterogeneous permeability (B x grad ln mu source at every site), 2000 steps: 52 B/site per launch (the
    # grad ln mu planes add 8 to the 44), two steps per launch by default, then single-step launches
    pm = W.heterogeneous_2d_mu(p.shape[0], seed=2, nsteps=2000)
    for key, spp_set in (("f32_mu_heterogeneous", 2), ("f32_mu_single_step", 1)):
        s = lbem.Solver(pm.shape, stream=stream.cuda_stream)
        if spp_set == 1:
            lbem.lbem_set_temporal_blocking(s.h, 1, -1)
        ms, v, spp = _time_run(lbem, torch, s, pm, 2000, stream)
        shape_mu = lbem.lbem_get_temporal_blocking(s.h)[1]
        s.close()
        per = ms / (2000 // spp)
        gbs = 52 * n / (per * 1e-3) / 1e9
        kern = ("step2d_ss2<MU>" if shape_mu == 2 else f"step2d_tb2<MU> (tile shape {shape_mu})") if spp == 2 \
            else f"step2d<f32, MU> (variant {v})"
        out[key] = {"mlups": n * 2000 / (ms * 1e-3) / 1e6, "ms_per_launch": per, "achieved_gbs": gbs,
                    "frac": gbs / peak, "bytes_per_site_per_launch": 52, "steps_per_launch": spp, "variant": v,
                    "lb_steps": 2000, "kernel": kern}
    # the same medium in a PEC box with a 32-site absorbing layer, 2000 steps: the stream-collide launches plus
    # the edge kernel after each (44 algorithmic B/site per launch; the edge recompute counts as overhead)
    pw = W.heterogeneous_2d_walls(p.shape[0], seed=2, nsteps=2000)
    s = lbem.Solver(pw.shape, stream=stream.cuda_stream)
    ms, v, spp = _time_run(lbem, torch, s, pw, 2000, stream)
    s.close()
    per = ms / (2000 // spp)
    gbs = 44 * n / (per * 1e-3) / 1e9
    out["f32_walls_absorbing"] = {"mlups": n * 2000 / (ms * 1e-3) / 1e6, "ms_per_launch": per, "achieved_gbs": gbs,
                                  "frac": gbs / peak, "bytes_per_site_per_launch": 44, "steps_per_launch": spp,
                                  "variant": v, "lb_steps": 2000, "bc": list(pw.bc), "layer": pw.layer,
                                  "gamma_max": pw.gamma_max}
    # the same medium with a lossy Drude cylinder (one dispersive pole per site), 2000 steps: 44 B/site plus the
    # pole's J and P read and written (16) and its three parameters read (12) = 72 B/site per launch; two steps
    # per launch by default (the tile kernel carrying the pole), then single-step launches of the general kernel
    pd = W.heterogeneous_2d_drude(p.shape[0], seed=2, nsteps=2000)
    for key, spp_set in (("f32_drude_dispersive", 2), ("f32_drude_single_step", 1)):
        s = lbem.Solver(pd.shape, stream=stream.cuda_stream)
        if spp_set == 1:
            lbem.lbem_set_temporal_blocking(s.h, 1, -1)
        ms, v, spp = _time_run(lbem, torch, s, pd, 2000, stream)
        s.close()
        per = ms / (2000 // spp)
        gbs = 72 * n / (per * 1e-3) / 1e9
        out[key] = {"mlups": n * 2000 / (ms * 1e-3) / 1e6, "ms_per_launch": per, "achieved_gbs": gbs,
                    "frac": gbs / peak, "bytes_per_site_per_launch": 72, "steps_per_launch": spp, "lb_steps": 2000,
                    "kernel": "step2d_tb2<POLE>" if spp == 2 else "step2d_gen"}
    # the same medium made uniaxial, mu = diag(2, 1) (per-axis lattice weights), 2000 steps: 44 B/site per
    # launch, two steps per launch by default (the strip or the tile kernel with per-axis weights, as autotuned),
    # then single-step launches of the general kernel
    pa = W.heterogeneous_2d_aniso(p.shape[0], seed=2, nsteps=2000)
    for key, spp_set in (("f32_anisotropic", 2), ("f32_anisotropic_single_step", 1)):
        s = lbem.Solver(pa.shape, stream=stream.cuda_stream)
        if spp_set == 1:
            lbem.lbem_set_temporal_blocking(s.h, 1, -1)
        ms, v, spp = _time_run(lbem, torch, s, pa, 2000, stream)
        shape_an = lbem.lbem_get_temporal_blocking(s.h)[1]
        s.close()
        per = ms / (2000 // spp)
        gbs = 44 * n / (per * 1e-3) / 1e9
        kern = ("step2d_ss2<AN>" if shape_an == 1 else "step2d_tb2<AN>") if spp == 2 else "step2d_gen"
        out[key] = {"mlups": n * 2000 / (ms * 1e-3) / 1e6, "ms_per_launch": per, "achieved_gbs": gbs,
                    "frac": gbs / peak, "bytes_per_site_per_launch": 44, "steps_per_launch": spp, "lb_steps": 2000,
                    "kernel": kern, "mu_tensor": list(pa.aniso)}
    # 192^3 in a PEC box with a 16-site absorbing layer (walls applied by the one-site-per-thread 3D kernel),
    # 500 steps: 172 B/site
    qb = W.heterogeneous_3d(192, nsteps=500)
    qb.bc, qb.layer, qb.gamma_max = (1, 1, 1), 16, 0.2
    s = lbem.Solver(qb.shape, stream=stream.cuda_stream)
    ms, v, _ = _time_run(lbem, torch, s, qb, 500, stream)
    s.close()
    n3 = int(np.prod(qb.shape))
    per = ms / 500
    gbs = 172 * n3 / (per * 1e-3) / 1e9
    out["het3d_192_box"] = {"mlups": n3 * 500 / (ms * 1e-3) / 1e6, "ms_per_launch": per, "achieved_gbs": gbs,
                            "frac": gbs / peak, "bytes_per_site": 172, "variant": v, "lb_steps": 500,
                            "steps_per_launch": 1,
                            "bc": list(qb.bc), "layer": qb.layer}
    q = W.heterogeneous_3d(192, nsteps=1000)
    s = lbem.Solver(q.shape, stream=stream.cuda_stream)
    ms, v, _ = _time_run(lbem, torch, s, q, 1000, stream)
    # adjoint: forward with a checkpoint every 100 steps, then the reverse-time pass (segment recompute +
    # adjoint kernel, FP64 gradient accumulation), cotangent = the traces themselves; the faster of the
    # two one-site-per-thread adjoint shapes (3D variants 1 and 2) on a short trial
    trial = {}
    for v3 in (1, 2):
        lbem.lbem_set_variant(s.h, v3)
        lbem.lbem_set_fields(s.h)
        lbem.lbem_forward_record(s.h, 50, 25)
        c0 = torch.zeros(q.rec_site.size * 50, dtype=torch.float32, device="cuda")
        g0 = torch.empty(192 ** 3, dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lbem.lbem_adjoint(s.h, c0, g0)
        torch.cuda.synchronize()
        trial[v3] = time.perf_counter() - t0
    v_adj = min(trial, key=trial.get)
    lbem.lbem_set_variant(s.h, v_adj)
    lbem.lbem_set_fields(s.h)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record(stream)
    lbem.lbem_forward_record(s.h, 1000, 100)
    ev[1].record(stream)
    cot = torch.empty(q.rec_site.size * 1000, dtype=torch.float32, device="cuda")
    lbem.lbem_traces(s.h, cot)
    grad = torch.empty(192 ** 3, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    ev[2].record(stream)
    lbem.lbem_adjoint(s.h, cot, grad)
    ev[3].record(stream)
    torch.cuda.synchronize()
    s.close()
    t_fwd, t_adj = ev[0].elapsed_time(ev[1]), ev[2].elapsed_time(ev[3])
    n3 = 192 ** 3
    per = ms / 1000
    gbs = 172 * n3 / (per * 1e-3) / 1e9
    out["het3d_192"] = {"mlups": n3 * 1000 / (ms * 1e-3) / 1e6, "ms_per_launch": per, "achieved_gbs": gbs,
                        "frac": gbs / peak, "bytes_per_site": 172, "variant": v, "steps_per_launch": 1}
    # backward pass bytes: recompute of 900 forward steps (172 B/site) + 1000 adjoint steps (272 B/site:
    # lambda 84 read + state 84 read + c_L^2 4 + FP64 gradient 16 read/write + lambda 84 write)
    bwd_bytes = (900 * 172 + 1000 * 272) * n3
    out["adjoint_192"] = {"lb_steps": 1000, "checkpoint_every": 100, "variant": v_adj, "ms_forward_record": t_fwd,
                          "ms_backward": t_adj, "mlups_forward_plus_backward": n3 * 1000 / ((t_fwd + t_adj) * 1e-3) / 1e6,
                          "backward_achieved_gbs": bwd_bytes / (t_adj * 1e-3) / 1e9,
                          "backward_frac": bwd_bytes / (t_adj * 1e-3) / 1e9 / peak}
    return out


def _crop_pole(p, crop):
    """The workload's dispersive pole on a crop of its grid (None without one)."""
    if p.D != 2 or p.wp2 is None:
        return None
    f = lambda a: np.asarray(np.broadcast_to(0.0 if a is None else a, p.shape)[crop], np.float32).astype(np.float64)
    return dict(wp2=f(p.wp2), wr2=f(p.wr2), gamma=f(p.gamma))


def cpu_baseline(p, budget_s=12.0):
    """Time the FP64 oracle (as it stands) on a bounded sample: a 1024^2 crop of the medium centred on the
    source, as many steps as fit in about budget_s seconds of CPU work."""
    import oracle as O

    n = min(1024 if p.D == 2 else 64, p.shape[0])
    c0 = (p.shape[0] - n) // 2
    crop = tuple(slice(c0, c0 + n) for _ in range(p.D))
    eps = np.asarray(p.eps_r[crop], np.float32).astype(np.float64)
    m = O.medium(p.D, eps, bc=p.bc, layer=min(p.layer, n // 2), gamma_max=p.gamma_max, dispersion=_crop_pole(p, crop),
                 aniso=p.aniso)
    g = O.init_state(m)
    pole = O.pole_state(m) if m.wp2 is not None else None
    shape = (n,) * p.D
    src = dict(site=np.array([W.flat_index(shape, (n // 2,) * p.D)]), comp=np.array([2]),
               amp=np.asarray(p.src_amp, np.float32).astype(np.float64))
    t0 = time.perf_counter()
    O.run(m, g, 10, sources=src, pole=pole)
    dt10 = time.perf_counter() - t0
    steps = int(max(10, min(p.nsteps - 10, budget_s / max(dt10 / 10, 1e-6))))
    t0 = time.perf_counter()
    O.run(m, g, steps, t0=10, sources=src, pole=pole)
    dt = time.perf_counter() - t0
    return {"value": n ** p.D * steps / dt / 1e6, "unit": "Mlups", "cores": O.threads(), "kind": "oracle",
            "sample": f"FP64 oracle, {n}^{p.D} crop of the workload's medium, point source, {steps} steps "
                      f"({dt:.1f} s)"}


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform string)."""
    import platform

    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


def crop512(p):
    """The config-2 accuracy case (reading R11): the 512^2 centre crop of the 4096^2 medium run as its own periodic
    problem, Ricker source at its centre, 64 receivers on a circle of radius 128, 5000 steps."""
    c0 = (p.shape[0] - 512) // 2
    eps = np.asarray(p.eps_r[c0:c0 + 512, c0:c0 + 512], np.float64)
    recs = W.circle_receivers((256, 256), 128, 64)
    return W.point_source_problem(2, (512, 512), np.sqrt(eps), 5000, (256, 256), 64, recs, name="crop512")


# rel-L2 bars of the benchmark spec: FP32 storage <= 1e-4 after 5000 steps, reduced-precision storage <= 1e-3
TOL = {"f32": 1e-4, "f16": 1e-3, "bf16": 1e-3, "i16b": 1e-3}


def accuracy_cases(p, spl):
    """Per form, the problem its rel-L2 against the FP64 oracle is stated on, and how the GPU runs it:
    {form: (problem, storage, steps per launch or None for the library default, bar)}.  spl maps a form to the
    steps per launch its timed run used, so the accuracy run takes the same kernels.  The storage forms share
    the 512^2 crop (reading R11); the other forms use their own recipe at 256^2 (3D: 32^3), whose oracle runs fit
    the benchmark's CPU budget; the batch uses its four smallest members."""
    c = crop512(p)
    cases = {"f32": (c, "f32", spl.get("f32"), TOL["f32"])}
    for st in ("f16", "bf16", "i16b"):
        cases[st] = (c, st, spl.get(st), TOL[st])
    cases["f32_single_step"] = (c, "f32", 1, TOL["f32"])
    cases["f32_1024"] = (W.heterogeneous_2d(256, seed=1, nsteps=5000, name="het2d_1024_recipe_256"), "f32",
                         spl.get("f32_1024"), TOL["f32"])
    small = {"f32_mu": W.heterogeneous_2d_mu(256, seed=2, nsteps=1000),
             "f32_walls_absorbing": W.heterogeneous_2d_walls(256, seed=2, nsteps=1000, layer=16),
             "f32_drude": W.heterogeneous_2d_drude(256, seed=2, nsteps=1000),
             "f32_anisotropic": W.heterogeneous_2d_aniso(256, seed=2, nsteps=1000)}
    for key, q in (("f32_mu_heterogeneous", small["f32_mu"]), ("f32_mu_single_step", small["f32_mu"]),
                   ("f32_walls_absorbing", small["f32_walls_absorbing"]), ("f32_drude_dispersive", small["f32_drude"]),
                   ("f32_drude_single_step", small["f32_drude"]), ("f32_anisotropic", small["f32_anisotropic"]),
                   ("f32_anisotropic_single_step", small["f32_anisotropic"])):
        cases[key] = (q, "f32", spl.get(key, 1 if key.endswith("single_step") else None), TOL["f32"])
    q3 = W.heterogeneous_3d(32, seed=4, nsteps=300, sigma=3.0, plane_dz=8, rec_grid=(4, 4))
    cases["het3d_192"] = (q3, "f32", None, TOL["f32"])
    qb = W.heterogeneous_3d(32, seed=4, nsteps=300, sigma=3.0, plane_dz=8, rec_grid=(4, 4))
    qb.bc, qb.layer, qb.gamma_max = (1, 1, 1), 4, 0.2
    qb.name = "het3d_box_32"
    cases["het3d_192_box"] = (qb, "f32", None, TOL["f32"])
    members = sorted(W.batch_2d(256, nsteps=2000), key=lambda q: int(np.prod(q.shape)))[:4]
    cases["batch256"] = (members, "f32", "batch", TOL["f32"])
    return cases


def _f32(a):
    return None if a is None else np.asarray(a, np.float32).astype(np.float64)


def _rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def gpu_result(lbem, torch, stream, q, storage, spl):
    """E, B ((3,) + grid) and traces of problem q run on the GPU library as a form runs it (float64 numpy)."""
    s = lbem.Solver(q.shape, storage=storage, stream=stream.cuda_stream)
    try:
        s.set_problem(q)
        if spl is not None:
            lbem.lbem_set_temporal_blocking(s.h, spl, -1)
        s.step(q.nsteps)
        E, B = s.fields()
        tr = s.traces(q.rec_site.size)
        torch.cuda.synchronize()
        return E.cpu().double().numpy(), B.cpu().double().numpy(), tr.cpu().double().numpy()
    finally:
        s.close()


def gpu_batch_result(lbem, torch, stream, members):
    """The members stepped together by the batched kernel: [(E, B, traces)] per member."""
    ss = []
    for q in members:
        s = lbem.Solver(q.shape, stream=stream.cuda_stream)
        s.set_problem(q)
        ss.append(s)
    b = lbem.lbem_batch_create([s.h for s in ss], stream.cuda_stream)
    lbem.lbem_batch_step(b, members[0].nsteps)
    out = []
    for s, q in zip(ss, members):
        E, B = s.fields()
        tr = s.traces(q.rec_site.size)
        torch.cuda.synchronize()
        out.append((E.cpu().double().numpy(), B.cpu().double().numpy(), tr.cpu().double().numpy()))
    lbem.lbem_batch_destroy(b)
    for s in ss:
        s.close()
    return out


def oracle_leg(p, cases, gpu_out):
    """The CPU-baseline leg: the FP64 oracle, as it stands, on the host cores.  It times the oracle on the config-2
    accuracy case (the 512^2 crop x 5000 steps, all cores), on one core (a 256^2 crop, 200 steps) and as an FP32
    build of the same source (the 512^2 crop, 500 steps), and runs the oracle on every other form's accuracy case;
    returns (cpu_baseline, {form: rel-L2 (E, B, traces)})."""
    import oracle as O

    def run(q):
        disp = None
        if q.D == 2 and q.wp2 is not None:
            full = lambda a: _f32(np.broadcast_to(0.0 if a is None else a, q.shape))
            disp = dict(wp2=full(q.wp2), wr2=full(q.wr2), gamma=full(q.gamma))
        m = O.medium(q.D, _f32(q.eps_r), _f32(q.mu_r), bc=q.bc, layer=q.layer, gamma_max=q.gamma_max,
                     dispersion=disp, aniso=q.aniso)
        g = O.init_state(m, _f32(q.E0), _f32(q.B0))
        pole = O.pole_state(m) if disp is not None else None
        src = q.sources()
        if src is not None:
            src = dict(src, amp=_f32(src["amp"]))
        t0 = time.perf_counter()
        tr = O.run(m, g, q.nsteps, sources=src, receivers=q.receivers(), pole=pole)
        dt = time.perf_counter() - t0
        E, B = O.fields(m, g, pole)
        return np.moveaxis(E, -1, 0), np.moveaxis(B, -1, 0), tr, dt

    cores = O.threads()
    done, samples, acc = {}, {}, {}
    for key, (q, st, spl, tol) in cases.items():
        qs = q if isinstance(q, list) else [q]
        res = []
        for qq in qs:
            if qq.name not in done:
                done[qq.name] = run(qq)
                samples[qq.name] = {"mlups": float(np.prod(qq.shape)) * qq.nsteps / done[qq.name][3] / 1e6,
                                    "seconds": done[qq.name][3]}
            res.append(done[qq.name])
        g = gpu_out.get(key)
        if g is None:
            continue
        gs = g if isinstance(q, list) else [g]
        e = [(_rel(a[0], r[0]), _rel(a[1], r[1]), _rel(a[2], r[2])) for a, r in zip(gs, res)]
        acc[key] = tuple(max(x[k] for x in e) for k in range(3))
    main = done["crop512"]
    c = crop512(p)
    value = 512 * 512 * c.nsteps / main[3] / 1e6
    # one core, a 256^2 crop of the same medium, 200 steps
    q1 = crop512(p)
    q1.eps_r = q1.eps_r[128:384, 128:384]
    q1.shape, q1.nsteps = (256, 256), 200
    q1.src_site = np.array([W.flat_index((256, 256), (128, 128))], np.int64)
    q1.rec_site = np.zeros(0, np.int64)
    q1.rec_comp = np.zeros(0, np.int32)
    q1.name = "crop256_1core"
    O.set_threads(1)
    try:
        one = run(q1)[3]
    finally:
        O.set_threads(cores)
    # FP32 build of the same source, all cores, the 512^2 crop for 500 steps
    dt32, cores32 = O.time_fp32(c.eps_r, 500, int(c.src_site[0]), c.src_amp[0], threads_=cores)
    cpu = {"value": value, "unit": "Mlups", "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
           "sample": f"FP64 oracle, 512^2 centre crop of the {p.shape[0]}^2 medium (config 2's accuracy case), "
                     f"Ricker at the crop centre, 64 receivers, {c.nsteps} steps ({main[3]:.1f} s)",
           "one_core": {"value": 256 * 256 * 200 / one / 1e6, "unit": "Mlups", "cores": 1,
                        "sample": f"FP64 oracle, 256^2 crop of the same medium, 200 steps ({one:.1f} s)"},
           "fp32_build": {"value": 512 * 512 * 500 / dt32 / 1e6, "unit": "Mlups", "cores": cores32,
                          "sample": f"the same oracle source built with float, 512^2 crop, 500 steps ({dt32:.1f} s)"},
           "accuracy_samples": samples}
    return cpu, acc


def slab_problem(rank, world, n=4096, nsteps=5000, halo=2):
    """Rank `rank`'s slab of the weak-scaled workload: a (n world) x n grid whose rows [r n, (r + 1) n) hold the n^2
    heterogeneous recipe with seed 2 + r (Ricker source at the slab centre, 64 receivers), periodic along y across
    the ranks.  Returns the slab with `halo` ghost rows on either side (the neighbours' rows of the medium)."""
    from dataclasses import replace

    own = W.heterogeneous_2d(n, seed=2 + rank, nsteps=nsteps)
    below = own if world == 1 else W.heterogeneous_2d(n, seed=2 + (rank - 1) % world, nsteps=nsteps)
    above = own if world == 1 else W.heterogeneous_2d(n, seed=2 + (rank + 1) % world, nsteps=nsteps)
    eps = np.concatenate([below.eps_r[-halo:], own.eps_r, above.eps_r[:halo]])
    loc = replace(own, shape=(n + 2 * halo, n), eps_r=eps, name=f"het2d_{n}_slab{rank}of{world}")
    loc.src_site = own.src_site + halo * n
    loc.rec_site = own.rec_site + halo * n
    return loc


def slab_pass(lbem, torch, slab, eps_d, E_d, B_d, tr_d, u_d, rank, world, nsteps, host=False, ev=None,
              stream=None):
    """One pass of the decomposed path on this rank: medium upload, initial state, nsteps steps with a halo exchange
    after every two-step launch, fields, traces and the FP64 field energy of the real rows all-reduced over the
    ranks.  Returns the energy."""
    from paper_1108_2651_gb300 import decomp

    h = slab.s.h
    lbem.lbem_set_medium(h, eps_d)
    lbem.lbem_set_fields(h)
    if ev is not None:
        ev[0].record(stream)
    decomp.step_dist(slab, rank, world, nsteps, host=host)
    if ev is not None:
        ev[1].record(stream)
    lbem.lbem_fields(h, E_d, B_d)
    lbem.lbem_traces(h, tr_d)
    lbem.lbem_energy_flux(h, u_d, None)
    nx, hl = slab.nx, slab.halo
    en = u_d.view(-1, nx)[hl:hl + slab.count].double().sum().reshape(1)
    if world > 1:
        import torch.distributed as dist

        if host:
            en = en.cpu()
        dist.all_reduce(en)
    return float(en.item())


def run_slabs_main(args, lbem, torch, rank, world, local, peak, peak_kind):
    """The N-GPU run: this rank's slab of the weak-scaled grid (slab_problem), exchanging over NCCL."""
    import torch.distributed as dist

    from paper_1108_2651_gb300 import decomp

    n, halo = 4096, 2
    nsteps = args.lb_steps or 5000
    loc = slab_problem(rank, world, n, nsteps, halo)
    stream = torch.cuda.current_stream()
    slab = decomp.LbemSlab(loc, n, halo=halo)
    h = slab.s.h
    nsite = slab.s.nsite
    eps_d = torch.as_tensor(np.ascontiguousarray(loc.eps_r, np.float32).ravel(), device="cuda")
    E_d = torch.empty(3 * nsite, dtype=torch.float32, device="cuda")
    B_d = torch.empty_like(E_d)
    u_d = torch.empty(nsite, dtype=torch.float32, device="cuda")
    tr_d = torch.empty(loc.rec_site.size * nsteps, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        slab_pass(lbem, torch, slab, eps_d, E_d, B_d, tr_d, u_d, rank, world, nsteps)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        start.record(stream)
        for k in range(args.steps):
            en = slab_pass(lbem, torch, slab, eps_d, E_d, B_d, tr_d, u_d, rank, world, nsteps, ev=evs[k],
                           stream=stream)
        stop.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    total_ms = dist_max(start.elapsed_time(stop), world)
    step_ms = dist_max(float(np.mean([a.elapsed_time(b) for a, b in evs])), world)
    launches = nsteps // 2 + nsteps % 2
    ms_per_launch = step_ms / launches  # the stepping region: launches and halo exchanges
    ms_per_step = total_ms / args.steps
    real = n * n
    value = world * real * nsteps / (ms_per_step * 1e-3) / 1e6
    achieved = 44 * nsite / (ms_per_launch * 1e-3) / 1e9
    # end to end: the medium from pinned host memory, fields and traces back to it, every pass
    eps_h = torch.from_numpy(np.ascontiguousarray(loc.eps_r, np.float32).ravel()).pin_memory()
    E_h = torch.empty(3 * nsite, dtype=torch.float32).pin_memory()
    B_h = torch.empty(3 * nsite, dtype=torch.float32).pin_memory()
    tr_h = torch.empty(loc.rec_site.size * nsteps, dtype=torch.float32).pin_memory()
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    slab_pass(lbem, torch, slab, eps_h, E_h, B_h, tr_h, u_d, rank, world, nsteps)
    torch.cuda.synchronize()
    dt = dist_max(time.perf_counter() - t0, world)
    nb = lambda t: t.numel() * t.element_size()
    slab.close()
    if rank == 0:
        per_exchange = 2 * 5 * n * 4  # bytes each rank sends per two-step launch (5 rows up, 5 down)
        line = {"metric": "Mlups", "value": value, "unit": "Mlups", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"het2d_4096 weak-scaled: {n * world} x {n} grid, {world} slabs of {n} rows "
                                       f"(medium seeds 2 .. {1 + world}, one Ricker source each)",
                           "grid": [n * world, n], "lb_steps": nsteps, "storage": "f32",
                           "parallelism": f"slabs{world} (two-row halo, NCCL send/recv after every two-step launch, "
                                          f"{per_exchange} B per rank per exchange)",
                           "l2": "inputs larger than L2, no flush"},
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": None,
                             "kernel": "step2d_tb2 on each slab, two steps per launch (time per launch includes the "
                                       "halo exchange)", "steps_per_launch": 2, "ms_per_launch": ms_per_launch,
                             "algorithmic_bytes_per_site_per_launch": 44, "peak_kind": peak_kind},
                "cpu_baseline": None,
                "e2e": {"value": world * real * nsteps / dt / 1e6, "unit": "Mlups", "host_memory": "pinned",
                        "h2d_bytes_per_step": int(nb(eps_h)), "d2h_bytes_per_step": int(nb(E_h) + nb(B_h) + nb(tr_h))},
                "gpu_launches": args.steps * (launches * 5 + 7), "clocks": clk.summary(), "energy_last": en}
        print(json.dumps(line), flush=True)
    dist.destroy_process_group()


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if args.impl != "reference" else "gloo"
        dist.init_process_group(backend)
    return rank, world


def dist_max(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def run_reference(args, rank, world):
    if rank != 0:
        return
    p = workload(args.workload)
    cores = None
    times = []
    steps_per = max(5, int(args.ref_steps))
    import oracle as O

    n = min(1024, p.shape[0])
    c0 = (p.shape[0] - n) // 2
    eps = np.asarray(p.eps_r[c0:c0 + n, c0:c0 + n], np.float32).astype(np.float64)
    crop = (slice(c0, c0 + n), slice(c0, c0 + n))
    m = O.medium(2, eps, bc=p.bc, layer=min(p.layer, n // 2), gamma_max=p.gamma_max, dispersion=_crop_pole(p, crop),
                 aniso=p.aniso)
    src = dict(site=np.array([W.flat_index((n, n), (n // 2, n // 2))]), comp=np.array([2]),
               amp=np.asarray(p.src_amp, np.float32).astype(np.float64))
    for k in range(args.warmup + args.steps):
        g = O.init_state(m)
        pole = O.pole_state(m) if m.wp2 is not None else None
        t0 = time.perf_counter()
        O.run(m, g, steps_per, sources=src, pole=pole)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    cores = O.threads()
    value = n * n * steps_per / (sum(times) / len(times)) / 1e6
    line = {"impl": "reference", "metric": "Mlups", "value": value, "unit": "Mlups", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": p.name, "grid": [n, n], "crop_of": list(p.shape), "lb_steps": steps_per,
                       "storage": "f64-oracle"},
            "cpu_baseline": {"value": value, "unit": "Mlups", "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
                             "sample": f"FP64 oracle, {n}x{n} centre crop of the workload's {p.shape[0]}^2 medium, "
                                       f"{steps_per} steps per benchmark step"},
            "e2e": {"value": value, "unit": "Mlups", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lbem", choices=["lbem", "reference"])
    ap.add_argument("--workload", default="het2d_4096",
                    choices=["het2d_4096", "het2d_1024", "het2d_walls_4096", "het2d_drude_4096",
                             "het2d_aniso_4096", "het3d_192", "het3d_box_192", "batch256", "adjoint3d_96"])
    ap.add_argument("--storage", default="f32", choices=list(BYTES_PER_SITE))
    ap.add_argument("--lb-steps", type=int, default=None, help="override the workload's step count (profiling)")
    ap.add_argument("--ref-steps", type=int, default=40)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--variant", type=int, default=None,
                    help="force a launch shape of the single-step stream-collide kernel (every step single)")
    ap.add_argument("--steps-per-pass", type=int, default=None, choices=[1, 2],
                    help="1: single-step launches; 2: two steps per launch (the library default where it applies)")
    ap.add_argument("--tile-shape", type=int, default=None, help="tile shape of the two-step kernel")
    ap.add_argument("--no-forms", action="store_true", help="skip the 16-bit, batched and 3D forms")
    args = ap.parse_args()
    rank, world = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch

    from paper_1108_2651_gb300 import lbem

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    lbem.load()
    if world > 1:  # the path shards: slabs of a weak-scaled grid with halo exchanges over NCCL
        peak, peak_kind = measured_peak_gbs()
        run_slabs_main(args, lbem, torch, rank, world, local, peak, peak_kind)
        return
    if args.workload == "batch256":
        peak, peak_kind = measured_peak_gbs()
        run_batch_main(args, lbem, torch, torch.cuda.Stream(), peak, peak_kind)
        return
    if args.workload == "adjoint3d_96":
        peak, peak_kind = measured_peak_gbs()
        run_adjoint_main(args, lbem, torch, torch.cuda.Stream(), peak, peak_kind)
        return
    p = workload(args.workload)
    if p.D == 3:
        args.storage = "f32"
        args.no_forms = True
    if args.lb_steps:
        p.nsteps = args.lb_steps
        p.src_amp = p.src_amp[:, : p.nsteps]
    nsteps = p.nsteps
    stream = torch.cuda.Stream()
    eps_d = torch.as_tensor(np.ascontiguousarray(p.eps_r, np.float32).ravel(), device="cuda")
    with torch.cuda.stream(stream):
        s = lbem.Solver(p.shape, storage=args.storage, stream=stream.cuda_stream)
    h = s.h
    state_mb = lbem.lbem_info(h)[1] / 1e6
    aniso = p.D == 2 and p.aniso is not None

    def upload_medium(eps):
        if aniso:
            lbem.lbem_set_medium_aniso(h, eps, *p.aniso)
        else:
            lbem.lbem_set_medium(h, eps)

    upload_medium(eps_d)
    walls = any(p.bc)
    if walls:
        lbem.lbem_set_boundaries(h, p.bc, p.layer, p.gamma_max)
    disp = p.D == 2 and p.wp2 is not None
    if disp:
        dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32).ravel(), device="cuda")
        lbem.lbem_set_dispersion(h, dev(p.wp2), dev(p.wr2), dev(p.gamma))
    lbem.lbem_set_sources(h, p.src_site, p.src_comp, p.src_amp)
    lbem.lbem_set_receivers(h, p.rec_site, p.rec_comp, nsteps)
    variant = lbem.lbem_get_variant(h)[0]
    if args.variant is not None:  # a single-step launch shape: every step runs it
        lbem.lbem_set_temporal_blocking(h, 1, -1)
    if args.steps_per_pass is not None or args.tile_shape is not None:
        lbem.lbem_set_temporal_blocking(h, args.steps_per_pass or 2, -1 if args.tile_shape is None else args.tile_shape)
    if args.autotune:
        lbem.lbem_set_fields(h)
        variant = lbem.lbem_autotune(h, 50)
    if args.variant is not None:
        lbem.lbem_set_variant(h, args.variant)
        variant = args.variant
    spp, tile_shape, _ = lbem.lbem_get_temporal_blocking(h)
    nsite = s.nsite
    E_d = torch.empty(3 * nsite, dtype=torch.float32, device="cuda")
    B_d = torch.empty_like(E_d)
    tr_d = torch.empty(p.rec_site.size * nsteps, dtype=torch.float32, device="cuda")

    def one_pass(ev=None):
        upload_medium(eps_d)
        lbem.lbem_set_fields(h)
        if ev is not None:
            ev[0].record(stream)
        lbem.lbem_step(h, nsteps)
        if ev is not None:
            ev[1].record(stream)
        lbem.lbem_fields(h, E_d, B_d)
        lbem.lbem_traces(h, tr_d)
        return lbem.lbem_diagnostics(h)

    for _ in range(args.warmup):
        one_pass()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        start.record(stream)
        for k in range(args.steps):
            diag = one_pass(evs[k])
        stop.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    total_ms = start.elapsed_time(stop)
    total_ms = dist_max(total_ms, world)
    kern_ms = [a.elapsed_time(b) for a, b in evs]
    # stream-collide launches per run: pairs of steps (plus an odd last step) or single steps
    step_launches = nsteps // 2 + nsteps % 2 if spp == 2 else nsteps
    ms_per_launch = float(np.mean(kern_ms)) / step_launches
    ms_per_step = total_ms / args.steps
    value = world * nsite * nsteps / (ms_per_step * 1e-3) / 1e6

    peak, peak_kind = measured_peak_gbs()
    bps = (72 if disp else BYTES_PER_SITE[args.storage]) if p.D == 2 else 172
    achieved = bps * nsite / (ms_per_launch * 1e-3) / 1e9
    if spp == 2 and args.storage == "f32" and tile_shape >= 9:
        kname, kid = f"step2d_ss2 (strip streaming, tile shape {tile_shape}, 2 steps per launch)", f"tb2-{tile_shape}"
    elif spp == 2 and args.storage == "f32" and tile_shape >= 7:
        kname, kid = f"step2d_rs2 (register streaming, tile shape {tile_shape}, 2 steps per launch)", f"tb2-{tile_shape}"
    elif spp >= 2:
        kern = {2: "step2d_tb2", 3: "step2d_tb3"}[spp] + ("" if args.storage == "f32" else f"h<{args.storage}>")
        kname, kid = f"{kern} (tile shape {tile_shape}, {spp} steps per launch)", f"tb{spp}-{tile_shape}"
    else:
        kname = (f"step2d<{args.storage}>" if p.D == 2 else "step3d") + f" (variant {variant})"
        kid = variant
    if disp and spp == 1:
        kname, kid = "step2d_gen (one dispersive pole per site, single steps)", "disp"
    elif disp:
        kname, kid = "step2d_tb2<POLE> (one dispersive pole per site, tile shape 0, 2 steps per launch)", "tb2pole"
    elif aniso and spp == 1:
        kname, kid = "step2d_gen (anisotropic medium, single steps)", "gen"
    elif aniso and tile_shape == 1:
        kname, kid = "step2d_ss2<AN> (anisotropic medium, strip streaming, 2 steps per launch)", "ss2an"
    elif aniso:
        kname, kid = "step2d_tb2<AN> (anisotropic medium, tile shape 0, 2 steps per launch)", "tb2an"
    elif walls and p.D == 2:
        kname += " + edge2d (walls and layers)"
    elif walls:
        kname = "step3d_site (walls and layers applied in the kernel)"
    traffic = NCU_TRAFFIC.get((args.workload, args.storage, kid)) if args.lb_steps is None else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": kname, "steps_per_launch": spp,
                "algorithmic_bytes_per_site_per_launch": bps, "ms_per_launch": ms_per_launch,
                "peak_kind": peak_kind}

    # end to end through the C ABI with host buffers (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        # pinned host buffers: the medium goes in, the fields and traces come out, every pass
        eps_h = torch.from_numpy(np.ascontiguousarray(p.eps_r, np.float32).ravel()).pin_memory()
        E_h = torch.empty(3 * nsite, dtype=torch.float32).pin_memory()
        B_h = torch.empty(3 * nsite, dtype=torch.float32).pin_memory()
        tr_h = torch.empty(p.rec_site.size * nsteps, dtype=torch.float32).pin_memory()
        def e2e_pass():
            upload_medium(eps_h)
            lbem.lbem_set_sources(h, p.src_site, p.src_comp, p.src_amp)
            lbem.lbem_set_fields(h)
            lbem.lbem_step(h, nsteps)
            lbem.lbem_fields(h, E_h, B_h)
            lbem.lbem_traces(h, tr_h)
            lbem.lbem_diagnostics(h)

        e2e_pass()  # warm-up: the library's host staging buffer is allocated on the first host-buffer call
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reps = max(1, min(args.steps, 2))
        for _ in range(reps):
            e2e_pass()
        dt = (time.perf_counter() - t0) / reps
        dt = dist_max(dt, world)
        nb = lambda t: t.numel() * t.element_size()
        e2e = {"value": world * nsite * nsteps / dt / 1e6, "unit": "Mlups", "host_memory": "pinned",
               "h2d_bytes_per_step": int(nb(eps_h) + p.src_amp.size * 4 + p.src_site.size * 12),
               "d2h_bytes_per_step": int(nb(E_h) + nb(B_h) + nb(tr_h) + 24)}

    forms = None
    if not args.no_forms and args.lb_steps is None and args.workload == "het2d_4096":
        forms = other_forms(lbem, torch, p, peak, stream)
    cpu, acc = None, {}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        if args.workload == "het2d_4096" and args.lb_steps is None:
            # every form's accuracy against the FP64 oracle, on the GPU kernels the form's timed run used
            spl = {k: v.get("steps_per_launch") for k, v in (forms or {}).items()}
            spl[args.storage] = spp
            cases = accuracy_cases(p, spl)
            if forms is None:
                cases = {args.storage: cases[args.storage]}
            gpu_out = {}
            for key, (q, st, sp, _) in cases.items():
                if sp == "batch":
                    gpu_out[key] = gpu_batch_result(lbem, torch, stream, q)
                else:
                    gpu_out[key] = gpu_result(lbem, torch, stream, q, st, sp)
            cpu, acc = oracle_leg(p, cases, gpu_out)
            for key, e in acc.items():
                if forms and key in forms:
                    forms[key]["rel_l2"] = {"E": e[0], "B": e[1], "traces": e[2], "case": cases[key][0].name
                                            if not isinstance(cases[key][0], list) else "4 smallest batch members",
                                            "bar": cases[key][3], "within_bar": max(e) <= cases[key][3]}
        else:
            cpu = cpu_baseline(p)
            cpu["cpu_model"] = cpu_model()
    s.close()
    if rank == 0:
        # per pass: the step launches (plus the edge kernel after each with 2D walls on the tile path), the medium
        # upload's check and write (plus the pole's re-check, and the wall-aware grad ln mu with walls and mu),
        # init, fields, the FP64 diagnostics and its reduction
        launches = args.steps * (step_launches * (2 if walls and p.D == 2 and not (disp or aniso) else 1) + 6 +
                                 (1 if args.storage == "f16" else 0) + (1 if disp else 0) +
                                 (1 if walls and p.mu_r is not None else 0))
        line = {"metric": "Mlups", "value": value, "unit": "Mlups", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32" if args.storage == "f32" else f"f32-math/{args.storage}-storage",
                "data": "synthetic",
                "config": {"workload": p.name, "grid": list(p.shape), "lb_steps": nsteps, "storage": args.storage,
                           "sources": int(p.src_site.size), "receivers": int(p.rec_site.size),
                           "l2": f"inputs larger than L2 (2 x {state_mb:.0f} MB distributions), no flush",
                           "parallelism": "single GPU"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk.summary(), "diagnostics_last": list(diag)}
        main_acc = acc.get(args.storage)
        if main_acc is not None:
            line["accuracy"] = {"E": main_acc[0], "B": main_acc[1], "traces": main_acc[2],
                                "case": "512^2 centre crop x 5000 steps vs FP64 oracle (config 2, reading R11)",
                                "bar": TOL[args.storage], "within_bar": max(main_acc) <= TOL[args.storage]}
        line["forms"] = forms
        # last, so that it survives a truncated tail of the output: one compact entry per form
        summ = {"legend": "[kMlups, frac of measured HBM copy rate at the form's algorithmic bytes per launch, "
                          "steps per launch, rel-L2 E/B/traces vs FP64 oracle on the form's accuracy case, bar]"}

        def entry(mlups, frac, spl_, e, bar):
            r = None if e is None else "/".join(f"{x:.1e}" for x in e)
            verdict = None if e is None else (f"<={bar:g} met" if max(e) <= bar else f"<={bar:g} MISSED")
            return [round(mlups / 1e3, 1), None if frac is None else round(frac, 3), spl_, r, verdict]

        summ[f"{args.storage} (main)"] = entry(value, roofline["frac"], spp, main_acc, TOL[args.storage])
        for k, v in (forms or {}).items():
            if k == "adjoint_192":
                summ[k] = [round(v["mlups_forward_plus_backward"] / 1e3, 1), round(v["backward_frac"], 3), 1,
                           "vs FD and oracle adjoint in tests", None]
                continue
            e = acc.get(k)
            bar = TOL.get(k, TOL["f32"])
            summ[k] = entry(v["mlups"], v.get("frac"), v.get("steps_per_launch"), e, bar)
        line["forms_summary"] = summ
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
