#!/usr/bin/env python
"""Benchmark of the batched heat-kernel Sinkhorn on a 720 x 1440 Gauss-Legendre grid.

One step = one iteration of Algorithm 1 (u-step, v-step, gauge) for every problem of
the batch, with the marginal check every C = 10 iterations, inside one
shot_divergence call (8 measure pairs -> 24 OT problems -> 48 heat convolutions of
all 24 fields per iteration), followed by the final objective and S of every pair.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16x3|tf32x3|fp32]
                    [--impl ours|reference]

The headline is the split-precision (BF16x3) form; the same run also times the plain FP32
form on the same fields and reports the speedup and the S agreement between the two
(also for --precision tf32x3, the tf32 hi/lo split at FP32-class accuracy).

--impl reference times the FP64 CPU oracle on the host cores (the only other place this
file runs oracle code besides the cpu_baseline leg).  Prints one JSON line on rank 0.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "heat-Sinkhorn iters/s at 720x1440 GL grid, batched; split-prec vs FP32 at 1e-4"
DTYPE = {"fp32": "f32", "bf16x3": "bf16x3 (bf16 hi/lo products, f32 accumulate; f32 elsewhere)",
         "tf32x3": "tf32x3 (tf32 hi/lo products, f32 accumulate; f32 elsewhere)"}
NLAT, NLON, T_HEAT, PAIRS, CHECK_EVERY = 720, 1440, 1e-4, 8, 10
EPS = 4.0 * T_HEAT
RECIPE = "paper_uniform"
SEED = 5000


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16x3", choices=["bf16x3", "tf32x3", "fp32"])
    ap.add_argument("--workload", default="divergence", choices=["divergence", "multi", "grad"],
                    help="divergence: the headline (720x1440, 24 problems); multi: 4 grids x 3 tau x 8 pairs "
                         "in one shot_divergence_multi solve; grad: shot_divergence_grad at 256x512, 16 pairs")
    ap.add_argument("--no-compare", action="store_true", help="skip the FP32 comparison pass")
    ap.add_argument("--legendre", default="table", choices=["table", "recurrence"])
    ap.add_argument("--tau", type=float, default=math.inf)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--nlat", type=int, default=NLAT, help=argparse.SUPPRESS)
    ap.add_argument("--quadrature", default="gl", choices=["gl", "cc", "healpix"],
                    help="grid (cc: equiangular Clenshaw-Curtis; healpix: HEALPix rings, with --nside); "
                         "the headline line is gl")
    ap.add_argument("--nside", type=int, default=64, help="HEALPix resolution (the paper's climate grid: 64)")
    ap.add_argument("--t", type=float, default=None,
                    help="heat time t = eps/4 (default 1e-4; the climate setting eps = 0.01 is t = 2.5e-3)")
    args = ap.parse_args()
    global T_HEAT, EPS
    if args.t is not None:
        T_HEAT = args.t
        EPS = 4.0 * T_HEAT
    return args


def grid_dims(args):
    """(rings, longest ring, nodes per field) of the benchmarked grid."""
    if args.quadrature == "healpix":
        return 4 * args.nside - 1, 4 * args.nside, 12 * args.nside * args.nside
    return args.nlat, 2 * args.nlat, args.nlat * 2 * args.nlat


def oracle_grid(args):
    if args.quadrature == "healpix":
        from oracle.healpix import HealpixGrid
        return HealpixGrid(args.nside)
    from oracle.grid import Grid
    return Grid(args.nlat, quadrature=args.quadrature)


def oracle_nodes(og):
    """(x, nlon, a_ring) of an oracle GL/CC grid; None for HEALPix (fields drawn per pixel)."""
    return (og.x, og.nlon, og.a_ring) if hasattr(og, "nlon") else None


def bench_fields(args, og_or_nodes, npairs, base_seed, dtype=np.float32):
    """The workload's p, q: U(0,1) per node with unit mass (Sec. 4.1), on the grid's nodes;
    HEALPix fields are flat [pairs, 1, N] (oracle layout)."""
    from paper_2605_18389_gb300 import inputs
    if args.quadrature == "healpix":
        npix = 12 * args.nside * args.nside
        area = 4.0 * np.pi / npix
        def one(seed):
            f = np.random.default_rng(seed).uniform(size=npix)
            return (f / (area * f.sum()))[None]
        p = np.stack([one([base_seed, 2 * i]) for i in range(npairs)]).astype(dtype)
        q = np.stack([one([base_seed, 2 * i + 1]) for i in range(npairs)]).astype(dtype)
        return p, q
    x, nlon, a_ring = og_or_nodes
    return inputs.pairs(RECIPE, base_seed, npairs, x, nlon, a_ring, dtype=dtype)


def config(args, nlat, nlon):
    quad = {"gl": "GL", "cc": "Clenshaw-Curtis", "healpix": "HEALPix"}[args.quadrature]
    shape = (f"nside {args.nside} ({12 * args.nside ** 2} pixels, lmax {3 * args.nside - 1})"
             if args.quadrature == "healpix" else f"{nlat}x{nlon} (lmax {nlat - 1})")
    return {"workload": f"heat-Sinkhorn divergence, {quad} {shape}, t={T_HEAT:g} "
                        f"(eps={EPS:g}), {PAIRS} pairs -> {3 * PAIRS} OT problems, "
                        f"{'balanced' if math.isinf(args.tau) else f'tau={args.tau:g}'}, check every "
                        f"{CHECK_EVERY}",
            "nlat": nlat, "nlon": nlon, "pairs": PAIRS, "problems": 3 * PAIRS, "t": T_HEAT,
            "tau": None if math.isinf(args.tau) else args.tau, "precision": args.precision,
            "legendre": args.legendre, "quadrature": args.quadrature,
            "nside": args.nside if args.quadrature == "healpix" else None,
            "fields": f"{RECIPE} (Sec. 4.1 workload: U(0,1) per node, unit mass), seed {SEED}",
            "l2": "working set > L2 every iteration (fields 2x100 MB, spectra 150 MB, table 0.37 GB)"}


def dist_env():
    from paper_2605_18389_gb300 import dist as sd
    return sd.env()


class ClockSampler:
    """nvidia-smi samples (200 ms) taken while the timed region runs."""
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 10:
                continue
            try:
                sm.append(float(f[2]))
                smax = float(f[3])
                power.append(float(f[4]))
            except ValueError:
                continue
            for nm, val in zip(names, f[6:10]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


def legendre_flops_per_launch(nlat, lmax, nfields):
    """Algorithmic FLOPs of ONE Legendre launch (analysis or synthesis) over nfields
    fields with the hemisphere fold: 2 * (sum over (m,p) blocks of rows) * nh * 2 nfields
    = 2 * T * ceil(nlat/2) * 2 nfields, T = (lmax+1)(lmax+2)/2."""
    T = (lmax + 1) * (lmax + 2) // 2
    nh = (nlat + 1) // 2
    return 2.0 * T * nh * 2 * nfields


def fp32_simt_peak_tflops():
    """152 SMs x 128 FP32 lanes x 2 FLOP (FMA) x 2.070 GHz (max SM clock)."""
    return 152 * 128 * 2 * 2.070e9 / 1e12


def algorithmic_work(kind, nlat, npix, lmax, nfields):
    """(bytes, flops) one launch of a kernel kind must move / compute at minimum.

    npix nodes per field, nh = ceil(nlat/2) ring pairs, T = (lmax+1)(lmax+2)/2 degrees
    and orders; the folded table holds T*nh entries (4 B in FP32 and TF32x3, 2+2 B as bf16
    hi/lo), read once per launch in every precision.
    """
    n = npix
    nh = (nlat + 1) // 2
    L = lmax + 1
    T = L * (L + 1) // 2
    field = nfields * n * 4.0                     # one FP32 field batch
    spec = 2 * L * nh * 2 * nfields * 4.0         # folded ring spectra X or Y (FP32)
    coef = T * 2 * nfields * 4.0                  # coefficients (FP32, or bf16 hi+lo)
    table = T * nh * 4.0
    if kind == "ring_dft":
        return field + spec, 0.0
    if kind == "inverse_dft_epilogue":
        # the fused half-step: Y in, marginal in, spectra X of the new scaling out; the last two
        # of a block's 2C half-steps also store the scaling (averaged over the block)
        return 2 * spec + field + field / CHECK_EVERY, 0.0
    if kind == "check_final":
        # marginal check: Y in, marginal in, u in
        return spec + 2 * field, 0.0
    if kind == "legendre_analysis":
        return table + spec + coef, legendre_flops_per_launch(nlat, lmax, nfields)
    if kind == "legendre_synthesis":
        return table + coef + spec, legendre_flops_per_launch(nlat, lmax, nfields)
    return 0.0, 0.0


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) from ncu --set full
# captures of this file's 720 x 1440, 24-field runs (profiles/ncu_k_idft_720x1440.md,
# ncu_k_legendre_tc_720x1440.md, ncu_k_legendre_tf32_720x1440.md); valid only for that workload,
# precision and the kernels as captured.
NCU_TRAFFIC = {("inverse_dft_epilogue", "bf16x3"): (18 * 227.7e6 + 2 * 311.4e6) / 20,
               ("legendre_analysis", "bf16x3"): 532.7e6, ("legendre_synthesis", "bf16x3"): 521.7e6,
               ("legendre_analysis", "tf32x3"): 528.5e6, ("legendre_synthesis", "tf32x3"): 612.9e6}


def roofline(kind, avg_ms, nlat, npix, lmax, nfields, prec):
    by, fl = algorithmic_work(kind, nlat, npix, lmax, nfields)
    fp32 = prec == "fp32"
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    src = "of measured (MEASURED_PEAKS.json hbm_gbs, burst copy)"
    if hbm is None:
        hbm, src = 6800.0, "of fallback (6.8 TB/s)"
    s = avg_ms / 1e3
    if kind.startswith("legendre") and fp32:
        peak = fp32_simt_peak_tflops()
        ach = fl / s / 1e12
        return {"kernel": kind, "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": None,
                "peak_source": "FP32 FFMA, derived: 152 SMs x 128 lanes x 2 FLOP x 2.070 GHz",
                "algorithmic_per_launch": fl, "avg_launch_ms": avg_ms}
    ach = by / s / 1e9
    traffic = NCU_TRAFFIC.get((kind, prec)) if (nlat, npix, nfields) == (720, 720 * 1440, 24) else None
    out = {"kernel": kind, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
           "traffic": traffic, "peak_source": src, "algorithmic_per_launch": by, "avg_launch_ms": avg_ms}
    if kind.startswith("legendre"):
        bf = peaks.get("bf16_tflops_sustained", 1700.0)
        if prec == "tf32x3":   # dense TF32 runs at half the bf16 rate (nominal 1.1 vs 2.25 PFLOP/s)
            out["tensor"] = {"issued_tflops": 3 * fl / s / 1e12, "peak_tf32_tflops": bf / 2,
                             "frac": 3 * fl / s / 1e12 / (bf / 2),
                             "note": "TF32x3 issues 3 MMAs per product; peak = measured bf16 x 1/2"}
        else:
            out["tensor"] = {"issued_tflops": 3 * fl / s / 1e12, "peak_bf16_tflops": bf,
                             "frac": 3 * fl / s / 1e12 / bf, "note": "BF16x3 issues 3 MMAs per product"}
    return out


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def run_reference(args):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample of the workload."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import sinkhorn as sk
    og = oracle_grid(args)
    og.pbar()
    p, q = bench_fields(args, oracle_nodes(og), 1, SEED)
    p = p.astype(np.float64)
    q = q.astype(np.float64)
    # one step = one Alg. 1 iteration of ONE (p,q) problem (a 1/24 sample of a batch step)
    sk.sinkhorn(og, p, q, EPS, args.tau, T=max(1, args.warmup), C=0)
    t0 = time.perf_counter()
    sk.sinkhorn(og, p, q, EPS, args.tau, T=args.steps, C=0)
    dt = time.perf_counter() - t0
    value = args.steps / dt / (3 * PAIRS)
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config(args, *grid_dims(args)[:2]),
            "cpu_baseline": {"kind": "oracle", "cores": cores, "value": value, "unit": "iters/s",
                             "sample": f"each step = 1 Alg. 1 iteration of 1 of the {3 * PAIRS} problems "
                                       f"(numpy FP64, OpenBLAS on {cores} threads); value = problem-iterations/s "
                                       f"/ {3 * PAIRS}"},
            "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def make_grid(shot, args, prec, mode):
    if args.quadrature == "healpix":
        return shot.shot_grid_init_healpix(args.nside, -1, prec, mode)
    quad = shot.SHOT_QUAD_GAUSS_LEGENDRE if args.quadrature == "gl" else shot.SHOT_QUAD_CLENSHAW_CURTIS
    return shot.shot_grid_init_quad(quad, args.nlat, 2 * args.nlat, -1, prec, mode)


def fp32_compare(args, shot, torch, quad, nlat, nlon, mode, pt, qt, S_split):
    """The plain FP32 form on the same fields and steps (graph path, CUDA events): its
    iters/s, the split form's speedup over it, and the relative S difference."""
    g = make_grid(shot, args, shot.SHOT_FP32, mode)
    shot.shot_grid_reserve(g, 3 * PAIRS)
    u3 = torch.empty((3 * PAIRS,) + tuple(pt.shape[1:]), device="cuda")
    v3 = torch.empty_like(u3)
    kw = dict(tau=args.tau, tol=0.0, check_every=CHECK_EVERY, u3=u3, v3=v3)
    shot.shot_divergence(g, pt, qt, EPS, max_iter=args.warmup, **kw)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    _, res = shot.shot_divergence(g, pt, qt, EPS, max_iter=args.steps, **kw)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    shot.shot_grid_free(g)
    v32 = args.steps / (ms / 1e3)
    S32 = np.asarray(res["S"], dtype=np.float64)
    d = np.abs(np.asarray(S_split, dtype=np.float64) - S32)
    ot_pq = np.abs(np.asarray(res["ot3"], dtype=np.float64)[:PAIRS])
    # S = OT(p,q) - (OT(p,p) + OT(q,q))/2 cancels: the split form's error scales with |OT|,
    # so the difference is also stated relative to |OT(p,q)|
    return {"value": v32, "unit": "iters/s", "ms_per_step": ms / args.steps,
            "split_speedup": None, "S_max_rel_diff": float(np.max(d / np.maximum(np.abs(S32), 1e-300))),
            "S_max_diff_over_OT": float(np.max(d / np.maximum(ot_pq, 1e-300)))}


def cpu_baseline(args, x, w, a_ring):
    """Oracle on a bounded sample (~10-30 s): 2 iterations of the full 24-problem batch."""
    from oracle import sinkhorn as sk
    og = oracle_grid(args)
    og.pbar()
    p, q = bench_fields(args, oracle_nodes(og), PAIRS, SEED)
    P = np.concatenate([p, p, q]).astype(np.float64)
    Q = np.concatenate([q, p, q]).astype(np.float64)
    iters = 2
    t0 = time.perf_counter()
    sk.sinkhorn(og, P, Q, EPS, args.tau, T=iters, C=0)
    dt = time.perf_counter() - t0
    return {"value": iters / dt, "unit": "iters/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{iters} Alg. 1 iterations of the full {3 * PAIRS}-problem batch on the same "
                      f"grid (FP64 numpy, OpenBLAS threads = {os.cpu_count()}); "
                      f"grid/table set-up excluded", "seconds": dt}


def timed_calls(torch, fn, warmup, steps, index):
    """warm-up calls, then `steps` calls between CUDA events on the current stream with the
    clocks sampled meanwhile; returns (ms per call, clocks)."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk = ClockSampler(index)
    clk.start()
    e0.record(st)
    for _ in range(steps):
        fn()
    e1.record(st)
    torch.cuda.synchronize()
    clocks = clk.stop()
    return e0.elapsed_time(e1) / steps, clocks


def run_multi(args):
    """Many pair sets on uneven grids in one solve (shot_divergence_multi): grids 64x128, 96x192,
    128x256, 180x360; tau in {0.1, 1, 10} with masses U[0.5, 2] per field; 8 pairs per
    (grid, tau) -> 96 pairs, 288 OT problems; t = 2.5e-3 (eps = 0.01); the paper's runtime-
    experiment fields (Sec. 4.1: U(0, 1) per node); a fixed number of iterations (no convergence
    stop).  One step = one Alg. 1 iteration of all 288 problems.  (At tau = 10 and mass ratios
    up to 4 the scalings reach e^{+-700}: the solver carries that factor in FP64.  Sharp vMF
    mixtures at this eps spread the potentials by hundreds of eps across the sphere, beyond
    any FP32 scaling: App. C.4.)"""
    import torch
    from paper_2605_18389_gb300 import shot, inputs
    prec = {"fp32": shot.SHOT_FP32, "bf16x3": shot.SHOT_BF16X3, "tf32x3": shot.SHOT_TF32X3}[args.precision]
    t = 2.5e-3
    eps = 4 * t
    T = 200
    grids, sets = [], []
    for gi, nlat in enumerate((64, 96, 128, 180)):
        g = shot.shot_grid_init(nlat, 2 * nlat, -1, prec)
        grids.append(g)
        x, w, a = shot.shot_grid_nodes(g)
        for ti, tau in enumerate((0.1, 1.0, 10.0)):
            p, q = inputs.pairs("paper_uniform", 3000 + 10 * gi + ti, 8, x, 2 * nlat, a, masses=True,
                                dtype=np.float32)
            sets.append(dict(grid=g, p=torch.from_numpy(p).cuda(), q=torch.from_numpy(q).cuda(), eps=eps, tau=tau))
    ms, clocks = timed_calls(torch, lambda: shot.shot_divergence_multi(sets, max_iter=T, tol=0.0, check_every=10),
                             1, max(1, args.steps // T), 0)
    rc, outs = shot.shot_divergence_multi(sets, max_iter=T, tol=0.0, check_every=10)
    for g in grids:
        shot.shot_grid_free(g)
    print(json.dumps({"metric": "multi-grid heat-Sinkhorn iters/s (288 problems on 4 grids, one solve)",
                      "value": T / (ms / 1e3), "unit": "iters/s", "ms_per_solve": ms, "iterations_per_solve": T,
                      "problem_iters_per_s": 288 * T / (ms / 1e3), "dtype": DTYPE[args.precision],
                      "data": "synthetic", "config": {"workload": "multi: grids 64/96/128/180 (nlon = 2 nlat), "
                                                                  "tau 0.1/1/10, masses U[0.5, 2], 8 pairs each, "
                                                                  "t = 2.5e-3, paper_uniform"},
                      "clocks": clocks, "status": {"rc": int(rc), "S_finite": bool(all(np.all(np.isfinite(o["S"]))
                                                                                       for o in outs)),
                                                   "failed_pairs_per_set": [int(np.sum(o["status"] < 0))
                                                                            for o in outs]}}))
    return 0


def run_grad(args):
    """The gradient of the Sinkhorn divergence (shot_divergence_grad, unrolled through T = 400
    iterations with checkpoints every 20) at 256x512 for 16 pairs (48 forward problems),
    t = 1e-3, the paper's runtime-experiment fields (Sec. 4.1)."""
    import torch
    from paper_2605_18389_gb300 import shot, inputs
    prec = {"fp32": shot.SHOT_FP32, "bf16x3": shot.SHOT_BF16X3, "tf32x3": shot.SHOT_TF32X3}[args.precision]
    nlat, T, ck = 256, 400, 20
    g = shot.shot_grid_init(nlat, 2 * nlat, -1, prec)
    x, w, a = shot.shot_grid_nodes(g)
    p, q = inputs.pairs("paper_uniform", 4000, 16, x, 2 * nlat, a, dtype=np.float32)
    pt, qt = torch.from_numpy(p).cuda(), torch.from_numpy(q).cuda()
    res = {}

    def call():
        res["r"] = shot.shot_divergence_grad(g, pt, qt, 4e-3, max_iter=T, checkpoint_every=ck,
                                             mode=shot.SHOT_GRAD_UNROLLED)
    ms, clocks = timed_calls(torch, call, 1, max(1, min(args.steps, 5)), 0)
    rc, r = res["r"]
    ok = bool(np.all(np.isfinite(r["grad"].cpu().numpy())))
    shot.shot_grid_free(g)
    print(json.dumps({"metric": "divergence gradients/s (256x512, 16 pairs, T = 400 unrolled, checkpoints every 20)",
                      "value": 1e3 / ms, "unit": "gradients/s", "ms_per_gradient": ms,
                      "forward_iters_per_s": T / (ms / 1e3), "dtype": DTYPE[args.precision], "data": "synthetic",
                      "config": {"workload": "grad: 256x512 GL, t = 1e-3, 16 pairs -> 48 forward problems, "
                                             "paper_uniform"},
                      "clocks": clocks, "status": {"rc": int(rc), "grad_finite": ok}}))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "multi":
        return run_multi(args)
    if args.workload == "grad":
        return run_grad(args)
    import torch
    from paper_2605_18389_gb300 import shot, inputs
    from paper_2605_18389_gb300 import dist as sd

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    prec = {"fp32": shot.SHOT_FP32, "bf16x3": shot.SHOT_BF16X3, "tf32x3": shot.SHOT_TF32X3}[args.precision]
    nlat, nlon, npix = grid_dims(args)
    mode = shot.SHOT_TABLE if args.legendre == "table" else shot.SHOT_RECURRENCE
    quad = None
    g = make_grid(shot, args, prec, mode)
    x, w, a_ring = shot.shot_grid_nodes(g)
    p, q = bench_fields(args, (x, nlon, a_ring), PAIRS, sd.pair_seed(SEED, rank))
    pt = torch.from_numpy(p).cuda()
    qt = torch.from_numpy(q).cuda()
    u3 = torch.empty((3 * PAIRS,) + tuple(pt.shape[1:]), device="cuda")
    v3 = torch.empty_like(u3)
    shot.shot_grid_reserve(g, 3 * PAIRS)
    kw = dict(tau=args.tau, tol=0.0, check_every=CHECK_EVERY, u3=u3, v3=v3)

    # warm-up (untimed)
    shot.shot_divergence(g, pt, qt, EPS, max_iter=args.warmup, **kw)
    torch.cuda.synchronize()

    def barrier():
        if pg is not None:
            pg.barrier()

    # timed region: device-resident inputs, the solver as a user runs it (CUDA graphs)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    n0 = shot.shot_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    rc, res = shot.shot_divergence(g, pt, qt, EPS, max_iter=args.steps, **kw)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = shot.shot_launch_count() - n0
    barrier()
    clk = clocks.stop()
    ms = sd.max_over_ranks(e0.elapsed_time(e1), device="cuda")
    value = sd.job_throughput(args.steps, ms / 1e3, ws)

    # per-kernel times: the same K steps again with a CUDA event pair around every launch
    # (no graph capture in this pass)
    shot.shot_profile_enable(True)
    shot.shot_divergence(g, pt, qt, EPS, max_iter=args.steps, **kw)
    torch.cuda.synchronize()
    shot.shot_profile_enable(False)
    prof = shot.shot_profile_read()

    # end to end through the public call with host buffers: H2D of p, q inside the region
    ph = torch.from_numpy(p).pin_memory()
    qh = torch.from_numpy(q).pin_memory()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pd = ph.to("cuda", non_blocking=True)
    qd = qh.to("cuda", non_blocking=True)
    rc2, res2 = shot.shot_divergence(g, pd, qd, EPS, max_iter=args.steps, **kw)   # S, status -> host
    torch.cuda.synchronize()
    e2e_s = sd.max_over_ranks(time.perf_counter() - t0, device="cuda")
    e2e = {"value": sd.job_throughput(args.steps, e2e_s, ws), "unit": "iters/s",
           "h2d_bytes_per_step": (p.nbytes + q.nbytes) / args.steps,
           "d2h_bytes_per_step": (res2["S"].nbytes + res2["S_dual"].nbytes + res2["status"].nbytes
                                  + res2["ot3"].nbytes + res2["iters3"].nbytes) / args.steps}

    # roofline of the dominant kernel over the timed region
    kinds = {k: v for k, v in prof.items() if v[1] > 0}
    dom = max(kinds, key=lambda k: kinds[k][0])
    dom_ms, dom_n = kinds[dom]
    lmax = 3 * args.nside - 1 if args.quadrature == "healpix" else nlat - 1
    roof = roofline(dom, dom_ms / dom_n, nlat, npix, lmax, 3 * PAIRS, args.precision)
    roof["launches"] = dom_n
    roof["timing"] = ("CUDA events around every launch on the solver's stream, over a second "
                      "pass of the timed K steps")
    share = {k: round(v[0] / sum(x[0] for x in kinds.values()), 4) for k, v in kinds.items()}
    per_kind = {k: {"avg_launch_ms": round(v[0] / v[1], 5), "launches": v[1]} for k, v in kinds.items()}

    compare = None
    if args.precision != "fp32" and not args.no_compare and ws == 1:
        compare = fp32_compare(args, shot, torch, quad, nlat, nlon, mode, pt, qt, res["S"])
    line = {"metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[args.precision],
            "data": "synthetic",
            "config": config(args, nlat, nlon), "e2e": e2e, "gpu_launches": launches, "clocks": clk,
            "roofline": roof, "kernel_share": share, "kernels": per_kind,
            "status": {"rc": int(rc), "S_finite": bool(np.all(np.isfinite(res["S"])))}}
    if compare is not None:
        compare["split_speedup"] = value / compare["value"]
        line["fp32_compare"] = compare
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline(args, x, w, a_ring)
    shot.shot_grid_free(g)
    if rank == 0:
        print(json.dumps(line))
    if pg is not None:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
