#!/usr/bin/env python
"""Benchmark of the batched heat-kernel Sinkhorn on a 720 x 1440 Gauss-Legendre grid.

One step = one iteration of Algorithm 1 (u-step, v-step, gauge) for every problem of
the batch, with the marginal check every C = 10 iterations, inside one
shot_divergence call (8 measure pairs -> 24 OT problems -> 48 heat convolutions of
all 24 fields per iteration), followed by the final objective and S of every pair.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16x3|tf32x3|fp32]
                    [--impl ours|reference]

The headline is --precision (default: the split form that meets the 1e-4 accuracy bar at
this shape); the same run times the other precisions on the same fields ("forms"), and the
cpu_baseline leg runs the FP64 oracle on a bounded sample (one pair, 20 iterations) that is
also the reference of every precision's accuracy on that sample ("accuracy"); the split
form's speedup over FP32 is stated only when it meets its bar.

--impl reference times the FP64 CPU oracle on the host cores (the only other place this
file runs oracle code besides the cpu_baseline leg).  --gpus N without a torchrun
environment starts N ranks itself.  Prints one JSON line on rank 0.
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
    ap.add_argument("--precision", default="tf32x3", choices=["bf16x3", "tf32x3", "fp32"])
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


def algorithmic_work(kind, nlat, npix, lmax, nfields, legendre="table"):
    """(bytes, flops) one launch of a kernel kind must move / compute at minimum.

    npix nodes per field, nh = ceil(nlat/2) ring pairs, T = (lmax+1)(lmax+2)/2 degrees
    and orders; the folded table holds T*nh entries (4 B in FP32 and TF32x3, 2+2 B as bf16
    hi/lo), read once per launch in every precision.  In recurrence mode the TF32x3 kernels
    read the checkpoints instead (4 FP32 values per 16 degrees and node: T*nh/4 entries).
    """
    n = npix
    nh = (nlat + 1) // 2
    L = lmax + 1
    T = L * (L + 1) // 2
    field = nfields * n * 4.0                     # one FP32 field batch
    spec = 2 * L * nh * 2 * nfields * 4.0         # folded ring spectra X or Y (FP32)
    coef = T * 2 * nfields * 4.0                  # coefficients (FP32, or bf16 hi+lo)
    table = T * nh * 4.0 if legendre == "table" else T * nh * 4.0 / 4
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


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) from ncu captures of
# this file's 720 x 1440, 24-field TF32x3 runs of the kernels as they are (profiles/
# ncu_k_idft_720x1440.md, ncu_k_legendre_tf32_720x1440.md); valid only for that workload and those
# kernels.  The update kernel stores the scaling in 2 of a block's 20 half-steps.  Forms whose
# kernels changed since their last capture (BF16x3, the recurrence mode) report null.
NCU_TRAFFIC = {("inverse_dft_epilogue", "*", "*"): (18 * 223.2e6 + 2 * 313.5e6) / 20,   # same kernel in every form
               ("legendre_analysis", "tf32x3", "table"): 524.6e6, ("legendre_synthesis", "tf32x3", "table"): 611.5e6}


def roofline(kind, avg_ms, nlat, npix, lmax, nfields, prec, legendre="table"):
    by, fl = algorithmic_work(kind, nlat, npix, lmax, nfields, legendre)
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
    traffic = (NCU_TRAFFIC.get((kind, prec, legendre), NCU_TRAFFIC.get((kind, "*", "*")))
               if (nlat, npix, nfields) == (720, 720 * 1440, 24) else None)
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


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the baseline lines."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu part")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def blas_threads():
    """Threads numpy's BLAS runs on (the oracle's only parallelism)."""
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        if os.environ.get(k, "").isdigit():
            return int(os.environ[k])
    return os.cpu_count()


def oracle_batch(args, og, nprob):
    """The first nprob problems of the workload's batch [(p,q)] + [(p,p)] + [(q,q)] (FP64)."""
    p, q = bench_fields(args, oracle_nodes(og), PAIRS, SEED)
    P = np.concatenate([p, p, q]).astype(np.float64)[:nprob]
    Q = np.concatenate([q, p, q]).astype(np.float64)[:nprob]
    return P, Q


def run_reference(args):
    """The FP64 oracle as it stands, on the host cores: W warm-up steps, then K timed steps,
    each one Alg. 1 iteration of the workload's batch (all 24 problems when K such steps fit
    in about two minutes, else the largest leading subset that does; the line states it)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import sinkhorn as sk
    og = oracle_grid(args)
    og.pbar()
    nprob = 3 * PAIRS
    # size the sample from one iteration of one problem
    P1, Q1 = oracle_batch(args, og, 1)
    t0 = time.perf_counter()
    sk.sinkhorn(og, P1, Q1, EPS, args.tau, T=1, C=0)
    per_problem = time.perf_counter() - t0
    nsub = int(max(1, min(nprob, 120.0 / max(1e-9, per_problem * max(1, args.steps)))))
    P, Q = oracle_batch(args, og, nsub)
    for _ in range(args.warmup):
        sk.sinkhorn(og, P, Q, EPS, args.tau, T=1, C=0)
    # one sinkhorn call per step (a fresh T = 1 call iterates from u = v = 1: same work per step)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sk.sinkhorn(og, P, Q, EPS, args.tau, T=1, C=0)
    dt = time.perf_counter() - t0
    frac = nsub / nprob                      # share of one batch iteration per step
    value = args.steps * frac / dt
    cores = blas_threads()
    sample = (f"each step = 1 Alg. 1 iteration of {nsub} of the {nprob} problems of the batch "
              f"(numpy FP64, BLAS threads = {cores}, {cpu_model()}); value = batch iterations/s "
              f"= steps x {nsub}/{nprob} / time; grid and table set-up excluded")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config(args, *grid_dims(args)[:2]),
            "cpu_baseline": {"kind": "oracle", "cores": cores, "cpu_model": cpu_model(), "value": value,
                             "unit": "iters/s", "sample": sample},
            "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def make_grid(shot, args, prec, mode):
    if args.quadrature == "healpix":
        return shot.shot_grid_init_healpix(args.nside, -1, prec, mode)
    quad = shot.SHOT_QUAD_GAUSS_LEGENDRE if args.quadrature == "gl" else shot.SHOT_QUAD_CLENSHAW_CURTIS
    return shot.shot_grid_init_quad(quad, args.nlat, 2 * args.nlat, -1, prec, mode)


# the timed and accuracy-checked forms: (precision of the Legendre contractions, Legendre mode)
FORMS = {"fp32": ("fp32", "table"), "tf32x3": ("tf32x3", "table"), "tf32x3_rec": ("tf32x3", "recurrence"),
         "bf16x3": ("bf16x3", "table")}
TARGET = {"fp32": 1e-5, "tf32x3": 1e-4, "tf32x3_rec": 1e-4, "bf16x3": 1e-4}
ACC_ITERS = 20   # iterations of the accuracy sample (one pair, the oracle's bounded sample)


def prec_code(shot, prec):
    return {"fp32": shot.SHOT_FP32, "bf16x3": shot.SHOT_BF16X3, "tf32x3": shot.SHOT_TF32X3}[prec]


def mode_code(shot, legendre):
    return shot.SHOT_TABLE if legendre == "table" else shot.SHOT_RECURRENCE


def form_name(precision, legendre):
    return precision + ("_rec" if legendre == "recurrence" else "")


def form_grid(shot, args, form):
    prec, leg = FORMS[form]
    return make_grid(shot, args, prec_code(shot, prec), mode_code(shot, leg))


def time_form(args, shot, torch, form, pt, qt):
    """Another form on the same fields and steps (graph path, CUDA events): iters/s."""
    g = form_grid(shot, args, form)
    shot.shot_grid_reserve(g, 3 * PAIRS)
    u3 = torch.empty((3 * PAIRS,) + tuple(pt.shape[1:]), device="cuda")
    v3 = torch.empty_like(u3)
    kw = dict(tau=args.tau, tol=0.0, check_every=CHECK_EVERY, u3=u3, v3=v3)
    shot.shot_divergence(g, pt, qt, EPS, max_iter=args.warmup, **kw)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    shot.shot_divergence(g, pt, qt, EPS, max_iter=args.steps, **kw)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    shot.shot_grid_free(g)
    return {"value": args.steps / (ms / 1e3), "unit": "iters/s", "ms_per_step": ms / args.steps}


def accuracy_sample_gpu(args, shot, torch, p, q):
    """Every form on the accuracy sample: the first pair of the batch (3 problems),
    ACC_ITERS iterations; returns S, S_dual, OT and the scalings per form (host)."""
    out = {}
    pt = torch.from_numpy(np.ascontiguousarray(p[:1])).cuda()
    qt = torch.from_numpy(np.ascontiguousarray(q[:1])).cuda()
    for prec in FORMS:
        g = form_grid(shot, args, prec)
        u3 = torch.empty((3,) + tuple(pt.shape[1:]), device="cuda")
        v3 = torch.empty_like(u3)
        rc, r = shot.shot_divergence(g, pt, qt, EPS, args.tau, max_iter=ACC_ITERS, tol=0.0, check_every=CHECK_EVERY,
                                     u3=u3, v3=v3)
        r["rc"] = int(rc)
        r["u"] = u3.cpu().numpy().astype(np.float64)
        r["v"] = v3.cpu().numpy().astype(np.float64)
        shot.shot_grid_free(g)
        out[prec] = r
    return out


def cpu_baseline(args, gpu_sample):
    """The oracle on a bounded sample (~10-30 s on the host cores): ACC_ITERS Alg. 1 iterations
    of the first pair of the batch (3 of its 24 problems), timed; the same oracle run is the
    reference of the per-precision accuracy of that sample (the GPU's results for it come in
    gpu_sample).  Returns (cpu_baseline, accuracy)."""
    from oracle import sinkhorn as sk
    from oracle import sht as osht
    og = oracle_grid(args)
    og.pbar()
    p, q = bench_fields(args, oracle_nodes(og), 1, SEED)
    p64, q64 = p.astype(np.float64), q.astype(np.float64)
    t0 = time.perf_counter()
    ref = sk.divergence(og, p64, q64, EPS, args.tau, T=ACC_ITERS, C=CHECK_EVERY)
    dt = time.perf_counter() - t0
    nprob = 3 * PAIRS
    base = {"value": ACC_ITERS * (3 / nprob) / dt, "unit": "iters/s", "cores": blas_threads(),
            "cpu_model": cpu_model(), "kind": "oracle",
            "sample": f"{ACC_ITERS} Alg. 1 iterations (with the check every {CHECK_EVERY} and the final "
                      f"objective) of 1 pair = 3 of the {nprob} problems of the batch, on the same grid "
                      f"(FP64 numpy, BLAS threads = {blas_threads()}); value = batch iterations/s = "
                      f"{ACC_ITERS} x 3/{nprob} / time; grid and table set-up excluded", "seconds": dt}
    runs = ref["runs"]
    ot_pq = np.abs(runs["ot"][:1])
    P = np.concatenate([p64, p64, q64])

    def s_rel(a, b):
        return float(np.max(np.abs(np.asarray(a) - b) / np.maximum(np.abs(b), 1e-3 * ot_pq)))

    acc = {"sample": f"pair 0 of the batch (3 problems), {ACC_ITERS} iterations, FP64 oracle of the "
                     f"same run as cpu_baseline",
           "metric": {"S": "|dS| / max(|S|, 1e-3 |OT(p,q)|)",
                      "potentials": "max |d phi~| / max |phi~| (gauge-fixed, App. C.2 phi = eps log u)",
                      "scalings_elementwise": "max |u_gpu / u_ref - 1| over u and v (= max |d phi| / eps)",
                      "marginal_err": "|e_gpu - e_ref| of App. C.3's relative error, e_gpu recomputed "
                                      "by the oracle from the GPU's u, v"},
           "S_ref": float(ref["S"][0]), "S_over_OT": float(abs(ref["S"][0]) / ot_pq[0])}
    rp, rs = sk.gauge_fixed(og, runs["phi"], runs["psi"])
    heat = (lambda f: og.heat_apply(f, EPS / 4.0)) if hasattr(og, "heat_apply") else \
        (lambda f: osht.heat_apply(og, f, EPS / 4.0))
    for prec, r in gpu_sample.items():
        r["u"] = r["u"].reshape(runs["u"].shape)
        r["v"] = r["v"].reshape(runs["v"].shape)
        phi, psi = EPS * np.log(r["u"]), EPS * np.log(r["v"])
        gp, gs = sk.gauge_fixed(og, phi, psi)
        pot = max(float(np.max(np.abs(gp - rp)) / np.max(np.abs(rp))),
                  float(np.max(np.abs(gs - rs)) / np.max(np.abs(rs))))
        elem = max(float(np.max(np.abs(r["u"] / runs["u"] - 1.0))), float(np.max(np.abs(r["v"] / runs["v"] - 1.0))))
        e_gpu = sk.marginal_error(og, r["u"], heat(r["v"]), P)
        marg = float(np.max(np.abs(e_gpu - runs["err"])))
        e = {"S": s_rel(r["S"], ref["S"]), "S_dual": s_rel(r["S_dual"], ref["S_dual"]), "potentials": pot,
             "scalings_elementwise": elem, "marginal_err": marg, "target": TARGET[prec]}
        e["meets_target"] = bool(max(e["S"], e["S_dual"], pot, marg) <= TARGET[prec])
        acc[prec] = e
    return base, acc


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
    any FP32 scaling: App. C.4.)

    Under torchrun the 96 pairs are split across the ranks by the static cost model
    3 nlat^3 T (strong scaling: the whole set is fixed), each rank solves its share in one
    shot_divergence_multi call, and S and status of every pair are gathered on the host."""
    import torch
    from paper_2605_18389_gb300 import shot, inputs
    from paper_2605_18389_gb300 import dist as sd
    ws, rank, local = sd.env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    prec = {"fp32": shot.SHOT_FP32, "bf16x3": shot.SHOT_BF16X3, "tf32x3": shot.SHOT_TF32X3}[args.precision]
    t = 2.5e-3
    eps = 4 * t
    T = 200
    nlats, taus = (64, 96, 128, 180), (0.1, 1.0, 10.0)
    pairs = [(gi, ti, k) for gi in range(len(nlats)) for ti in range(len(taus)) for k in range(8)]
    parts = sd.partition_by_cost([sd.pair_cost(nlats[gi], T) for gi, _, _ in pairs], ws)
    mine = parts[rank]
    grids, sets, set_pairs = {}, [], []
    for gi, nlat in enumerate(nlats):
        for ti, tau in enumerate(taus):
            ks = [i for i in mine if pairs[i][0] == gi and pairs[i][1] == ti]
            if not ks:
                continue
            if gi not in grids:
                grids[gi] = shot.shot_grid_init(nlat, 2 * nlat, -1, prec)
            g = grids[gi]
            x, w, a = shot.shot_grid_nodes(g)
            p, q = inputs.pairs("paper_uniform", 3000 + 10 * gi + ti, 8, x, 2 * nlat, a, masses=True,
                                dtype=np.float32)
            sel = [pairs[i][2] for i in ks]
            sets.append(dict(grid=g, p=torch.from_numpy(np.ascontiguousarray(p[sel])).cuda(),
                             q=torch.from_numpy(np.ascontiguousarray(q[sel])).cuda(), eps=eps, tau=tau))
            set_pairs.append(ks)

    def solve():
        return shot.shot_divergence_multi(sets, max_iter=T, tol=0.0, check_every=10) if sets else (0, [])
    solve()
    torch.cuda.synchronize()
    reps = max(1, args.steps // T)
    clk = ClockSampler(local)
    clk.start()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        rc, outs = solve()
    e1.record(st)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = clk.stop()
    ms = sd.max_over_ranks(e0.elapsed_time(e1) / reps, device="cuda")
    local_res = {}
    for ks, o in zip(set_pairs, outs):
        for j, i in enumerate(ks):
            local_res[i] = (float(o["S"][j]), int(o["status"][j]))
    allres = sd.gather_by_index(local_res, len(pairs))
    rcs = sd.gather_by_index({rank: int(rc)}, ws)
    for g in grids.values():
        shot.shot_grid_free(g)
    if rank == 0:
        S = np.array([r[0] for r in allres])
        stat = np.array([r[1] for r in allres])
        failed = [int(np.sum(stat[[i for i, pr in enumerate(pairs) if pr[:2] == (gi, ti)]] < 0))
                  for gi in range(len(nlats)) for ti in range(len(taus))]
        print(json.dumps({"metric": "multi-grid heat-Sinkhorn iters/s (288 problems on 4 grids, one solve)",
                          "value": T / (ms / 1e3), "unit": "iters/s", "n_gpus": ws, "ms_per_solve": ms,
                          "iterations_per_solve": T, "problem_iters_per_s": 288 * T / (ms / 1e3),
                          "scaling": "strong", "dtype": DTYPE[args.precision], "data": "synthetic",
                          "config": {"workload": "multi: grids 64/96/128/180 (nlon = 2 nlat), tau 0.1/1/10, "
                                                 "masses U[0.5, 2], 8 pairs each, t = 2.5e-3, paper_uniform",
                                     "sharding": f"96 pairs over {ws} rank(s) by cost 3 nlat^3 T (LPT)",
                                     "rank_loads": sd.loads([sd.pair_cost(nlats[gi], T) for gi, _, _ in pairs],
                                                            parts)},
                          "clocks": clocks, "status": {"rc": min(rcs), "S_finite": bool(np.all(np.isfinite(S))),
                                                       "failed_pairs_per_set": failed}}))
    if ws > 1:
        dist.destroy_process_group()
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


def relaunch(n):
    """`--gpus N` without a torchrun environment: start this file again as N ranks, one
    process per GPU (torch.distributed.run on 127.0.0.1); rank 0 prints the line."""
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr", "127.0.0.1", f"--master-port={port}", os.path.abspath(__file__), *sys.argv[1:]]
    return subprocess.run(cmd).returncode


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        return relaunch(args.gpus)
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
    roof = roofline(dom, dom_ms / dom_n, nlat, npix, lmax, 3 * PAIRS, args.precision, args.legendre)
    roof["launches"] = dom_n
    roof["timing"] = ("CUDA events around every launch on the solver's stream, over a second "
                      "pass of the timed K steps")
    share = {k: round(v[0] / sum(x[0] for x in kinds.values()), 4) for k, v in kinds.items()}
    per_kind = {k: {"avg_launch_ms": round(v[0] / v[1], 5), "launches": v[1]} for k, v in kinds.items()}

    head = form_name(args.precision, args.legendre)
    forms = {head: {"value": value, "unit": "iters/s", "ms_per_step": ms / args.steps}}
    if not args.no_compare and ws == 1:
        for f in FORMS:
            if f != head:
                forms[f] = time_form(args, shot, torch, f, pt, qt)
    line = {"metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[args.precision],
            "data": "synthetic",
            "config": config(args, nlat, nlon), "e2e": e2e, "gpu_launches": launches, "clocks": clk,
            "roofline": roof, "kernel_share": share, "kernels": per_kind,
            "status": {"rc": int(rc), "S_finite": bool(np.all(np.isfinite(res["S"])))},
            "forms": forms}
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        sample = accuracy_sample_gpu(args, shot, torch, p, q)
        line["cpu_baseline"], acc = cpu_baseline(args, sample)
        line["accuracy"] = {"vs_oracle": acc}
        # the speedup of a split form over FP32 counts only where the split form meets its bar
        for f in forms:
            if f in acc:
                forms[f]["meets_target"] = acc[f]["meets_target"]
        if "fp32" in forms:
            for f in forms:
                if f != "fp32":
                    forms[f]["speedup_over_fp32"] = forms[f]["value"] / forms["fp32"]["value"]
            if head != "fp32" and head in acc:
                line["split_speedup"] = (forms[head]["value"] / forms["fp32"]["value"]
                                         if acc[head]["meets_target"] else None)
    shot.shot_grid_free(g)
    if rank == 0:
        print(json.dumps(line))
    if pg is not None:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
