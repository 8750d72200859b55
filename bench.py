"""Benchmark: MBIR slice-iterations per second on the full synthetic volume.

Workload (one GPU): 1024 slices of 2048 x 2048, 128 angles over [0, pi),
2896 detector bins, kernel width 7, oversampling 2; Poisson data at I0 = 1e4
from analytic ellipsoid line integrals (pixel size 1/N); weights = counts/I0;
26-neighbour qGGMRF prior (p = 1.2, sigma = 1/0.7, c = 1e-4).  One step is one
accelerated-gradient iteration over the whole resident volume: A, residual,
A^T, prior, FP64 reductions and the update.  Inputs (17 GB per volume array)
are far larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N --steps K --warmup W]      # CUDA path
  python bench.py --impl reference ...                  # FP64 oracle on host cores

Prints one JSON line (rank 0).  Under torchrun each rank solves its own
replica volume (no collective on the data path; weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MBIR slice-iter/s 2048²×128ang batched vs plain (err≤1e-4); A/Aᵀ HBM frac"
UNIT = "slice-iter/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--angles", type=int, default=128)
    ap.add_argument("--det", type=int, default=2896)
    ap.add_argument("--slices", type=int, default=1024)
    ap.add_argument("--chunk", type=int, default=64, help="slices per launch (plan max_batch)")
    ap.add_argument("--plain-slices", type=int, default=32)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--normal-slices", type=int, default=64,
                    help="slices of the unweighted 1024^2 solve comparing the Toeplitz-plus-Hankel "
                         "normal operator with the gridded operators (0: skip)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--profile-steps", type=int, default=3,
                    help="iterations of the separate per-kernel event pass")
    ap.add_argument("--step", type=float, default=None,
                    help="use this step instead of deriving it (profiling runs skip the power iteration)")
    ap.add_argument("--power-iter", type=int, default=30,
                    help="power iterations of the library-derived step (first, untimed call)")
    ap.add_argument("--uneven-slices", type=int, default=512,
                    help="slices of the uneven-size batching measurement (0 skips it)")
    ap.add_argument("--cpu-angles", type=int, default=16,
                    help="angles of one slice timed by the oracle for the CPU baseline")
    ap.add_argument("--oracle-configs", action="store_true",
                    help="instead of the headline: time the FP64 oracle's MBIR solve on the host cores and "
                         "the library on the GPU for the single-slice 128^2 and the noisy 16 x 512^2 configurations")
    ap.add_argument("--oracle-iters2", type=int, default=3,
                    help="--oracle-configs: oracle iterations timed on one noisy 512^2 slice (of the 50)")
    ap.add_argument("--workload", default=None,
                    choices=["volume_2048x1024", "tb25_shape", "tb86_shape"],
                    help="set n, angles, det and slices from a named synthetic workload")
    args = ap.parse_args()
    if args.workload:
        from paper_2304_12934_gb300 import synth
        wl = synth.WORKLOADS[args.workload]
        args.n, args.angles, args.det, args.slices = wl.n, wl.n_angles, wl.n_det, wl.slices
    return args


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float, device=None) -> float:
    """Largest value over all ranks (the job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(rank: int) -> int:
    """Each rank solves its own replica volume, seeded by its rank."""
    from paper_2304_12934_gb300 import synth
    return synth.BASE_SEED + 1000 * rank


# ------------------------------------------------------------- clocks ------
class ClockSampler:
    """nvidia-smi SM clock / throttle-reason samples during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                      "--format=csv,noheader,nounits"], capture_output=True,
                                     text=True, timeout=5).stdout.strip()
                if out:
                    self.samples.append([v.strip() for v in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self._t:
            self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if len(s) > 3 + i and s[3 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


# ------------------------------------------------------ roofline bytes -----
def algorithmic_bytes(name, N, A, D, w, B):
    """Compulsory HBM bytes of one launch over B slices: each kernel's inputs
    read once and outputs written once (tables and L2-resident vectors not
    counted)."""
    R = N + w  # grid rows touched by the half-plane polar points (jmin..jmax)
    Mh = D // 2 + 1
    AM = A * Mh
    img, sino = 4 * N * N, 4 * A * D
    grid_rows = 8 * R * N
    part = 8 * w * AM
    per = {
        "k_fwd_col": img + grid_rows,
        "k_fwd_row": grid_rows + part,
        "k_fwd_det": part + 3 * sino,
        "k_adj_det": sino + 8 * AM,
        "k_adj_row": 8 * AM + grid_rows,
        "k_adj_col": grid_rows + img,
        "k_prior": 4 * img,  # f, g read + g written, and x_prev for the fused restart dots
        # the solver's fused form: f, g, x_prev read; x_{k+1} and the momentum point written
        "k_prior_next": 5 * img,
        "k_dots_gzx_gg": 3 * img,
        "k_update": 5 * img,  # solver without a prior: x, z, g read; x_{k+1} and z_{k+1} written
        # normal operator A^T A (Toeplitz-plus-Hankel embedding): half-plane rows ky = 0..N
        "k_nrm_col_fwd": img + 8 * (N + 1) * N,
        "k_nrm_row": 2 * 8 * (N + 1) * N,
        "k_nrm_col_adj": 8 * (N + 1) * N + 2 * img,  # rows in; gradient out, A^T b in
    }
    return per.get(name, 0) * B


def prior_roofline(api, dev, name, N, units, dims, avg_s, hbm, timing):
    """The prior kernel's roof is the special-function unit, not HBM: every
    unordered neighbour pair costs one lg2, one ex2 and one rcp per cell
    (13 pairs per voxel with 26 neighbours, 4 with 8), and 20 bytes per voxel
    would stream in a third of that time.  The unit's rates are measured here
    (tc_sfu_throughput); the peak is the pair rate they allow,
    1 / (1/r_lg2 + 1/r_ex2 + 1/r_rcp).  The HBM view is kept beside it."""
    r = {op: api.sfu_throughput(op, dev) for op in ("lg2", "ex2", "rcp")}
    peak = 1.0 / sum(1.0 / v for v in r.values())
    pairs = (13 if dims == 3 else 4) * N * N * units
    ach = pairs / avg_s
    return {"bound": "alu", "kernel": name, "achieved": round(ach / 1e9, 1), "peak": round(peak / 1e9, 1),
            "unit": "Gpair/s", "frac": round(ach / peak, 4), "traffic": hbm["traffic"],
            "pairs_per_launch": pairs,
            "peak_kind": ("special-function unit, measured in this run (lane-ops/s: "
                          + ", ".join(f"{k} {v:.3e}" for k, v in r.items())
                          + "); one lg2, ex2 and rcp per unordered pair and cell"),
            "timing": timing,
            "hbm": {"achieved": hbm["achieved"], "peak": hbm["peak"], "unit": "GB/s", "frac": hbm["frac"],
                    "alg_bytes_per_launch": hbm["alg_bytes_per_launch"], "peak_kind": hbm["peak_kind"]}}


def launch_units(name, B_total, chunk):
    """Slices processed by one launch of each kernel."""
    if name in ("k_prior", "k_prior_next", "k_dots_gzx_gg", "k_update", "k_restart_fixup"):
        return B_total
    return chunk


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_sources_sha256(files):
    """sha256 over the concatenated source files that define a kernel."""
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2304_12934_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def traffic_for(name, units):
    """DRAM bytes of one launch of `name` over `units` slices, from the committed
    ncu counters (bytes per slice), or None when one of the kernel's source
    files changed since those counters were taken."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(path) as fh:
            ent = json.load(fh)["kernels"][name]
        if kernel_sources_sha256(ent["source_files"]) != ent["source_sha256"]:
            return None
        return int(ent["bytes_per_slice"] * units)
    except Exception:
        return None


# ------------------------------------------------------------ CPU oracle ---
def oracle_slice_iter_seconds(N, A, D, n_ang_sample):
    """Time the FP64 oracle (as it stands) on a bounded sample: A and A^T of one
    N x N slice restricted to n_ang_sample angles, plus the 26-neighbour prior
    on a 3-slice stack; scaled to one slice-iteration over all A angles."""
    import numpy as np
    import oracle
    from paper_2304_12934_gb300 import synth
    oracle.build()
    th = oracle.default_angles(A)[:: max(1, A // n_ang_sample)][:n_ang_sample]
    f = synth.rasterize(N, synth.random_ellipses(N, synth.BASE_SEED, scale=1.0 / N))
    t0 = time.perf_counter()
    y = oracle.radon_fwd(f, th.shape[0], D, th)
    t1 = time.perf_counter()
    oracle.radon_adj(y, N, th)
    t2 = time.perf_counter()
    vol = np.stack([f, f, f])
    oracle.prior_value_grad(vol, 3)
    t3 = time.perf_counter()
    scale = A / th.shape[0]
    per_slice = (t1 - t0) * scale + (t2 - t1) * scale + (t3 - t2) / 3.0
    return per_slice, dict(fwd_s=t1 - t0, adj_s=t2 - t1, prior_s=t3 - t2, angles=int(th.shape[0]))


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    N, A, D = args.n, args.angles, args.det
    nang = max(1, min(args.cpu_angles // 4, A))
    cores = os.cpu_count()
    times, walls = [], []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        per_slice, info = oracle_slice_iter_seconds(N, A, D, nang)
        if i >= args.warmup:
            times.append(per_slice)
            walls.append(time.perf_counter() - t0)
    per_slice = statistics.mean(times)
    value = 1.0 / per_slice
    sample = (f"per step: oracle A and A^T of one {N}x{N} slice over {nang} of {A} angles "
              f"(D={D}) plus the 26-neighbour prior on 3 slices (ms_per_step is that sample's "
              f"wall time); value scales it to one slice-iteration over all {A} angles")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.mean(walls) * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"volume {N}x{N}x{args.slices}, {A} angles, {D} bins (sampled)",
                       "n": N, "angles": A, "det": D},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------- oracle against library timings ---
def oracle_configs(args):
    """FP64 oracle MBIR on the host cores next to the library on the GPU.

    Single slice: 128^2 random-ellipse phantom, 90 angles, 184 bins, noise-free
    b = A x_true with W = I, 8-neighbour prior, 20 iterations; the oracle runs
    all of them (and its power iteration for the step) and the library runs
    the same solve with the oracle's step.  Noisy: 16 slices of 512^2, 180
    angles, 724 bins, Poisson data at I0 = 1e4 with count weights, 50
    iterations; the library runs all 16 slices, the oracle one slice for
    --oracle-iters2 iterations (its per-iteration cost is constant), and the
    library's iterate of that slice after as many iterations is compared."""
    import numpy as np
    import torch
    import oracle
    from paper_2304_12934_gb300 import api, synth
    oracle.build()
    api.load()
    dev = torch.device("cuda:0")
    lam = 1e-2
    out = {"mode": "oracle_configs", "cores": os.cpu_count()}

    def gpu_solve(plan, b, w, iters, step, prior, reps=3):
        ts = []
        for _ in range(reps):
            x = torch.zeros((b.shape[0], plan.n, plan.n), device=dev)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = api.mbir_solve(plan, b, w, x, iters, step, prior)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        return x, st, min(ts)

    # ---- single slice, noise-free, 20 iterations
    N, A, D, it1 = 128, 90, 184, 20
    ells = synth.random_ellipses(N, synth.BASE_SEED, scale=1.0 / N)
    f = synth.rasterize(N, ells)[None]
    t0 = time.perf_counter()
    b = oracle.radon_fwd(f[0], A, D)[None]
    w = np.ones_like(b)
    lam_max = oracle.power_norm(N, A, D, None, synth.random_start((1, N, N), synth.BASE_SEED + 1), 30)
    step = 1.0 / (1.05 * lam_max + lam * oracle.prior_lipschitz(**oracle.PAPER_PRIOR))
    t1 = time.perf_counter()
    xo = oracle.mbir_solve(b, w, N, it1, step, lam=lam, prior=oracle.PAPER_PRIOR, dims=2)
    t2 = time.perf_counter()
    prior = api.Prior(lam=lam, dims=2)
    with api.Plan(N, A, D, max_batch=1, device=dev) as plan:
        bt = torch.tensor(b, dtype=torch.float32, device=dev)
        wt = torch.tensor(w, dtype=torch.float32, device=dev)
        xg, st, tg = gpu_solve(plan, bt, wt, it1, step, prior)
    err = float(np.linalg.norm(xg.cpu().double().numpy() - xo) / np.linalg.norm(xo))
    out["single_128"] = {"workload": f"1 slice {N}^2, {A} angles, {D} bins, noise-free, W = I, 8-nbr prior, "
                                     f"{it1} iterations", "oracle_data_and_step_s": round(t1 - t0, 3),
                         "oracle_solve_s": round(t2 - t1, 3), "gpu_solve_s": round(tg, 5),
                         "speedup": round((t2 - t1) / tg, 1), "rel_l2_gpu_vs_oracle": err}
    print(json.dumps(out), flush=True)

    # ---- noisy, 16 slices of 512^2, 50 iterations
    N, A, D, B, it2 = 512, 180, 724, 16, 50
    th = oracle.default_angles(A)
    _, ells = synth.phantom_slices(N, B, scale=1.0 / N, seed0=synth.BASE_SEED + 512)
    p = np.stack([synth.ellipse_line_integrals(e, th, D) for e in ells])
    b, w = synth.poisson_measurement(p, 1e4, synth.BASE_SEED + 513)
    prior = api.Prior(lam=lam, dims=2)
    with api.Plan(N, A, D, max_batch=B, device=dev) as plan:
        bt = torch.tensor(b, dtype=torch.float32, device=dev)
        wt = torch.tensor(w, dtype=torch.float32, device=dev)
        x = torch.zeros((B, N, N), device=dev)
        st = api.mbir_solve(plan, bt, wt, x, 0, None, prior)   # the library derives the step
        torch.cuda.synchronize()
        step = st.step
        _, st, tg = gpu_solve(plan, bt, wt, it2, step, prior)
    k = max(1, args.oracle_iters2)
    b0, w0 = b[:1].astype(np.float32).astype(np.float64), w[:1].astype(np.float32).astype(np.float64)
    t0 = time.perf_counter()
    xo = oracle.mbir_solve(b0, w0, N, k, step, lam=lam, prior=oracle.PAPER_PRIOR, dims=2)
    to = time.perf_counter() - t0
    with api.Plan(N, A, D, max_batch=1, device=dev) as plan:
        xk, _, _ = gpu_solve(plan, torch.tensor(b0, dtype=torch.float32, device=dev),
                             torch.tensor(w0, dtype=torch.float32, device=dev), k, step, prior, reps=1)
    err = float(np.linalg.norm(xk.cpu().double().numpy() - xo) / np.linalg.norm(xo))
    per_it = to / k
    out["noisy_512x16"] = {"workload": f"{B} slices {N}^2, {A} angles, {D} bins, Poisson I0=1e4, count weights, "
                                       f"8-nbr prior, {it2} iterations",
                           "gpu_solve_s": round(tg, 4), "gpu_slice_iter_s": round(B * it2 / tg, 1),
                           "oracle_sample": f"1 slice, {k} of {it2} iterations, step from the library",
                           "oracle_s": round(to, 2), "oracle_s_per_slice_iter": round(per_it, 3),
                           "oracle_slice_iter_s": round(1.0 / per_it, 5),
                           "oracle_full_run_s_projected": round(per_it * B * it2, 1),
                           "speedup": round(per_it * B * it2 / tg, 1),
                           "rel_l2_gpu_vs_oracle_slice0": err}
    print(json.dumps(out), flush=True)


# ------------------------------------------------- uneven-size batching ---
def uneven_batch(api, synth, dev, n_slices, reps=3):
    """Gradient evaluations (A, A^T, 8-neighbour prior) of n_slices slices of
    uneven side (256..2048) and angle count (64..256), seeded: per geometry
    one plan over all its slices, the whole batch captured in one CUDA graph;
    against the plain form, one slice per launch through plans of one slice."""
    import numpy as np
    import torch
    rng = np.random.default_rng(synth.BASE_SEED + 3)
    sides = rng.choice([256, 512, 1024, 2048], n_slices)
    angs = rng.choice([64, 128, 256], n_slices)
    groups = sorted(set(zip(sides.tolist(), angs.tolist())))
    prior = api.Prior(lam=1e-2, dims=2)
    bufs = []
    for n, a in groups:
        cnt = int(np.sum((sides == n) & (angs == a)))
        d = synth.det_for(n)
        g = torch.Generator(device=dev)
        g.manual_seed(n * 1000 + a)
        x = torch.rand((cnt, n, n), device=dev, generator=g)
        b = torch.rand((cnt, a, d), device=dev, generator=g)
        w = torch.rand((cnt, a, d), device=dev, generator=g)
        bufs.append(dict(n=n, a=a, d=d, cnt=cnt, x=x, b=b, w=w, grad=torch.empty_like(x),
                         obj=torch.zeros(2, dtype=torch.float64, device=dev),
                         pb=api.Plan(n, a, d, max_batch=min(cnt, 64), device=dev),
                         p1=api.Plan(n, a, d, max_batch=1, device=dev)))

    def batched():
        for q in bufs:
            api.mbir_grad(q["pb"], q["x"], q["b"], q["w"], prior, grad=q["grad"], obj=q["obj"])

    def plain():
        for q in bufs:
            for k in range(q["cnt"]):
                api.mbir_grad(q["p1"], q["x"][k:k + 1], q["b"][k:k + 1], q["w"][k:k + 1], prior,
                              grad=q["grad"][k:k + 1], obj=q["obj"])

    # the same batch as one plan group: one launch per stage and geometry class
    # over the work list of its (geometry, slice, tile) items, one CTA per item,
    # the call captured in a graph
    grp = api.PlanGroup([(q["n"], q["a"], q["d"]) for q in bufs], [q["cnt"] for q in bufs], device=dev)
    gx = torch.cat([q["x"].flatten() for q in bufs])
    gb = torch.cat([q["b"].flatten() for q in bufs])
    gw = torch.cat([q["w"].flatten() for q in bufs])
    ggrad = torch.empty_like(gx)
    gobj = torch.zeros((len(bufs), 2), dtype=torch.float64, device=dev)

    def grouped():
        api.mbir_grad_group(grp, gx, gb, gw, prior, grad=ggrad, obj=gobj)

    stream = torch.cuda.current_stream(dev)
    batched()
    grouped()
    torch.cuda.synchronize()
    ref = torch.cat([q["grad"].flatten() for q in bufs])
    rel_grouped = float((ggrad - ref).norm() / ref.norm())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        batched()
    ggraph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(ggraph):
        grouped()
    res = {}
    for name, fn in (("graph", graph.replay), ("grouped", ggraph.replay), ("plain", plain)):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        res[name] = n_slices * reps / (e0.elapsed_time(e1) / 1e3)
    for q in bufs:
        q["pb"].close()
        q["p1"].close()
    grp.close()
    return {"metric": "slice-gradients/s (A, A^T, 8-neighbour prior)", "slices": n_slices,
            "geometries": len(groups), "plan_group": round(res["grouped"], 1),
            "graph_batched": round(res["graph"], 1),
            "plain_one_slice_per_launch": round(res["plain"], 1),
            "speedup": round(res["graph"] / res["plain"], 3),
            "speedup_grouped_vs_plain": round(res["grouped"] / res["plain"], 3),
            "grouped_vs_per_plan_rel_l2": rel_grouped,
            "sizes": "sides {256,512,1024,2048}, angles {64,128,256}, D = 2 round(N/sqrt 2), seeded"}


def normal_operator(api, synth, dev, n_slices, iters=3):
    """Unweighted MBIR (noise-free analytic data, W = I, 26-neighbour prior) on
    n_slices slices of 1024^2 with 360 angles and 1448 bins: the data term's
    Hessian through the gridded A and A^T against the Toeplitz-plus-Hankel normal
    operator (no gridding).  Both solves start from zero with the same step."""
    import numpy as np
    import torch
    N, A, D = 1024, 360, 1448
    theta = np.arange(A) * (math.pi / A)
    b = synth.ellipsoid_sinogram_torch(N, n_slices, theta, D, dev, scale=1.0 / N, seed=synth.BASE_SEED + 5)
    prior = api.Prior(lam=1e-2, dims=3)
    stream = torch.cuda.current_stream(dev)
    out = {"workload": f"{n_slices} slices of {N}x{N}, {A} angles, {D} bins, noise-free, W = I, "
                       f"26-nbr qGGMRF", "iterations": iters}
    with api.Plan(N, A, D, max_batch=n_slices, device=dev) as plan:
        t0 = time.perf_counter()
        plan.prepare_normal()
        out["prepare_s"] = round(time.perf_counter() - t0, 3)
        x0 = torch.zeros((n_slices, N, N), device=dev)
        st0 = api.SolveState(x0)
        api.mbir_solve(plan, b, None, x0, 0, None, prior, state=st0, power_iter=15)
        step = st0.step
        del st0, x0
        xs, prof = {}, {}
        for mode in (False, True):
            x = torch.zeros((n_slices, N, N), device=dev)
            st = api.SolveState(x)
            api.mbir_solve(plan, b, None, x, 1, step, prior, state=st, normal=mode)
            torch.cuda.synchronize()
            api.profile_enable(True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            api.mbir_solve(plan, b, None, x, iters, step, prior, state=st, normal=mode)
            e1.record(stream)
            torch.cuda.synchronize()
            prof[mode] = api.profile_collect()
            api.profile_enable(False)
            out["normal_slice_iter_s" if mode else "gridded_slice_iter_s"] = round(
                n_slices * iters / (e0.elapsed_time(e1) / 1e3), 1)
            xs[mode] = x
        out["speedup"] = round(out["normal_slice_iter_s"] / out["gridded_slice_iter_s"], 3)
        out["rel_diff_x"] = float((xs[True] - xs[False]).norm() / xs[False].norm().clamp(min=1e-30))
        out["kernels_normal"] = {k: {"launches": c, "ms_per_launch": round(m / c, 4),
                                     "gbs_alg": round(algorithmic_bytes(k, N, A, D, plan.kernel_width,
                                                                        n_slices) / (m / c / 1e3) / 1e9, 1)
                                     if k.startswith("k_nrm") else None}
                                 for k, (c, m) in sorted(prof[True].items(), key=lambda kv: -kv[1][1])}
    return out


def normal_vs_gridded_operator(api, plan, x, reps=3):
    """A^T A on one launch of slices of the main workload: gridded A then A^T
    against the Toeplitz-plus-Hankel embedding (device ms per launch)."""
    import torch
    stream = torch.cuda.current_stream(x.device)
    t0 = time.perf_counter()
    plan.prepare_normal()
    prep = time.perf_counter() - t0
    y = api.radon_fwd(plan, x)
    g = api.radon_adj(plan, y)
    nx = api.radon_normal(plan, x)
    torch.cuda.synchronize()
    res = {}
    for name, fn in (("gridded_ms", lambda: api.radon_adj(plan, api.radon_fwd(plan, x, y=y), x=g)),
                     ("normal_ms", lambda: api.radon_normal(plan, x, out=nx))):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        res[name] = round(e0.elapsed_time(e1) / reps, 3)
    res["speedup"] = round(res["gridded_ms"] / res["normal_ms"], 3)
    res["rel_diff"] = float((nx - g).norm() / g.norm().clamp(min=1e-30))
    res["slices"] = x.shape[0]
    res["prepare_s"] = round(prep, 3)
    return res


# ------------------------------------------------------------- CUDA path ---
def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2304_12934_gb300 import api, synth

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    N, A, D, B, MB = args.n, args.angles, args.det, args.slices, min(args.chunk, args.slices)
    theta = np.arange(A) * (math.pi / A)

    # ---- inputs (untimed): replica volume per rank, seeded by rank
    seed = replica_seed(rank)
    p_true = synth.ellipsoid_sinogram_torch(N, B, theta, D, dev, scale=1.0 / N, seed=seed)
    b, wgt = synth.poisson_measurement_torch(p_true, 1e4, seed + 1)
    del p_true
    torch.cuda.empty_cache()
    prior = api.Prior(lam=1e-2, dims=3)
    plan = api.Plan(N, A, D, max_batch=MB, device=dev)

    x = torch.zeros((B, N, N), device=dev)
    st = api.SolveState(x)

    # ---- warm-up; the first call derives the step inside the library (power
    # iteration over the whole volume plus the prior's curvature bound)
    t_step = time.perf_counter()
    if args.step is None:
        api.mbir_solve(plan, b, wgt, x, 0, None, prior, state=st, power_iter=args.power_iter)
        torch.cuda.synchronize()
        step = st.step
    else:
        step = args.step
    t_step = time.perf_counter() - t_step
    api.mbir_solve(plan, b, wgt, x, args.warmup, step, prior, state=st)
    torch.cuda.synchronize()

    # ---- timed region: exactly K iterations, events on the launch stream (the
    # library's per-kernel event profiler is off here)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = api.launch_count()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0.record(stream)
        api.mbir_solve(plan, b, wgt, x, args.steps, step, prior, state=st)
        e1.record(stream)
        torch.cuda.synchronize()
    gpu_launches = api.launch_count() - launches0
    if ws > 1:
        dist.barrier()
    ms = max_over_ranks(e0.elapsed_time(e1), dev)
    ms_per_step = ms / args.steps
    value = ws * B * args.steps / (ms / 1e3)

    # ---- per-kernel split: the same iterations again with every library launch
    # bracketed by CUDA events on its stream (a separate pass, so the events do
    # not perturb the headline)
    prof_steps = max(1, min(args.steps, args.profile_steps))
    api.profile_enable(True)
    p0 = time.perf_counter()
    api.mbir_solve(plan, b, wgt, x, prof_steps, step, prior, state=st)
    torch.cuda.synchronize()
    prof_wall = time.perf_counter() - p0
    prof = api.profile_collect()
    api.profile_enable(False)

    # ---- roofline of the dominant kernel
    peak, peak_kind = measured_peaks()
    dom = max(prof.items(), key=lambda kv: kv[1][1])
    dname, (dcnt, dms) = dom
    units = launch_units(dname, B, MB)
    alg = algorithmic_bytes(dname, N, A, D, plan.kernel_width, units)
    avg_s = dms / dcnt / 1e3
    achieved = alg / avg_s / 1e9
    kernels = {k: {"launches": c, "ms_total": round(m, 3), "share": round(m / sum(v[1] for v in prof.values()), 4),
                   "gbs_alg": round(algorithmic_bytes(k, N, A, D, plan.kernel_width,
                                                      launch_units(k, B, MB)) / (m / c / 1e3) / 1e9, 1)}
               for k, (c, m) in sorted(prof.items(), key=lambda kv: -kv[1][1])}
    timing = (f"CUDA events around each launch, separate pass of {prof_steps} iterations "
              f"({prof_wall:.2f} s) right after the timed region")
    roofline = {"bound": "hbm", "kernel": dname, "achieved": round(achieved, 1), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic_for(dname, units),
                "alg_bytes_per_launch": alg, "peak_kind": f"{peak_kind} hbm_gbs (burst copy)",
                "timing": timing}
    if dname in ("k_prior", "k_prior_next"):
        roofline = prior_roofline(api, dev, dname, N, units, prior.dims, avg_s, roofline, timing)

    # ---- batched vs plain on a subset (same inputs, same iteration)
    plain = None
    if rank == 0 and args.plain_slices > 0:
        S = min(args.plain_slices, B)
        with api.Plan(N, A, D, max_batch=1, device=dev) as p1:
            xs = [torch.zeros((S, N, N), device=dev) for _ in range(2)]
            bs, ws_ = b[:S].contiguous(), wgt[:S].contiguous()
            res = []
            for pl, xx in ((p1, xs[0]), (plan, xs[1])):
                s2 = api.SolveState(xx)
                api.mbir_solve(pl, bs, ws_, xx, 1, step, prior, state=s2)
                torch.cuda.synchronize()
                a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a0.record(stream)
                api.mbir_solve(pl, bs, ws_, xx, 2, step, prior, state=s2)
                a1.record(stream)
                torch.cuda.synchronize()
                res.append(S * 2 / (a0.elapsed_time(a1) / 1e3))
            err = float((xs[0] - xs[1]).norm() / xs[1].norm().clamp(min=1e-30))
            plain = {"plain_slice_iter_s": round(res[0], 2), "batched_slice_iter_s": round(res[1], 2),
                     "slices": S, "rel_err_batched_vs_plain": err,
                     "speedup": round(res[1] / res[0], 3)}
            del xs

    # ---- end to end through the host-buffer entry point (pinned memory)
    e2e = None
    if not args.no_e2e:
        bh = b.cpu().pin_memory()
        wh = wgt.cpu().pin_memory()
        xh = x.cpu().pin_memory()
        devbuf = {"b": b, "w": wgt, "x": x}
        st_e = api.SolveState(x)
        api.mbir_solve_host(plan, bh, wh, xh, 1, step, prior, state=st_e, dev=devbuf)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            api.mbir_solve_host(plan, bh, wh, xh, 1, step, prior, state=st_e, dev=devbuf)
        t_e2e = max_over_ranks(time.perf_counter() - t0, dev)
        e2e = {"value": ws * B * args.steps / t_e2e, "unit": UNIT,
               "h2d_bytes_per_step": int(bh.numel() * 4 + wh.numel() * 4 + xh.numel() * 4),
               "d2h_bytes_per_step": int(xh.numel() * 4),
               "call": "mbir_solve_host(n_iter=1) per step: H2D b, w, x; one iteration; D2H x"}

    # ---- normal operator (Toeplitz-plus-Hankel) against the gridded pair
    normal = None
    if rank == 0 and args.normal_slices > 0:
        normal = {"headline_operator": normal_vs_gridded_operator(api, plan, x[:MB].contiguous()),
                  "unweighted_solve": normal_operator(api, synth, dev, args.normal_slices)}
        torch.cuda.empty_cache()

    # ---- uneven sizes: one CUDA graph over per-geometry batches vs one slice per launch
    uneven = None
    if rank == 0 and args.uneven_slices > 0:
        uneven = uneven_batch(api, synth, dev, args.uneven_slices)

    # ---- CPU oracle baseline (rank 0, N = 1)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        per_slice, info = oracle_slice_iter_seconds(N, A, D, args.cpu_angles)
        cpu = {"value": 1.0 / per_slice, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": (f"oracle A and A^T of one {N}x{N} slice over {info['angles']} of {A} "
                          f"angles (D={D}; {info['fwd_s']:.1f}+{info['adj_s']:.1f} s) plus the "
                          f"26-neighbour prior on 3 slices ({info['prior_s']:.1f} s), scaled to "
                          f"one slice-iteration over all {A} angles")}

    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32 (FP64 reductions)", "data": "synthetic",
                "config": {"workload": f"volume {N}x{N}x{B}, {A} angles, {D} bins, Poisson I0=1e4, "
                                       f"26-nbr qGGMRF, 1 MBIR iteration per step",
                           "name": args.workload or "custom" if (N, A, D, B) != (2048, 128, 2896, 1024)
                           else "volume_2048x1024",
                           "n": N, "angles": A, "det": D, "slices_per_gpu": B,
                           "slices_per_launch": MB, "kernel_width": plan.kernel_width,
                           "oversample": 2, "l2": f"inputs {4 * N * N * B / 1e9:.1f} GB per volume array >> L2 (129 MB); no flush",
                           "parallelism": f"replicas x{ws}"},
                "roofline": roofline, "kernels": kernels, "batched_vs_plain": plain,
                "e2e": e2e, "cpu_baseline": cpu, "gpu_launches": int(gpu_launches),
                "uneven_batch": uneven, "normal_operator": normal,
                "clocks": clk.summary(), "solver": {"step": step, "restarts": st.n_restarts,
                                                    "obj": list(st.obj),
                                                    "step_derivation_s": round(t_step, 2)}}
        print(json.dumps(line), flush=True)
    plan.close()
    if ws > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.oracle_configs:
        oracle_configs(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
