"""Benchmark of the EFGP hot path on GB300.

One step = the whole path on one synthetic problem: bin sort + type-1 spread
+ fine FFT + Toeplitz transform (set-up), the CG solve with the FFT Toeplitz
product, and the type-2 evaluation of the posterior mean at the targets.
Default workload: 2D Matern-3/2, l = 0.05, sigma = 0.5, eps = 1e-3,
N = 10^9 points (float32), 1000^2 grid targets.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank solves its
own independent problem (weak scaling, no collective on the data path);
value = all ranks' points / max-over-ranks time.
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
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthdata  # noqa: E402

METRIC = "points/s end-to-end EFGP at stated mean error; spread/interp GB/s vs HBM peak"
UNIT = "points/s"


CSRC = os.path.join(ROOT, "paper_2210_10210_gb300", "csrc")
KERNEL_NAMES = {"spread": ("spread.cu", "spread_pair_kernel("), "bin_scatter": ("spread.cu", "bin_scatter_big_kernel("),
                "bin_count": ("setup_fused.cu", "fused_count_kernel(")}


def kernel_fingerprint(key):
    """SHA-1 of one kernel's source text (template header or qualifiers to the
    closing brace); DRAM counters recorded for another fingerprint are stale."""
    fname, marker = KERNEL_NAMES[key]
    text = open(os.path.join(CSRC, fname)).read()
    i = text.index(marker)
    start = text.rfind("\n\n", 0, i) + 2
    depth, j = 0, text.index("{", i)
    while j < len(text):
        if text[j] == "{":
            depth += 1
        elif text[j] == "}":
            depth -= 1
            if depth == 0:
                break
        j += 1
    import hashlib
    return hashlib.sha1(text[start:j + 1].encode()).hexdigest()


def traffic_for(kernel, n_points, path):
    """DRAM bytes per launch scaled from an ncu capture, or None when absent or stale."""
    try:
        t = json.load(open(path))["kernels"][kernel]
    except Exception:
        return None
    if t.get("src_sha1") != kernel_fingerprint(kernel):
        return None
    return t["dram_bytes_per_point"] * n_points


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1])]
        mx = [num(r[2]) for r in rows if num(r[2])]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for i, n in enumerate(names):
                if r[5 + i].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def max_over_ranks(x, dist, device):
    """Largest value of x over all ranks (x itself without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(points_per_rank, world, ms_per_step):
    """Whole-job points/s: every rank's points over the slowest rank's step time."""
    return world * points_per_rank / (ms_per_step / 1000.0)


def rank_recipe(name, n, rank):
    """The workload of one rank: same shape, its own seed (independent problems)."""
    rec = synthdata.config(name, n=n)
    rec.seed += 1000 * rank
    return rec


def workload_desc(name, rec, model):
    fam, nu, ell, sigma, eps = model
    kern = "SE" if fam == "se" else f"Matern-{nu:g}"
    tg = f"{rec.n_targets_1d}^{rec.d} grid" if rec.targets == "grid" else f"{rec.n_targets} iid"
    return f"{name}: {rec.d}D {kern} l={ell} sigma={sigma} eps={eps} N={rec.n} targets {tg}"


def n_targets(rec):
    return rec.n_targets_1d ** rec.d if rec.targets == "grid" else rec.n_targets


# ------------------------------------------------------------------ CPU oracle leg
def oracle_sample(name, n_sample, q_sample):
    """The FP64 oracle (direct sums + dense Cholesky + direct evaluation) on a
    bounded sample of the workload: the first n_sample points and q_sample
    targets, same kernel and tolerance (hence the same h and m)."""
    from oracle import efgp_oracle as O
    rec = synthdata.config(name, n=n_sample)
    x, y, z = synthdata.make_np(rec)
    z = z[:q_sample]
    fam, nu, ell, sigma, eps = synthdata.MODELS[name]
    t0 = time.perf_counter()
    O.efgp(x, y, z, O.Kernel(fam, nu, ell), sigma, eps)
    dt = time.perf_counter() - t0
    return n_sample / dt, dt


def cpu_efgp_sample(name, n_sample, q_sample):
    """The multithreaded FP64 CPU EFGP (ES-kernel NUFFTs, FFT Toeplitz CG,
    scipy.fft on all host cores) on the first n_sample points and q_sample
    targets of the workload."""
    import cpu_efgp as C
    from oracle import efgp_oracle as O
    rec = synthdata.config(name, n=n_sample)
    x, y, z = synthdata.make_np(rec)
    z = z[:q_sample]
    fam, nu, ell, sigma, eps = synthdata.MODELS[name]
    t0 = time.perf_counter()
    _, info = C.efgp(x, y, z, O.Kernel(fam, nu, ell), sigma, eps)
    dt = time.perf_counter() - t0
    return n_sample / dt, dt, info


def cpu_efgp_sample_size(name):
    return {"se1d": 10_000, "matern2d": 1_000_000, "se3d": 1_000_000, "matern2d_1e9": 10_000_000,
            "matern2d_table4": 2_000_000, "matern2d_table5": 2_000_000}.get(name, 1_000_000)


def cpu_sample_size(name):
    return {"se1d": 10_000, "matern2d": 200_000, "se3d": 20_000, "matern2d_1e9": 500_000,
            "matern2d_table4": 50_000, "matern2d_table5": 50_000}.get(name, 100_000)


# se1d asks for eps = 1e-6, beyond the FP32 path: plain FP64.  At N = 1e9
# with sigma = 0.1 (N / sigma^2 = 1e11) the FP32 error of the Toeplitz product
# (~1e-7 N max D^2) exceeds sigma^2, so the all-FP32-FFT operator is not
# positive definite and CG breaks down: the set-up stays FP32, the Toeplitz
# products and CG run in FP64 (mixed_cg64).
DEFAULT_PRECISION = {"se1d": "fp64", "matern2d_table4": "mixed_cg64"}

# Jacobi-preconditioned CG where it was measured to pay on these workloads
# (the 2D Matern ones: 4-40x fewer iterations at N = 1e6-1e9, means within
# the criterion at full size); the 3D SE workload takes more iterations with it.
DEFAULT_PRECOND = {"matern2d": 1, "matern2d_1e9": 1, "matern2d_table4": 1, "matern2d_table5": 1, "batch": 1}

# The paper's total run times (set-up, solve and the mean on the 1000^2 target
# grid) for the exact N = 1e9 workloads of Sec. 5.4, on its 12-core desktop:
# Table 4 (l = 0.1, sigma = 0.1, eps = 1e-5, m = 94) and Table 5 (same with
# sigma = 1.83, N / sigma^2 = 3e8).  points/s = N / seconds.
PAPER_TOTAL_S = {"matern2d_table4": 103.0, "matern2d_table5": 121.0}


def paper_ratio(name, n, value):
    if name in PAPER_TOTAL_S and n == synthdata.config(name).n:
        return value / (n / PAPER_TOTAL_S[name])
    return None


def setup_roofline(rec, d, coord_b, val_b, rec_bytes, tot, hbm, src, traffic_json):
    """Roofline of the set-up (tile count, sorting scatter, spread): its
    algorithmic bytes are each point's coordinates and value read once
    (d*4 + 4 = 12 B per point for 2D FP32); extra sort traffic is not
    algorithmic and counts against the fraction.  Per-kernel figures (each
    kernel's own reads and writes over its own time) are kept beside it."""
    setup_ms = tot["bin_count_ms"] + tot["bin_scatter_ms"] + tot["spread_ms"]
    alg = rec.n * (d * coord_b + val_b)
    achieved = alg / (setup_ms / 1000.0) / 1e9 if setup_ms > 0 else None
    per = {
        "bin_count": rec.n * d * coord_b,
        "bin_scatter": rec.n * (d * coord_b + val_b) + rec.n * (d + 1) * rec_bytes,
        "spread": rec.n * (d + 1) * rec_bytes,
    }
    per_kernel = {}
    traffic = 0.0
    for k, b in per.items():
        ms = tot[k + "_ms"]
        t = traffic_for(k, rec.n, traffic_json) if traffic_json else None
        traffic = None if (t is None or traffic is None) else traffic + t
        per_kernel[k] = {"alg_bytes": b, "ms": ms, "gbs": b / (ms / 1000) / 1e9 if ms > 0 else None,
                         "frac": b / (ms / 1000) / 1e9 / hbm if ms > 0 else None, "traffic": t}
    return {"kernel": "setup: tile count + sorting scatter + spread", "bound": "hbm", "achieved": achieved,
            "peak": hbm, "unit": "GB/s", "frac": (achieved / hbm) if achieved else None, "traffic": traffic,
            "peak_source": src, "alg_bytes_per_launch": alg, "ms_per_launch": setup_ms, "per_kernel": per_kernel}


_DIRECT_CACHE = {}


def accuracy_record(E, x, y, z, kern, sigma, eps, prec, name, setup_path=0, max_dense_M=12000, n_targets=2000,
                    precond=0):
    """Mean error of the GPU path, the way tests/test_gpu_full_size.py checks it
    (CPU test infrastructure, outside any timed region): sampled entries of w
    (eq. 88) and b (eq. rhs) against FP64 direct sums over all points; then
    the dense solve of the GPU's own (verified) system and the direct mean at
    sampled targets against the GPU's CG + type-2 mean, relative to max|y|."""
    import numpy as np
    from oracle import efgp_oracle as O
    h = E.setup(x, y, kern, sigma, eps, precision=prec, setup_path=setup_path, precond=precond)
    info = h.solve()
    mu = h.predict(z).double().cpu().numpy()
    w, b = h.system()
    par = h.params()
    h.close()
    fam, nu, ell, _, _ = synthdata.MODELS[name]
    okern = O.Kernel(fam, nu, ell)
    d = x.shape[1] if x.dim() > 1 else 1
    hh, m = O.choose_h_m(okern, d, eps)
    D = O.spectral_weights(okern, d, hh, m)
    xh, yh = x.cpu().numpy(), y.cpu().numpy()
    n = xh.shape[0]
    rng = np.random.default_rng(2024)
    # one random entry of each (every entry is a sum over all N points: at
    # N = 1e9 that is ~20 s of host time per entry; the full-size test checks more)
    kw = np.array([list(rng.integers(-2 * m, 2 * m + 1, d))])
    kb = np.array([list(rng.integers(-m, m + 1, d))])
    t0 = time.perf_counter()
    key = (name, n, m)
    if key not in _DIRECT_CACHE:    # the same points for every form: sum once
        _DIRECT_CACHE[key] = (O.direct_modes(xh, 1.0, hh, kw), O.direct_modes(xh, yh, hh, kb))
    wd, bd = _DIRECT_CACHE[key]
    n1 = 2 * m + 1
    w_err = max(abs(w[tuple(k + 2 * m)] - r) for k, r in zip(kw, wd)) / n
    jb = [int(np.ravel_multi_index(tuple(k + m), (n1,) * d)) for k in kb]
    ysum = float(np.abs(yh).sum(dtype=np.float64))
    b_err = max(abs(b[j] / D[j] - r) for j, r in zip(jb, bd)) / ysum
    ymax = float(np.abs(yh).max())
    out = {"w_err_rel_n": float(w_err), "b_err_rel_sum_abs_y": float(b_err), "nufft_tol": eps / 10,
           "cg_iters": info["iters"], "true_rel_residual": info["true_rel_residual"], "criterion": 10 * eps,
           "method": "a random w and b entry vs FP64 direct sums over all points; dense solve of the GPU's "
                     f"system and direct mean at {n_targets} sampled targets vs the GPU mean, / max|y|"}
    if par["M"] <= max_dense_M:
        A = O.system_matrix(w, D, sigma, m, d)
        beta = np.linalg.solve(A, b)
        del A
        idx = rng.choice(mu.shape[0], min(n_targets, mu.shape[0]), replace=False)
        ref = O.mean_at(z[idx].cpu().numpy().astype(np.float64), beta, D, hh, m).real
        out["mean_error"] = float(np.abs(mu[idx] - ref).max() / ymax)
    else:
        out["mean_error"] = None
        out["note"] = f"M = {par['M']} is beyond the dense solve ({max_dense_M})"
    out["check_s"] = time.perf_counter() - t0
    return out


def oracle_single_core(name, n_sample, q_sample):
    """The oracle on one host core (BLAS and thread pools limited to one
    thread, in a child process so the limit holds from interpreter start)."""
    code = ("import sys, json; sys.path.insert(0, %r); import bench; "
            "v, dt = bench.oracle_sample(%r, %d, %d); print(json.dumps([v, dt]))" % (ROOT, name, n_sample, q_sample))
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
    v, dt = json.loads(r.stdout.strip().splitlines()[-1])
    return v, dt


def time_variant(E, x, y, z, kern, sigma, eps, prec, setup_path, steps, warmup=1, precond=0):
    """ms per whole step (set-up, solve, predict) of another form of the path
    on the same device inputs, CUDA events on the current stream."""
    import torch

    def one():
        h = E.setup(x, y, kern, sigma, eps, precision=prec, setup_path=setup_path, profile=1, precond=precond)
        info = h.solve()
        h.predict(z)
        pt = h.phase_times()
        h.close()
        return info, pt
    for _ in range(warmup):
        one()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    outs = [one() for _ in range(steps)]
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    ph = {k.replace("_ms", ""): round(sum(o[1][k] for o in outs) / steps, 4)
          for k in ("bin_count_ms", "bin_scatter_ms", "spread_ms", "cg_ms")}
    return ms, [o[0]["iters"] for o in outs], ph


def run_reference(args, rank, world):
    """Reference arm: the oracle on the host cores, a bounded sample per step."""
    if rank != 0:
        return
    ns = cpu_sample_size(args.config)
    qs = 10_000
    for _ in range(args.warmup):
        oracle_sample(args.config, max(ns // 10, 1000), 1000)
    vals, times = [], []
    for _ in range(args.steps):
        v, dt = oracle_sample(args.config, ns, qs)
        vals.append(v)
        times.append(dt)
    value = statistics.median(vals)
    rec = synthdata.config(args.config)
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000 * statistics.median(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(args.config, rec, synthdata.MODELS[args.config])},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"first {ns} points of the workload, {qs} targets, same h and m"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU leg
def run_batch(args, rank, world):
    """The heterogeneous batch: 64 independent 2D Matern problems of uneven
    size set up, CG-solved together (one persistent launch with a cluster per
    problem, or graph branches) and evaluated at 1e4 targets each."""
    import torch
    import paper_2210_10210_gb300 as E
    from paper_2210_10210_gb300 import build
    build.build()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    precond = args.precond if args.precond >= 0 else DEFAULT_PRECOND.get("batch", 0)
    probs = synthdata.batch_problems(seed=6 + 1000 * rank, count=args.batch_count)
    items, targets, npts = [], [], 0
    for rec, model in probs:
        fam, nu, ell, sigma, eps = model
        x, y = synthdata.make_torch(rec, dev)
        items.append(dict(x=x, y=y, kernel=E.Kernel(fam, nu, ell), sigma=sigma, eps=eps))
        targets.append(torch.from_numpy(synthdata.targets_np(rec)).to(dev))
        npts += rec.n
    torch.cuda.synchronize()

    def step():
        B = E.batch_setup(items, precision=args.precision or "mixed", cg_mode=args.cg_mode, autotune=args.autotune,
                          precond=precond)
        infos = B.solve()
        for i in range(len(items)):
            B.predict(i, targets[i])
        iters = [i["iters"] for i in infos]
        B.close()
        return iters, infos[0]["solve_ms"]

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record()
        solve_ms = []
        for _ in range(args.steps):
            iters, sms = step()
            solve_ms.append(sms)
        ev1.record()
        torch.cuda.synchronize()
    ms = max_over_ranks(ev0.elapsed_time(ev1), dist, dev) / args.steps
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": job_throughput(npts, world, ms), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if (args.precision or "mixed") == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": f"batch of {len(items)} 2D Matern-1/2 and 3/2 problems, N log-uniform "
                                   f"[1e4, 1e7] (total {npts}), l U[0.03, 0.3], sigma U[0.1, 1], eps 1e-4, "
                                   "1e4 iid targets each", "problems": len(items), "points": npts},
            "cg_iters_max": max(iters), "cg_iters_median": sorted(iters)[len(iters) // 2],
            "cg_iters_total": sum(iters), "cg_ms": sum(solve_ms) / len(solve_ms), "cg_mode": args.cg_mode,
            "cg_iters_per_s": sum(iters) / (sum(solve_ms) / len(solve_ms) / 1000),
            "precision": args.precision or "mixed", "precond": precond,
            "clocks": clk.summary(),
        }), flush=True)
    if dist:
        dist.destroy_process_group()


def toeplitz_matvec_timing(E, h, par, d, sigma, dev, reps=50):
    """Per-matvec device time of the library's fused Stockham Toeplitz product
    (efgp_apply_system_device) beside a cuFFT form of the same product
    (torch.fft: pad, FFT, w-hat product, inverse FFT, crop, D and sigma^2),
    FP32 grid, captured in a CUDA graph.  The baseline's D is a stand-in
    (timing only); its w-hat comes from the handle's Toeplitz vector."""
    import torch
    M, L, m = int(par["M"]), int(par["L"]), int(par["m"])
    n1 = 2 * m + 1
    g = torch.Generator(device=dev).manual_seed(0)
    v = torch.randn(M, dtype=torch.complex128, device=dev, generator=g)
    out = torch.empty_like(v)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(3):
        h.apply_system_device(v, out)
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(reps):
        h.apply_system_device(v, out)
    ev1.record()
    torch.cuda.synchronize()
    ours = ev0.elapsed_time(ev1) * 1000 / reps

    w, _ = h.system()
    wt = torch.from_numpy(w).to(dev)
    ks = torch.arange(-2 * m, 2 * m + 1, device=dev) % L
    grid = torch.zeros((L,) * d, dtype=torch.complex128, device=dev)
    grid[torch.meshgrid(*([ks] * d), indexing="ij")] = wt
    what = (torch.fft.fftn(grid).real / L ** d).float()
    del grid
    Dv = torch.rand(M, dtype=torch.float64, device=dev, generator=g) + 0.5
    buf = torch.zeros((L,) * d, dtype=torch.complex64, device=dev)
    crop = (slice(0, n1),) * d
    s2 = sigma * sigma

    def matvec():
        buf.zero_()
        buf[crop] = (Dv * v).to(torch.complex64).reshape((n1,) * d)
        U = torch.fft.fftn(buf)
        U *= what
        y = torch.fft.ifftn(U, norm="forward")
        return Dv * y[crop].reshape(-1).to(torch.complex128) + s2 * v

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(3):
            matvec()
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        matvec()
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(reps):
        graph.replay()
    ev1.record()
    torch.cuda.synchronize()
    cufft = ev0.elapsed_time(ev1) * 1000 / reps
    return {"L": L, "grid": f"{L}^{d}", "ours_us": ours, "cufft_graph_us": cufft,
            "note": "per product A v; cuFFT form via torch.fft in a CUDA graph, FP32 grid, stand-in D"}


def run_ours(args, rank, world):
    import torch
    import paper_2210_10210_gb300 as E
    from paper_2210_10210_gb300 import build
    build.build()

    local = int(os.environ.get("LOCAL_RANK", "0"))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    name = args.config
    rec = rank_recipe(name, args.n, rank)    # independent problem per rank
    model = synthdata.MODELS[name]
    fam, nu, ell, sigma, eps = model
    kern = E.Kernel(fam, nu, ell)
    prec = args.precision or DEFAULT_PRECISION.get(name, "mixed")
    precond = args.precond if args.precond >= 0 else DEFAULT_PRECOND.get(name, 0)

    if rec.cluster_frac > 0:       # clustered recipes are drawn on the host
        xn, yn = synthdata.points_np(rec), None
        yn = synthdata.values_np(rec, xn)
        x, y = torch.from_numpy(xn).to(dev), torch.from_numpy(yn).to(dev)
        del xn, yn
    else:
        x, y = synthdata.make_torch(rec, dev)
    z = torch.from_numpy(synthdata.targets_np(rec)).to(dev)
    q = z.shape[0]
    torch.cuda.synchronize()

    def step(profile=0):
        h = E.setup(x, y, kern, sigma, eps, precision=prec, profile=profile, cg_mode=args.cg_mode,
                    autotune=args.autotune, setup_path=args.setup_path, precond=precond,
                    cg_tol=args.cg_tol or None, upsampfac=args.upsampfac or None, es_width=args.es_width or None)
        info = h.solve()
        mu = h.predict(z)
        pt = h.phase_times()
        par = h.params()
        h.close()
        return info, mu, pt, par

    if args.once:                     # one untimed pass (a target for profilers)
        info, mu, pt, par = step()
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"once": True, "workload": workload_desc(name, rec, model), "cg_iters": info["iters"],
                              "launches": pt["launches"]}), flush=True)
        if dist:
            dist.destroy_process_group()
        return
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos, pts = [], []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(args.steps):
            info, mu, pt, par = step(profile=1)
            infos.append(info)
            pts.append(pt)
        ev1.record()
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1), dist, dev)
    ms_step = ms / args.steps
    value = job_throughput(rec.n, world, ms_step)

    # phase shares and the set-up's roofline
    keys = ["bin_count_ms", "bin_scatter_ms", "spread_ms", "fine_fft_ms", "what_ms", "cg_ms", "predict_fft_ms",
            "interp_ms"]
    tot = {k: sum(p[k] for p in pts) / args.steps for k in keys}
    launches = sum(p["launches"] for p in pts)
    iters = [i["iters"] for i in infos]
    hbm, src = _peaks()
    d = rec.d
    rec_bytes = 8 if prec == "fp64" else 4
    coord_b = 4 if rec.coord_dtype == "float32" else 8
    val_b = 4 if rec.value_dtype == "float32" else 8
    roofline = setup_roofline(rec, d, coord_b, val_b, rec_bytes, tot, hbm, src, args.traffic_json)

    # end to end through the C ABI from pinned host buffers (first after the
    # timed region: the cuFFT baseline's plans and graphs slow later copies)
    e2e = None
    if not args.no_e2e:
        xh = torch.empty(x.shape, dtype=x.dtype, pin_memory=True)
        yh = torch.empty(y.shape, dtype=y.dtype, pin_memory=True)
        zh = torch.empty(z.shape, dtype=z.dtype, pin_memory=True)
        xh.copy_(x)
        yh.copy_(y)
        zh.copy_(z)
        xn, yn, zn = xh.numpy(), yh.numpy(), zh.numpy()
        mu_h = torch.empty(q, dtype=torch.float32 if rec.value_dtype == "float32" else torch.float64,
                           pin_memory=True).numpy()

        def e2e_step():
            h = E.setup(xn, yn, kern, sigma, eps, precision=prec, precond=precond)
            h.solve()
            h.predict(zn, out=mu_h)
            h.close()

        for _ in range(max(3, args.warmup)):     # the device pool grows on the first steps
            e2e_step()
        torch.cuda.synchronize()
        # each step timed on its own; the host link and host memory are shared
        # with other jobs on the machine, so the median step is the figure and
        # every sample is reported beside it
        ke = max(3, min(args.steps, 5))
        samples = []
        for _ in range(ke):
            t0 = time.perf_counter()
            e2e_step()
            torch.cuda.synchronize()
            samples.append(time.perf_counter() - t0)
        te = max_over_ranks(statistics.median(samples), dist, dev)
        # the host link alone: the same pinned x and y copied to the device
        # (same values) with nothing else running, median of three
        copies = []
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            x.copy_(xh, non_blocking=True)
            y.copy_(yh, non_blocking=True)
            torch.cuda.synchronize()
            copies.append(time.perf_counter() - t0)
        tc = statistics.median(copies)
        e2e = {"value": job_throughput(rec.n, world, 1000 * te), "unit": UNIT,
               "h2d_bytes_per_step": int(xn.nbytes + yn.nbytes + zn.nbytes), "d2h_bytes_per_step": int(mu_h.nbytes),
               "ms_per_step": 1000 * te, "statistic": "median of %d steps" % ke,
               "mean_ms": 1000 * statistics.mean(samples), "samples_ms": [round(1000 * v, 2) for v in samples],
               "h2d_copy_ms": 1000 * tc, "h2d_link_gbs": (xh.nbytes + yh.nbytes) / tc / 1e9,
               "over_copy": te / tc}

    accuracy = None
    # other forms of the same step, outside the timed region: the bitwise
    # reproducible fused set-up, and the plain FP64 form (precision pattern)
    variants = {}
    if not args.no_variants:
        if d == 2 and prec != "fp64" and rec.coord_dtype == "float32":
            ms_f, it_f, ph_f = time_variant(E, x, y, z, kern, sigma, eps, prec, 2, max(1, min(args.steps, 3)),
                                            precond=precond)
            variants["fused_deterministic_setup"] = {"ms_per_step": ms_f, "value": job_throughput(rec.n, world, ms_f),
                                                     "cg_iters": it_f, "phase_ms": ph_f}
        if prec != "fp64":
            ms_d, it_d, ph_d = time_variant(E, x, y, z, kern, sigma, eps, "fp64", 0, 2, precond=precond)
            variants["fp64_form"] = {"ms_per_step": ms_d, "value": job_throughput(rec.n, world, ms_d),
                                     "cg_iters": it_d, "phase_ms": ph_d}

    # the Toeplitz product beside a cuFFT form of it
    matvec = None
    if not args.no_fft_baseline:
        hm = E.setup(x, y, kern, sigma, eps, precision=prec)
        matvec = toeplitz_matvec_timing(E, hm, hm.params(), d, sigma, dev)
        hm.close()

    # posterior mean at all N training points (type-2 with q = N)
    at_data = None
    if args.at_data:
        h = E.setup(x, y, kern, sigma, eps, precision=prec, profile=1, precond=precond)
        h.solve()
        mu_all = torch.empty(rec.n, dtype=y.dtype, device=dev)
        h.predict(x, out=mu_all)
        torch.cuda.synchronize()
        t0 = h.phase_times()
        reps = 3
        for _ in range(reps):
            h.predict(x, out=mu_all)
        torch.cuda.synchronize()
        t1 = h.phase_times()
        h.close()
        ims = (t1["interp_ms"] - t0["interp_ms"]) / reps
        fms = (t1["predict_fft_ms"] - t0["predict_fft_ms"]) / reps
        ib = rec.n * (d * coord_b + val_b)
        at_data = {"points": rec.n, "interp_ms": ims, "grid_ms": fms,
                   "interp_gbs": ib / (ims / 1000) / 1e9, "interp_frac_hbm": ib / (ims / 1000) / 1e9 / hbm,
                   "alg_bytes": ib}
        del mu_all

    # accuracy of the measured form (and of the FP64 form), by the CPU
    # reference leg's procedure: outside every timed region, rank 0 at N = 1,
    # after the end-to-end leg (its host work would slow the pinned copies)
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.no_accuracy:
        accuracy = accuracy_record(E, x, y, z, kern, sigma, eps, prec, name, precond=precond)
        if "fp64_form" in variants:
            variants["fp64_form"]["accuracy"] = accuracy_record(E, x, y, z, kern, sigma, eps, "fp64", name,
                                                                precond=precond)

    cpu = cpu_efgp = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ns = cpu_sample_size(name)
        v, dt = oracle_sample(name, ns, 10_000)
        cpu = {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"first {ns} points of the workload, 10000 targets, same h and m ({dt:.1f} s)"}
        try:
            n1c = max(ns // 8, 1000)
            v1, dt1 = oracle_single_core(name, n1c, 2_000)
            cpu["single_core"] = {"value": v1, "unit": UNIT, "cores": 1,
                                  "sample": f"first {n1c} points, 2000 targets ({dt1:.1f} s)"}
        except Exception as exc:   # reported, not fatal: the all-core figure stands
            cpu["single_core"] = {"value": None, "error": str(exc)[:200]}
        ne = cpu_efgp_sample_size(name)
        ve, dte, inf = cpu_efgp_sample(name, ne, 10_000)
        cpu_efgp = {"value": ve, "unit": UNIT, "cores": os.cpu_count(), "kind": "cpu_efgp",
                    "sample": f"first {ne} points of the workload, 10000 targets, same h and m, "
                              f"{inf['iters']} CG iterations ({dte:.1f} s)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": paper_ratio(name, rec.n, value), "dtype": "f64" if prec == "fp64" else "f32+f64",
            "data": "synthetic",
            "config": {"workload": workload_desc(name, rec, model), "precision": prec, "precond": precond,
                       "cg_tol": args.cg_tol or "default",
                       "m": par["m"],
                       "M": par["M"], "L": par["L"], "nf1": par["nf1"], "w1": par["w1"], "nf2": par["nf2"],
                       "w2": par["w2"], "l2_flush": "inputs larger than L2 (%.1f GB)" % (
                           rec.n * (d * coord_b + val_b) / 1e9), "parallelism": f"independent problem per GPU x{world}"},
            "cg_iters": iters, "cg_rel_residual": [i["rel_residual"] for i in infos],
            "cg_iters_per_s": (sum(iters) / len(iters)) / (tot["cg_ms"] / 1000) if tot.get("cg_ms") else None,
            "phase_ms": {k.replace("_ms", ""): round(v, 4) for k, v in tot.items()},
            "clocks": clk.summary(), "e2e": e2e, "gpu_launches": launches, "roofline": roofline,
            "cpu_baseline": cpu,
        }
        if accuracy:
            line["mean_error"] = accuracy.get("mean_error")
            line["accuracy"] = accuracy
        line.update(variants)
        if at_data:
            line["mean_at_data"] = at_data
        if matvec:
            line["toeplitz_matvec"] = matvec
        if cpu_efgp:
            line["cpu_efgp"] = cpu_efgp
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="matern2d_1e9")
    ap.add_argument("--n", type=int, default=None, help="override the point count")
    ap.add_argument("--precision", default=None, choices=[None, "mixed", "fp64", "mixed_cg64"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--once", action="store_true", help="run one untimed step and exit (profiling target)")
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--no-fft-baseline", action="store_true",
                    help="skip timing the Toeplitz product beside its cuFFT form")
    ap.add_argument("--autotune", type=int, default=0, choices=[0, 1],
                    help="time candidate line batches per Toeplitz pass before the CG graph is captured")
    ap.add_argument("--cg-mode", type=int, default=0, choices=[0, 1, 2, 3, 4],
                    help="CG launch form (0 chooses; see efgp_options.cg_mode)")
    ap.add_argument("--upsampfac", type=float, default=0.0, help="NUFFT upsampling factor (0: the planner's)")
    ap.add_argument("--es-width", type=int, default=0, help="ES kernel width (0: the planner's)")
    ap.add_argument("--cg-tol", type=float, default=0.0,
                    help="CG stopping residual rho (0: the library's default)")
    ap.add_argument("--precond", type=int, default=-1, choices=[-1, 0, 1],
                    help="Jacobi-preconditioned CG (efgp_options.precond; -1: the workload's default)")
    ap.add_argument("--setup-path", type=int, default=0, choices=[0, 1, 2],
                    help="set-up kernels (0 chooses; 1 three passes; 2 fused chunked; see efgp_options.setup_path)")
    ap.add_argument("--at-data", action="store_true",
                    help="also time the posterior mean at all N training points (type-2 with q = N)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the mean-error check of the CPU leg")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip timing the fused deterministic set-up and the FP64 form beside the measured step")
    ap.add_argument("--traffic-json", default=os.path.join(ROOT, "profiles", "traffic.json"))
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.config == "batch":
        run_batch(args, rank, world)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()
