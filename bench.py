#!/usr/bin/env python3
"""Benchmark of NFFT-accelerated Sinkhorn on GB300.

One step = one Sinkhorn iteration (the u half-step and the v half-step, each a
fast summation: spread, FFT, multiply, inverse FFT, interpolation, FP64
update) on the workload "ball3d_n1e6_eps0.02_fp32": n = m = 1e6 points i.i.d.
uniform in the radius-0.2 ball in R^3 (seeds 1, 2), uniform weights,
squared Euclidean cost (r = 2), eps = 0.02, bandwidth N = 64, sigma = 2,
Kaiser-Bessel cutoff m = 4, FP32 fast summation with FP64 updates.

Reported: iterations/s (whole job over all ranks), the same through the C ABI
with host buffers (e2e, plan build and copies included), the direct-summation
Sinkhorn on the same GPU, the per-stage roofline of the dominant kernel, and
the FP64 CPU oracle timed on a bounded sample on the host cores.

--impl reference times the CPU oracle (the reference arm of this project) on
bounded samples of the same workload.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Sinkhorn iters/s at n=m=1e6,d=3 (NFFT vs direct on same GB300, ≤1e-5 rel err)"
METRIC_OTHER = "Sinkhorn iters/s, workload %s (NFFT vs direct on same GB300)"
UNIT = "iters/s"
L2_FLUSH_BYTES = 512 * 1024 * 1024


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.strip().split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if sm:
            sm.sort()
            out["sm_mhz"] = sm[len(sm) // 2]
            out["sm_max_mhz"] = max(mx)
        out["reasons"] = sorted(reasons)
        out["samples"] = len(sm)
        return out


# ------------------------------------------------------------------ CPU oracle legs
_POOL_STATE = {}


def _oracle_pool_init(workload):
    """Per-process set-up outside the timed region: one thread, the
    workload's points and weights generated once."""
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    from paper_2201_07524_gb300 import workloads as wl
    w = _workloads(wl)[workload]
    x, y = w.points()
    a, b = w.marginals()
    _POOL_STATE.update(w=w, x=x, y=y, a=a, b=b)


def _oracle_rows_job(args):
    """The oracle's exact kernel products (Eqs. (matexp)/(matexpt)) and FP64
    updates for `rows` sampled rows of K v and `rows` columns of K^T u, from
    u = v = 1; returns the number of rows and columns done."""
    import numpy as np
    from oracle import sinkhorn as osk
    rows, seed = args
    w, x, y, a, b = (_POOL_STATE[k] for k in ("w", "x", "y", "a", "b"))
    rng = np.random.default_rng(seed)
    ri = rng.choice(w.n, rows, replace=False)
    ci = rng.choice(w.m, rows, replace=False)
    u_new = a[ri] / osk.kernel_apply(x[ri], y, np.ones(w.m), w.eps, w.r, chunk=4)
    v_new = b[ci] / osk.kernel_apply(y[ci], x, np.ones(w.n), w.eps, w.r, chunk=4)
    assert np.all(np.isfinite(u_new)) and np.all(np.isfinite(v_new))
    return 2 * rows


class OraclePool:
    """The FP64 oracle on every host core: one single-threaded process per
    core (spawned, so no CUDA state is inherited), each with the workload's
    points already generated."""

    def __init__(self, workload):
        import multiprocessing as mp
        self.cores = os.cpu_count() or 1
        self.workload = workload
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_oracle_pool_init, initargs=(workload,))
        self.pool.map(_oracle_rows_job, [(1, 10_000 + k) for k in range(self.cores)])   # warm-up

    def sample(self, rows_per_core, seed):
        """Wall seconds for rows_per_core rows and as many columns on every
        core, and the full-iteration time they extrapolate to."""
        from paper_2201_07524_gb300 import workloads as wl
        w = _workloads(wl)[self.workload]
        t0 = time.perf_counter()
        done = sum(self.pool.map(_oracle_rows_job, [(rows_per_core, seed * 1000 + k) for k in range(self.cores)]))
        wall = time.perf_counter() - t0
        return wall, wall * (w.n + w.m) / done, done

    def close(self):
        self.pool.close()
        self.pool.join()


def _full_small_run():
    """The smallest workload (2000 points per side, 2-D, 100 iterations,
    dense FP64 oracle, Alg. 1), run in full; returns seconds."""
    from oracle import sinkhorn as osk
    from paper_2201_07524_gb300 import workloads as wl
    w = wl.SMALL_2D
    x, y = w.points()
    a, b = w.marginals()
    t0 = time.perf_counter()
    out = osk.sinkhorn_dense(x, a, y, b, w.eps, w.r, w.iters)
    return time.perf_counter() - t0, out["s"]


def _workloads(wl):
    return {"headline": wl.HEADLINE_3D, "gmm2d": wl.GMM_2D, "r1": wl.BALL3D_R1}


def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_2201_07524_gb300 import workloads as wl
    w = _workloads(wl)[args.workload]
    pool = OraclePool(args.workload)
    try:
        for k in range(args.warmup):
            pool.sample(args.ref_rows, 100 + k)
        walls, secs, done = [], [], 0
        t_all = time.perf_counter()
        for k in range(args.steps):
            wall, sec, dn = pool.sample(args.ref_rows, k)
            walls.append(wall)
            secs.append(sec)
            done += dn
        wall_all = time.perf_counter() - t_all
    finally:
        pool.close()
    sec = sum(secs) / len(secs)
    value = 1.0 / sec
    frac = done / args.steps / (w.n + w.m)
    sample = ("each step: %d sampled rows of K v and %d columns of K^T u on each of %d host cores (exact FP64 "
              "numpy sums over all %.0e points, one thread per core), a fraction %.2e of one iteration; value "
              "extrapolated to a full iteration, ms_per_step is the measured step" %
              (args.ref_rows, args.ref_rows, pool.cores, float(w.n), frac))
    line = {
        "impl": "reference", "metric": METRIC if args.workload == "headline" else METRIC_OTHER % w.name,
        "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(walls) / len(walls),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "n": w.n, "m": w.m, "d": w.d, "r": w.r, "eps": w.eps,
                   "kernel": "exact FP64 sums (oracle)",
                   "extrapolated": "value from %d sampled rows + columns per step (fraction %.2e of an iteration)"
                                   % (done // args.steps, frac)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": wall_all,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
def algorithmic_counts(w, n_os):
    """Algorithmic work per launch of the two point stages of one product over
    n points (n = m here), as stated in the design notes:
      flops: 2 W^d per point (one multiply forming each tap weight, one add into
        the grid or into the sum), W = 2 m;
      bytes: spreading reads d FP32 coordinates and one FP64 weight per point
        and writes the n_os^d FP32 grid once; interpolation reads the grid once
        and, per point, d FP32 coordinates, u and a (FP64), and writes u."""
    d, W = w.d, 2 * w.m_w
    n = w.n
    taps = W ** d
    grid_bytes = 4.0 * n_os ** d
    return {"spread": (2.0 * taps * n, n * (4 * d + 8) + grid_bytes),
            "interp": (2.0 * taps * n, grid_bytes + n * (4 * d + 8 * 3))}


def kernel_name(stage, w, tensor_cores):
    W = 2 * w.m_w
    if w.d == 3:
        if stage == "interp" and tensor_cores:
            return "k_interp3_tc<%d>" % W
        return "k_%s3_col<%d, float>" % (stage, W)
    if w.d == 2:
        if stage == "interp" and tensor_cores:
            return "k_interp2_tc<%d>" % W
        return ("k_spread2_col<%d, float>" if stage == "spread" else "k_interp2_strip<%d, float>") % W
    return None


def measured_traffic(kname):
    """DRAM bytes per launch of `kname` from the committed ncu record, or None
    when there is none or the kernel's sources changed since the capture."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f).get(kname)
        if not rec:
            return None
        h = hashlib.sha1()
        for src in rec["sources"]:
            with open(os.path.join(ROOT, src), "rb") as f:
                h.update(f.read())
        return rec["dram_bytes_per_launch"] if h.hexdigest() == rec["sha1"] else None
    except Exception:
        return None


def reduce_max_ms(ms, world, device="cpu"):
    """The timed region's length as the maximum over ranks (ranks run
    independent problems; the job ends when the slowest rank does)."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(ms_max, steps, world):
    """Iterations per second of the whole job: every rank ran `steps`
    iterations of its own problem within ms_max milliseconds."""
    return world * steps / (ms_max / 1e3)


def replica_workload(w, rank):
    """Rank r solves its own problem: the same workload (every field kept)
    with seeds shifted by 1000 r."""
    import dataclasses
    return dataclasses.replace(w, seed_x=w.seed_x + 1000 * rank, seed_y=w.seed_y + 1000 * rank)


def fp32_peak(sk):
    """The FP32 roofline denominator, measured on this GPU (sk_fp32_peak: FMA
    chains on every SM, scalar and packed FP32x2 forms); the larger of the two
    is the peak.  Returns (peak TFLOP/s, record)."""
    scalar, sms = sk.sk_fp32_peak(False, 200000)
    packed, _ = sk.sk_fp32_peak(True, 100000)
    rec = {"scalar_tflops": scalar, "packed_tflops": packed, "sms": sms,
           "method": "sk_fp32_peak: 8 independent FMA chains per thread, every SM filled, CUDA events"}
    return max(scalar, packed), rec


def small_full_run(sk, T, dev, stream):
    """The smallest workload, ball2d_n2000_eps0.05_fp64 (2000 points per side,
    2-D, r = 2, eps = 0.05, 100 iterations, FP64 fast summation), run in full
    on the GPU and by the dense FP64 oracle on the host (Alg. 1, numpy with its
    default threads); both values and times."""
    import torch
    from paper_2201_07524_gb300 import workloads as wl
    w = wl.SMALL_2D
    x, y = w.points()
    a, b = w.marginals()
    prm = sk.sk_default_params(N=w.N, m_w=w.m_w, sigma=w.sigma, precision=sk.SK_FP64)
    plan = sk.sk_init(T(x), T(a), T(y), T(b), w.eps, w.r, prm)
    sk.sk_solve(plan, 2, result=False)                      # warm-up (graph capture)
    sk.sk_set_state(plan)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    sk.sk_solve(plan, w.iters, result=False)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    gpu_ms = ev0.elapsed_time(ev1)
    _, res = sk.sk_solve(plan, 0)
    plan.close()
    cpu_s, s_oracle = _full_small_run()
    return {"workload": w.name, "iters": w.iters, "gpu_ms": gpu_ms, "cpu_oracle_s": cpu_s,
            "cpu_cores": os.cpu_count(), "s_gpu": res["s"], "s_oracle": s_oracle,
            "s_rel_err": abs(res["s"] - s_oracle) / abs(s_oracle)}


def run_ours(args, rank, world):
    import numpy as np
    import torch
    from paper_2201_07524_gb300 import sk
    from paper_2201_07524_gb300 import workloads as wl

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    # each rank solves its own independent problem (replicas; seeds offset by rank)
    base = _workloads(wl)[args.workload]
    w = replica_workload(base, rank)
    x, y = w.points()
    a, b = w.marginals()
    T = lambda z: torch.as_tensor(z, dtype=torch.float64, device=dev)
    prm = sk.sk_default_params(N=w.N, m_w=w.m_w, sigma=w.sigma, precision=sk.SK_FP32)
    if "eps_I" in w.extra:
        prm.eps_I = w.extra["eps_I"]
    plan = sk.sk_init(T(x), T(a), T(y), T(b), w.eps, w.r, prm)
    info = sk.sk_plan_info(plan)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    # warm-up
    for _ in range(args.warmup):
        sk.sk_solve(plan, 1, result=False)
    barrier()

    # timed: K steps, each bracketed by events on the launching stream, L2 flushed between steps
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = sk.sk_launch_count(plan)
    barrier()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        starts[k].record(stream)
        sk.sk_solve(plan, 1, result=False)
        ends[k].record(stream)
    barrier()
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    launches = sk.sk_launch_count(plan) - launches0
    ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    ms_max = reduce_max_ms(ms, world, dev)
    value = whole_job_rate(ms_max, args.steps, world)

    # per-stage times over the same number of steps (a replayed graph with stage events)
    sk.sk_stage_times(plan, 1)
    for k in range(args.steps):
        flush.zero_()
        sk.sk_solve(plan, 1, result=False)
    stages = sk.sk_stage_times(plan, 0)
    torch.cuda.synchronize(dev)

    # equal-accuracy comparison with the direct-summation Sinkhorn (Eqs. (matexp),
    # (matexpt) summed exactly, FP32 kernel values, FP64 across tiles) on the
    # same GPU and plan: both methods run the same number of iterations from
    # u = v = 1, and the values s (Alg. 3 result line) are compared
    K = max(2, args.direct_iters)
    sk.sk_set_state(plan)
    _, res_nfft = sk.sk_solve(plan, K)
    v_test = wl.positive_vector(w.m, 36)
    t_gpu = torch.zeros(w.n, dtype=torch.float64, device=dev)
    sk.sk_kernel_apply(plan, 0, T(v_test), t_gpu)
    direct = None
    t_dir = None
    if args.direct_iters > 0:
        sk.sk_set_state(plan)
        sk.sk_set_method(plan, sk.SK_METHOD_DIRECT)
        sk.sk_solve(plan, 1, result=False)            # iteration 1 of K, untimed (graph capture)
        torch.cuda.synchronize(dev)
        ds = [torch.cuda.Event(enable_timing=True) for _ in range(K - 1)]
        de = [torch.cuda.Event(enable_timing=True) for _ in range(K - 1)]
        for k in range(K - 1):
            ds[k].record(stream)
            sk.sk_solve(plan, 1, result=False)
            de[k].record(stream)
        torch.cuda.synchronize(dev)
        dms = sum(s0.elapsed_time(e0) for s0, e0 in zip(ds, de)) / (K - 1)
        _, res_dir = sk.sk_solve(plan, 0)                 # value of the state after K iterations
        t_dir = torch.zeros(w.n, dtype=torch.float64, device=dev)
        sk.sk_kernel_apply(plan, 0, T(v_test), t_dir)
        sk.sk_set_method(plan, sk.SK_METHOD_NFFT)
        rel = abs(res_nfft["s"] - res_dir["s"]) / abs(res_dir["s"])
        direct = {"value": 1e3 / dms, "unit": UNIT, "ms_per_step": dms, "steps": K - 1,
                  "speedup_nfft_over_direct": (value / world) / (1e3 / dms),
                  "s_after_iters": res_dir["s"], "marg_err_after_iters": res_dir["marg_err"]}
    res = res_nfft

    # end to end through the C ABI with host buffers: pinned inputs -> sk_init
    # (copies, sort, tables) -> K iterations -> u, v, result read back to the host
    e2e = None
    if args.e2e:
        pin = lambda z: torch.as_tensor(z, dtype=torch.float64).pin_memory()
        xh, yh, ah, bh = pin(x), pin(y), pin(a), pin(b)
        uh = torch.empty(w.n, dtype=torch.float64).pin_memory()
        vh = torch.empty(w.m, dtype=torch.float64).pin_memory()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        plan2 = sk.sk_init(xh, ah, yh, bh, w.eps, w.r, prm)
        sk.sk_solve(plan2, args.steps, u_out=uh, v_out=vh, result=True)
        torch.cuda.synchronize(dev)
        e2e_s = time.perf_counter() - t0
        plan2.close()
        h2d = (x.nbytes + y.nbytes + a.nbytes + b.nbytes) / args.steps
        d2h = (uh.numel() + vh.numel()) * 8 / args.steps
        e2e = {"value": world * args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "includes": "plan build (sort, tables) and copies",
               "wall_s": e2e_s}

    # roofline of the dominant kernel
    pk, pk_kind = peaks()
    counts = algorithmic_counts(w, info["n_os"])
    per_launch = {k: (stages[k][0] / stages[k][1] if stages[k][1] else 0.0) for k in stages}
    dominant = max(("spread", "interp"), key=lambda k: per_launch[k])
    kname = kernel_name(dominant, w, info.get("tensor_cores", 0))
    flops, bytes_ = counts[dominant]
    dur_s = per_launch[dominant] / 1e3
    alu_peak, peak_rec = fp32_peak(sk)
    achieved = flops / dur_s / 1e12
    stage_report = {}
    for k in ("spread", "fft", "interp", "near", "other"):
        if stages[k][1]:
            ent = {"ms_per_launch": per_launch[k], "launches": stages[k][1],
                   "share": stages[k][0] / max(1e-12, sum(v[0] for v in stages.values()))}
            if k in counts:
                ent["tflops"] = counts[k][0] / (per_launch[k] / 1e3) / 1e12
                ent["gbs"] = counts[k][1] / (per_launch[k] / 1e3) / 1e9
                ent["hbm_frac"] = ent["gbs"] / pk["hbm_gbs"]
            stage_report[k] = ent

    # sampled accuracy of the products used in this run: exact FP64 sums of
    # the oracle on 32 rows
    if rank == 0:
        from oracle import sinkhorn as osk
        rows = np.random.default_rng(37).choice(w.n, 32, replace=False)
        exact = osk.kernel_apply(x[rows], y, v_test, w.eps, w.r, chunk=4)
        efs = lambda t: float(np.max(np.abs(t.cpu().numpy()[rows] - exact)) / np.max(np.abs(exact)))
        efs_sample = efs(t_gpu)
        efs_direct = efs(t_dir) if t_dir is not None else None
    accuracy = {"efs_sampled_rows": efs_sample if rank == 0 else None, "iters_compared": K,
                "s_nfft": res_nfft["s"], "marg_err_nfft": res_nfft["marg_err"]}
    if args.workload == "r1" and rank == 0:
        # the r = 1 workload's check: E_fs on 2e4 random targets against exact
        # FP64 sums over all sources (the FP64 direct method on a plan whose
        # targets are the subsample)
        sub = np.random.default_rng(54).choice(w.n, 20000, replace=False)
        ref_plan = sk.sk_init(T(x[sub]), T(wl.uniform_weights(len(sub))), T(y), T(b), w.eps, w.r,
                              sk.sk_default_params(precision=sk.SK_FP64, eps_I=w.extra["eps_I"]))
        sk.sk_set_method(ref_plan, sk.SK_METHOD_DIRECT)
        exact = torch.zeros(len(sub), dtype=torch.float64, device=dev)
        sk.sk_kernel_apply(ref_plan, 0, T(v_test), exact)
        ref_plan.close()
        exact = exact.cpu().numpy()
        accuracy["efs_2e4_subsample_vs_fp64_direct"] = float(
            np.max(np.abs(t_gpu.cpu().numpy()[sub] - exact)) / np.max(exact))
    if direct is not None:
        accuracy.update({"s_direct": direct["s_after_iters"], "s_rel_err_vs_direct": rel,
                         "s_rel_err_gate": 1e-5, "s_rel_err_ok": bool(rel <= 1e-5),
                         "efs_direct_sampled_rows": efs_direct if rank == 0 else None})
    cpu = None
    small = None
    if rank == 0 and world == 1 and args.cpu_rows > 0:
        pool = OraclePool(args.workload)
        try:
            wall_cpu, sec, done = pool.sample(args.cpu_rows, 7)
        finally:
            pool.close()
        cpu = {"value": 1.0 / sec, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
               "sample": "%d sampled rows of K v and %d columns of K^T u on each of %d host cores (exact FP64 numpy "
                         "sums over all %.0e points, one thread per core, %d rows + columns in %.2f s wall), "
                         "extrapolated to one full iteration" %
                         (args.cpu_rows, args.cpu_rows, pool.cores, float(w.n), done, wall_cpu)}
        small = small_full_run(sk, T, dev, stream)

    if rank == 0:
        line = {
            "metric": METRIC if args.workload == "headline" else METRIC_OTHER % w.name, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "n": w.n, "m": w.m, "d": w.d, "r": w.r, "eps": w.eps, "N": w.N,
                       "sigma": w.sigma, "m_w": w.m_w, "fast_summation": "fp32", "updates": "fp64",
                       "points": ("source: 8-component Gaussian mixture (sigma 0.03, means uniform in a radius-0.15 "
                                  "ball), target: uniform in a radius-0.2 ball" if w.source == "gmm"
                                  else "uniform in radius-0.2 ball") + ", weights " + w.weights
                                 + ", seeds %d/%d (+1000*rank)" % (base.seed_x, base.seed_y),
                       "l2": "flushed between timed steps (512 MB write outside the timed events)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"],
                       "samples": clk["samples"]},
            "gpu_launches": int(launches),
            "roofline": {"bound": "alu", "kernel": kname or dominant, "achieved": achieved,
                         "peak": alu_peak, "unit": "TFLOP/s", "frac": achieved / alu_peak,
                         "traffic": measured_traffic(kname),
                         "peak_source": "measured on this GPU (FP32 FMA chains; of measured)",
                         "peak_measurement": peak_rec,
                         "algorithmic_flops_per_launch": flops, "algorithmic_bytes_per_launch": bytes_,
                         "hbm_frac": bytes_ / dur_s / 1e9 / pk["hbm_gbs"], "hbm_peak_source": pk_kind},
            "stages": stage_report,
            "direct": direct,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "accuracy": accuracy,
            "small_full_run": small,
            "wall_s": wall,
        }
        print(json.dumps(line), flush=True)
    plan.close()


def batch_problems(count, seed):
    """The batching workload: independent problems, d in {2, 3}, n and m
    log-uniform in [1e3, 2e5], uniform-ball clouds (radius 0.2), uniform
    weights, r = 2, eps uniform in [0.01, 0.1] (seeded)."""
    import numpy as np
    from paper_2201_07524_gb300 import workloads as wl
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        d = int(rng.integers(2, 4))
        n, m = (int(np.exp(rng.uniform(np.log(1e3), np.log(2e5)))) for _ in range(2))
        eps = float(rng.uniform(0.01, 0.1))
        out.append((d, n, m, eps, seed * 100003 + 2 * k))
    return out


def run_batch(args):
    """512 independent problems solved together (sk_solve_batch, one graph
    per iteration holding every problem) against the same plans solved one
    after another (sk_solve); FP32 fast summation, N and m_w chosen per
    problem by sk_init.  Prints one JSON line (problem-iterations/s)."""
    import numpy as np
    import torch
    from paper_2201_07524_gb300 import sk
    from paper_2201_07524_gb300 import workloads as wl
    dev = torch.device("cuda", 0)
    T = lambda z: torch.as_tensor(z, dtype=torch.float64, device=dev)
    probs = batch_problems(args.batch, 5)
    t0 = time.perf_counter()
    plans, grids = [], []
    for d, n, m, eps, seed in probs:
        x = wl.uniform_ball(n, d, 0.2, seed)
        y = wl.uniform_ball(m, d, 0.2, seed + 1)
        prm = sk.sk_default_params(precision=sk.SK_FP32)
        prm.N = 0
        prm.m_w = 0
        plans.append(sk.sk_init(T(x), T(wl.uniform_weights(n)), T(y), T(wl.uniform_weights(m)), eps, 2.0, prm))
        info = sk.sk_plan_info(plans[-1])
        grids.append((info["N"], info["m_w"]))
    torch.cuda.synchronize(dev)
    build_s = time.perf_counter() - t0
    # the autotuner keeps, per problem, the faster interpolation kernel kind
    t0 = time.perf_counter()
    chosen = [sk.sk_autotune(p) for p in plans] if args.autotune else []
    tune_s = time.perf_counter() - t0

    def timed(fn):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        ev0.record()
        fn()
        ev1.record()
        torch.cuda.synchronize(dev)
        return ev0.elapsed_time(ev1)

    k1, k2 = args.warmup, args.warmup + args.steps
    sk.sk_solve_batch(plans, args.warmup, result=False)                       # warm-up
    b1 = timed(lambda: sk.sk_solve_batch(plans, k1, result=False))
    b2 = timed(lambda: sk.sk_solve_batch(plans, k2, result=False))
    per_iter_batch = (b2 - b1) / (k2 - k1)                                   # the capture cancels
    for p in plans:
        sk.sk_solve(p, 1, result=False)                                     # each plan's own graph
    s1 = timed(lambda: [sk.sk_solve(p, k1, result=False) for p in plans])
    s2 = timed(lambda: [sk.sk_solve(p, k2, result=False) for p in plans])
    per_iter_seq = (s2 - s1) / (k2 - k1)
    st, res = sk.sk_solve_batch(plans, 1)
    pts = sum(n + m for _, n, m, _, _ in probs)
    Ns = sorted(set(g[0] for g in grids))
    line = {
        "metric": "batched Sinkhorn problem-iterations/s (%d independent problems)" % len(plans),
        "value": len(plans) * 1000.0 / per_iter_batch,
        "unit": "problem-iters/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": per_iter_batch, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batch%d" % len(plans), "d": [2, 3], "n_m": "log-uniform [1e3, 2e5]",
                   "eps": "uniform [0.01, 0.1]", "r": 2.0, "points_total": pts,
                   "N_chosen": Ns, "m_w_chosen": sorted(set(g[1] for g in grids))},
        "one_by_one": {"value": len(plans) * 1000.0 / per_iter_seq, "ms_per_step": per_iter_seq,
                       "speedup_batch": per_iter_seq / per_iter_batch},
        "capture_ms": b1 - k1 * per_iter_batch,
        "plan_build_s": build_s,
        "autotune": ({"s": tune_s, "tensor_cores": sum(1 for c in chosen if c == sk.SK_KERNELS_TENSOR),
                      "cuda_cores": sum(1 for c in chosen if c == sk.SK_KERNELS_SIMT)} if args.autotune else None),
        "all_finite": bool(all(np.isfinite(r["s"]) for r in res)),
    }
    print(json.dumps(line), flush=True)


def run_grad(args):
    """The differentiation workload: Sinkhorn divergence S = s(x, y) - s(x, x)/2
    - s(y, y)/2 and its gradient with respect to the weights and positions
    (sk_divergence, FP32 fast summation), n = m = 2^18 points of two
    8-component Gaussian mixtures in R^3 (sigma 0.03, means in a radius-0.15
    ball), uniform weights, r = 2, eps = 0.02, 200 iterations per solve.

    The gradient is the envelope gradient of the dual at the final state (the
    gradient of the converged value).  It is checked by central differences
    with step 1e-4 on 64 random position coordinates: each difference solves
    s(x', y) and s(x', x') with FP64 fast summation from the unperturbed
    converged state until the row residual is below 1e-13, all plans on one
    fixed torus geometry.  Prints one JSON line."""
    import numpy as np
    import torch
    from paper_2201_07524_gb300 import sk
    from paper_2201_07524_gb300 import workloads as wl
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    T = lambda z: torch.as_tensor(np.ascontiguousarray(z), dtype=torch.float64, device=dev)
    n, d, eps, r, iters, h, ncoord = 2 ** 18, 3, 0.02, 2.0, 200, 1e-4, 64
    x = wl.gaussian_mixture(n, d, 8, 0.03, 0.15, 11)
    y = wl.gaussian_mixture(n, d, 8, 0.03, 0.15, 12)
    a, b = wl.uniform_weights(n), wl.uniform_weights(n)
    # one geometry for every plan, with room for the perturbed points
    pts = np.concatenate([x, y])
    c = 0.5 * (pts.min(0) + pts.max(0))
    scale = (0.25 - 0.05) / (np.max(np.linalg.norm(pts - c, axis=1)) + 1e-3)

    def params(precision):
        prm = sk.sk_default_params(N=64, m_w=4, precision=precision)
        prm.user_geometry = 1
        prm.scale = float(scale)
        for t in range(3):
            prm.center[t] = float(c[t])
        return prm

    xd, yd, ad, bd = T(x), T(y), T(a), T(b)
    grads = {}

    def divergence(precision):
        ga, gb = torch.zeros(n, dtype=torch.float64, device=dev), torch.zeros(n, dtype=torch.float64, device=dev)
        gx, gy = torch.zeros((n, d), dtype=torch.float64, device=dev), torch.zeros((n, d), dtype=torch.float64,
                                                                                  device=dev)
        out = sk.sk_divergence(xd, ad, yd, bd, eps, r, iters, 0.0, params(precision), grad_a=ga, grad_b=gb,
                               grad_x=gx, grad_y=gy)
        return out, gx, ga

    divergence(sk.SK_FP32)                                        # warm-up
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(1, args.steps)
    t_wall = time.perf_counter()
    ev0.record(stream)
    for _ in range(reps):
        out32, gx32, ga32 = divergence(sk.SK_FP32)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t_wall
    ms = ev0.elapsed_time(ev1) / reps
    t0 = time.perf_counter()
    out64, gx64, ga64 = divergence(sk.SK_FP64)
    torch.cuda.synchronize(dev)
    fp64_s = time.perf_counter() - t0

    # the converged FP64 states of the two terms that depend on x
    def solve(xp, yp, u0=None, v0=None, tol=0.0, max_iter=iters):
        pl = sk.sk_init(T(xp), ad, T(yp), bd if yp is y else ad, eps, r, params(sk.SK_FP64))
        if u0 is not None:
            sk.sk_set_state(pl, u0, v0)
        st, res = sk.sk_solve(pl, max_iter, tol=tol, check_every=5)
        u, v = np.zeros(n), np.zeros(n)
        sk.sk_get_state(pl, u, v)
        pl.close()
        return res, u, v

    res_xy, u_xy, v_xy = solve(x, y)
    res_xx, u_xx, v_xx = solve(x, x)
    rng = np.random.default_rng(13)
    coords = [(int(i), int(t)) for i, t in zip(rng.choice(n, ncoord, replace=False), rng.integers(0, d, ncoord))]
    fd = []
    t0 = time.perf_counter()
    for i, t in coords:
        vals = []
        for sgn in (1.0, -1.0):
            xp = x.copy()
            xp[i, t] += sgn * h
            rxy, _, _ = solve(xp, y, u_xy, v_xy, tol=1e-13, max_iter=400)
            rxx, _, _ = solve(xp, xp, u_xx, v_xx, tol=1e-13, max_iter=400)
            vals.append(rxy["s"] - 0.5 * rxx["s"])                 # s(y, y) does not depend on x
        fd.append((vals[0] - vals[1]) / (2 * h))
    fd_s = time.perf_counter() - t0
    fd = np.array(fd)
    g64 = np.array([gx64[i, t].item() for i, t in coords])
    g32 = np.array([gx32[i, t].item() for i, t in coords])
    scale_g = np.max(np.abs(fd))
    line = {
        "metric": "Sinkhorn divergence + gradient evaluations/s (n=m=2^18, d=3, 200 iterations per solve)",
        "value": 1e3 / ms, "unit": "evals/s", "n_gpus": 1, "steps": reps, "warmup": 1, "ms_per_step": ms,
        "higher_is_better": True, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "grad_gmm3d_n2^18_eps0.02", "n": n, "m": n, "d": d, "r": r, "eps": eps,
                   "iters": iters, "N": 64, "m_w": 4,
                   "points": "8-component Gaussian mixtures (sigma 0.03, means uniform in a radius-0.15 ball), "
                             "seeds 11 (x) and 12 (y), uniform weights"},
        "iterations_per_s": 3 * iters * 1e3 / ms,
        "value_fp32": out32[0], "value_fp64": out64[0],
        "value_rel_err_fp32_vs_fp64": abs(out32[0] - out64[0]) / abs(out64[0]),
        "residual_after_200": {"s_xy_err_row": res_xy["err_row"], "s_xx_err_row": res_xx["err_row"],
                               "norm_a": float(np.linalg.norm(a))},
        "fd": {"coords": ncoord, "step": h, "solves": 4 * ncoord, "seconds": fd_s,
               "max_abs_fd": float(scale_g),
               "max_err_fp64_grad": float(np.max(np.abs(g64 - fd)) / scale_g),
               "max_err_fp32_grad": float(np.max(np.abs(g32 - fd)) / scale_g),
               "errors_relative_to": "max |finite difference| over the 64 coordinates"},
        "grad_fp32_vs_fp64": {"x_max_rel": float((gx32 - gx64).abs().max().item() / gx64.abs().max().item()),
                              "a_max_rel": float((ga32 - ga64).abs().max().item() / ga64.abs().max().item())},
        "fp64_divergence_s": fp64_s, "wall_s": wall,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--direct-iters", type=int, default=10,
                    help="iterations of the NFFT and the direct method compared from u = v = 1 (direct timed)")
    ap.add_argument("--cpu-rows", type=int, default=8, help="oracle rows (and columns) per host core")
    ap.add_argument("--ref-rows", type=int, default=8, help="reference arm: oracle rows (and columns) per core")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--workload", default="headline", choices=["headline", "gmm2d", "r1", "batch", "grad"],
                    help="headline: the 1e6-point 3-D workload; gmm2d: the 1e6-point 2-D Gaussian mixture; "
                         "r1: the 4e6-point 3-D workload with r = 1 (near field); batch: --batch independent problems; "
                         "grad: Sinkhorn divergence and its gradient at 2^18 points, checked by finite differences")
    ap.add_argument("--batch", type=int, default=512)
    ap.add_argument("--autotune", action="store_true",
                    help="batch: let sk_autotune pick each plan's interpolation kernels (measured no faster)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        elif args.workload == "batch":
            if rank == 0:
                run_batch(args)
        elif args.workload == "grad":
            if rank == 0:
                run_grad(args)
        else:
            run_ours(args, rank, world)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
