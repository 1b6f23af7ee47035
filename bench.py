"""Benchmark: 7-point explicit heat, 512^3 FP64, r = 0.125, 200 sweeps per step.

One step is one pass of the hot path over the workload: region analysis of
the interior loop nest (host), specialisation (a cache hit after warm-up) and
one graph launch of 200 ping-pong sweeps, each with its fused max-abs
residual.  Inputs stay resident in HBM; the two 1 GiB fields exceed L2.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line (rank 0).  With torchrun (N > 1) every rank runs an
independent replica (the path has no exchange step); value = total updates
of all ranks / max-over-ranks time.
"""
import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 512
R = 0.125
SWEEPS = 200
LUP_PER_SWEEP = (N - 2) ** 3


def launches_per_step(info):
    """Kernels of one jacc_sweep sequence: the sweeps, the max-abs pre-pass of a
    fixed-point field and, for one of at least 2^22 points and two sweeps or
    more, the in-place conversion that lets the first sweep skip converting."""
    fixed = bool(info["fixed_point"])
    return SWEEPS + (1 if fixed else 0) + (1 if fixed and N ** 3 >= 2 ** 22 and SWEEPS >= 2 else 0)


def set_size(n, sweeps):
    global N, SWEEPS, LUP_PER_SWEEP, WORKLOAD
    N, SWEEPS, LUP_PER_SWEEP = n, sweeps, (n - 2) ** 3
    WORKLOAD = f"heat3d 7-point FP64 {n}^3, r=0.125, zero Dirichlet, {sweeps} sweeps per CUDA graph"
BYTES_PER_LUP = 16  # one FP64 read + one FP64 write per interior point
# DRAM bytes (read + write) per update of the intermediate-sweep kernel, from
# an ncu capture of the same kernel on a 384^3 grid (882.8 MB for 382^3
# updates); scaled to a launch by its updates.
DRAM_BYTES_PER_LUP = 15.837
METRIC = "stencil GLUP/s"
WORKLOAD = "heat3d 7-point FP64 512^3, r=0.125, zero Dirichlet, 200 sweeps per CUDA graph"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        # the raw samples go to BENCH_CLOCKS_DIR (default: the system's temporary directory)
        d = os.environ.get("BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"bench_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], 0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(ms_local, units_local, device=None):
    """Whole-job rate over ranks: every rank runs its own replica; the job's
    time is the slowest rank's and its work the sum over ranks.  Returns
    (max ms, total units).  Single process: the inputs unchanged."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms_local, units_local
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    u = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def region_nest():
    I3 = [[1, 0, 0], [0, 1, 0], [0, 0, 1]]
    refs = [dict(array=0, coef=I3, off=o) for o in
            ([-1, 0, 0], [1, 0, 0], [0, -1, 0], [0, 1, 0], [0, 0, -1], [0, 0, 1], [0, 0, 0])]
    refs.append(dict(array=1, write=True, coef=I3, off=[0, 0, 0]))
    return [(1, N - 2, 1)] * 3, refs, [[N, N, N], [N, N, N]]


def cpu_model():
    """The host CPU's model name (x86 /proc/cpuinfo, else lscpu, else the machine type)."""
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def _oracle_rate(u, nsweeps, threads):
    """GLUP/s of the oracle running nsweeps of the 512^3 heat sequence on `threads` threads."""
    import oracle
    with oracle.threads(threads):
        t0 = time.perf_counter()
        oracle.heat3d_run(u, R, nsweeps)
        dt = time.perf_counter() - t0
    return LUP_PER_SWEEP * nsweeps / dt / 1e9, dt


def cpu_baseline_oracle(single_sweeps=5, threaded_sweeps=40):
    """The oracle, as it stands, on the full 512^3 grid: a few sweeps on one
    thread and more on every host core (its threaded run splits each sweep's
    planes across threads, bit-identical to one thread)."""
    import oracle
    from paper_2110_14340_gb300 import inputs
    oracle.build()
    u = inputs.heat3d_field(N, seed=2)
    cores = os.cpu_count() or 1
    v1, t1 = _oracle_rate(u, single_sweeps, 1)
    vn, tn = _oracle_rate(u, threaded_sweeps, cores)
    return {"value": vn, "unit": "GLUP/s", "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
            "sample": f"{N}^3 grid, {threaded_sweeps} sweeps (of {SWEEPS}) of the plain C oracle on {cores} threads "
                      f"({tn:.1f} s)",
            "single_thread": {"value": v1, "unit": "GLUP/s", "cores": 1,
                              "sample": f"{N}^3 grid, {single_sweeps} sweeps on one thread ({t1:.1f} s)"}}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2110_14340_gb300 import inputs
    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    u = inputs.heat3d_field(N, seed=2)
    for _ in range(args.warmup):
        oracle.heat3d_sweep(u, R)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        u, _ = oracle.heat3d_sweep(u, R)
        times.append(time.perf_counter() - t0)
    dt = sum(times)
    value = LUP_PER_SWEEP * args.steps / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GLUP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "step": f"1 sweep of the {N}^3 grid by the CPU oracle on {cores} threads"},
            "cpu_baseline": {"value": value, "unit": "GLUP/s", "cores": cores, "kind": "oracle",
                             "cpu_model": cpu_model(),
                             "sample": f"{args.steps} single sweeps of the {N}^3 grid, each on {cores} threads"},
            "e2e": {"value": value, "unit": "GLUP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gpu(args):
    import numpy as np
    import torch

    from paper_2110_14340_gb300 import build, inputs, jacc

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    jacc.lib()

    u_host = inputs.heat3d_field(N, seed=2)
    a = torch.from_numpy(u_host).to(dev)
    b = torch.empty_like(a)
    resid = torch.zeros(SWEEPS, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    loops, refs, arrays = region_nest()

    # Set-up (untimed): the exhaustive autotuner picks the tile for this shape
    # (remembered by the library, so tile_id = -1 resolves to it), then the
    # constant-folded NVRTC variant of that tile is compiled and cached.
    tune = None
    if args.tile < 0 and not args.no_tune:
        t0 = time.perf_counter()
        # 10-sweep sequences: like the timed 200-sweep graph, mostly intermediate
        # (resident fixed-point) sweeps
        r = jacc.autotune(dict(stencil=jacc.STENCIL_7PT, dtype=jacc.F64, nx=N, ny=N, nz=N, coeffs=(R,)), a, b,
                          sweeps_per_rep=10, reps=3)
        tune = {"best_tile": r["best_tile"], "best_ms_per_sweep": r["best_ms"], "seconds": time.perf_counter() - t0}
        a.copy_(torch.from_numpy(u_host))
    jit = not args.no_jit

    def step(x, y):
        st, _ = jacc.region_analyze(loops, refs, arrays)
        assert st == 0
        k = jacc.Kernel(jacc.STENCIL_7PT, jacc.F64, N, N, N, coeffs=(R,), tile_id=args.tile, jit=jit)
        fb = jacc.sweep(k, x, y, SWEEPS, resid, graph=True)
        k.release()
        return fb

    def step_host(u_in, out, x, y, r, r_host, stream, wait_event, done_event):
        """The same step from and to host memory: one jacc_sweep_host call."""
        st, _ = jacc.region_analyze(loops, refs, arrays)
        assert st == 0
        k = jacc.Kernel(jacc.STENCIL_7PT, jacc.F64, N, N, N, coeffs=(R,), tile_id=args.tile, jit=jit)
        fb = jacc.sweep_host(k, u_in, out, x, y, SWEEPS, r, r_host, graph=True, stream=stream,
                             wait_event=wait_event, done_event=done_event)
        k.release()
        return fb

    keep = jacc.Kernel(jacc.STENCIL_7PT, jacc.F64, N, N, N, coeffs=(R,), tile_id=args.tile,
                       jit=jit)  # holds the cache entry
    info = keep.info()
    bufs = [a, b]
    for _ in range(args.warmup):
        fb = step(bufs[0], bufs[1])
        if fb == 1:
            bufs.reverse()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        fb = step(bufs[0], bufs[1])
        if fb == 1:
            bufs.reverse()
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    ms, total_lup = aggregate(ms, LUP_PER_SWEEP * SWEEPS * args.steps, device=dev)
    value = total_lup / (ms * 1e-3) / 1e9
    ms_step = ms / args.steps

    # Roofline of the dominant kernel (the 7-point sweep): algorithmic bytes
    # per launch / average launch time.  The step's time also holds one
    # max-abs pre-pass (1 GiB read) and, for a fixed-point field of at least
    # 2^22 points, its in-place conversion (1 GiB read and written), so this is
    # a lower bound on the kernel's rate.
    peak, peak_kind = peaks()
    achieved = LUP_PER_SWEEP * BYTES_PER_LUP / (ms_step / SWEEPS * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": args.traffic if args.traffic is not None else DRAM_BYTES_PER_LUP * LUP_PER_SWEEP,
            "traffic_source": "command line" if args.traffic is not None else
            "ncu dram read+write bytes of a 382^3 launch of the same kernel, 15.837 B per update, x updates per launch",
            "peak_kind": peak_kind,
            "per_unit": f"16 B per interior point per sweep (8 B read + 8 B write), {N - 2}^3 points per launch"}

    # End to end through the public API with host buffers: pinned H2D of the
    # input field, the 200-sweep graph, D2H of the result field and residuals.
    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(step_host, a, b, resid, u_host, args, ws)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GLUP/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "int64", "storage_dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "grid": [N, N, N], "sweeps_per_step": SWEEPS, "r": R,
                           "tile": info["tile_id"], "fixed_point": info["fixed_point"], "jit": info["jit"],
                           "jit_compile_ms": info["compile_ms"], "autotune": tune,
                           "l2": f"inputs larger than L2 (two {N ** 3 * 8 / 2 ** 20:.0f} MiB fields)",
                           "parallelism": "replicas" if ws > 1 else "single GPU"},
                "roofline": roof, "e2e": e2e, "gpu_launches": launches_per_step(info) * args.steps,
                "clocks": clk}
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_oracle()
        if not args.no_secondary and N == 512:
            line["secondary"] = secondary(dev)
        print(json.dumps(line), flush=True)
    keep.release()
    if ws > 1:
        torch.distributed.destroy_process_group()


def measure_e2e(step_host, a, b, resid, u_host, args, ws):
    """Whole-job rate from host memory: every step copies its input field (1 GiB,
    page-locked) to the device, runs the 200-sweep sequence and copies the result
    field and the residuals back, in one jacc_sweep_host call.  Consecutive steps
    rotate over three streams and three sets of device buffers, the sweeps kept in
    order by events, so one step's copy back and the next copy into the same
    buffers have two other steps' sweeps to overlap (the host link is shared with
    other jobs on the machine, and its rate varies); the timed region is host wall
    time from the first call to the completion of the last copy."""
    import numpy as np
    import torch
    nsets = 3
    pin_in = torch.from_numpy(u_host).pin_memory()
    outs = [torch.empty_like(pin_in).pin_memory() for _ in range(nsets)]
    res_host = [torch.empty(SWEEPS, dtype=torch.float64).pin_memory() for _ in range(nsets)]
    sets = [(a, b, resid)] + [(torch.empty_like(a), torch.empty_like(b), torch.zeros_like(resid))
                              for _ in range(nsets - 1)]
    streams = [torch.cuda.Stream() for _ in range(nsets)]
    done = [torch.cuda.Event() for _ in range(nsets)]
    # the first copy in and the last copy out overlap nothing: a run of at least
    # 30 steps keeps them a small part of the whole job
    e_steps = max(30, min(args.steps, 60))

    def run(nsteps):
        # step i: copy in on stream i % nsets at once, sweeps after step i-1's
        # sweeps (events), copy out after its own sweeps
        for i in range(nsteps):
            j = i % nsets
            x, y, r = sets[j]
            step_host(pin_in, outs[j], x, y, r, res_host[j], streams[j],
                      done[(i - 1) % nsets] if i else None, done[j])
        torch.cuda.synchronize()

    run(nsets)  # captures the sequence graph of each buffer set
    # the host link's rate on this machine, for the record: one 1 GiB copy each way
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record()
    a.copy_(pin_in, non_blocking=True)
    ev[1].record()
    outs[0].copy_(a, non_blocking=True)
    ev[2].record()
    torch.cuda.synchronize()
    link = {"h2d_GB/s": pin_in.numel() * 8 / ev[0].elapsed_time(ev[1]) / 1e6,
            "d2h_GB/s": pin_in.numel() * 8 / ev[1].elapsed_time(ev[2]) / 1e6}
    t0 = time.perf_counter()
    run(e_steps)
    e2e_s = (time.perf_counter() - t0) / e_steps
    e2e = {"value": LUP_PER_SWEEP * SWEEPS * ws / e2e_s / 1e9, "unit": "GLUP/s",
           "h2d_bytes_per_step": int(pin_in.numel() * 8), "d2h_bytes_per_step": int(outs[0].numel() * 8 + SWEEPS * 8),
           "ms_per_step": 1e3 * e2e_s, "steps": e_steps, "host_link": link,
           "overlap": "three streams, three device buffer sets, sweeps kept in order by events; each step's copies "
                      "overlap the neighbouring steps' sweeps"}
    for rh in res_host:
        assert np.isfinite(rh.numpy()).all()
    return e2e


def region_analysis_c_us(n=256, calls=200000):
    """Microseconds per jacc_region_analyze call of the n x n 5-point interior
    nest, timed by a plain C program (tests/c/region_timing.c) linked with
    libjacc.so: no Python in the loop.  None if it cannot be built here."""
    from paper_2110_14340_gb300 import build
    libdir = os.path.dirname(build.LIB)
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "region_timing")
        try:
            subprocess.run(["gcc", "-O2", "-std=c11", os.path.join(ROOT, "tests", "c", "region_timing.c"), "-o", exe,
                            "-I" + os.path.join(ROOT, "include"), "-L" + libdir, "-ljacc", "-Wl,-rpath," + libdir,
                            "-L/usr/local/cuda/lib64", "-lcudart", "-Wl,-rpath,/usr/local/cuda/lib64"],
                           check=True, capture_output=True, text=True, timeout=120)
            r = subprocess.run([exe, str(n), str(calls)], capture_output=True, text=True, timeout=120, check=True)
            return float(r.stdout.splitlines()[1].split()[1])
        except Exception:
            return None


def _time_ms(fn, reps=3):
    """Best of `reps` CUDA-event timings of fn() on the current stream (after one warm-up call)."""
    import torch
    fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    best = float("inf")
    for _ in range(reps):
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def secondary(dev):
    """The other workloads of the path, measured on the same GPU (not part of the timed step):
    Jacobi 256^2 x100 (graph and cluster-resident), 64 batched Jacobi grids x500 (persistent vs
    64 plain graphs), the 27-point FP32 1024^3 x100 periodic stencil (plain vs temporally
    blocked), and the variable-coefficient 19-point FP32 stencil on a 512 x 512 x 1024 grid."""
    import numpy as np
    import torch

    from paper_2110_14340_gb300 import inputs, jacc
    out = {}
    # Jacobi 2D 5-point FP64 256^2, 100 sweeps, one graph; region analysis of [1,254]^2 on the host
    u = inputs.jacobi2d_field(256, 256, seed=1)
    a = torch.from_numpy(u).to(dev)
    b = torch.empty_like(a)
    r = jacc.autotune(dict(stencil=5, dtype=64, nx=256, ny=256), a, b, sweeps_per_rep=20, reps=3)
    a.copy_(torch.from_numpy(u))
    k = jacc.Kernel(5, 64, 256, 256, 1, jit=True)
    res = torch.zeros(100, dtype=torch.float64, device=dev)
    ms = _time_ms(lambda: jacc.sweep(k, a, b, 100, res), reps=10)
    I = [[1, 0], [0, 1]]
    refs = [dict(array=0, coef=I, off=o) for o in ([-1, 0], [1, 0], [0, -1], [0, 1], [0, 0])]
    refs.append(dict(array=1, write=True, coef=I, off=[0, 0]))
    t0 = time.perf_counter()
    for _ in range(1000):
        jacc.region_analyze([(1, 254, 1), (1, 254, 1)], refs, [[256, 256], [256, 256]])
    ra_us = (time.perf_counter() - t0) * 1e3
    # the same sequence in one cluster-resident launch (fields in distributed shared memory)
    kc = jacc.Kernel(5, 64, 256, 256, 1, cluster=True)
    a.copy_(torch.from_numpy(u))
    msc = _time_ms(lambda: jacc.sweep(kc, a, b, 100, res), reps=10)
    out["jacobi2d_256_x100"] = {"ms": ms, "us_per_sweep": 1e3 * ms / 100, "GLUP/s": 254 * 254 * 100 / ms / 1e6,
                                "tile": k.info()["tile_id"], "cluster_ms": msc,
                                "cluster_us_per_sweep": 1e3 * msc / 100,
                                "cluster_GLUP/s": 254 * 254 * 100 / msc / 1e6,
                                "region_analysis_us_via_python": ra_us,
                                "region_analysis_us_from_c": region_analysis_c_us()}
    k.release()
    kc.release()
    # 64 batched grids x 500 sweeps: one persistent launch vs 64 plain graph launches
    shapes = inputs.batched_shapes(64, seed=3)
    hosts = inputs.batched_fields(shapes, seed=4)
    fields = [(torch.from_numpy(h).to(dev), torch.zeros(h.shape, dtype=torch.float64, device=dev)) for h in hosts]
    lup = sum((nx - 2) * (ny - 2) for nx, ny in shapes) * 500
    ks = [jacc.Kernel(5, 64, nx, ny, 1) for nx, ny in shapes]
    rp = torch.zeros(64, 500, dtype=torch.float64, device=dev)
    plain = _time_ms(lambda: [jacc.sweep(ks[g], fa, fb, 500, rp[g]) for g, (fa, fb) in enumerate(fields)])
    bt = jacc.Batch(fields)
    cfg, _ = bt.tune(probe_sweeps=40)
    rb = torch.zeros(64 * 500, dtype=torch.float64, device=dev)
    batched = _time_ms(lambda: bt.sweep(500, rb))
    bt.status()
    out["batched_64_grids_x500"] = {"plain_ms": plain, "batched_ms": batched, "speedup": plain / batched,
                                    "plain_GLUP/s": lup / plain / 1e6, "batched_GLUP/s": lup / batched / 1e6,
                                    "schedule": cfg}
    for kk in ks:
        kk.release()
    bt.release()
    del fields
    # 27-point FP32 1024^3, 100 sweeps, periodic: plain (autotuned tile, precompiled and
    # constant-folded) vs temporal blocking
    n = 1024
    w = tuple(float(x) for x in inputs.box27_weights())
    a = inputs.uniform_torch(6, n ** 3, dev, torch.float32).mul_(2).sub_(1).view(n, n, n)
    b = torch.empty_like(a)
    r = jacc.autotune(dict(stencil=27, dtype=32, nx=n, ny=n, nz=n, coeffs=w), a, b, sweeps_per_rep=1, reps=3)
    kp = jacc.Kernel(27, 32, n, n, n, coeffs=w)
    res = torch.zeros(100, dtype=torch.float64, device=dev)
    c5 = {}
    c5["plain_ms"] = _time_ms(lambda: jacc.sweep(kp, a, b, 100, res), reps=2)
    c5["plain_tile"] = kp.info()["tile_id"]
    # the same tile with extents and weights folded as constants (NVRTC)
    kj = jacc.Kernel(27, 32, n, n, n, coeffs=w, jit=True)
    c5["jit_ms"] = _time_ms(lambda: jacc.sweep(kj, a, b, 100, res), reps=2)
    for T in (2,):
        kt = jacc.Kernel(27, 32, n, n, n, coeffs=w, tblock=T)
        c5[f"tb{T}_ms"] = _time_ms(lambda: jacc.sweep(kt, a, b, 100, res), reps=2)
        kt.release()
    best = min(c5["plain_ms"], c5["jit_ms"], c5["tb2_ms"])
    c5["GLUP/s"] = n ** 3 * 100 / best / 1e6
    c5["effective_GB/s_8B_per_point"] = n ** 3 * 100 * 8 / best / 1e6
    # sum conservation on a fresh field: S_100 = W^100 S_0 (W = sum of the FP32 weights, in FP64)
    a.copy_(inputs.uniform_torch(6, n ** 3, dev, torch.float32).mul_(2).sub_(1).view(n, n, n))
    s0 = float(a.double().sum().item())
    sabs = float(a.abs().double().sum().item())
    jacc.sweep(kj, a, b, 100, res)  # the constant-folded single-sweep kernel (every sweep's sum)
    torch.cuda.synchronize()
    kj.release()
    Wsum = sum(float(np.float32(x)) * c for x, c in zip(w, (1, 6, 12, 8)))
    rr = res.cpu().numpy()
    c5["sum_check_rel_to_sum_abs"] = abs(rr[-1] - Wsum ** 100 * s0) / sabs
    c5["sum_check_tolerance"] = 1e-6
    kp.release()
    out["box27_f32_1024_x100"] = c5
    del a, b
    torch.cuda.empty_cache()
    # region-driven scheduler: 32 independent 32^3 heat grids x 40 sweeps, one
    # stream back to back vs spread over 8 streams (no conflicts between them)
    side, ns, G = 32, 40, 32
    hosts = [inputs.heat3d_field(side, seed=90 + g) for g in range(G)]
    k7 = jacc.Kernel(7, 64, side, side, side, coeffs=(0.125,))
    sb = [(torch.from_numpy(h).to(dev), torch.empty((side,) * 3, dtype=torch.float64, device=dev)) for h in hosts]

    def seq():
        for u0, u1 in sb:
            jacc.sweep(k7, u0, u1, ns)

    def sched():
        sc = jacc.Sched(nstreams=8)
        for u0, u1 in sb:
            sc.sweep(k7, u0, u1, ns)
        sc.join()
        sc.release()

    out["sched_32_grids_32cubed_x40"] = {"one_stream_ms": _time_ms(seq, reps=3),
                                          "scheduled_8_streams_ms": _time_ms(sched, reps=3)}
    out["sched_32_grids_32cubed_x40"]["speedup"] = (out["sched_32_grids_32cubed_x40"]["one_stream_ms"]
                                                    / out["sched_32_grids_32cubed_x40"]["scheduled_8_streams_ms"])
    k7.release()
    del sb
    # variable-coefficient 19-point (Himeno-like) FP32, the paper's XL grid size
    # (512 x 512 x 1024 points, 14 fields = 15 GB), 20 graph-launched sweeps
    nx, ny, nz = 512, 512, 1024
    p, fields = inputs.var19_problem_torch(nx, ny, nz, dev, seed=7)
    q = torch.empty_like(p)
    k19 = jacc.Kernel(jacc.STENCIL_19PT, jacc.F32, nx, ny, nz, coeffs=(0.8,))
    r19 = torch.zeros(20, dtype=torch.float64, device=dev)
    ms19 = _time_ms(lambda: jacc.sweep_coeffs(k19, p, q, 20, fields, r19), reps=3) / 20
    lup19 = (nx - 2) * (ny - 2) * (nz - 2)
    out["var19_f32_512x512x1024_x20"] = {
        "ms_per_sweep": ms19, "GLUP/s": lup19 / ms19 / 1e6,
        "GB/s_56B_per_update": lup19 * 56 / ms19 / 1e6,
        "frac_of_measured_hbm": lup19 * 56 / ms19 / 1e6 / peaks()[0],
        "residual_first_last": [float(r19[0]), float(r19[-1])]}
    k19.release()
    del p, q, fields
    return out


def profile_case(args):
    """A 27-point FP32 periodic (or 19-point variable-coefficient) sweep sequence on an n^3 cube,
    nothing else (for ncu captures)."""
    import torch

    from paper_2110_14340_gb300 import build, inputs, jacc
    build.build()
    n = args.n
    if args.profile_case == "jacobi2d":
        u = inputs.jacobi2d_field(n, n, seed=1)
        a = torch.from_numpy(u).to("cuda")
        b = torch.empty_like(a)
        k = jacc.Kernel(5, 64, n, n, 1, tile_id=args.tile, jit=True)
        kc = jacc.Kernel(5, 64, n, n, 1, cluster=True)
        res = torch.zeros(args.sweeps, dtype=torch.float64, device="cuda")
        for _ in range(args.warmup + args.steps):
            jacc.sweep(k, a, b, args.sweeps, res)
            jacc.sweep(kc, a, b, args.sweeps, res)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": args.profile_case, "n": n, "sweeps": args.sweeps,
                          "runs": args.warmup + args.steps, "tile": k.info()["tile_id"]}))
        return
    if args.profile_case == "batched":
        shapes = inputs.batched_shapes(64, seed=3)
        hosts = inputs.batched_fields(shapes, seed=4)
        fields = [(torch.from_numpy(h).to("cuda"), torch.zeros(h.shape, dtype=torch.float64, device="cuda"))
                  for h in hosts]
        cfg = dict(item_points=args.item_points, group_bytes=args.group_bytes)
        bt = jacc.Batch(fields, **cfg)
        res = torch.zeros(64 * args.sweeps, dtype=torch.float64, device="cuda")
        for _ in range(args.warmup + args.steps):
            bt.sweep(args.sweeps, res)
        bt.status()
        print(json.dumps({"profile_case": args.profile_case, "sweeps": args.sweeps, "config": bt.config(),
                          "runs": args.warmup + args.steps}))
        return
    if args.profile_case == "var19":
        p, fields = inputs.var19_problem_torch(n, n, n, "cuda", seed=7)
        q = torch.empty_like(p)
        k = jacc.Kernel(jacc.STENCIL_19PT, jacc.F32, n, n, n, coeffs=(0.8,))
        res = torch.zeros(args.sweeps, dtype=torch.float64, device="cuda")
        for _ in range(args.warmup + args.steps):
            jacc.sweep_coeffs(k, p, q, args.sweeps, fields, res)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": args.profile_case, "n": n, "sweeps": args.sweeps,
                          "runs": args.warmup + args.steps}))
        return
    w = tuple(float(x) for x in inputs.box27_weights())
    a = inputs.uniform_torch(6, n ** 3, "cuda", torch.float32).mul_(2).sub_(1).view(n, n, n)
    b = torch.empty_like(a)
    T = {"box27-tb2": 2, "box27-tb3": 3}.get(args.profile_case, 0)
    k = jacc.Kernel(27, 32, n, n, n, coeffs=w, tile_id=3 if args.tile < 0 else args.tile, tblock=T,
                    jit=args.profile_case == "box27-jit")
    res = torch.zeros(args.sweeps, dtype=torch.float64, device="cuda")
    for _ in range(args.warmup + args.steps):
        jacc.sweep(k, a, b, args.sweeps, res)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": args.profile_case, "n": n, "sweeps": args.sweeps,
                      "runs": args.warmup + args.steps}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tile", type=int, default=-1)
    ap.add_argument("--no-jit", action="store_true", help="use the precompiled kernel instead of the NVRTC variant")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner; use the library's default tile")
    ap.add_argument("--no-secondary", action="store_true", help="skip the other workloads' measurements")
    ap.add_argument("--profile-case", choices=["box27", "box27-jit", "box27-tb2", "box27-tb3", "var19", "jacobi2d",
                                               "batched"], default=None,
                    help="run only one sweep sequence (27-point FP32 or 19-point on an --n cube; jacobi2d: 5-point FP64 --n squared, graph and cluster launch) for profilers, and exit")
    ap.add_argument("--traffic", type=float, default=None,
                    help="ncu dram bytes per launch of the sweep kernel, if captured for this build")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--n", type=int, default=512, help="grid side (profiling of small cases)")
    ap.add_argument("--sweeps", type=int, default=200)
    ap.add_argument("--item-points", type=int, default=16384, help="batched profile case: points per item")
    ap.add_argument("--group-bytes", type=int, default=-1, help="batched profile case: L2 budget per group")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    set_size(args.n, args.sweeps)
    if args.profile_case:
        profile_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
