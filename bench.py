"""Benchmark: cell-updates/s per RK stage of the ES van der Waals moving-mesh scheme on GB300.

Workload (default): the 2D four-quadrant van der Waals Riemann problem on an
adaptive moving mesh, 200 x 200 nodes, outflow boundaries, seeded states near
the critical point, monitor with the fundamental derivative (alpha = 1200 x 3,
5 filter passes, 5 Jacobi sweeps), SSP-RK3 at CFL 0.4, FP64.  One step = the
whole hot path: CFL time step, mesh redistribution, three fused RK stages.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

The reference arm (--impl reference) times the plain FP64 CPU oracle on the
same workload on the host cores.  Multi-GPU runs (torchrun) are independent
replicas (the hot path has no cross-rank exchange here); value = all ranks'
cell updates / the slowest rank's time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s per RK stage"
RESTART_EVERY = 40          # steps; the state restarts from t = 0 (outside the timed region)
SEED = 5                    # quadrant states with a G < 0 region (non-classical waves)
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=200)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--tile", type=int, default=0,
                    help="fixed stage-tile shape 1..5 of the main form (default 0: the autotuner chooses)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-chosen", action="store_true", help="skip the mixed-precision comparison run")
    ap.add_argument("--batch-problems", type=int, default=4096, help="batched-form problems (0: skip)")
    ap.add_argument("--batch-steps", type=int, default=10)
    ap.add_argument("--no-matched-error", action="store_true",
                    help="skip the default matched-error comparison (1D sine 50..200, vortex 128^2..256^2, both forms)")
    ap.add_argument("--precision-sweep", action="store_true",
                    help="also run the precision-form sweep: 1D sine 50..1600, 2D sine 1024^2 and the vortex 128^2..2048^2, "
                         "both forms")
    ap.add_argument("--mach-reflection", action="store_true",
                    help="also run Example 5.4's Mach reflection (P1, D1) to its final time: MM, MM1, UM, FP64")
    ap.add_argument("--learned", action="store_true",
                    help="also train and evaluate the learned warm start (512^2, about 3 minutes)")
    ap.add_argument("--nn-inference", type=int, default=0,
                    help="also time the warm-start network's inference on one n x n image (0: skip)")
    ap.add_argument("--three-d", type=int, default=96,
                    help="also time the 3D FP64 path on the moving-mesh 3D sine wave at n^3 (0: skip)")
    ap.add_argument("--three-d-steps", type=int, default=5)
    ap.add_argument("--large-n", type=int, default=1024,
                    help="also time the mixed stage kernel on the n x n Riemann problem (0: skip)")
    ap.add_argument("--mesh-n", type=int, default=4096,
                    help="also time the mesh redistribution alone on an n x n mesh, both forms (0: skip)")
    ap.add_argument("--learned-n", type=int, default=512)
    ap.add_argument("--learned-seeds", type=int, default=20, help="plain runs; the last two are held out")
    ap.add_argument("--learned-steps", type=int, default=100)
    ap.add_argument("--learned-epochs", type=int, default=8)
    ap.add_argument("--learned-tols", default="0.02,0.01,0.005,0.0025",
                    help="Jacobi tolerances (cells) of the matched-accuracy comparison; the first is the training one")
    return ap.parse_args()


def max_over_ranks(value, device):
    """The largest of the ranks' values (the slowest rank's time); the value itself on one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(n):
    from paper_2407_05568_gb300 import workloads as wl
    w = wl.riemann_2d(n, seed=SEED)
    w["t_end"] = 1e30        # steps are the unit of work; restarts keep the run on the t <= 0.2 solution
    return w


def config(n, precision, flush):
    return {"workload": f"2D vdW four-quadrant Riemann problem, adaptive moving mesh, {n}x{n} nodes, "
                        f"monitor with G, 5 filter passes, 5 Jacobi sweeps, SSP-RK3 CFL 0.4",
            "nodes": n * n, "rk_stages_per_step": 3, "precision_form": precision,
            "l2": flush, "restart_every_steps": RESTART_EVERY}


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- oracle
def oracle_state(w):
    from oracle import operator as op
    from oracle import stepper, thermo
    g = thermo.Gas(**w["gas"])
    sch = op.Scheme(gas=g, dim=w["dim"], bc=w["bc"], dxi=w["dxi"], period=w["period"])
    J = op.node_jacobian(sch, w["x"])
    JU = thermo.prim_to_cons(g, w["rho"], w["v"], w["p"]) * J
    mc = stepper.MeshControl(moving=True, **w["mesh"])
    return sch, mc, JU, J, w["x"].copy()


def time_oracle(w, nsteps):
    """Oracle steps from t = 0; returns (seconds, steps)."""
    from oracle import stepper
    sch, mc, JU, J, x = oracle_state(w)
    t = 0.0
    t0 = time.perf_counter()
    for _ in range(nsteps):
        JU, J, x, t, _ = stepper.step(sch, mc, JU, J, x, t, 1e30, w["cfl"])
    return time.perf_counter() - t0, nsteps


def cpu_cores():
    return 1   # numpy element-wise kernels run on one thread; no BLAS on this path


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    w = workload(args.n)
    nodes = args.n * args.n
    time_oracle(w, max(0, min(args.warmup, 1)))
    sec, k = time_oracle(w, args.steps)
    value = nodes * 3 * k / sec
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "cell-updates/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sec / k, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": config(args.n, "fp64", "host"),
            "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": f"{k} full steps of the {args.n}x{args.n} workload from t = 0"},
            "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- GPU arm
def measure_form(args, precision, dev, stream, world):
    """Time K steps of one arithmetic form; returns a dict of the measurements."""
    import torch
    import torch.distributed as dist

    from paper_2407_05568_gb300 import es
    w = workload(args.n)
    nodes = args.n * args.n
    with torch.cuda.stream(stream):
        tile = args.tile if precision == args.precision else 0
        ctx = es.es_create(es.make_params(w, precision=precision, tile=tile), stream)
        x0 = torch.tensor(w["x"], dtype=torch.float64, device=dev)
        J0 = es.state_empty(ctx, w["x"].shape[1:], dev)
        es.es_init_mesh(ctx, x0, J0)
        JU0 = es.state_empty(ctx, (4,) + w["x"].shape[1:], dev)
        es.es_prim_to_cons(ctx, torch.tensor(w["rho"], device=dev), torch.tensor(w["v"], device=dev),
                           torch.tensor(w["p"], device=dev), J0, JU0)
        JU, J, x = JU0.clone(), J0.clone(), x0.clone()
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream.synchronize()

    def restart():
        with torch.cuda.stream(stream):
            JU.copy_(JU0)
            J.copy_(J0)
            x.copy_(x0)
        stream.synchronize()
        es.es_set_time(ctx, 0.0)

    restart()
    if tile:                                             # fixed by --tile
        tile_ms = None
    else:
        tile, tile_ms = es.es_autotune(ctx, JU, J, x)    # stage tile shape for this problem size
    done = 0
    for _ in range(args.warmup):
        es.es_steps(ctx, JU, J, x, 1, w["t_end"])
        done += 1
    stream.synchronize()
    if es.es_check(ctx):
        raise RuntimeError(es.es_last_error(ctx))

    # device-timed region: K steps, L2 flushed before each (outside the events)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = ctx.launches
    with ClockSampler(dev.index) as clk:
        for k in range(args.steps):
            if done and done % RESTART_EVERY == 0:
                restart()
            with torch.cuda.stream(stream):
                flush.fill_(float(k))
                starts[k].record(stream)
            es.es_steps(ctx, JU, J, x, 1, w["t_end"])
            ends[k].record(stream)
            done += 1
        torch.cuda.synchronize()
    launches = ctx.launches - launches0
    if world > 1:
        dist.barrier()
    ms = max_over_ranks(sum(s.elapsed_time(e) for s, e in zip(starts, ends)) / args.steps, dev)
    if es.es_check(ctx):
        raise RuntimeError(es.es_last_error(ctx))
    roof = stage_roofline(es, ctx, JU, J, x, stream, w, nodes, precision, tile)
    roof["autotune_ms_per_shape"] = tile_ms

    # end to end through the C ABI with host buffers (copies inside the timed region)
    hJU, hJ, hx = (pin(np.ascontiguousarray(t.cpu().numpy())) for t in (JU0, J0, x0))
    es.es_set_time(ctx, 0.0)
    es.es_run_host(ctx, hJU, hJ, hx, 1, w["t_end"])          # warm (captures the host-buffer graph)
    e2e_t = []
    for _ in range(max(3, args.steps // 2)):
        t0 = time.perf_counter()
        es.es_run_host(ctx, hJU, hJ, hx, 1, w["t_end"])
        e2e_t.append(time.perf_counter() - t0)
    # the state after the same number of steps from t = 0, for the error between forms
    restart()
    es.es_steps(ctx, JU, J, x, min(args.steps, RESTART_EVERY), w["t_end"])
    stream.synchronize()
    state = JU.double() if precision == "fp64" else (JU[0].double() + JU[1].double())
    return dict(ms=ms, value=world * nodes * 3 / (ms * 1e-3), roof=roof, clocks=clk.summary(),
                launches=int(launches), e2e=world * nodes * 3 / statistics.median(e2e_t),
                io_bytes=hJU.nbytes + hJ.nbytes + hx.nbytes, state=state.cpu().numpy())


def measure_batch(args, dev, stream):
    """The batched form: 4096 1D vdW shock tubes, lengths U{200..8000}, moving mesh, one persistent
    launch per K steps (mixed arithmetic).  The packed state (~2 GB) is larger than L2."""
    import torch

    from paper_2407_05568_gb300 import es
    from paper_2407_05568_gb300 import workloads as wl
    batch = wl.shock_tube_batch(nprob=args.batch_problems)
    b = es.es_batch_create(es.batch_params(batch["gas"]), batch["lengths"], stream)
    with torch.cuda.stream(stream):
        rho, v, p = (torch.tensor(a, dtype=torch.float64, device=dev) for a in wl.batch_fields(batch))
        es.es_batch_set_prim(b, rho, v, p)
    bt, probe_ms = es.es_batch_autotune(b)                # CTA shape: one probe step per shape
    es.es_batch_steps(b, args.batch_steps, 1e30)          # warm-up launch (captures the graph)
    if es.es_batch_check(b):
        raise RuntimeError("batched form: device status")
    st = torch.cuda.Event(enable_timing=True)
    en = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    st.record(stream)
    es.es_batch_steps(b, args.batch_steps, 1e30)
    en.record(stream)
    en.synchronize()
    if es.es_batch_check(b):
        raise RuntimeError("batched form: device status")
    ms = st.elapsed_time(en)
    cells = b.ntot * 3 * args.batch_steps
    from paper_2407_05568_gb300 import perfmodel
    _, f32 = measured_alu_peaks(es, stream)
    achieved = cells * perfmodel.flops_per_node_stage(1) / (ms * 1e-3) / 1e12
    roof = {"bound": "alu", "kernel": "batch_kernel", "achieved": achieved, "peak": f32, "unit": "TFLOP/s",
            "frac": achieved / f32, "ops_per_node_stage": perfmodel.flops_per_node_stage(1),
            "traffic": None, "launch_ms": ms,
            "peak_source": "measured in this run: es_selftest_peaks, FMA chains on every SM, best of 5 launches "
                           "(FP32); of measured"}
    return {"workload": f"{b.nprob} independent 1D vdW shock tubes, lengths U{{200..8000}} "
                        f"({b.ntot} nodes), moving mesh, one persistent launch per {args.batch_steps} steps",
            "value": cells / (ms * 1e-3), "unit": "cell-updates/s", "ms_per_launch": ms,
            "steps_per_launch": args.batch_steps, "nodes": b.ntot, "dtype": "f32",
            "autotune": {"threads_per_cta": bt, "probe_ms_128_256_512": probe_ms},
            "roofline": roof, "l2": "state (2 GB) larger than L2"}


def measure_large_stage(args, dev, stream):
    """The mixed stage kernel alone on the n x n vdW Riemann problem (the 200 x 200 recipe at n x n): shape from
    es_autotune, duration over 20 launches, against the measured FP32 rate."""
    from paper_2407_05568_gb300 import es
    n = args.large_n
    ctx, JU, J, x = es.setup_workload(workload(n), "mixed", dev, stream=stream)
    tile, tile_ms = es.es_autotune(ctx, JU, J, x)
    roof = stage_roofline(es, ctx, JU, J, x, stream, workload(n), n * n, "mixed", tile)
    roof["autotune_ms_per_shape"] = tile_ms
    mb = (JU.numel() + J.numel()) * 4 * 2 / 1e6
    return {"workload": f"2D vdW four-quadrant Riemann problem, {n}x{n} nodes, one RK stage (mixed form)",
            "roofline": roof, "l2": f"state {mb:.0f} MB in and out per launch; bound by the FP32 pipe, no flush"}


def measure_mesh(args, dev, stream):
    """The mesh redistribution alone (es_mesh_redistribute: monitor with G, 5 filter passes, 5 Jacobi sweeps,
    limiter, mesh velocity) on the n x n vdW Riemann problem, both forms, against the measured HBM copy rate with
    the kernel sequence's compulsory bytes (perfmodel.mesh_bytes_per_node).  The state is larger than L2."""
    import torch

    from paper_2407_05568_gb300 import es, perfmodel
    n = args.mesh_n
    w = workload(n)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm = peaks.get("hbm_gbs")
    source = "MEASURED_PEAKS.json hbm_gbs (STREAM-style copy); of measured"
    if hbm is None:
        hbm, source = 6800.0, "profiling recipe's fallback 6.8 TB/s; of fallback"
    m = w.get("mesh", {})
    passes, sweeps = m.get("filter_passes", 5), m.get("sweeps", 5)
    out = {"workload": f"mesh redistribution of the 2D vdW Riemann problem, {n}x{n} nodes, {passes} filter passes, "
                       f"{sweeps} Jacobi sweeps (es_mesh_redistribute)"}
    for prec in ("mixed", "fp64"):
        ctx, JU, J, x = es.setup_workload(w, prec, dev, stream=stream)
        with torch.cuda.stream(stream):
            xdot = torch.empty_like(x)
        dt, reps = 1e-4, 10
        for _ in range(3):
            es.es_mesh_redistribute(ctx, JU, J, x, dt, xdot, stats=False)
        st = torch.cuda.Event(enable_timing=True)
        en = torch.cuda.Event(enable_timing=True)
        launches0 = ctx.launches
        st.record(stream)
        for _ in range(reps):
            es.es_mesh_redistribute(ctx, JU, J, x, dt, xdot, stats=False)
        en.record(stream)
        launches = (ctx.launches - launches0) // reps
        en.synchronize()
        if es.es_check(ctx):
            raise RuntimeError(es.es_last_error(ctx))
        ms = st.elapsed_time(en) / reps
        bpn = perfmodel.mesh_bytes_per_node(prec, passes, sweeps)
        achieved = bpn * n * n / (ms * 1e-3) / 1e9
        out[prec] = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": None, "bytes_per_node": bpn, "ms_per_call": ms,
                     "gpu_launches_per_call": int(launches), "peak_source": source}
        del ctx, JU, J, x, xdot
        torch.cuda.empty_cache()
    return out


def _three_d_form(w, precision, args, dev, stream):
    """Whole steps through es_steps and the operator alone, for one precision form."""
    import torch

    from paper_2407_05568_gb300 import es
    ctx, JU, J, x = es.setup_workload(w, precision, dev, stream=stream)
    shape, shape_ms = es.es_autotune(ctx, JU, J, x)         # pencil shape of the direction kernels
    es.es_steps(ctx, JU, J, x, max(args.warmup, 1), w["t_end"])
    stream.synchronize()
    if es.es_check(ctx):
        raise RuntimeError(es.es_last_error(ctx))
    K = args.three_d_steps
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = ctx.launches
    e0.record(stream)
    es.es_steps(ctx, JU, J, x, K, w["t_end"])
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / K
    launches = (ctx.launches - launches0) // K
    if es.es_check(ctx):
        raise RuntimeError(es.es_last_error(ctx))
    # the operator alone (metrics, node fields, three direction kernels) on the current state
    with torch.cuda.stream(stream):
        xd = torch.zeros_like(x)
        dU, dJ = torch.empty_like(JU), torch.empty_like(J)
    for _ in range(2):
        es.es_rhs(ctx, JU, J, x, xd, dU, dJ)
    e0.record(stream)
    for _ in range(5):
        es.es_rhs(ctx, JU, J, x, xd, dU, dJ)
    e1.record(stream)
    e1.synchronize()
    ms_rhs = e0.elapsed_time(e1) / 5
    if es.es_check(ctx):
        raise RuntimeError(es.es_last_error(ctx))
    return ms, launches, ms_rhs, shape, list(shape_ms[:4])


def measure_three_d(args, dev, stream):
    """The 3D path: Example 5.6's 3D sine wave on the moving mesh at n^3 (smooth monitor, 20
    filter passes, 10 Jacobi sweeps), whole steps through es_steps and the operator alone, in
    the FP64 form and in the mixed form."""
    from paper_2407_05568_gb300 import workloads as wl
    n = args.three_d
    w = wl.sine_3d(n, moving=True)
    nodes = n ** 3
    pencils = {"fp64": {1: "16 nodes x 16 lines", 2: "16 nodes x 8 lines", 3: "16 nodes x 4 lines",
                        4: "32 nodes x 4 lines"},
               "mixed": {1: "16 nodes x 16 lines", 2: "32 nodes x 8 lines", 3: "16 nodes x 8 lines",
                         4: "32 nodes x 4 lines"}}
    out = {"workload": f"3D sine wave (Example 5.6 setup), periodic [0,1)^3, {n}^3 nodes, moving mesh "
                       "(smooth monitor alpha = (20, 15), 20 filter passes, 10 Jacobi sweeps), MR-WENO weights 1/3",
           "unit": "cell-updates/s"}
    for prec in ("fp64", "mixed"):
        ms, launches, ms_rhs, shape, shape_ms = _three_d_form(w, prec, args, dev, stream)
        r = {"value": nodes * 3 / (ms * 1e-3), "ms_per_step": ms, "steps": args.three_d_steps,
             "gpu_launches_per_step": launches, "operator_ms": ms_rhs,
             "operator_cell_updates_per_s": nodes / (ms_rhs * 1e-3),
             "pencil": pencils[prec][shape], "autotune_ms_per_shape": shape_ms}
        if prec == "fp64":
            out.update(precision_form="fp64", **r)
        else:
            out["mixed"] = dict(precision_form="mixed (f32 operator, double-float state)", **r)
    out["l2"] = f"working set {nodes * 8 * 66 / 1e9:.1f} GB (larger than L2); no flush"
    return out


def run_to_end(w, precision, dev, dt_fixed=0.0):
    """Advance a workload to its t_end with es_steps (graph replays); returns the density at the end
    (float64 numpy), the steps taken, the device time and the autotuned tile shape."""
    import torch

    from paper_2407_05568_gb300 import es
    ctx, JU, J, x = es.setup_workload(w, precision, dev, dt_fixed=dt_fixed)
    tile, _ = es.es_autotune(ctx, JU, J, x)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = 0
    es.es_steps(ctx, JU, J, x, 1, w["t_end"])        # capture the step graph
    steps += 1
    torch.cuda.synchronize()
    ms = 0.0
    t, dt = es.es_get_time(ctx)
    while t < w["t_end"] * (1 - 1e-14):
        k = max(1, min(2000, int((w["t_end"] - t) / max(dt, 1e-300)) + 1))
        e0.record()
        es.es_steps(ctx, JU, J, x, k, w["t_end"])
        e1.record()
        e1.synchronize()
        ms += e0.elapsed_time(e1)
        steps += k
        t, dt = es.es_get_time(ctx)
    if es.es_check(ctx):
        raise RuntimeError(es.es_last_error(ctx))
    if JU.dtype == torch.float64:
        rho = (JU[0] / J).cpu().numpy()
    else:
        rho = ((JU[0, 0].double() + JU[1, 0].double()) / (J[0].double() + J[1].double())).cpu().numpy()
    return rho, steps, ms, tile


def matched_error(rows, levels=(1e-4, 1e-5, 1e-6, 1e-7, 1e-8)):
    """Per target level of L1(rho) against the exact solution and per form, the smallest grid of
    a sweep that meets it, with its time to solution and throughput (None: no grid meets it)."""
    out = []
    for lv in levels:
        row = {"l1_level": lv}
        for prec in ("fp64", "mixed"):
            ok = [r for r in rows if r[prec]["l1_vs_exact"] <= lv]
            if not ok:
                row[prec] = None
                continue
            r = min(ok, key=lambda r: r["n"])
            row[prec] = {"n": r["n"], "time_to_solution_ms": r[prec]["ms"],
                         "cell_updates_per_s": r[prec]["cell_updates_per_s"]}
        if row["fp64"] and row["mixed"]:
            row["time_ratio_fp64_over_mixed"] = row["fp64"]["time_to_solution_ms"] / row["mixed"]["time_to_solution_ms"]
        out.append(row)
    return out


# the default line's matched-error comparison: the smallest grids of the two accuracy sweeps
QUICK_SWEEP = [("sine1d", 50), ("sine1d", 100), ("sine1d", 200), ("vortex", 128), ("vortex", 256)]


def measure_precision_sweep(args, dev, cases=None):
    """The precision form against the plain FP64 form: L1(rho) against the exact solution and
    against the FP64 run, throughput and time to solution, on the 1D sine wave (50 .. 1600 nodes,
    fixed mesh, dt = 0.4 dxi^(5/3), t = 0.1), the 2D sine wave (1024^2, t = 0.1) and the
    ideal-gas isentropic vortex (128^2 .. 2048^2 on the box of side 20, t = 1); then, per sweep, the smallest grid of
    each form that meets each error level (matched error)."""
    from paper_2407_05568_gb300 import workloads as wl
    out = []
    if cases is None:
        cases = ([("sine1d", n) for n in (50, 100, 200, 400, 800, 1600)] + [("sine2d", 1024)]
                 + [("vortex", n) for n in (128, 256, 512, 1024, 2048)])
    for name, n in cases:
        dt_fixed = 0.0
        if name == "sine1d":
            w = wl.sine_1d(n)
            dt_fixed = 0.4 * w["dxi"][0] ** (5.0 / 3.0)
            X = w["x"][0]
            exact = 0.5 + 0.2 * np.sin(2 * np.pi * (X - w["t_end"]))
        elif name == "sine2d":
            w = wl.sine_2d(n)
            X, Y = w["x"]
            exact = 0.5 + 0.2 * np.sin(2 * np.pi * (X + Y - w["t_end"]))
        else:
            w = wl.isentropic_vortex(n)
            X, Y = w["x"]
            exact = wl.vortex_density(X, Y, w["t_end"])
        nodes = int(np.prod(w["x"].shape[1:]))
        row = {"case": name, "n": n, "t_end": w["t_end"]}
        res = {}
        for prec in ("fp64", "mixed"):
            rho, steps, ms, tile = run_to_end(w, prec, dev, dt_fixed=dt_fixed)
            res[prec] = rho
            bx, by, _ = TILES[prec][tile] if w["dim"] == 2 else (254, 1, 256)
            row[prec] = {"l1_vs_exact": float(np.abs(rho - exact).mean()), "steps": steps, "ms": ms,
                         "cell_updates_per_s": nodes * 3 * (steps - 1) / (ms * 1e-3) if ms > 0 else None,
                         "tile": f"{bx}x{by}"}
        row["mixed_rel_l1_vs_fp64"] = float(np.abs(res["mixed"] - res["fp64"]).sum() / np.abs(res["fp64"]).sum())
        out.append(row)
    matched = {}
    for case in ("sine1d", "vortex"):
        rows = [r for r in out if r["case"] == case]
        for a, b in zip(rows, rows[1:]):
            for prec in ("fp64", "mixed"):
                b[prec]["order_vs_previous"] = float(np.log2(a[prec]["l1_vs_exact"] / b[prec]["l1_vs_exact"]))
        if rows:
            matched[case] = matched_error(rows)
    return {"runs": out, "matched_error": matched}


# Table 5.3: the paper's CPU times (4 Xeon E5-2697A v4 cores) of Example 5.4, in seconds
TABLE_5_3 = {"P1": {"MM": 233, "MM1": 199, "UM": 37, "UM600": 657}, "D1": {"MM": 240, "MM1": 217, "UM": 47, "UM600": 789}}


def measure_mach(args, dev):
    """Example 5.4's Mach reflection (one reading of its geometry, see workloads.mach_reflection), FP64:
    MM, MM1 and UM on 200 x 100 and UM on 600 x 300, each advanced to its final time through es_steps;
    time to solution beside the paper's CPU times (context: other hardware, and for P1 another final
    time)."""
    from paper_2407_05568_gb300 import workloads as wl
    out = {}
    for case in ("P1", "D1"):
        rows = {}
        for variant, (n1, n2) in (("MM", (200, 100)), ("MM1", (200, 100)), ("UM", (200, 100)), ("UM600", (600, 300))):
            w = wl.mach_reflection(case, n1, n2, "UM" if variant == "UM600" else variant)
            _, steps, ms, tile = run_to_end(w, "fp64", dev)
            rows[variant] = {"grid": f"{n1}x{n2}", "steps": steps, "time_to_solution_ms": ms,
                             "cell_updates_per_s": n1 * n2 * 3 * (steps - 1) / (ms * 1e-3) if ms > 0 else None,
                             "paper_cpu_s": TABLE_5_3[case][variant]}
        out[case] = {"t_end": float(wl.mach_reflection(case, 8, 8, "UM")["t_end"]), "runs": rows}
    return out


def measure_learned(args, dev):
    """The learned warm start on the 2D vdW Riemann problem: snapshots of plain runs (Jacobi to
    max change < 0.02 cells, at most 300 sweeps), training, and the plain against the
    warm-started solve on held-out seeds (same states, then two full runs)."""
    import time

    import torch

    from paper_2407_05568_gb300 import learned
    n, eps, mu = args.learned_n, 0.02, 300
    seeds = list(range(100, 100 + args.learned_seeds))
    train_seeds, test_seeds = seeds[:-2], seeds[-2:]
    t0 = time.perf_counter()
    feats, tgts, sw = learned.snapshots(train_seeds, n, args.learned_steps, eps, mu, device=dev)
    torch.cuda.synchronize()
    t_snap = time.perf_counter() - t0
    net = learned.WarmStartNet(hidden=32, layers=4, seed=0, in_scale=learned.feature_scale(feats), device=dev)
    t0 = time.perf_counter()
    hist = learned.train(net, feats, tgts, epochs=args.learned_epochs, batch=4, lr=2e-3, lr_final=1e-4)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    iters = args.learned_epochs * (feats.shape[0] // 4)
    del feats, tgts
    torch.cuda.empty_cache()
    # inference time of the network alone (four conv launches on one n x n image): the tensor-core
    # path the solver uses, and the FP32 CUDA-core forward of the training path
    x = torch.zeros((1, 4, n, n), dtype=torch.float32, device=dev)
    t_inf = {}
    for name, fn in (("tensor_cores_bf16_inputs", net.infer), ("cuda_cores_fp32", net.forward)):
        for _ in range(3):
            fn(x)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(20):
            fn(x)
        e1.record()
        torch.cuda.synchronize()
        t_inf[name] = e0.elapsed_time(e1) / 20
    cmp = learned.compare_solves(net, test_seeds, n, args.learned_steps, eps, mu, device=dev)
    run = learned.compare_runs(net, test_seeds[0], n, args.learned_steps, eps, mu, device=dev)
    # matched accuracy: both solves against the converged mesh of the same states, then full runs with the plain
    # tolerance that gives the plain solve the warm solve's mean distance to it
    tols = [float(t) for t in args.learned_tols.split(",")]
    mres, ref_sw = learned.compare_matched(net, test_seeds, n, args.learned_steps, tols, mu, device=dev)
    per_tol = {str(t): {k: float(v.mean()) for k, v in r.items()} | {"dist_plain_max_max": float(r["dist_plain_max"].max()),
                                                                     "dist_warm_max_max": float(r["dist_warm_max"].max())}
               for t, r in mres.items()}
    matched = {"reference": f"Jacobi from x^n to a change below 1e-5 cells (at most 20000 sweeps; "
                            f"mean {ref_sw.mean():.0f}, max {ref_sw.max()} sweeps)",
               "per_tolerance": per_tol}
    dw = float(mres[tols[0]]["dist_warm_mean"].mean())
    at = learned.plain_at(mres, dw)
    if at is not None:
        tol_p, sw_p = at
        matched["warm_at_training_tolerance"] = {"tolerance": tols[0], "dist_mean": dw,
                                                 "sweeps_warm": float(mres[tols[0]]["sweeps_warm"].mean()),
                                                 "plain_tolerance_at_same_dist": tol_p, "sweeps_plain_at_same_dist": sw_p}
        matched["full_runs"] = learned.compare_runs(net, test_seeds[0], n, args.learned_steps, tol_p, mu,
                                                    device=dev, eps_warm=tols[0])
    return {"workload": f"2D vdW Riemann problem {n}x{n}, moving mesh, Jacobi to max change < {eps} cells "
                        f"(at most {mu} sweeps); network 4 conv3x3 layers, 32 channels, bf16 weights",
            "snapshots": int(len(sw)), "train_seeds": f"{train_seeds[0]}..{train_seeds[-1]}",
            "test_seeds": test_seeds, "steps_per_seed": args.learned_steps,
            "snapshot_seconds": t_snap, "train_seconds": t_train, "train_iterations": iters,
            "loss_first_epoch": hist[0], "loss_last_epoch": hist[-1],
            "guard_ratio": learned.GUARD_RATIO,
            "same_states": {"sweeps_plain": float(cmp["sweeps_plain"].mean()),
                            "sweeps_warm": float(cmp["sweeps_warm"].mean()),
                            "sweeps_saved_frac": float(1 - cmp["sweeps_warm"].mean() / cmp["sweeps_plain"].mean()),
                            "warm_kept_frac": float(cmp["picked"].mean()),
                            "mesh_dev_cells_max": float(cmp["dev_cells"].max()),
                            "mesh_dev_cells_mean": float(cmp["dev_cells"].mean())},
            "full_runs": run, "matched_accuracy": matched, "nn_inference_ms": t_inf}


def measure_nn_inference(n, dev):
    """The warm-start network (4 conv3x3 layers, 32 channels, seeded weights) on one n x n feature
    image: tensor-core path and FP32 CUDA-core path, CUDA events over 20 inferences."""
    import torch

    from paper_2407_05568_gb300 import learned
    net = learned.WarmStartNet(hidden=32, layers=4, seed=0, device=dev)
    g = torch.Generator(device="cpu").manual_seed(0)
    x = torch.randn((1, 4, n, n), generator=g).to(dev)
    res = {"n": n, "flops_per_inference": 2 * 9 * (4 * 32 + 32 * 32 * 2 + 32 * 2) * n * n}
    for name, fn in (("tensor_cores_bf16_inputs", net.infer), ("cuda_cores_fp32", net.forward)):
        for _ in range(3):
            fn(x)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(20):
            fn(x)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 20
        res[name] = {"ms": ms, "tflops": res["flops_per_inference"] / (ms * 1e-3) / 1e12}
    return res


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2407_05568_gb300 import build
    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    stream = torch.cuda.Stream(device=dev)
    nodes = args.n * args.n
    main_form = measure_form(args, args.precision, dev, stream, world)
    other = None
    if not args.no_chosen and args.precision == "fp64":
        other = measure_form(args, "mixed", dev, stream, world)
    batched = None
    if args.batch_problems > 0 and rank == 0:
        batched = measure_batch(args, dev, stream)
    three_d = measure_three_d(args, dev, stream) if args.three_d > 0 and rank == 0 else None
    large = measure_large_stage(args, dev, stream) if args.large_n > 0 and rank == 0 else None
    mesh_res = measure_mesh(args, dev, stream) if args.mesh_n > 0 and rank == 0 else None
    learned_res = measure_learned(args, dev) if args.learned and rank == 0 else None
    sweep_res = measure_precision_sweep(args, dev) if args.precision_sweep and rank == 0 else None
    quick = None
    if sweep_res is None and not args.no_matched_error and rank == 0:
        quick = measure_precision_sweep(args, dev, QUICK_SWEEP)
    nn_res = measure_nn_inference(args.nn_inference, dev) if args.nn_inference > 0 and rank == 0 else None
    mach_res = measure_mach(args, dev) if args.mach_reflection and rank == 0 else None
    if rank == 0:
        m = main_form
        line = {"metric": METRIC, "value": m["value"], "unit": "cell-updates/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": m["ms"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32",
                "data": "synthetic", "config": config(args.n, args.precision,
                                                      "flushed before each timed step (512 MB write)"),
                "roofline": m["roof"], "clocks": m["clocks"], "gpu_launches": m["launches"],
                "e2e": {"value": m["e2e"], "unit": "cell-updates/s", "h2d_bytes_per_step": m["io_bytes"],
                        "d2h_bytes_per_step": m["io_bytes"]}}
        if other is not None:
            ref = m["state"]
            diff = float(np.abs(other["state"] - ref).sum() / np.abs(ref).sum())
            line["chosen"] = {"form": "mixed (FP32 pipe, compensated-float state)", "value": other["value"],
                              "unit": "cell-updates/s", "ms_per_step": other["ms"],
                              "speedup_vs_fp64": other["value"] / m["value"],
                              "rel_l1_vs_fp64_same_steps": diff,
                              "steps_compared": min(args.steps, RESTART_EVERY),
                              "roofline": other["roof"], "gpu_launches": other["launches"],
                              "e2e": {"value": other["e2e"], "unit": "cell-updates/s"}}
        if batched is not None:
            line["batched"] = batched
        if three_d is not None:
            line["three_d"] = three_d
        if large is not None:
            line["chosen_large"] = large
        if mesh_res is not None:
            line["mesh"] = mesh_res
        if learned_res is not None:
            line["learned"] = learned_res
        if sweep_res is not None:
            line["precision_sweep"] = sweep_res
            line["matched_error"] = sweep_res["matched_error"]
        elif quick is not None:
            # the metric's comparison at matched L1(rho) against the exact solution: per level, the
            # smallest grid of each form that reaches it and its time to solution (to t_end)
            line["matched_error"] = dict(quick["matched_error"],
                                         cases="1D sine 50/100/200 nodes to t = 0.1 (dt = 0.4 dxi^(5/3)), "
                                               "ideal-gas isentropic vortex 128^2/256^2 (box of side 20) to t = 1, both forms")
        if nn_res is not None:
            line["nn_inference"] = nn_res
        if mach_res is not None:
            line["mach_reflection"] = mach_res
        if not args.no_cpu_baseline:
            sec, k = time_oracle(workload(args.n), 24)
            line["cpu_baseline"] = {"value": nodes * 3 * k / sec, "unit": "cell-updates/s", "cores": cpu_cores(),
                                    "kind": "oracle",
                                    "sample": f"{k} full steps of the same {args.n}x{args.n} workload from t = 0"}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def pin(a):
    import torch
    t = torch.from_numpy(a).pin_memory()
    return t.numpy()


# (nodes along xi_1, along xi_2, threads) of each tile shape; the mixed 384- and 320-thread shapes give two lanes
# to each face
TILES = {"fp64": {1: (32, 8, 288), 2: (25, 11, 384), 3: (16, 16, 288), 4: (32, 12, 416), 5: (20, 10, 224)},
         "mixed": {1: (20, 8, 384), 2: (25, 6, 192), 3: (20, 8, 192), 4: (20, 14, 608), 5: (16, 8, 160)}}
# dram__bytes_read.sum + dram__bytes_write.sum per launch at 200 x 200, from one ncu capture of each
# kernel as it is now (a kernel changed since its capture has no entry); other sizes were not captured
TRAFFIC_200 = {"stage_kernel_fp64<2,25,11,384>": 3032064 + 0}


def stage_roofline(es, ctx, JU, J, x, stream, w, nodes, precision, tile):
    """Mean device time of the stage kernel (stage 2 form) over 20 back-to-back launches, timed by the library
    with CUDA events on the bench stream (es_time_stage: no host work between the launches)."""
    ms = es.es_time_stage(ctx, JU, J, x, stage=2, dt=1e-4, reps=20)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    from paper_2407_05568_gb300 import perfmodel
    flops = perfmodel.stage_flops(dim=2, nodes=nodes, precision=precision)
    f64, f32 = measured_alu_peaks(es, stream)
    peak = f64 if precision == "fp64" else f32
    nominal = perfmodel.fp64_peak_tflops(peaks) if precision == "fp64" else perfmodel.fp32_peak_tflops(peaks)
    achieved = flops / (ms * 1e-3) / 1e12
    bx, by, nt = TILES[precision][tile]
    kname = ("stage_kernel_fp64" if precision == "fp64" else "stage_kernel_mixed") + f"<2,{bx},{by},{nt}>"
    return {"bound": "alu", "kernel": kname, "tile": f"{bx}x{by}/{nt}",
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": TRAFFIC_200.get(kname) if nodes == 200 * 200 else None, "launch_ms": ms,
            "flops_per_launch": flops,
            "peak_source": ("measured in this run: es_selftest_peaks, FMA chains on every SM, best of 5 launches "
                            f"({'FP64' if precision == 'fp64' else 'FP32'}); of measured"),
            "nominal_peak": nominal}


_PEAKS = None


def measured_alu_peaks(es, stream):
    """(FP64, FP32) TFLOP/s of this GPU from the library's FMA-chain probe, measured once per run."""
    global _PEAKS
    if _PEAKS is None:
        _PEAKS = es.es_selftest_peaks(stream)
    return _PEAKS


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
