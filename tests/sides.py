"""Test helpers: build the same seeded problem on the oracle side and on the CUDA side.

Each side converts the generator's primitive fields with its own arithmetic;
nothing computed by one side is fed to the other.
"""
import numpy as np

from oracle import operator as op
from oracle import stepper, thermo


def oracle_setup(w, dissipation=True, x=None):
    g = thermo.Gas(**w["gas"])
    sch = op.Scheme(gas=g, dim=w["dim"], bc=tuple(w["bc"]), dxi=tuple(w["dxi"]), period=tuple(w["period"]),
                    dissipation=dissipation, weno_gammas=tuple(w.get("weno_gammas", (0.005, 0.045, 0.95))))
    x = w["x"] if x is None else x
    J = op.node_jacobian(sch, x)
    JU = thermo.prim_to_cons(g, w["rho"], w["v"], w["p"]) * J
    mc = stepper.MeshControl(moving=bool(w.get("moving", False)), **w.get("mesh", {}))
    return sch, mc, JU, J, x


def gpu_setup(w, precision="fp64", dissipation=True, x=None, dt_fixed=0.0):
    import torch

    from paper_2407_05568_gb300 import es
    dev = torch.device("cuda:0")
    p = es.make_params(w, precision=precision, dissipation=dissipation, dt_fixed=dt_fixed)
    ctx = es.es_create(p)
    x = w["x"] if x is None else x
    xt = torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device=dev)
    J = es.state_empty(ctx, x.shape[1:], dev)
    es.es_init_mesh(ctx, xt, J)
    rho = torch.tensor(w["rho"], dtype=torch.float64, device=dev)
    v = torch.tensor(np.ascontiguousarray(w["v"]), dtype=torch.float64, device=dev)
    pr = torch.tensor(w["p"], dtype=torch.float64, device=dev)
    JU = es.state_empty(ctx, (w["dim"] + 2,) + x.shape[1:], dev)
    es.es_prim_to_cons(ctx, rho, v, pr, J, JU)
    return ctx, JU, J, xt


def rel_l1(a, b):
    """sum |a - b| / sum |b|."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).sum() / max(np.abs(b).sum(), 1e-300))


def to_np(t):
    """float64 numpy values of a state tensor (mixed form: hi plane + lo plane)."""
    a = t.detach().cpu()
    if a.dtype == torch_float32():
        return a[0].double().numpy() + a[1].double().numpy()
    return a.double().numpy()


def torch_float32():
    import torch
    return torch.float32


def batch_trajectory(args):
    """The oracle's states (JU, J, x_1, t) at every step of problem k of a shock-tube batch, from t = 0 to t_end
    (a process-pool worker: its arguments and result are plain arrays)."""
    batch, k, t_end = args
    from paper_2407_05568_gb300 import workloads as wl
    w = wl.batch_problem(batch, k)
    sch, mc, JU, J, x = oracle_setup(w)
    t = 0.0
    traj = [(JU, J, x[0], t)]
    while t < t_end * (1.0 - 1e-14):
        JU, J, x, t, _ = stepper.step(sch, mc, JU, J, x, t, t_end, w["cfl"])
        traj.append((JU, J, x[0], t))
    return traj


def batch_trajectories(batch, t_end):
    """batch_trajectory for every problem, in a pool of fresh interpreters (spawned: safe beside a CUDA context)."""
    import multiprocessing as mp
    import os
    jobs = [(batch, k, t_end) for k in range(batch["lengths"].size)]
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        return pool.map(batch_trajectory, jobs)


def riemann_perturbed_final(args):
    """Final state (JU, J, x) of an Example 5.2 oracle run whose initial JU is perturbed by `size` (relative,
    seeded normal); a process-pool worker."""
    name, variant, n, size, seed = args
    import numpy as np
    from paper_2407_05568_gb300 import workloads as wl
    w = wl.riemann_1d(name, n=n, moving=variant != "UM")
    if variant == "MM1":
        w = wl.mm1(w)
    sch, mc, JU, J, x = oracle_setup(w)
    if size > 0.0:
        JU = JU * (1.0 + size * np.random.default_rng(seed).standard_normal(JU.shape))
    JU, J, x, _ = stepper.run(sch, mc, JU, J, x, w["t_end"], w["cfl"])
    return JU, J, x


def pool_map(fn, jobs):
    """fn over jobs in a pool of fresh interpreters (spawned: safe beside a CUDA context)."""
    import multiprocessing as mp
    import os
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1, len(jobs))) as pool:
        return pool.map(fn, jobs)
