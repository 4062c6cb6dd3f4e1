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
