"""Parity at the benchmark configurations' full sizes, in the launch configurations the
bench times (autotuned tiles, graph-replayed steps, the persistent batched launch).

Where the oracle cannot finish a full-size case in seconds (the 1024^2 sine step takes
about 100 s), the check is on a sample or on a property: the FP64 path at 256^2 on the
same code path against the oracle, and the mixed form at 1024^2 against the FP64 path.
"""
import numpy as np
import pytest

from oracle import stepper, warmstart
from paper_2407_05568_gb300 import workloads as wl

from sides import gpu_setup, oracle_setup, rel_l1, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_05568_gb300 import build
    build.build()


def _gpu_steps(w, precision, nsteps):
    from paper_2407_05568_gb300 import es
    ctx, JU, J, xt = gpu_setup(w, precision=precision)
    es.es_set_time(ctx, 0.0)
    es.es_steps(ctx, JU, J, xt, nsteps, w["t_end"])
    assert es.es_check(ctx) == 0, es.es_last_error(ctx)
    return to_np(JU), to_np(J), to_np(xt)


def _oracle_steps(w, nsteps):
    sch, mc, JU, J, x = oracle_setup(w)
    t = 0.0
    for _ in range(nsteps):
        JU, J, x, t, _ = stepper.step(sch, mc, JU, J, x, t, w["t_end"], w["cfl"])
    return JU, J, x


def test_bench_workload_mixed_one_step():
    """The bench's chosen form on its workload (200^2 moving-mesh Riemann problem, seed 5)."""
    w = wl.riemann_2d(200, seed=5)
    JU, J, x = _gpu_steps(w, "mixed", 1)
    JUo, Jo, xo = _oracle_steps(w, 1)
    assert rel_l1(JU, JUo) < 2e-6, rel_l1(JU, JUo)
    assert rel_l1(J, Jo) < 1e-6
    assert rel_l1(x, xo) < 1e-6


def test_sine_256_fp64_one_step():
    """The precision config's FP64 path (periodic sine wave, fixed mesh) at 256^2 against the oracle."""
    w = wl.sine_2d(256)
    JU, J, x = _gpu_steps(w, "fp64", 1)
    JUo, Jo, xo = _oracle_steps(w, 1)
    assert rel_l1(JU, JUo) < 1e-12
    assert rel_l1(J, Jo) < 1e-13


def test_sine_1024_mixed_against_fp64():
    """At the precision config's full size (1024^2) the mixed form stays within 1e-6 of the FP64 path
    after 5 steps (the FP64 path is pinned to the oracle per step at every smaller size)."""
    w = wl.sine_2d(1024)
    JU64, _, _ = _gpu_steps(w, "fp64", 5)
    JU32, _, _ = _gpu_steps(w, "mixed", 5)
    assert rel_l1(JU32, JU64) < 1e-6, rel_l1(JU32, JU64)


def test_batch_full_size_sampled():
    """The batched config at full size (4096 tubes, 16.8 M nodes, autotuned CTA shape), two steps;
    the longest, the shortest and six seeded problems checked one by one against the oracle."""
    import torch

    from paper_2407_05568_gb300 import es
    dev = torch.device("cuda:0")
    batch = wl.shock_tube_batch()
    b = es.es_batch_create(es.batch_params(batch["gas"]), batch["lengths"])
    rho, v, p = (torch.tensor(a, dtype=torch.float64, device=dev) for a in wl.batch_fields(batch))
    es.es_batch_set_prim(b, rho, v, p)
    es.es_batch_autotune(b)
    es.es_batch_steps(b, 2, 1e30)
    assert es.es_batch_check(b) == 0
    JU = torch.empty((3, b.ntot), dtype=torch.float64, device=dev)
    J = torch.empty(b.ntot, dtype=torch.float64, device=dev)
    x = torch.empty(b.ntot, dtype=torch.float64, device=dev)
    es.es_batch_get(b, JU, J, x)
    JU, J, x = JU.cpu().numpy(), J.cpu().numpy(), x.cpu().numpy()
    L = np.asarray(batch["lengths"])
    rng = np.random.default_rng(2024)
    picks = {int(np.argmax(L)), int(np.argmin(L))} | set(int(k) for k in rng.choice(L.size, 6, replace=False))
    offs = np.concatenate([[0], np.cumsum(L)[:-1]])
    for k in sorted(picks):
        w = wl.batch_problem(batch, k)
        sch, mc, JUo, Jo, xo = oracle_setup(w)
        t = 0.0
        for _ in range(2):
            JUo, Jo, xo, t, _ = stepper.step(sch, mc, JUo, Jo, xo, t, 1e30, 0.4)
        sl = slice(offs[k], offs[k] + L[k])
        assert rel_l1(JU[:, sl], JUo) < 1e-4, (k, rel_l1(JU[:, sl], JUo))
        assert rel_l1(x[sl], xo[0]) < 1e-6


def test_learned_config_features_and_solve_512():
    """The learned config at full size (512^2 Riemann problem, Jacobi to 0.02 cells, at most 64
    sweeps): the features and the plain mesh solve against the oracle at t = 0."""
    import torch

    from paper_2407_05568_gb300 import es
    w = wl.riemann_2d(512, seed=118)
    w["mesh"] = dict(w["mesh"], sweeps=64, eps=0.02 * w["dxi"][0])
    sch, mc, JU_o, J_o, x = oracle_setup(w)
    ctx, JU, J, xt = gpu_setup(w)
    feat = torch.empty((4,) + x.shape[1:], dtype=torch.float32, device="cuda")
    es.es_mesh_features(ctx, JU, J, xt, feat)
    ref = warmstart.features(sch, mc, JU_o, J_o, x)
    f = feat.double().cpu().numpy()
    for c in range(4):
        assert np.abs(f[c] - ref[c]).max() <= 1e-6 * max(1.0, np.abs(ref[c]).max()), c
    xo, ko, _ = warmstart.solve(sch, mc, JU_o, J_o, x)
    xg = torch.empty_like(xt)
    kg, _ = es.es_mesh_solve(ctx, JU, J, xt, None, xg)
    assert kg == ko
    assert np.abs(xg.cpu().numpy() - xo).max() <= 1e-12 * w["dxi"][0] * ko
