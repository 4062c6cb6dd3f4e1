"""The learned warm start on the GPU against the oracle: the network kernels
(forward, backward, MSE, Adam), the features, the warm start and the guarded
mesh solve, and a training run that shows what the network saves.

Tolerances: the network runs in FP32 with bf16 weights; the oracle evaluates the
same bf16 weights in float64, so a layer agrees to a few FP32 roundings of its
largest partial sums (<= 2e-5 of the output scale for 288-term sums).  The mesh
solve is FP64 on both sides (<= 1e-12 cells)."""
import numpy as np
import pytest

from oracle import convnet, mesh, stepper, warmstart
from paper_2407_05568_gb300 import workloads as wl

from sides import gpu_setup, oracle_setup
from test_gpu_parity import _ragged_riemann

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_05568_gb300 import build
    build.build()


def _t(a, dtype="float32"):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=getattr(torch, dtype), device="cuda")


def _bf16_weights(rng, shape, scale):
    """Seeded weights already on the bf16 grid (float64 values), and the bf16 device tensor."""
    w = convnet.bf16_round((rng.standard_normal(shape) * scale).astype(np.float32))
    return w, _t(w, "bfloat16")


def _np(t):
    return t.detach().double().cpu().numpy()


@pytest.mark.parametrize("cin,cout,act", [(4, 32, True), (32, 32, True), (32, 2, False), (2, 4, False)])
def test_conv_forward_vs_oracle(cin, cout, act):
    import torch

    from paper_2407_05568_gb300 import es
    rng = np.random.default_rng(10 + cin + cout)
    B, H, W = 2, 37, 50                               # several 16-pixel tiles and ragged tails
    a = rng.standard_normal((B, cin, H, W)).astype(np.float32)
    w, wt = _bf16_weights(rng, (cout, cin, 3, 3), 1.0 / np.sqrt(9 * cin))
    b = rng.standard_normal(cout).astype(np.float32) * 0.1
    out = torch.empty((B, cout, H, W), dtype=torch.float32, device="cuda")
    ws = torch.empty(es.es_nn_workspace_bytes(B, cin, cout, H, W) // 4 + 1, dtype=torch.float32, device="cuda")
    es.es_nn_conv_forward(_t(a), wt, _t(b), out, act, ws)
    torch.cuda.synchronize()
    z = convnet.conv3x3(a.astype(np.float64), w, b.astype(np.float64))
    ref = np.tanh(z) if act else z
    scale = np.abs(z).max()
    assert np.abs(_np(out) - ref).max() <= 2e-5 * scale


@pytest.mark.parametrize("cin,cout,act", [(4, 32, True), (32, 32, True), (32, 2, False), (2, 4, False)])
def test_conv_forward_tensor_cores_vs_oracle(cin, cout, act):
    """The inference layer on the tensor cores: the correlation of the bf16-rounded input with bf16
    weights, FP32 accumulation (several 16 x 16 tiles and ragged tails, batch of 2)."""
    import torch

    from paper_2407_05568_gb300 import es
    rng = np.random.default_rng(30 + cin + cout)
    B, H, W = 2, 37, 50
    a = rng.standard_normal((B, cin, H, W)).astype(np.float32)
    w, wt = _bf16_weights(rng, (cout, cin, 3, 3), 1.0 / np.sqrt(9 * cin))
    b = rng.standard_normal(cout).astype(np.float32) * 0.1
    out = torch.empty((B, cout, H, W), dtype=torch.float32, device="cuda")
    es.es_nn_conv_forward_bf16(_t(a), wt, _t(b), out, act)
    torch.cuda.synchronize()
    z = convnet.conv3x3(convnet.bf16_round(a), w, b.astype(np.float64))
    ref = np.tanh(z) if act else z
    assert np.abs(_np(out) - ref).max() <= 2e-5 * np.abs(z).max()


@pytest.mark.parametrize("cin,cout,act", [(4, 32, True), (32, 32, True), (32, 2, False)])
def test_conv_backward_vs_oracle(cin, cout, act):
    import torch

    from paper_2407_05568_gb300 import es
    rng = np.random.default_rng(20 + cin + cout)
    B, H, W = 3, 33, 21
    a = rng.standard_normal((B, cin, H, W)).astype(np.float32)
    w, wt = _bf16_weights(rng, (cout, cin, 3, 3), 1.0 / np.sqrt(9 * cin))
    b = np.zeros(cout, dtype=np.float32)
    go = rng.standard_normal((B, cout, H, W)).astype(np.float32)
    dev = "cuda"
    out = torch.empty((B, cout, H, W), dtype=torch.float32, device=dev)
    ws = torch.empty(es.es_nn_workspace_bytes(B, cin, cout, H, W) // 4 + 1, dtype=torch.float32, device=dev)
    es.es_nn_conv_forward(_t(a), wt, _t(b), out, act, ws)
    g = _t(go)
    gin = torch.empty((B, cin, H, W), dtype=torch.float32, device=dev)
    gw = torch.empty((cout, cin, 3, 3), dtype=torch.float32, device=dev)
    gb = torch.empty(cout, dtype=torch.float32, device=dev)
    es.es_nn_conv_backward(_t(a), wt, out, g, gin, gw, gb, act, ws)
    torch.cuda.synchronize()
    z = convnet.conv3x3(a.astype(np.float64), w)
    gz = go * (1.0 - np.tanh(z) ** 2) if act else go.astype(np.float64)
    rw, rb, ra = convnet.conv3x3_backward(a.astype(np.float64), w, gz)
    n_terms = B * H * W
    for got, ref, terms in ((_np(gw), rw, n_terms), (_np(gb), rb, n_terms), (_np(gin), ra, 9 * cout)):
        tol = 4e-7 * np.sqrt(terms) * np.abs(ref).max() + 1e-6 * np.abs(ref).max()
        assert np.abs(got - ref).max() <= tol, (np.abs(got - ref).max(), tol)


def test_backward_is_deterministic():
    """The weight gradient is reduced over tiles in a fixed order: two calls agree bit for bit."""
    import torch

    from paper_2407_05568_gb300 import es
    rng = np.random.default_rng(5)
    B, H, W, cin, cout = 2, 64, 48, 32, 32
    a = _t(rng.standard_normal((B, cin, H, W)))
    _, wt = _bf16_weights(rng, (cout, cin, 3, 3), 0.06)
    ws = torch.empty(es.es_nn_workspace_bytes(B, cin, cout, H, W) // 4 + 1, dtype=torch.float32, device="cuda")
    g0 = rng.standard_normal((B, cout, H, W))
    res = []
    for _ in range(2):
        g = _t(g0)
        gw = torch.empty((cout, cin, 3, 3), dtype=torch.float32, device="cuda")
        gb = torch.empty(cout, dtype=torch.float32, device="cuda")
        es.es_nn_conv_backward(a, wt, None, g, None, gw, gb, False, ws)
        res.append((gw.clone(), gb.clone()))
    assert torch.equal(res[0][0], res[1][0]) and torch.equal(res[0][1], res[1][1])


def test_mse_and_adam_vs_oracle():
    import torch

    from paper_2407_05568_gb300 import es
    rng = np.random.default_rng(6)
    p = rng.standard_normal(10007).astype(np.float32)
    t = rng.standard_normal(10007).astype(np.float32)
    grad = torch.empty(10007, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    es.es_nn_mse(_t(p), _t(t), grad, loss)
    L, g = convnet.mse(p, t)
    assert abs(loss.item() - L) <= 1e-5 * L
    assert np.abs(_np(grad) - g).max() <= 1e-6 * np.abs(g).max()
    # three Adam steps from given gradients
    th = rng.standard_normal(4099).astype(np.float32)
    gs = [rng.standard_normal(4099).astype(np.float32) for _ in range(3)]
    master = _t(th)
    wb = torch.empty(4099, dtype=torch.bfloat16, device="cuda")
    m = torch.zeros(4099, dtype=torch.float32, device="cuda")
    v = torch.zeros_like(m)
    thr, mr, vr = th.astype(np.float64), np.zeros(4099), np.zeros(4099)
    for k, gk in enumerate(gs, start=1):
        es.es_nn_adam(master, wb, _t(gk), m, v, 1e-3, 0.9, 0.999, 1e-8, k)
        thr, mr, vr = convnet.adam(thr, gk.astype(np.float64), mr, vr, k, 1e-3)
    torch.cuda.synchronize()
    assert np.abs(_np(master) - thr).max() <= 1e-6 * np.abs(thr).max()
    assert np.abs(_np(m) - mr).max() <= 1e-6 * np.abs(mr).max()
    # the bf16 copy is the master rounded to nearest even
    assert np.array_equal(_np(wb), convnet.bf16_round(master.cpu().numpy()))


# ------------------------------------------------------------------ mesh side
def _riemann(n1=70, n2=45, sweeps=30, eps_cells=0.02):
    """Ragged 2D Riemann problem (n1 x n2 nodes), Jacobi to eps_cells cells or `sweeps`."""
    w = _ragged_riemann(n1, n2, seed=5)
    w["mesh"] = dict(w["mesh"], sweeps=sweeps, eps=eps_cells * w["dxi"][0])
    return w


def test_features_vs_oracle():
    import torch

    from paper_2407_05568_gb300 import es
    w = _riemann()
    sch, mc, JU_o, J_o, x = oracle_setup(w)
    ctx, JU, J, xt = gpu_setup(w)
    feat = torch.empty((4,) + x.shape[1:], dtype=torch.float32, device="cuda")
    es.es_mesh_features(ctx, JU, J, xt, feat)
    ref = warmstart.features(sch, mc, JU_o, J_o, x)
    for c in range(4):
        assert np.abs(_np(feat[c]) - ref[c]).max() <= 1e-6 * max(1.0, np.abs(ref[c]).max()), c


def test_warm_start_kernel_vs_oracle():
    import torch

    from paper_2407_05568_gb300 import es
    w = _riemann()
    sch, mc, JU_o, J_o, x = oracle_setup(w)
    ctx, JU, J, xt = gpu_setup(w)
    rng = np.random.default_rng(8)
    out = (rng.standard_normal(x.shape) * 0.3).astype(np.float32)
    out[1, 4, 7] = np.nan
    out[0, 9, 2] = np.inf
    xs = torch.empty_like(xt)
    es.es_mesh_warm_start(ctx, xt, _t(out), xs)
    ref = warmstart.warm_start(sch, x, out.astype(np.float64))
    assert np.abs(_np(xs) - ref).max() <= 4e-16 * np.abs(ref).max()   # dxi o vs o / (1/dxi): an ulp


@pytest.mark.parametrize("start,ratio", [("none", 1.0), ("good", 1.0), ("bad", 1.0), ("bad", 4.0),
                                         ("noisy", 1.0), ("noisy", 4.0)])
def test_mesh_solve_vs_oracle(start, ratio):
    import torch

    from paper_2407_05568_gb300 import es
    w = _riemann()
    sch, mc, JU_o, J_o, x = oracle_setup(w)
    ctx, JU, J, xt = gpu_setup(w)
    x_start = None
    if start == "good":
        om, _ = warmstart.filtered_monitor(sch, mc, JU_o, J_o)
        x_start, _ = mesh.jacobi(sch, x, om, 12)          # a start partway along the plain path
    elif start == "bad":
        rng = np.random.default_rng(9)
        x_start = warmstart.warm_start(sch, x, rng.standard_normal(x.shape) * 0.4)
    elif start == "noisy":                               # the good start with small grid-scale noise
        om, _ = warmstart.filtered_monitor(sch, mc, JU_o, J_o)
        x12, _ = mesh.jacobi(sch, x, om, 12)
        rng = np.random.default_rng(12)
        x_start = warmstart.warm_start(sch, x12, rng.standard_normal(x.shape) * 0.1)
    xo, ko, po = warmstart.solve(sch, mc, JU_o, J_o, x, x_start, guard_ratio=ratio)
    xg = torch.empty_like(xt)
    dg = torch.empty(x.shape, dtype=torch.float32, device="cuda")
    kg, pg = es.es_mesh_solve(ctx, JU, J, xt, None if x_start is None else _t(x_start, "float64"), xg, dg,
                              guard_ratio=ratio)
    assert (kg, pg) == (ko, po)
    h = w["dxi"][0]
    assert np.abs(_np(xg) - xo).max() <= 1e-12 * h * max(1, ko)
    d_ref = (xo - x) / np.asarray(w["dxi"])[:, None, None]          # cells, per direction
    assert np.abs(_np(dg) - d_ref).max() <= 1e-6 * max(1.0, np.abs(d_ref).max())
    assert po == {"none": 0, "good": 1, "bad": 0, "noisy": int(ratio > 1.0)}[start]


def test_redistribute_with_registered_network_vs_oracle():
    """es_mesh_redistribute with a registered network = oracle features -> network ->
    warm start -> guarded solve -> limiter, to the network's FP32 rounding."""
    import torch

    from paper_2407_05568_gb300 import es
    w = _riemann(sweeps=25)
    sch, mc, JU_o, J_o, x = oracle_setup(w)
    ctx, JU, J, xt = gpu_setup(w)
    rng = np.random.default_rng(11)
    chans = [4, 4, 4, 2]
    ws = [convnet.bf16_round((rng.standard_normal((chans[l + 1], chans[l], 3, 3)) * 0.2).astype(np.float32))
          for l in range(3)]
    bs = [(rng.standard_normal(chans[l + 1]) * 0.05).astype(np.float32) for l in range(3)]
    es.es_set_warm_start(ctx, _t(np.concatenate([a.ravel() for a in ws]), "bfloat16"),
                         _t(np.concatenate(bs)), 3, 4, 1.0)
    dt = 0.004
    xdot = torch.empty_like(xt)
    sw, gam = es.es_mesh_redistribute(ctx, JU, J, xt, dt, xdot)
    f = warmstart.features(sch, mc, JU_o, J_o, x)
    out = convnet.forward(ws, [b.astype(np.float64) for b in bs], f[None], bf16_inputs=True)[-1][0]
    xs = warmstart.warm_start(sch, x, out)
    xo, ko, po = warmstart.solve(sch, mc, JU_o, J_o, x, xs, guard_ratio=1.0)
    assert po == 0                                       # an untrained network's start is refused
    gam_o = mesh.limiter(sch, x, xo - x)
    xdot_o = gam_o * (xo - x) / dt
    assert sw == ko
    assert abs(gam - gam_o) <= 1e-5 * gam_o
    assert np.abs(_np(xdot) - xdot_o).max() <= 1e-5 * np.abs(xdot_o).max()
    # removing the network restores the plain path exactly
    es.es_set_warm_start(ctx, None, None, 0, 0)
    sw2, gam2 = es.es_mesh_redistribute(ctx, JU, J, xt, dt, xdot)
    xdot_p, sw_p, gam_p = stepper.redistribute(sch, mc, JU_o, J_o, x, dt)
    assert sw2 == sw_p and abs(gam2 - gam_p) <= 1e-12 * gam_p


def test_training_gain():
    """Train on plain-run snapshots (64^2, 4 seeds) and compare, on a held-out seed, the
    sweeps to tolerance of the plain and the warm-started solve of the same states."""
    from paper_2407_05568_gb300 import learned
    n, eps, mu = 64, 0.02, 200
    feats, tgts, sw = learned.snapshots([100, 101, 102, 103], n, 40, eps, mu)
    net = learned.WarmStartNet(hidden=32, layers=4, seed=0, in_scale=learned.feature_scale(feats))
    hist = learned.train(net, feats, tgts, epochs=30, batch=8, lr=2e-3, lr_final=2e-4)
    assert hist[-1] < 0.5 * hist[0]
    cmp = learned.compare_solves(net, [118], n, 30, eps, mu)
    plain, warm = cmp["sweeps_plain"].mean(), cmp["sweeps_warm"].mean()
    assert warm < 0.8 * plain, (plain, warm)
    assert cmp["dev_cells"].max() < 0.5
