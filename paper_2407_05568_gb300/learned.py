"""Learned warm start of the mesh iteration: the network, its training, snapshot
generation from plain runs, and evaluation against the plain method.

The Jacobi iteration of Sec. 4 moves the mesh towards the equidistribution of the
monitor.  A 3x3 convolutional network (BF16 weights, FP32 activations and
accumulation) reads the features the library computes at the current mesh
(ln omega, G/(1+|G|), the mesh displacement in cells) and predicts the
displacement, in cells, that the plain iteration reaches; the iteration then
starts from that prediction and always finishes the solve (es_mesh_solve,
es_set_warm_start).

Every arithmetic step -- features, targets, forward and backward passes, loss,
Adam -- runs in the library's kernels; torch only holds device memory and the
stream, and gathers training batches (a copy).
"""
import numpy as np

from . import es
from . import workloads as wl


# The warm start is kept when its first Jacobi sweep changes the mesh by less than
# GUARD_RATIO times the plain start's first sweep.  A trained network's start has a
# larger first residual than the plain start (its error has grid-scale content) yet
# needs fewer sweeps to the tolerance; noise at the grid scale, which the plain sweep
# does not damp, shows ratios of 8 and more and is refused.
GUARD_RATIO = 4.0


def _torch():
    import torch
    return torch


class WarmStartNet:
    """Conv net 4 -> hidden -> ... -> hidden -> 2 with tanh between layers.

    Flat parameter buffers: FP32 master weights and their BF16 copy (layer by layer,
    each [Cout][Cin][3][3]), FP32 biases, Adam moments, gradients."""

    def __init__(self, hidden=32, layers=4, cin=4, cout=2, seed=0, in_scale=None, device="cuda"):
        torch = _torch()
        self.hidden, self.layers, self.cin, self.cout = hidden, layers, cin, cout
        chans = [cin] + [hidden] * (layers - 1) + [cout]
        self.shapes = [(chans[l + 1], chans[l], 3, 3) for l in range(layers)]
        rng = np.random.default_rng(seed)
        ws, bs = [], []
        for l, (co, ci, _, _) in enumerate(self.shapes):
            w = rng.standard_normal((co, ci, 3, 3)) / np.sqrt(9.0 * ci)       # LeCun scale for tanh
            if l == 0 and in_scale is not None:
                w = w / np.maximum(1.0, np.asarray(in_scale, dtype=np.float64))[None, :, None, None]
            if l == layers - 1:
                w = w * 0.1                                                  # start near the plain start
            ws.append(w.ravel())
            bs.append(np.zeros(co))
        dev = torch.device(device)
        f32 = torch.float32
        self.w = torch.tensor(np.concatenate(ws), dtype=f32, device=dev)
        self.b = torch.tensor(np.concatenate(bs), dtype=f32, device=dev)
        self.wb = torch.empty(self.w.numel(), dtype=torch.bfloat16, device=dev)
        es.es_nn_to_bf16(self.w, self.wb)
        self.gw = torch.zeros_like(self.w)
        self.gb = torch.zeros_like(self.b)
        self.mw, self.vw = torch.zeros_like(self.w), torch.zeros_like(self.w)
        self.mb, self.vb = torch.zeros_like(self.b), torch.zeros_like(self.b)
        self.step = 0
        self._ws = None
        self._acts = None
        self.loss = torch.zeros(1, dtype=f32, device=dev)

    # views of layer l in the flat buffers
    def _offsets(self):
        wo, bo = [0], [0]
        for (co, ci, _, _) in self.shapes:
            wo.append(wo[-1] + co * ci * 9)
            bo.append(bo[-1] + co)
        return wo, bo

    def layer(self, l, flat, kind="w"):
        wo, bo = self._offsets()
        co, ci, _, _ = self.shapes[l]
        if kind == "w":
            return flat[wo[l]:wo[l + 1]].view(co, ci, 3, 3)
        return flat[bo[l]:bo[l + 1]]

    def numpy_layers(self):
        """(weights as the bf16 values in float64, biases) per layer, for checks."""
        wb = self.wb.float().cpu().double().numpy()
        b = self.b.cpu().double().numpy()
        wo, bo = self._offsets()
        ws = [wb[wo[l]:wo[l + 1]].reshape(self.shapes[l]) for l in range(self.layers)]
        bs = [b[bo[l]:bo[l + 1]] for l in range(self.layers)]
        return ws, bs

    def _buffers(self, B, H, W):
        torch = _torch()
        key = (B, H, W)
        if self._acts is None or self._acts[0] != key:
            dev = self.w.device
            acts = [None] + [torch.empty((B, co, H, W), dtype=torch.float32, device=dev) for (co, _, _, _) in
                             self.shapes]
            grads = [torch.empty((B, ci, H, W), dtype=torch.float32, device=dev) for (_, ci, _, _) in self.shapes]
            gout = torch.empty((B, self.cout, H, W), dtype=torch.float32, device=dev)
            nbytes = max(es.es_nn_workspace_bytes(B, ci, co, H, W) for (co, ci, _, _) in self.shapes)
            ws = torch.empty(nbytes // 4 + 1, dtype=torch.float32, device=dev)
            self._acts = (key, acts, grads, gout, ws)
        return self._acts[1:]

    def forward(self, x):
        """Network output [B][2][H][W] for features x [B][4][H][W] (float32, contiguous)."""
        B, _, H, W = x.shape
        acts, _, _, ws = self._buffers(B, H, W)
        acts[0] = x
        for l in range(self.layers):
            es.es_nn_conv_forward(acts[l], self.layer(l, self.wb), self.layer(l, self.b, "b"), acts[l + 1],
                                  l < self.layers - 1, ws)
        return acts[-1]

    def infer(self, x):
        """The inference path the context uses: every layer on the tensor cores (bf16 layer inputs)."""
        B, _, H, W = x.shape
        acts, _, _, _ = self._buffers(B, H, W)
        acts[0] = x
        for l in range(self.layers):
            es.es_nn_conv_forward_bf16(acts[l], self.layer(l, self.wb), self.layer(l, self.b, "b"), acts[l + 1],
                                       l < self.layers - 1)
        return acts[-1]

    def train_step(self, x, y, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        """One Adam step on the MSE of forward(x) against y; returns the loss tensor (device)."""
        B, _, H, W = x.shape
        out = self.forward(x)
        acts, grads, gout, ws = self._buffers(B, H, W)
        self.loss.zero_()
        es.es_nn_mse(out, y, gout, self.loss)
        g = gout
        for l in range(self.layers - 1, -1, -1):
            gin = grads[l] if l > 0 else None
            es.es_nn_conv_backward(acts[l], self.layer(l, self.wb), acts[l + 1], g, gin, self.layer(l, self.gw),
                                   self.layer(l, self.gb, "b"), l < self.layers - 1, ws)
            g = gin
        self.step += 1
        es.es_nn_adam(self.w, self.wb, self.gw, self.mw, self.vw, lr, beta1, beta2, eps, self.step)
        es.es_nn_adam(self.b, None, self.gb, self.mb, self.vb, lr, beta1, beta2, eps, self.step)
        return self.loss

    def register(self, ctx, guard_ratio=GUARD_RATIO):
        """Use this network as the warm start of ctx's mesh solves (the context copies it)."""
        es.es_set_warm_start(ctx, self.wb, self.b, self.layers, self.hidden, guard_ratio)


# ----------------------------------------------------------------------------- runs
def riemann_workload(n, seed, eps_cells, mu_max):
    """The 2D vdW four-quadrant Riemann problem on the moving mesh, with the Jacobi
    iteration run to max change < eps_cells cells (at most mu_max sweeps)."""
    w = wl.riemann_2d(n, seed=seed)
    w["mesh"] = dict(w["mesh"], sweeps=int(mu_max), eps=float(eps_cells) * w["dxi"][0])
    return w


def setup(w, precision="fp64", device="cuda"):
    """Context and device state (JU, J, x) of a workload description."""
    return es.setup_workload(w, precision, device)


def snapshots(seeds, n, steps, eps_cells, mu_max, every=1, precision="fp64", device="cuda"):
    """Features [S][4][n][n] and targets [S][2][n][n] (plain iteration's displacement in
    cells) along plain runs of the given seeds; also the plain sweeps of each snapshot."""
    torch = _torch()
    per = (steps + every - 1) // every
    S = per * len(seeds)
    feats = torch.empty((S, 4, n, n), dtype=torch.float32, device=device)
    tgts = torch.empty((S, 2, n, n), dtype=torch.float32, device=device)
    sweeps = []
    k = 0
    for seed in seeds:
        w = riemann_workload(n, seed, eps_cells, mu_max)
        ctx, JU, J, x = setup(w, precision, device)
        for s in range(steps):
            if s % every == 0:
                es.es_mesh_features(ctx, JU, J, x, feats[k])
                sw, _ = es.es_mesh_solve(ctx, JU, J, x, None, None, tgts[k])
                sweeps.append(sw)
                k += 1
            es.es_steps(ctx, JU, J, x, 1, w["t_end"])
        rc = es.es_check(ctx)
        if rc != 0:
            raise es.EsError(rc, es.es_last_error(ctx))
    return feats[:k], tgts[:k], np.array(sweeps)


def train(net, feats, tgts, epochs, batch, lr, seed=0, lr_final=None, log=None):
    """Adam on random batches of the snapshots; returns the per-epoch mean loss."""
    torch = _torch()
    S = feats.shape[0]
    rng = np.random.default_rng(seed)
    nb = max(1, S // batch)
    total = epochs * nb
    hist = []
    it = 0
    for ep in range(epochs):
        perm = rng.permutation(S)
        acc = torch.zeros(1, dtype=torch.float32, device=feats.device)
        for bi in range(nb):
            idx = torch.as_tensor(perm[bi * batch:(bi + 1) * batch], device=feats.device)
            x = feats.index_select(0, idx).contiguous()
            y = tgts.index_select(0, idx).contiguous()
            a = lr if lr_final is None else lr * (lr_final / lr) ** (it / max(1, total - 1))
            acc += net.train_step(x, y, a)
            it += 1
        hist.append(float(acc.item()) / nb)
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.4e}")
    return hist


def compare_solves(net, seeds, n, steps, eps_cells, mu_max, precision="fp64", device="cuda",
                   guard_ratio=GUARD_RATIO):
    """Along plain runs: the plain and the warm-started solve of the same state, per step.

    Returns dict of arrays: sweeps_plain, sweeps_warm, picked, dev_cells (max |x_warm - x_plain| / dxi)."""
    torch = _torch()
    out = dict(sweeps_plain=[], sweeps_warm=[], picked=[], dev_cells=[])
    for seed in seeds:
        w = riemann_workload(n, seed, eps_cells, mu_max)
        ctx, JU, J, x = setup(w, precision, device)
        xp = torch.empty_like(x)
        xw = torch.empty_like(x)
        feat = torch.empty((1, 4, n, n), dtype=torch.float32, device=device)
        xs = torch.empty_like(x)
        for s in range(steps):
            es.es_mesh_features(ctx, JU, J, x, feat[0])
            o = net.infer(feat)
            es.es_mesh_warm_start(ctx, x, o[0], xs)
            sp, _ = es.es_mesh_solve(ctx, JU, J, x, None, xp)
            sw, pk = es.es_mesh_solve(ctx, JU, J, x, xs, xw, guard_ratio=guard_ratio)
            out["sweeps_plain"].append(sp)
            out["sweeps_warm"].append(sw)
            out["picked"].append(pk)
            out["dev_cells"].append(float((xw - xp).abs().max().item()) / w["dxi"][0])
            es.es_steps(ctx, JU, J, x, 1, w["t_end"])
    return {k: np.array(v) for k, v in out.items()}


def compare_matched(net, seeds, n, steps, tols, mu_max, ref_tol=1e-5, ref_mu=20000, every=10, precision="fp64",
                    device="cuda", guard_ratio=GUARD_RATIO):
    """The plain and the warm-started solve measured against the converged mesh, along plain runs.

    Every `every` steps of a plain run (Jacobi to tols[0] cells), the state's mesh equation is solved from x^n until
    a sweep changes the mesh by less than ref_tol cells (at most ref_mu sweeps): x_ref.  Then, for each tolerance in
    tols, the plain solve and the warm-started solve of that state: sweeps, and the max and mean over nodes and
    components of |x - x_ref| / dxi.  Returns ({tol: {key: array over the sampled states}}, reference sweeps)."""
    torch = _torch()
    keys = ("sweeps_plain", "sweeps_warm", "picked", "dist_plain_max", "dist_plain_mean", "dist_warm_max",
            "dist_warm_mean")
    res = {t: {k: [] for k in keys} for t in tols}
    ref_sweeps = []
    for seed in seeds:
        w = riemann_workload(n, seed, tols[0], mu_max)
        dxi = w["dxi"][0]
        ctx, JU, J, x = setup(w, precision, device)
        solvers = {t: es.es_create(es.make_params(riemann_workload(n, seed, t, mu_max), precision=precision))
                   for t in tols}
        ref = es.es_create(es.make_params(riemann_workload(n, seed, ref_tol, ref_mu), precision=precision))
        xr, xp, xw, xs = (torch.empty_like(x) for _ in range(4))
        feat = torch.empty((1, 4, n, n), dtype=torch.float32, device=device)
        for s in range(steps):
            if s % every == 0:
                sr, _ = es.es_mesh_solve(ref, JU, J, x, None, xr)
                ref_sweeps.append(sr)
                es.es_mesh_features(ctx, JU, J, x, feat[0])
                o = net.infer(feat)
                es.es_mesh_warm_start(ctx, x, o[0], xs)
                for t, c in solvers.items():
                    sp, _ = es.es_mesh_solve(c, JU, J, x, None, xp)
                    sw, pk = es.es_mesh_solve(c, JU, J, x, xs, xw, guard_ratio=guard_ratio)
                    r = res[t]
                    r["sweeps_plain"].append(sp)
                    r["sweeps_warm"].append(sw)
                    r["picked"].append(pk)
                    dp = (xp - xr).abs() / dxi
                    dw = (xw - xr).abs() / dxi
                    r["dist_plain_max"].append(float(dp.max().item()))
                    r["dist_plain_mean"].append(float(dp.mean().item()))
                    r["dist_warm_max"].append(float(dw.max().item()))
                    r["dist_warm_mean"].append(float(dw.mean().item()))
            es.es_steps(ctx, JU, J, x, 1, w["t_end"])
        rc = es.es_check(ctx)
        if rc != 0:
            raise es.EsError(rc, es.es_last_error(ctx))
    return {t: {k: np.array(v) for k, v in r.items()} for t, r in res.items()}, np.array(ref_sweeps)


def plain_at(res, dist, key="mean"):
    """(tolerance, sweeps) of the plain solve at a given mean (or max) distance to the converged mesh: log-log
    interpolation of the plain solves' (distance, tolerance) and (distance, sweeps) over the tolerances; None
    outside their range."""
    pts = sorted((float(r[f"dist_plain_{key}"].mean()), t, float(r["sweeps_plain"].mean())) for t, r in res.items())
    d = np.log([p[0] for p in pts])
    x = np.log(dist)
    if x < d[0] - 1e-12 or x > d[-1] + 1e-12:
        return None
    tol = float(np.exp(np.interp(x, d, np.log([p[1] for p in pts]))))
    sweeps = float(np.exp(np.interp(x, d, np.log([p[2] for p in pts]))))
    return tol, sweeps


def compare_runs(net, seed, n, steps, eps_cells, mu_max, precision="fp64", device="cuda",
                 guard_ratio=GUARD_RATIO, eps_warm=None):
    """Two full runs from the same initial data, plain (Jacobi to eps_cells) and warm-started (to eps_warm, default
    eps_cells); sweeps, time, and the warm run's mesh and density against the plain run's after `steps` steps."""
    torch = _torch()
    res = {}
    states = {}
    for mode in ("plain", "warm"):
        eps = eps_cells if mode == "plain" or eps_warm is None else eps_warm
        w = riemann_workload(n, seed, eps, mu_max)
        ctx, JU, J, x = setup(w, precision, device)
        if mode == "warm":
            net.register(ctx, guard_ratio)
        es.es_steps(ctx, JU, J, x, 1, w["t_end"])          # capture the step graph
        es.es_mesh_stats(ctx, reset=True)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        es.es_steps(ctx, JU, J, x, steps - 1, w["t_end"])
        e1.record()
        torch.cuda.synchronize()
        rc = es.es_check(ctx)
        if rc != 0:
            raise es.EsError(rc, es.es_last_error(ctx))
        sw, solves, kept = es.es_mesh_stats(ctx)
        res[mode] = dict(ms_per_step=e0.elapsed_time(e1) / max(1, steps - 1), sweeps_per_step=sw / max(1, solves),
                         warm_kept=kept / max(1, solves))
        rho = JU[0] / J if JU.dtype == torch.float64 else (JU[0, 0].double() + JU[1, 0].double()) / (
            J[0].double() + J[1].double())
        states[mode] = (x.clone(), rho.clone())
        res["dxi"] = w["dxi"][0]
    xp, rp = states["plain"]
    xw, rw = states["warm"]
    res["mesh_dev_cells"] = float((xw - xp).abs().max().item()) / res["dxi"]
    res["rho_rel_l1"] = float(((rw - rp).abs().sum() / rp.abs().sum()).item())
    return res


def feature_scale(feats):
    """Per-channel RMS of the features (initial first-layer scaling)."""
    return np.sqrt(feats.double().pow(2).mean(dim=(0, 2, 3)).cpu().numpy())

