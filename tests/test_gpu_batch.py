"""The batched persistent form (many 1D shock tubes, one launch) against the oracle, problem by problem."""
import numpy as np
import pytest

from oracle import stepper
from paper_2407_05568_gb300 import workloads as wl

from sides import batch_trajectories, oracle_setup, rel_l1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_05568_gb300 import build
    build.build()


def _run_batch(batch, nsteps):
    import torch

    from paper_2407_05568_gb300 import es
    dev = torch.device("cuda:0")
    b = es.es_batch_create(es.batch_params(batch["gas"]), batch["lengths"])
    rho, v, p = (torch.tensor(a, dtype=torch.float64, device=dev) for a in wl.batch_fields(batch))
    es.es_batch_set_prim(b, rho, v, p)
    es.es_batch_steps(b, nsteps, 1e30)
    assert es.es_batch_check(b) == 0
    JU = torch.empty((3, b.ntot), dtype=torch.float64, device=dev)
    J = torch.empty(b.ntot, dtype=torch.float64, device=dev)
    x = torch.empty(b.ntot, dtype=torch.float64, device=dev)
    t = torch.empty(b.nprob, dtype=torch.float64, device=dev)
    es.es_batch_get(b, JU, J, x, t)
    assert es.es_batch_check(b) == 0
    return b, JU.cpu().numpy(), J.cpu().numpy(), x.cpu().numpy(), t.cpu().numpy()


def test_batch_matches_oracle_per_problem():
    """Ragged lengths (one to five 254-node chunks, and a short tube) after 3 steps.  The time agrees to 1e-4: the
    step is a stability bound, which the mixed form takes in FP32, and near the critical point its sound speed
    c^2 = (1 + delta) R T/(1 - b rho)^2 - 2 a rho cancels several digits (dt within a few 1e-5 of the oracle's)."""
    batch = wl.shock_tube_batch(lengths=[37, 200, 257, 600, 1023, 64], seed=7)
    nsteps = 3
    b, JU, J, x, t = _run_batch(batch, nsteps)
    for k in range(b.nprob):
        w = wl.batch_problem(batch, k)
        sch, mc, JUo, Jo, xo = oracle_setup(w)
        to = 0.0
        for _ in range(nsteps):
            JUo, Jo, xo, to, _ = stepper.step(sch, mc, JUo, Jo, xo, to, 1e30, 0.4)
        sl = slice(b.offsets[k], b.offsets[k] + b.lengths[k])
        assert abs(t[k] - to) <= 1e-4 * to
        assert rel_l1(JU[:, sl], JUo) < 1e-4, (k, rel_l1(JU[:, sl], JUo))
        assert rel_l1(x[sl], xo[0]) < 1e-6
        assert rel_l1(J[sl], Jo) < 1e-5


def test_batch_problems_are_independent():
    """A problem's result does not depend on which other problems share the launch."""
    batch = wl.shock_tube_batch(lengths=[300, 900, 120, 500], seed=9)
    b, JU, J, x, t = _run_batch(batch, 2)
    sub = dict(batch, lengths=batch["lengths"][[1, 3]], states=batch["states"][[1, 3]])
    b2, JU2, J2, x2, t2 = _run_batch(sub, 2)
    for kk, k in enumerate([1, 3]):
        a = slice(b.offsets[k], b.offsets[k] + b.lengths[k])
        c = slice(b2.offsets[kk], b2.offsets[kk] + b2.lengths[kk])
        assert np.array_equal(JU[:, a], JU2[:, c]) and np.array_equal(x[a], x2[c])


def test_batch_rejects_bad_lengths():
    from paper_2407_05568_gb300 import es
    with pytest.raises(es.EsError):
        es.es_batch_create(es.batch_params(wl.UNITS_A), [5, 100])


def test_autotune_restores_state_and_shapes_agree():
    """The autotuner leaves the state as it found it, and every CTA shape gives the same
    step bit for bit (per-node arithmetic does not depend on the chunking; the reductions are maxima)."""
    import torch

    from paper_2407_05568_gb300 import es
    dev = torch.device("cuda:0")
    batch = wl.shock_tube_batch(lengths=[37, 200, 257, 600, 1023, 64, 513, 130], seed=7)
    res = {}
    for tune in (False, True):
        b = es.es_batch_create(es.batch_params(batch["gas"]), batch["lengths"])
        rho, v, p = (torch.tensor(a, dtype=torch.float64, device=dev) for a in wl.batch_fields(batch))
        es.es_batch_set_prim(b, rho, v, p)
        es.es_batch_steps(b, 2, 1e30)
        JU0 = torch.empty((3, b.ntot), dtype=torch.float64, device=dev)
        J0 = torch.empty(b.ntot, dtype=torch.float64, device=dev)
        x0 = torch.empty(b.ntot, dtype=torch.float64, device=dev)
        es.es_batch_get(b, JU0, J0, x0)
        if tune:
            bt, ms = es.es_batch_autotune(b)
            assert bt in (128, 256, 512) and all(m > 0 for m in ms)
            JU1, J1, x1 = torch.empty_like(JU0), torch.empty_like(J0), torch.empty_like(x0)
            es.es_batch_get(b, JU1, J1, x1)
            assert torch.equal(JU0, JU1) and torch.equal(J0, J1) and torch.equal(x0, x1)
        es.es_batch_steps(b, 3, 1e30)
        assert es.es_batch_check(b) == 0
        es.es_batch_get(b, JU0, J0, x0)
        res[tune] = (JU0.cpu(), x0.cpu())
    assert torch.equal(res[False][0], res[True][0]) and torch.equal(res[False][1], res[True][1])


def _subset32():
    """The 32 shortest of the 4096 tubes of the benchmark recipe (lengths 200 to about 215): the recipe's
    states, at sizes the oracle runs to t = 0.1 in about a second each."""
    full = wl.shock_tube_batch()
    k = np.argsort(full["lengths"], kind="stable")[:32]
    return dict(full, lengths=full["lengths"][k], states=full["states"][k])


def test_batch_every_step_to_t01_against_the_oracle():
    """cfg4's accuracy check: 32 problems of the benchmark recipe to t = 0.1.  At every step each problem restarts
    from the oracle's state at that step (es_batch_set_state) and the batched kernel's step must equal the oracle's
    next state to 1e-5 relative L1 in JU, J and x (the mixed form's moving-mesh bar; its FP32 displacement and
    flux rounding), for every problem and every step (about 1000 to 2000 per problem)."""
    import torch

    from paper_2407_05568_gb300 import es
    dev = torch.device("cuda:0")
    batch = _subset32()
    t_end = 0.1
    trajs = batch_trajectories(batch, t_end)
    b = es.es_batch_create(es.batch_params(batch["gas"]), batch["lengths"])
    n = b.ntot
    JU = torch.empty((3, n), dtype=torch.float64, device=dev)
    J = torch.empty(n, dtype=torch.float64, device=dev)
    x = torch.empty(n, dtype=torch.float64, device=dev)
    t = torch.empty(b.nprob, dtype=torch.float64, device=dev)
    kmax = max(len(tr) for tr in trajs) - 1
    worst = 0.0
    for k in range(kmax):
        hJU = np.empty((3, n))
        hJ, hx, ht = np.empty(n), np.empty(n), np.empty(b.nprob)
        for p, tr in enumerate(trajs):
            s = tr[min(k, len(tr) - 1)]
            sl = slice(b.offsets[p], b.offsets[p] + b.lengths[p])
            hJU[:, sl], hJ[sl], hx[sl], ht[p] = s
        JU.copy_(torch.from_numpy(hJU))
        J.copy_(torch.from_numpy(hJ))
        x.copy_(torch.from_numpy(hx))
        t.copy_(torch.from_numpy(ht))
        es.es_batch_set_state(b, JU, J, x, t)
        es.es_batch_steps(b, 1, t_end)
        es.es_batch_get(b, JU, J, x, t)
        gJU, gJ, gx, gt = JU.cpu().numpy(), J.cpu().numpy(), x.cpu().numpy(), t.cpu().numpy()
        for p, tr in enumerate(trajs):
            o = tr[min(k + 1, len(tr) - 1)]
            sl = slice(b.offsets[p], b.offsets[p] + b.lengths[p])
            err = max(rel_l1(gJU[:, sl], o[0]), rel_l1(gJ[sl], o[1]), rel_l1(gx[sl], o[2]))
            worst = max(worst, err)
            assert err < 1e-5, (p, k, err)
            assert abs(gt[p] - o[3]) <= 1e-4 * o[3]
    assert es.es_batch_check(b) == 0
    assert kmax > 50 and worst > 0.0
