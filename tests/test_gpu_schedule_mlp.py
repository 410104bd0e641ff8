"""GPU parity of the adaptive annealing steps and of the schedule MLP.

- MLP forward, gradient and Adam kernels vs the fp64 oracle evaluating the same
  bf16-rounded network (fp32 accumulation on the GPU: relative 1e-4).
- Bisection and MLP schedules: the oracle replays the GPU's beta sequence bit
  for bit (spins, integer sums; ln Z to 1e-12) and re-derives every step's
  choice from its own population: the same kind of step every time (except a
  proposal whose overlap sits within 3e-5 of an edge of the acceptance band),
  dbeta to 1e-9 for bisection steps and to 3e-5 for proposals.
- What the trained network gains: most proposals are accepted by the overlap
  judge, and a step then costs 1 overlap evaluation instead of ~51.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from oracle import schedule as osch
from paper_1709_04394_gb300 import gbmc
from tests.gpu_common import ctx, spins_out, torch  # noqa: F401

pytestmark = pytest.mark.gpu


def _dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def _init_params(seed):
    rng = np.random.default_rng(seed)
    p = np.zeros(omlp.N_PARAMS)
    w = omlp.unpack(p)
    w["W1"][:] = rng.normal(0, 1 / math.sqrt(6), w["W1"].shape)
    w["W2"][:] = rng.normal(0, 1 / math.sqrt(64), w["W2"].shape)
    w["W3"][:] = rng.normal(0, 1 / math.sqrt(64), w["W3"].shape)
    return omlp.pack(w).astype(np.float32)


def _features(n, seed):
    rng = np.random.default_rng(seed)
    return np.stack([rng.uniform(-2, 0, n), rng.uniform(-3, 3, n), rng.uniform(-2, 2, n), rng.uniform(0, 1, n),
                     np.log(rng.choice([16, 32, 64, 128, 256], n)), np.log(rng.choice([1e3, 1e4, 1e5], n))], 1)


def test_mlp_forward_matches_oracle(ctx):
    p = _init_params(1)
    X = _features(300, 2).astype(np.float32)
    Y = torch.zeros(300, dtype=torch.float32, device="cuda")
    gbmc.mlp_forward(ctx, _dev(p), _dev(X), Y)
    ref, _ = omlp.forward(omlp.bf16_round(p), X.astype(np.float64))
    np.testing.assert_allclose(Y.cpu().numpy(), ref, rtol=1e-4, atol=1e-5)


def test_mlp_grad_matches_oracle(ctx):
    p = _init_params(3)
    X = _features(128, 4).astype(np.float32)
    T = np.random.default_rng(5).normal(size=128).astype(np.float32)
    g = torch.zeros(omlp.N_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    gbmc.mlp_grad(ctx, _dev(p), _dev(X), _dev(T), g, loss)
    pb = omlp.bf16_round(p)
    ref = omlp.grad(pb, X.astype(np.float64), T.astype(np.float64))
    got = g.cpu().numpy().astype(np.float64)
    assert float(loss.item()) == pytest.approx(omlp.loss(pb, X, T), rel=1e-5)
    # element by element, per tensor: the GPU sums B = 128 fp32 products (and
    # tanh in fp32) where the oracle sums fp64 ones over the same bf16 weights;
    # each element within 1e-3 of its value, with an absolute floor of 1e-5 of
    # the tensor's largest element for elements that cancel to near zero
    o = 0
    for name, shape in omlp.SIZES:
        n = int(np.prod(shape))
        r, gg = ref[o:o + n], got[o:o + n]
        floor = 1e-5 * float(np.abs(r).max())
        worst = float(np.max(np.abs(gg - r) / (1e-3 * np.abs(r) + floor)))
        assert worst <= 1.0, (name, worst)
        o += n


def test_mlp_adam_matches_oracle(ctx):
    rng = np.random.default_rng(6)
    p = _init_params(7)
    pd, m, v = _dev(p), torch.zeros(omlp.N_PARAMS, device="cuda"), torch.zeros(omlp.N_PARAMS, device="cuda")
    ref, rm, rv = p.astype(np.float64), np.zeros(omlp.N_PARAMS), np.zeros(omlp.N_PARAMS)
    for k in range(1, 5):
        g = rng.normal(0, 0.1, omlp.N_PARAMS).astype(np.float32)
        gbmc.mlp_adam(ctx, pd, _dev(g), m, v, k, 1e-3)
        ref, rm, rv = omlp.adam(ref, g.astype(np.float64), rm, rv, k, 1e-3)
    np.testing.assert_allclose(pd.cpu().numpy(), ref, rtol=1e-5, atol=1e-7)


def test_mlp_train_fits_a_smooth_target(ctx):
    X = _features(2048, 8).astype(np.float32)
    T = (0.5 * np.tanh(X[:, 1]) - 0.3 * X[:, 0] + 0.2 * X[:, 2] - 1.0).astype(np.float32)
    p = _dev(_init_params(9))
    losses = torch.zeros(60 * 16, dtype=torch.float32, device="cuda")
    gbmc.mlp_train(ctx, p, _dev(X), _dev(T), 60, 128, 3e-3, losses)
    l = losses.cpu().numpy().reshape(60, 16).mean(1)
    assert l[-1] < 0.05 * l[0], (l[0], l[-1])


def _adaptive_run(ctx, Ls, Rs, schedule, seed, params=None, theta=2, beta_f=1.0, dmax=0.1, cap=400):
    lats = [gbmc.lattice_init(ctx, 2, L, n_replicas=R, seed=seed, instance_base=i)
            for i, (L, R) in enumerate(zip(Ls, Rs))]
    pa = gbmc.pa_create(ctx, lats, theta, cap, schedule=schedule, beta_f=beta_f, target_overlap=0.85,
                        dbeta_max=dmax, mlp_params=params, overlap_lo=0.80, overlap_hi=0.90)
    stats, n = gbmc.pa_run(ctx, pa, capacity=cap + 1)
    out = []
    for i in range(len(lats)):
        out.append(dict(betas=gbmc.pa_betas(pa, i), log=gbmc.pa_schedule_log(pa, i), spins=spins_out(ctx, lats[i]),
                        stats=stats[:, i]))
    gbmc.pa_free(pa)
    for l in lats:
        gbmc.lattice_free(l)
    return out


# A proposal's realised overlap on the GPU and in the oracle can differ by the
# fp32 rounding of the network's inputs and sums (proposals agree to PROP_RTOL);
# only a proposal whose overlap lies within EDGE of an edge of the acceptance
# band may therefore be judged differently by the two sides.
PROP_RTOL = 3e-5
EDGE = 3e-5


def _check_replay(run, L, R, seed, inst, theta, params=None, dmax=0.1, beta_f=1.0, lo=0.80, hi=0.90):
    """The oracle replays the GPU's beta sequence and re-derives every step's
    choice from its own population. Returns (steps, boundary cases)."""
    betas = run["betas"]
    ref = oracle.pa_run(2, L, seed, inst, R, betas, theta, keep_energies=True)
    S = len(betas) - 1
    st = run["stats"][: S + 1]
    np.testing.assert_array_equal(st["sumE"], ref["sumE"])
    np.testing.assert_allclose(st["lnZ"], ref["lnZ"], rtol=1e-12)
    np.testing.assert_array_equal(run["spins"], ref["spins"])
    boundary = 0
    for i in range(1, S + 1):
        rec = run["log"][i - 1]
        levels, counts = osch.histogram(ref["E_steps"][i - 1])
        d = min(dmax, beta_f - betas[i - 1])
        ch = osch.choose_step(levels, counts, betas[i - 1], L, R, L * L, d, 0.85, params=params, lo=lo, hi=hi)
        # the network's inputs are the oracle's features rounded to fp32
        f = osch.features(levels, counts, betas[i - 1], L, R, L * L)
        np.testing.assert_allclose(rec["features"], f.astype(np.float32), rtol=1e-6, atol=1e-6, err_msg=str(i))
        if params is not None:
            assert rec["proposal"] == pytest.approx(ch["proposal"], rel=PROP_RTOL), (i, rec, ch)
        if ch["kind"] != rec["kind"]:
            a = ch["alpha_proposal"]
            assert min(abs(a - lo), abs(a - hi)) < EDGE, (i, rec, ch)
            boundary += 1
            continue
        if betas[i] < beta_f:
            tol = 1e-9 if rec["kind"] == 1 else PROP_RTOL
            assert rec["dbeta"] == pytest.approx(max(ch["dbeta"], 1e-7), rel=tol), (i, rec, ch)
            assert rec["alpha"] == pytest.approx(ch["alpha"], rel=1e-6, abs=1e-9)
    return S, boundary


def test_bisection_schedule_matches_oracle(ctx):
    runs = _adaptive_run(ctx, [16, 32], [800, 300], gbmc.GBMC_SCHED_BISECTION, seed=4)
    for i, (L, R) in enumerate(((16, 800), (32, 300))):
        run = runs[i]
        assert run["betas"][0] == 0.0 and run["betas"][-1] == 1.0
        assert all(r["kind"] == 1 for r in run["log"])
        S, boundary = _check_replay(run, L, R, 4, i, 2)
        assert S == len(run["log"]) and boundary == 0
        # every chosen step keeps the target overlap (unless capped)
        assert all(r["alpha"] >= 0.85 or r["clamped"] for r in run["log"])


def _training_set(runs):
    X, T = [], []
    for run in runs:
        for r in run["log"]:
            if r["kind"] == 1 and not r["clamped"]:
                X.append(r["features"])
                T.append(osch.target_from_dbeta(r["dbeta"], r["var"]))
    return np.array(X, dtype=np.float32), np.array(T, dtype=np.float32)


def test_mlp_schedule_matches_oracle_and_gains_over_bisection(ctx):
    # training data: bisection runs of the plain method on several sizes
    runs = []
    for seed in (11, 12, 13):
        runs += _adaptive_run(ctx, [16, 32, 64], [1000, 1000, 1000], gbmc.GBMC_SCHED_BISECTION, seed=seed)
    X, T = _training_set(runs)
    assert len(X) > 50
    p = _dev(_init_params(13))
    gbmc.mlp_train(ctx, p, _dev(X), _dev(T), 400, 64, 3e-3)
    params = p.cpu().numpy()
    # learned schedule on fresh seeds
    bis = _adaptive_run(ctx, [16, 32], [800, 300], gbmc.GBMC_SCHED_BISECTION, seed=21)
    ml = _adaptive_run(ctx, [16, 32], [800, 300], gbmc.GBMC_SCHED_MLP, seed=21, params=params)
    boundary = 0
    for i, (L, R) in enumerate(((16, 800), (32, 300))):
        boundary += _check_replay(ml[i], L, R, 21, i, 2, params=params)[1]
    # an overlap within EDGE of a band edge is rare: at most one such step
    assert boundary <= 1, boundary
    acc = np.mean([r["kind"] == 2 for run in ml for r in run["log"]])
    evals_ml = np.mean([r["evals"] for run in ml for r in run["log"]])
    evals_bis = np.mean([r["evals"] for run in bis for r in run["log"]])
    assert acc >= 0.6, acc
    assert evals_ml < 0.4 * evals_bis, (evals_ml, evals_bis)
    # both reach beta_f in a similar number of steps
    for a, b in zip(ml, bis):
        assert abs(len(a["betas"]) - len(b["betas"])) <= 0.3 * len(b["betas"]) + 2


def _stepwise_adaptive(ctx, L, R, schedule, seed, params, theta, dmax, sweep_checks, n_slots):
    """Anneal one L x L population step by step to beta = 1; before every step
    keep the population's energies (the histogram the schedule reads), and at
    the steps in `sweep_checks` the whole population too."""
    lat = gbmc.lattice_init(ctx, 2, L, n_replicas=R, seed=seed)
    pa = gbmc.pa_create(ctx, [lat], theta, 4000, schedule=schedule, beta_f=1.0, target_overlap=0.85,
                        dbeta_max=dmax, mlp_params=params, overlap_lo=0.85, overlap_hi=0.90)
    E = np.empty(R, dtype=np.int32)
    energies, rows, pops = [], [], {}
    while True:
        gbmc.pa_energies_out(ctx, pa, 0, E)
        k = len(energies) + 1
        if k in sweep_checks:
            pops[k] = spins_out(ctx, lat)
        energies.append(E.astype(np.int64))
        try:
            rows.append(gbmc.pa_step(ctx, pa)[0])
        except gbmc.GbmcError:
            energies.pop()
            break
        if k in pops:
            par = np.empty(R, dtype=np.uint32)
            gbmc.pa_parents_out(ctx, pa, 0, par)
            cur = spins_out(ctx, lat)
            beta = float(rows[-1]["beta"])
            for slot in np.random.default_rng(k).integers(R, size=n_slots):
                s = pops[k][par[slot]].copy()
                oracle.sweeps(2, L, s, None, beta, seed, 0, int(slot), (k - 1) * theta, theta)
                np.testing.assert_array_equal(cur[slot], s)
            pops[k] = None
    log = gbmc.pa_schedule_log(pa, 0)
    betas = gbmc.pa_betas(pa, 0)
    gbmc.pa_free(pa)
    gbmc.lattice_free(lat)
    return energies, rows, log, betas


def _rederive(L, R, energies, log, betas, params, dmax, lo, hi):
    """The oracle re-derives every step's choice from the GPU's energies."""
    boundary = 0
    for i, rec in enumerate(log):
        levels, counts = osch.histogram(energies[i])
        d = min(dmax, 1.0 - betas[i])
        ch = osch.choose_step(levels, counts, betas[i], L, R, L * L, d, 0.85, params=params, lo=lo, hi=hi)
        f = osch.features(levels, counts, betas[i], L, R, L * L)
        np.testing.assert_allclose(rec["features"], f.astype(np.float32), rtol=1e-6, atol=1e-6, err_msg=str(i))
        if params is not None:
            assert rec["proposal"] == pytest.approx(ch["proposal"], rel=PROP_RTOL), (i, rec, ch)
        if ch["kind"] != rec["kind"]:
            assert min(abs(ch["alpha_proposal"] - lo), abs(ch["alpha_proposal"] - hi)) < EDGE, (i, rec, ch)
            boundary += 1
            continue
        if betas[i + 1] < 1.0:
            tol = 1e-9 if rec["kind"] == 1 else PROP_RTOL
            assert rec["dbeta"] == pytest.approx(max(ch["dbeta"], 1e-7), rel=tol), (i, rec, ch)
            assert rec["alpha"] == pytest.approx(ch["alpha"], rel=1e-6, abs=1e-9)
    return boundary


def test_adaptive_schedules_at_full_size_l256_r50000(ctx):
    # the learned-schedule workload's largest lattice: 2D L = 256, R = 5 10^4,
    # theta = 10, beta 0 -> 1; bisection, then the MLP trained on the bisection
    # run's log (band [0.85, 0.90], the benchmark's), each step re-derived by the
    # oracle from the library's energies, resampling of sampled steps checked
    # whole and theta sweeps on sampled slots at two steps
    L, R, theta, dmax = 256, 50000, 10, 0.05
    E_b, rows_b, log_b, betas_b = _stepwise_adaptive(ctx, L, R, gbmc.GBMC_SCHED_BISECTION, 41, None, theta, dmax,
                                                     (2, 500), 3)
    assert betas_b[-1] == 1.0 and len(log_b) == len(betas_b) - 1 > 300
    assert _rederive(L, R, E_b, log_b, betas_b, None, dmax, 0.85, 0.90) == 0
    for i in (0, len(log_b) // 2, len(log_b) - 1):
        counts, lnQ = oracle.resample(E_b[i], betas_b[i + 1] - betas_b[i], 41, 0, i + 1)
        assert rows_b[i]["lnQ"] == pytest.approx(lnQ, rel=1e-12, abs=1e-13)
    # targets 0.97 x the bisection step, so that most proposals land inside the band
    X = np.array([r["features"] for r in log_b if r["kind"] == 1 and not r["clamped"]], dtype=np.float32)
    T = np.array([osch.target_from_dbeta(0.97 * r["dbeta"], r["var"]) for r in log_b
                  if r["kind"] == 1 and not r["clamped"]], dtype=np.float32)
    p = _dev(_init_params(17))
    gbmc.mlp_train(ctx, p, _dev(X), _dev(T), 300, 64, 3e-3)
    params = p.cpu().numpy()
    E_m, rows_m, log_m, betas_m = _stepwise_adaptive(ctx, L, R, gbmc.GBMC_SCHED_MLP, 42, params, theta, dmax,
                                                     (3, 400), 3)
    assert betas_m[-1] == 1.0
    boundary = _rederive(L, R, E_m, log_m, betas_m, params, dmax, 0.85, 0.90)
    assert boundary <= 2, boundary
    assert np.mean([r["kind"] == 2 for r in log_m]) > 0.5
