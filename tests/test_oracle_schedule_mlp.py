"""Pins for the oracle's adaptive-step helpers (histogram overlap, bisection,
moments) and the schedule MLP (forward, gradient, bf16 rounding, Adam)."""
import math

import numpy as np
import pytest
from scipy import stats
from scipy.special import erfc

from oracle import mlp, schedule


def _gauss_hist(sigma_bins=60, n=400001, mu=-5000):
    k = np.arange(-8 * sigma_bins, 8 * sigma_bins + 1)
    c = np.round(n * np.exp(-0.5 * (k / sigma_bins) ** 2) / (sigma_bins * math.sqrt(2 * math.pi)))
    keep = c > 0
    return (mu + 4 * k[keep]).astype(np.int64), c[keep].astype(np.float64)


def test_overlap_two_level_closed_form():
    levels = np.array([0, 4], dtype=np.int64)
    for a, b in ((3.0, 7.0), (10.0, 1.0), (5.0, 5.0)):
        counts = np.array([a, b])
        R = a + b
        for dbeta in (0.0, 0.01, 0.3, 2.0):
            q = math.exp(-4 * dbeta)
            # reweighting moves weight to the lower level: min picks P0 there, P1 above
            assert schedule.overlap(levels, counts, dbeta) == pytest.approx(a / R + b * q / (a + b * q), rel=1e-14)


def test_overlap_limits_and_monotonicity():
    levels, counts = _gauss_hist(20, 20001)
    assert schedule.overlap(levels, counts, 0.0) == pytest.approx(1.0, abs=1e-14)
    grid = [schedule.overlap(levels, counts, d) for d in np.linspace(0, 0.05, 60)]
    assert all(x >= y for x, y in zip(grid, grid[1:]))
    assert schedule.overlap(levels, counts, 50.0) == pytest.approx(counts[0] / counts.sum(), rel=1e-6)


def test_overlap_gaussian_limit():
    # a shift by dbeta sigma^2 of a Gaussian of width sigma overlaps by erfc(dbeta sigma / (2 sqrt 2))
    levels, counts = _gauss_hist(300, 4000001)
    _, var, _ = schedule.moments(levels, counts)
    sigma = math.sqrt(var)
    for x in (0.1, 0.378, 1.0):
        dbeta = x / sigma
        assert schedule.overlap(levels, counts, dbeta) == pytest.approx(erfc(x / (2 * math.sqrt(2))), abs=2e-3)


def test_bisection_brackets_the_target():
    levels, counts = _gauss_hist(80, 100001)
    d, clamped = schedule.bisect_dbeta(levels, counts, 0.85, 0.05)
    assert not clamped
    assert schedule.overlap(levels, counts, d) >= 0.85
    assert schedule.overlap(levels, counts, d + 0.05 * 2.0 ** -48) < 0.85
    narrow = (np.array([-8, -4]), np.array([100.0, 1.0]))
    d, clamped = schedule.bisect_dbeta(*narrow, 0.85, 0.05)
    assert clamped and d == 0.05


def test_moments_match_scipy_on_expanded_sample():
    rng = np.random.default_rng(5)
    E = -4 * rng.poisson(30, size=5000) - 100
    levels, counts = schedule.histogram(E)
    mean, var, skew = schedule.moments(levels, counts)
    assert mean == pytest.approx(E.mean(), rel=1e-13)
    assert var == pytest.approx(E.var(), rel=1e-12)
    assert skew == pytest.approx(stats.skew(E), rel=1e-10)
    f = schedule.features(levels, counts, 0.3, 64, 5000, 4096)
    assert f.shape == (6,) and f[3] == 0.3 and f[4] == pytest.approx(math.log(64))


def _params(seed=0, scale=0.5):
    return np.random.default_rng(seed).normal(0, scale, mlp.N_PARAMS)


def test_param_count():
    assert mlp.N_PARAMS == 6 * 64 + 64 + 64 * 64 + 64 + 64 + 1 == 4673


def test_forward_of_a_hand_built_network():
    w = {name: np.zeros(shape) for name, shape in mlp.SIZES}
    w["W1"][0, 2] = 0.5    # h1_0 = tanh(0.5 x2 + 0.1)
    w["b1"][0] = 0.1
    w["W2"][3, 0] = 2.0    # h2_3 = tanh(2 h1_0)
    w["W3"][3] = -1.5
    w["b3"][0] = 0.25
    x = np.array([[1.0, -2.0, 0.7, 0.0, 3.0, 9.0]])
    y, _ = mlp.forward(mlp.pack(w), x)
    assert y[0] == pytest.approx(-1.5 * math.tanh(2 * math.tanh(0.5 * 0.7 + 0.1)) + 0.25, rel=1e-15)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    p = _params(2, 0.3)
    X = rng.normal(size=(7, 6))
    T = rng.normal(size=7)
    g = mlp.grad(p, X, T)
    h = 1e-6
    idx = rng.choice(mlp.N_PARAMS, size=60, replace=False)
    idx = np.concatenate([idx, [0, 383, 384, 447, 448, 4543, 4544, 4607, 4608, 4671, 4672]])
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (mlp.loss(p + e, X, T) - mlp.loss(p - e, X, T)) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-10), i


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.normal(0, 3, 5000), [1.0, -0.0, 3.0e38, 1e-39],
                        # exact ties between two bf16 values
                        np.array([0x3F808000, 0x3F818000, 0xBF808000], dtype=np.uint32).view(np.float32)])
    x = x.astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16_round(x), ref)


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    p = rng.normal(size=50)
    t = torch.tensor(p.copy(), requires_grad=True)
    opt = torch.optim.Adam([t], lr=3e-3)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for k in range(1, 6):
        g = rng.normal(size=50)
        p, m, v = mlp.adam(p, g, m, v, k, 3e-3)
        opt.zero_grad()
        t.grad = torch.tensor(g)
        opt.step()
    np.testing.assert_allclose(p, t.detach().numpy(), rtol=1e-12, atol=1e-14)
