"""Pins of the weight-network oracle (CPU only): BF16 rounding against a
library conversion, softplus identities, gradients against central finite
differences, the closed-form optimum of the loss, feature closed forms and
training-target special cases."""
import math

import numpy as np
import pytest

import oracle as orc
from oracle import mlp


def test_bf16_matches_torch_and_ties_to_even():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(0, 3, 20000), rng.uniform(-1e-3, 1e-3, 2000),
                        [0.0, 1.0, -2.5, 1e30, -1e-30]]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x), ref)
    one_ulp = 2.0 ** -7
    assert mlp.bf16(np.float32(1.0 + one_ulp / 2)) == 1.0            # tie -> even (1.0)
    assert mlp.bf16(np.float32(1.0 + 1.5 * one_ulp)) == 1.0 + 2 * one_ulp   # tie -> even


def test_softplus_identities():
    o = np.linspace(-40, 40, 801)
    sp = mlp.softplus(o)
    assert abs(mlp.softplus(0.0) - math.log(2.0)) < 1e-15
    assert np.allclose(sp - mlp.softplus(-o), o, atol=1e-12)          # softplus(o) - softplus(-o) = o
    assert np.all(sp > 0) and np.all(np.diff(sp) > 0)
    assert np.allclose(mlp.sigmoid(o), 1 / (1 + np.exp(-o)), atol=1e-15)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gradients_match_central_differences(seed):
    rng = np.random.default_rng(seed)
    p = mlp.init_params(seed)
    p["b1"] = rng.normal(0, 0.1, 32)
    p["b2"] = rng.normal(0, 0.1, 32)
    x = rng.uniform(-1, 1, (64, 3))
    e2 = rng.uniform(0.1, 2.0, 64)
    mask = rng.uniform(size=64) > 0.2
    w, cache = mlp.forward(p, x, rounding=False)
    g = mlp.flatten(mlp.backward(p, cache, w, e2, mask))
    theta = mlp.flatten(p)
    h = 1e-6
    idx = rng.choice(len(theta), 120, replace=False)
    for k in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        lp = mlp.loss(mlp.forward(mlp.unflatten(tp), x, False)[0], e2, mask)
        lm = mlp.loss(mlp.forward(mlp.unflatten(tm), x, False)[0], e2, mask)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_loss_optimum_is_inverse_mean_residual():
    """With the network reduced to its output bias (W3 = 0), the mean NLL
    w e2 - ln w is minimised at w = 1 / mean(e2): the bias gradient vanishes
    there and has opposite signs on either side."""
    rng = np.random.default_rng(3)
    e2 = rng.uniform(0.01, 0.05, 500)
    x = rng.uniform(0, 1, (500, 3))
    mask = np.ones(500, bool)
    w_star = 1.0 / e2.mean()
    b_star = math.log(math.expm1(w_star))       # softplus^-1
    grads = []
    for b3 in (b_star - 0.5, b_star, b_star + 0.5):
        p = mlp.init_params(0)
        p["W3"][:] = 0.0
        p["b3"][0] = b3
        w, c = mlp.forward(p, x, rounding=False)
        assert np.allclose(w, mlp.softplus(b3))
        grads.append(mlp.backward(p, c, w, e2, mask)["b3"][0])
    assert grads[0] < 0 < grads[2] and abs(grads[1]) < 1e-12


def test_features_of_a_fronto_parallel_plane():
    """Pinhole view of the plane z = Z: range r = |P|, theta = angle between
    the pixel ray and the optical axis, variance 0 (constant depth)."""
    H, W, f, Z = 12, 16, 20.0, 3.0
    u, v = np.meshgrid(np.arange(W), np.arange(H))
    x = (u - (W - 1) / 2) / f * Z
    y = (v - (H - 1) / 2) / f * Z
    P = np.stack([x, y, np.full_like(x, Z)], -1).reshape(-1, 3).astype(np.float32)
    F = mlp.features(P, H, W, 0, 10.0).reshape(H, W, 3)
    r = np.linalg.norm(P.astype(np.float64), axis=1).reshape(H, W)
    assert np.allclose(F[..., 0], r / 10.0, rtol=1e-12)
    inner = np.s_[1:-1, 1:-1]
    th = np.arccos(Z / r)
    assert np.allclose(F[..., 1][inner], th[inner] / (math.pi / 2), atol=1e-7)
    assert np.allclose(F[..., 2], math.log(1e-8) / 10, atol=1e-6)
    assert (F[0, :, 1] == 0).all()          # border: no normal


def test_features_variance_of_a_depth_ramp():
    """Depth z = a + b*u: the 5x5 window variance is b^2 times the population
    variance of its five column offsets {-2..2} (= 2) away from the border."""
    H, W, f = 9, 11, 30.0
    u, v = np.meshgrid(np.arange(W), np.arange(H))
    z = 2.0 + 0.05 * u
    x = (u - (W - 1) / 2) / f * z
    y = (v - (H - 1) / 2) / f * z
    P = np.stack([x, y, z], -1).reshape(-1, 3)
    F = mlp.features(P, H, W, 0, 10.0).reshape(H, W, 3)
    var = np.exp(F[4, 5, 2] * 10) - 1e-8
    assert abs(var - 0.05 ** 2 * 2.0) < 1e-9
    Pn = P.copy()
    Pn[5] = np.nan
    Fn = mlp.features(Pn, H, W, 0, 10.0)
    assert (Fn[5] == 0).all()


def test_targets_zero_for_the_integrated_point_and_shift_squared():
    """A clean map of a single point: that point's residuals are 0; the same
    ray with the point moved by delta along it has residual delta^2 on every
    unclamped voxel."""
    T = np.array([1, 0, 0, 0.0625, 0, 1, 0, 0.0625, 0, 0, 1, 0.0625], np.float32)
    vs, tr = 0.125, 0.375
    m = orc.OracleSubmap(vs, tr)
    p = np.array([[1.0, 0.0, 0.0]], np.float32)
    m.integrate(p, T, sensor=1)
    keys, D, W = m.extract()
    e2, mask = mlp.targets(p, T, keys, D, W, vs, tr, sensor=1)
    assert mask[0] and e2[0] == 0.0
    q = np.array([[1.0 + 0.0625, 0.0, 0.0]], np.float32)   # moves every d by +0.0625
    e2, mask = mlp.targets(q, T, keys, D, W, vs, tr, sensor=1)
    # voxels 5..11 with the clean D; the shifted band covers 6..12; shared 6..11,
    # d_clean = 0.25, .., -0.375 and the shifted d = d_clean + 0.0625 clamped:
    d_clean = np.array([0.25, 0.125, 0.0, -0.125, -0.25, -0.375])
    d_new = np.clip(d_clean + 0.0625, -tr, tr)
    assert mask[0] and abs(e2[0] - np.mean((d_new - d_clean) ** 2)) < 1e-15


def test_adam_two_steps_hand_derived():
    """The oracle's Adam against a two-step sequence worked out by hand with
    exact fractions (tests/golden/adam_two_steps.json)."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "adam_two_steps.json")) as f:
        gold = json.load(f)
    opt = mlp.Adam(1, lr=gold["lr"], b1=gold["b1"], b2=gold["b2"], eps=gold["eps"])
    theta = np.array([gold["theta0"]])
    for g, expect in zip(gold["grads"], gold["theta"]):
        theta = opt.step(theta, np.array([g]))
        assert abs(theta[0] - expect) < 1e-15


def test_adam_constant_gradient_closed_form():
    """With a constant gradient g the bias corrections cancel exactly
    (m^ = g, v^ = g^2 at every step), so each step moves theta by
    lr g / (|g| + eps): after t steps theta = theta0 - t lr g / (|g| + eps)."""
    rng = np.random.default_rng(3)
    g = rng.normal(0, 2, 50)
    theta0 = rng.normal(0, 1, 50)
    opt = mlp.Adam(50, lr=1e-2)
    theta = theta0.copy()
    for t in range(1, 8):
        theta = opt.step(theta, g)
        assert np.allclose(theta, theta0 - t * 1e-2 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-13)
