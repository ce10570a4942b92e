"""Learned point weight on the GPU against the FP64 oracle (features,
inference, gradients, Adam, targets), and the gain of the trained network
over the plain weighting on a held-out scene (SDF RMSE)."""
import math

import numpy as np
import pytest

import oracle as orc
import scenegen as sg
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _scan(seed=21, W=96, H=72, noise=True):
    wl = sg.make_c2(seed=seed, n_frames=2, width=W, height=H, noise=noise)
    return wl


def test_features_match_oracle():
    import torch
    from paper_2410_21149_gb300 import weights
    wl = _scan()
    sc = wl.submaps[0].scans[1]
    f_gpu = weights.features(torch.from_numpy(sc.points).cuda(), sc.height, sc.width, 0, 10.0).cpu().numpy()
    f_orc = omlp.features(sc.points, sc.height, sc.width, 0, 10.0)
    assert np.abs(f_gpu[:, 0] - f_orc[:, 0]).max() < 1e-6
    assert np.abs(f_gpu[:, 1] - f_orc[:, 1]).max() < 2e-3
    assert np.abs(f_gpu[:, 2] - f_orc[:, 2]).max() < 2e-3
    assert (f_orc[:, 1] > 0).sum() > 0.5 * len(f_orc)


def _rand_params(seed):
    p = omlp.init_params(seed)
    rng = np.random.default_rng(seed)
    p["b1"] = rng.normal(0, 0.1, 32)
    p["b2"] = rng.normal(0, 0.1, 32)
    return p


def test_inference_matches_oracle():
    import torch
    from paper_2410_21149_gb300 import weights
    rng = np.random.default_rng(4)
    x = np.stack([rng.uniform(0, 1, 5000), rng.uniform(0, 1, 5000), rng.uniform(-1.9, 0, 5000)], 1)
    x = x.astype(np.float32)
    p = _rand_params(1)
    m = weights.WeightModel(omlp.flatten(p).astype(np.float32))
    w_gpu = m.infer(torch.from_numpy(x).cuda()).cpu().numpy()
    q = omlp.unflatten(omlp.flatten(p).astype(np.float32).astype(np.float64))
    w_orc, _ = omlp.forward(q, x.astype(np.float64))
    assert np.abs(w_gpu / w_orc - 1).max() < 2e-3
    m.close()


def test_gradient_loss_and_adam_match_oracle():
    import torch
    from paper_2410_21149_gb300 import weights
    rng = np.random.default_rng(5)
    n = 4099                                   # ragged last tile
    x = np.stack([rng.uniform(0, 1, n), rng.uniform(0, 1, n), rng.uniform(-1.9, 0, n)], 1).astype(np.float32)
    e2 = rng.uniform(1e-4, 1e-2, n).astype(np.float32)
    mask = (rng.uniform(size=n) > 0.1).astype(np.float32)
    p = _rand_params(2)
    theta0 = omlp.flatten(p).astype(np.float32)
    m = weights.WeightModel(theta0)
    X, E, M = (torch.from_numpy(a).cuda() for a in (x, e2, mask))
    m.train_step(X, E, M, 0.0)
    g_gpu, loss_gpu = m.last()
    q = omlp.unflatten(theta0.astype(np.float64))
    w, cache = omlp.forward(q, x.astype(np.float64))
    g_orc = omlp.flatten(omlp.backward(q, cache, w, e2.astype(np.float64), mask > 0))
    loss_orc = omlp.loss(w, e2.astype(np.float64), mask > 0)
    assert abs(loss_gpu - loss_orc) < 1e-4 * abs(loss_orc)
    for name, (a, b) in {"W1": (0, 96), "b1": (96, 128), "W2": (128, 1152), "b2": (1152, 1184),
                         "W3": (1184, 1216), "b3": (1216, 1217)}.items():
        scale = np.abs(g_orc[a:b]).max()
        assert np.abs(g_gpu[a:b] - g_orc[a:b]).max() <= 1e-2 * scale + 1e-7, name
    # three Adam steps checked against the oracle's Adam (pinned by a
    # hand-derived sequence) fed the gradients the GPU reports for each step
    # (a zero-rate step, as above, only evaluates: it leaves the optimiser's
    # step count and moments alone)
    opt = omlp.Adam(len(theta0))
    theta = theta0.astype(np.float64)
    for lr in (1e-3, 3e-3, 1e-3):
        m.train_step(X, E, M, lr)
        g_k, _ = m.last()
        opt.lr = lr
        theta = opt.step(theta, g_k.astype(np.float64))
        assert np.abs(m.params - theta).max() < 2e-6
    m.close()


def test_training_targets_match_oracle():
    import torch
    import paper_2410_21149_gb300 as cvx
    from paper_2410_21149_gb300 import weights
    clean = _scan(noise=False)
    noisy = _scan(noise=True)
    sm_c = clean.submaps[0]
    sub = cvx.Submap(sm_c.voxel_size, sm_c.trunc, 1e4)
    om = orc.OracleSubmap(sm_c.voxel_size, sm_c.trunc, 1e4)
    prm = cvx.integrate_params(0, 0, 0.1, 10.0, 0, sm_c.scans[0].height, sm_c.scans[0].width)
    for sc in sm_c.scans:
        sub.integrate(torch.from_numpy(sc.points).cuda(), sc.T_sub_sensor, prm)
        om.integrate(sc.points, sc.T_sub_sensor, None, 0, 0, 0.1, 10.0, 0)
    keys, D, W = om.extract()
    sc = noisy.submaps[0].scans[1]
    e2_g, m_g = weights.training_targets(sub, torch.from_numpy(sc.points).cuda(), sc.T_sub_sensor, prm)
    e2_o, m_o = omlp.targets(sc.points, sc.T_sub_sensor, keys, D, W, sm_c.voxel_size, sm_c.trunc, 0.1, 10.0, 0)
    e2_g, m_g = e2_g.cpu().numpy(), m_g.cpu().numpy()
    assert np.array_equal(m_g > 0, m_o)
    assert np.abs(e2_g - e2_o).max() < 1e-6 + 1e-3 * e2_o.max()
    assert m_o.sum() > 0.8 * np.isfinite(sc.points[:, 0]).sum()


def _rmse(wl, D, W, keys, vs, tr):
    b, l = np.nonzero((W > 0) & (np.abs(D) < tr))
    v = keys[b].astype(np.int64) * 8 + np.stack([l % 8, (l // 8) % 8, l // 64], 1)
    c = (v + 0.5) * np.float64(np.float32(vs))
    return float(np.sqrt(np.mean((D[b, l] - wl.scene.sdf(c, tr)) ** 2)))


def _fuse(cvx, torch, sm, scans_pts, weights_fn, mode, W, H, dropoff):
    sub = cvx.Submap(sm.voxel_size, sm.trunc, 1e4, max_blocks=1 << 17)
    for sc, pts in zip(sm.scans, scans_pts):
        wm = {"constant": 0, "quadratic": 1, "learned": 2}[mode]
        pw = weights_fn(sc) if mode == "learned" else None
        sub.integrate(pts, sc.T_sub_sensor, cvx.integrate_params(wm, dropoff, 0.1, 10.0, 0, H, W), pw)
    out = tuple(t.cpu().numpy() for t in sub.extract())
    sub.close()
    return out


def test_learned_weight_gain_over_plain_weighting():
    """Train on seeded buildings; evaluate on a held-out one with every
    weighting and the same behind-surface drop-off.

    The gain the network is trained for: the noise-induced TSDF error, the RMS
    difference between the TSDF fused from the noisy scans and the TSDF fused
    from the same scans without noise (same per-ray weights), is lower with
    the learned weight than with quadratic or constant weights.  Against the
    analytic scene the error is dominated by the projective-distance bias
    that every weighting shares; there the gate keeps the learned weight only
    if it lowers the SDF RMSE, and the learned weight must not be worse than
    the plain one by more than 2%."""
    import torch
    import paper_2410_21149_gb300 as cvx
    from paper_2410_21149_gb300 import weights
    W, H = 640, 480
    F, E, M = [], [], []
    for seed in (31, 32, 34):
        noisy = sg.make_c2(seed=seed, n_frames=8, width=W, height=H)
        clean = sg.make_c2(seed=seed, n_frames=8, width=W, height=H, noise=False)
        f, e, m = weights.build_training_set(noisy.submaps[0].scans, clean.submaps[0].scans, 0.05, 0.15, 10.0)
        F.append(f), E.append(e), M.append(m)
    F, E, M = torch.cat(F), torch.cat(E), torch.cat(M)
    E, _ = weights.normalise_targets(E, M)
    model = weights.WeightModel(seed=0)
    losses = weights.train(model, F, E, M, steps=1500, batch=65536, lr=3e-3)
    assert np.mean(losses[-50:]) < np.mean(losses[:50])
    ev = sg.make_c2(seed=33, n_frames=60, width=W, height=H)
    evc = sg.make_c2(seed=33, n_frames=60, width=W, height=H, noise=False)
    sm, smc = ev.submaps[0], evc.submaps[0]
    noisy_pts = [torch.from_numpy(sc.points).cuda() for sc in sm.scans]
    clean_pts = [torch.from_numpy(sc.points).cuda() for sc in smc.scans]
    wcache = {}

    def learned_w(sc):   # weights of the noisy scan's rays (used for both fusions)
        k = id(sc)
        if k not in wcache:
            i = [id(s) for s in sm.scans].index(k) if k in [id(s) for s in sm.scans] else \
                [id(s) for s in smc.scans].index(k)
            w = weights.learned_point_weights(model, noisy_pts[i], H, W, 0, 10.0)
            wcache[id(sm.scans[i])] = wcache[id(smc.scans[i])] = w
        return wcache[k]

    res = {}
    for mode in ("constant", "quadratic", "learned"):
        kn, Dn, Wn = _fuse(cvx, torch, sm, noisy_pts, learned_w, mode, W, H, ev.dropoff)
        kc, Dc, Wc = _fuse(cvx, torch, smc, clean_pts, learned_w, mode, W, H, ev.dropoff)
        rmse = _rmse(ev, Dn.astype(np.float64), Wn.astype(np.float64), kn, sm.voxel_size, sm.trunc)
        lut = {tuple(k): b for b, k in enumerate(kc)}
        diffs = []
        for b, k in enumerate(kn):
            bc = lut.get(tuple(k))
            if bc is None:
                continue
            m = (Wn[b] > 0) & (Wc[bc] > 0) & (np.abs(Dn[b]) < sm.trunc)
            diffs.append((Dn[b] - Dc[bc])[m].astype(np.float64))
        noise = float(np.sqrt(np.mean(np.concatenate(diffs) ** 2)))
        res[mode] = {"sdf_rmse": rmse, "noise_rmse": noise}
    print("weighting results", res)
    assert res["learned"]["noise_rmse"] < res["quadratic"]["noise_rmse"], res
    assert res["learned"]["noise_rmse"] < res["constant"]["noise_rmse"], res
    assert res["learned"]["sdf_rmse"] < 1.02 * res["quadratic"]["sdf_rmse"], res
    keep = weights.gate(res["learned"]["sdf_rmse"], res["quadratic"]["sdf_rmse"])
    assert keep == (res["learned"]["sdf_rmse"] < res["quadratic"]["sdf_rmse"])
    model.close()


def test_normalise_targets_on_device():
    """cvx_normalise_targets: e2 divided in place by its mean over the mask
    (the scale the learned weights are fitted at), deterministic."""
    import torch
    from paper_2410_21149_gb300 import weights
    rng = np.random.default_rng(9)
    n = 1_000_003
    e2 = rng.uniform(1e-5, 1e-2, n).astype(np.float32)
    mask = (rng.uniform(size=n) > 0.3).astype(np.float32)
    mean_ref = float((e2.astype(np.float64) * mask).sum() / mask.sum())
    out, mean = weights.normalise_targets(torch.from_numpy(e2).cuda(), torch.from_numpy(mask).cuda())
    assert abs(mean / mean_ref - 1) < 1e-6
    assert np.allclose(out.cpu().numpy(), e2 / np.float32(mean), rtol=2e-7, atol=0)
    out2, mean2 = weights.normalise_targets(torch.from_numpy(e2).cuda(), torch.from_numpy(mask).cuda())
    assert mean2 == mean and torch.equal(out, out2)


def test_fused_point_weights_match_features_then_inference():
    """cvx_weight_model_point_weights (features and network in one kernel,
    layer-to-layer activations in mma.sync fragments) against the two-kernel
    path (cvx_point_features, then cvx_weight_model_infer) and the FP64
    oracle, on a 640x480 frame (ragged tile rows) and a 64x1024 scan."""
    import torch
    from paper_2410_21149_gb300 import _capi, weights
    p = _rand_params(3)
    m = weights.WeightModel(omlp.flatten(p).astype(np.float32))
    q = omlp.unflatten(omlp.flatten(p).astype(np.float32).astype(np.float64))
    cases = [(_scan(seed=22, W=640, H=478).submaps[0].scans[1], 0, 10.0),
             (sg.make_c3(n_scans=2, scans_per_submap=2, n_boxes=300).submaps[0].scans[1], 1, 50.0)]
    for sc, sensor, max_range in cases:
        pts = torch.from_numpy(sc.points).cuda()
        fused = weights.learned_point_weights(m, pts, sc.height, sc.width, sensor, max_range).cpu().numpy()
        two = m.infer(weights.features(pts, sc.height, sc.width, sensor, max_range)).cpu().numpy()
        rel = np.abs(fused / two - 1)
        assert np.isfinite(fused).all() and rel.max() < 4e-3 and np.mean(rel > 1e-4) < 0.01, rel.max()
        f_orc = omlp.features(sc.points, sc.height, sc.width, sensor, max_range)
        w_orc, _ = omlp.forward(q, f_orc)
        valid = np.isfinite(sc.points).all(1)
        rel_o = np.abs(fused / w_orc - 1)[valid]
        assert np.quantile(rel_o, 0.999) < 1e-2, np.quantile(rel_o, 0.999)
    m.close()


def test_point_weights_of_many_frames_in_one_launch():
    """cvx_weight_model_point_weights_frames over five scans (one persistent
    launch over (frame, tile) items) equals the single-scan entry point on
    each scan, bit for bit: the same arithmetic per point."""
    import torch
    from paper_2410_21149_gb300 import weights
    m = weights.WeightModel(omlp.flatten(_rand_params(5)).astype(np.float32))
    wl = sg.make_c2(seed=23, n_frames=5, width=320, height=238)
    scans = wl.submaps[0].scans
    H, W = scans[0].height, scans[0].width
    pts = torch.from_numpy(np.stack([sc.points for sc in scans])).cuda()
    many = weights.learned_point_weights_frames(m, pts, H, W, 0, 10.0).cpu().numpy()
    for f in range(len(scans)):
        one = weights.learned_point_weights(m, pts[f], H, W, 0, 10.0).cpu().numpy()
        assert np.array_equal(many[f], one), f
    m.close()
