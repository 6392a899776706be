"""Pins of the oracle's extra channels (curvature map, depth distortion, median depth)
and of its Euclidean-density variant, each against something other than the oracle:
the Gaussian curvature from the fundamental forms of the parametrised surface, the
weighted-variance identity of the distortion, hand-worked planar stacks, distances
measured in world space, frame symmetries and finite differences."""
import math

import mpmath as mp
import numpy as np
import pytest
import torch

import oracle.qgs_oracle as O
from paper_2411_16392_gb300.scenes import Camera, Scene, f32_to_bf16_bits, scene_small

F64 = torch.float64


def t64(x):
    return torch.tensor(np.asarray(x, np.float64), dtype=F64)


# --------------------------------------------------------------------------- curvature
def _curvature_fundamental_forms(a, b, x, y):
    """K = (LN - M^2) / (EG - F^2) of r(u, v) = (u, v, a u^2 + b v^2), with every partial
    derivative taken numerically (mpmath, 40 digits)."""
    mp.mp.dps = 40

    def r(u, v):
        return [u, v, a * u * u + b * v * v]

    def d(i, j, u, v):
        return [mp.diff(lambda uu, vv: r(uu, vv)[k], (u, v), (i, j)) for k in range(3)]

    ru, rv = d(1, 0, x, y), d(0, 1, x, y)
    ruu, ruv, rvv = d(2, 0, x, y), d(1, 1, x, y), d(0, 2, x, y)
    n = [ru[1] * rv[2] - ru[2] * rv[1], ru[2] * rv[0] - ru[0] * rv[2], ru[0] * rv[1] - ru[1] * rv[0]]
    nn = mp.sqrt(sum(c * c for c in n))
    n = [c / nn for c in n]
    dot = lambda p, q: sum(pi * qi for pi, qi in zip(p, q))
    E, F, G = dot(ru, ru), dot(ru, rv), dot(rv, rv)
    L, M, N = dot(ruu, n), dot(ruv, n), dot(rvv, n)
    return float((L * N - M * M) / (E * G - F * F))


def test_curvature_matches_fundamental_forms():
    rng = np.random.default_rng(0)
    for _ in range(12):
        a, b = rng.uniform(-3, 3, 2)
        x, y = rng.uniform(-1, 1, 2)
        want = _curvature_fundamental_forms(mp.mpf(a), mp.mpf(b), mp.mpf(x), mp.mpf(y))
        got = float(O.gaussian_curvature(t64(x), t64(y), t64(a), t64(b)))
        assert abs(got - want) <= 1e-12 * max(1.0, abs(want)), (a, b, x, y)


def test_curvature_special_cases():
    """At the vertex K = 4ab (principal curvatures 2a, 2b); a cylinder (b = 0) and the
    plane have K = 0; a saddle (ab < 0) has K < 0 everywhere."""
    a, b = t64(1.5), t64(-0.5)
    assert float(O.gaussian_curvature(t64(0.0), t64(0.0), a, b)) == pytest.approx(4 * 1.5 * -0.5, abs=0)
    xs = t64(np.linspace(-2, 2, 9))
    assert torch.all(O.gaussian_curvature(xs, xs, t64(2.0), t64(0.0)) == 0)
    assert torch.all(O.gaussian_curvature(xs, xs.flip(0), a, b) < 0)


# --------------------------------------------------------------------------- distortion
def test_distortion_is_the_weighted_variance():
    """sum_i sum_{j<i} w_i w_j (t_i - t_j)^2 = W^2 Var_w(t), W = sum w (numpy's weighted
    average), and a plain pair loop on a tiny input."""
    rng = np.random.default_rng(1)
    w = rng.uniform(0, 0.3, (6, 40))
    w[:, 25:] = 0                      # pixels whose list ended early
    t = rng.uniform(1, 9, (6, 40))
    got = O._distortion(t64(w), t64(t), block=7).numpy()
    for p in range(6):
        W = w[p].sum()
        mean = np.average(t[p], weights=w[p])
        var = np.average((t[p] - mean) ** 2, weights=w[p])
        assert got[p] == pytest.approx(W * W * var, rel=1e-12)
        loop = sum(w[p, i] * w[p, j] * (t[p, i] - t[p, j]) ** 2 for i in range(40) for j in range(i))
        assert got[p] == pytest.approx(loop, rel=1e-12)


# --------------------------------------------------------------------------- planar stack
def _stack_scene(depths, opac, curv=(0.0, 0.0)):
    """Surfels facing the camera, centred on the ray of pixel (8, 8) of a 16x16 camera."""
    n = len(depths)
    cam = Camera(16, 16, 16.0, 16.0, 8.5, 8.5)      # pixel (8, 8) looks straight down +z
    mean = np.array([[0.0, 0.0, z] for z in depths], np.float32)
    quat = np.tile(np.array([1.0, 0, 0, 0], np.float32), (n, 1))
    scale = np.full((n, 2), 0.5, np.float32)
    cv = np.tile(np.array(curv, np.float32), (n, 1))
    sh = f32_to_bf16_bits(np.zeros((n, 48), np.float32))
    return Scene(mean, quat, scale, cv, np.array(opac, np.float32), sh), cam


def test_median_depth_and_distortion_of_a_planar_stack():
    """Three surfels hit head-on (G = 1, alpha = opacity) at t = 2, 3, 4 with alphas 0.3,
    0.4, 0.5: T before each is 1, 0.7, 0.42, so the median depth (largest t with
    T > 0.5) is 3; weights 0.3, 0.28, 0.21 give the distortion by hand."""
    sc, cam = _stack_scene([2.0, 3.0, 4.0], [0.3, 0.4, 0.5])
    r = O.render_pixels(sc, cam, [(8, 8)], extras=True)
    w = np.array([0.3, 0.7 * 0.4, 0.42 * 0.5])
    t = np.array([2.0, 3.0, 4.0])
    dist = w[1] * w[0] * 1.0 + w[2] * (w[0] * 4.0 + w[1] * 1.0)
    assert r["median_depth"][0] == pytest.approx(3.0, abs=1e-6)
    assert r["distortion"][0] == pytest.approx(dist, rel=1e-6)
    assert r["depth"][0] == pytest.approx((w * t).sum(), rel=1e-6)
    assert r["curvature"][0] == 0.0
    # the first surfel alone opaque enough: T drops to 0.4 after it, nothing else qualifies
    sc, cam = _stack_scene([2.0, 3.0, 4.0], [0.6, 0.4, 0.5])
    r = O.render_pixels(sc, cam, [(8, 8)], extras=True)
    assert r["median_depth"][0] == pytest.approx(2.0, abs=1e-6)


def test_curvature_map_of_a_curved_stack():
    """Head-on hits at the vertices: K_i = 4 a b exactly; the map is sum w_i K_i."""
    sc, cam = _stack_scene([2.0, 3.0], [0.5, 0.5], curv=(0.7, -0.2))
    r = O.render_pixels(sc, cam, [(8, 8)], extras=True)
    w = np.array([0.5, 0.25])
    a, b = float(np.float32(0.7)), float(np.float32(-0.2))     # the scene stores float32
    assert r["curvature"][0] == pytest.approx((w * 4 * a * b).sum(), rel=1e-9)


# --------------------------------------------------------------------------- Euclid variant
def _small_scene(n=150, W=32, seed=0):
    sc, cam = scene_small(seed, n)
    return sc, Camera(W, W, float(W), float(W), W / 2, W / 2)


def test_euclid_density_uses_the_world_space_distance():
    """For every hit of the Euclidean variant, alpha = min(0.99, o exp(-|p - mu|^2 /
    (2 sigma(theta)^2))) with p the world-space hit point c + t d_w, |p - mu| and the
    angle theta measured in world space (projections on the primitive's axes)."""
    sc, cam = _small_scene(seed=2)
    prm = O.Params(sc)
    c64 = O.CamF64(cam)
    b = O.bin_fp32(sc, cam)
    Rcw = cam.R_cw.astype(np.float64)
    c_w = -Rcw.T @ cam.t_cw.astype(np.float64)
    checked = 0
    for tile in range(b.tiles_x * b.tiles_y):
        checked += _check_euclid_tile(sc, cam, prm, c64, b, tile, Rcw, c_w)
    assert checked > 40


def _check_euclid_tile(sc, cam, prm, c64, b, tile, Rcw, c_w):
    s, e = b.ranges[tile]
    idx = torch.from_numpy(b.vals[s:e].astype(np.int64))
    xs, ys = O._tile_pixels(cam, tile, b.tiles_x)
    pe = O._eval_pairs(prm, c64, idx, t64(xs), t64(ys), density="euclid")
    checked = 0
    for p in range(len(xs)):
        d_cam = np.array([(xs[p] + 0.5 - np.float32(cam.cx)) / np.float32(cam.fx),
                          (ys[p] + 0.5 - np.float32(cam.cy)) / np.float32(cam.fy), 1.0])
        d_w = Rcw.T @ d_cam
        for j in range(len(idx)):
            if not bool(pe["valid"][p, j]):
                continue
            i = int(idx[j])
            q = sc.quat[i].astype(np.float64)
            q /= np.linalg.norm(q)
            w_, qx, qy, qz = q
            ru = np.array([1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy + w_ * qz), 2 * (qx * qz - w_ * qy)])
            rv = np.array([2 * (qx * qy - w_ * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz + w_ * qx)])
            hit = c_w + float(pe["t"][p, j]) * d_w - sc.mean[i].astype(np.float64)
            u, v = ru @ hit, rv @ hit
            su, sv = sc.scale[i].astype(np.float64)
            th = math.atan2(v, u)
            sig2 = (su * sv) ** 2 / ((sv * math.cos(th)) ** 2 + (su * math.sin(th)) ** 2)
            al = min(0.99, float(sc.opacity[i]) * math.exp(-(hit @ hit) / (2 * sig2)))
            assert float(pe["alpha"][p, j]) == pytest.approx(al, rel=1e-9, abs=1e-12)
            checked += 1
    return checked


def test_euclid_equals_geodesic_in_the_planar_limit_and_is_never_smaller():
    sc, cam = _small_scene(seed=4)
    planar = sc.copy()
    planar.curv[:] = 0
    g = O.render(planar, cam)
    e = O.render(planar, cam, density="euclid")
    for k in ("rgb", "alpha", "depth", "normal"):
        assert np.abs(g[k] - e[k]).max() < 1e-12, k
    # chord <= arc: the Euclidean weight of a given hit is never below the geodesic one
    x = t64(np.linspace(-0.3, 0.3, 13))
    a, b, s1, s2 = t64(4.0), t64(-2.5), t64(0.1), t64(0.15)
    Gg, lg, _ = O.geodesic_gaussian(x, x.flip(0), a, b, s1, s2)
    Ge, le, _ = O.euclid_gaussian(x, x.flip(0), a, b, s1, s2)
    assert torch.all(le <= lg + 1e-15) and torch.all(Ge >= Gg - 1e-15)


# --------------------------------------------------------------------------- symmetries
def _compose_rot(q, r):
    w1, x1, y1, z1 = q.T
    w2, x2, y2, z2 = r
    return np.stack([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                     w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                     w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2], 1).astype(np.float32)


@pytest.mark.parametrize("density", ["geodesic", "euclid"])
def test_extra_channels_are_frame_symmetric(density):
    """A half turn about the local x axis with both curvatures negated describes the same
    surface: every channel, curvature included (K = 4ab keeps its sign), is unchanged."""
    sc, cam = _small_scene(n=200, W=40, seed=6)
    ref = O.render(sc, cam, density=density, extras=True)
    s2 = sc.copy()
    s2.quat = _compose_rot(sc.quat, np.array([0.0, 1, 0, 0]))
    s2.curv = -sc.curv
    got = O.render(s2, cam, density=density, extras=True)
    ok = (np.minimum(ref["margin"], ref["margin_median"]) > 1e-6) & \
         (np.minimum(got["margin"], got["margin_median"]) > 1e-6)
    assert ok.mean() > 0.98
    for k in ("rgb", "alpha", "depth", "normal", "distortion", "median_depth"):
        assert np.abs(ref[k] - got[k])[..., ok].max() < 1e-9, k
    kerr = np.abs(ref["curvature"] - got["curvature"]) / np.maximum(1.0, ref["curvature_scale"])
    assert kerr[ok].max() < 1e-9


# --------------------------------------------------------------------------- gradients
def _tiny_grad_scene(seed):
    rng = np.random.default_rng(seed)
    n = 5
    s = rng.uniform(0.12, 0.3, (n, 2))
    kap = rng.uniform(-1.5, 1.5, (n, 2))
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    sc = Scene(np.stack([rng.uniform(-0.4, 0.4, n), rng.uniform(-0.4, 0.4, n), rng.uniform(1.8, 2.6, n)],
                        1).astype(np.float32),
               q.astype(np.float32), s.astype(np.float32), (kap / s).astype(np.float32),
               rng.uniform(0.3, 0.9, n).astype(np.float32),
               f32_to_bf16_bits(rng.normal(0, 0.3, (n, 48)).astype(np.float32)))
    return sc, Camera(20, 20, 17.0, 17.0, 10.0, 10.0)


@pytest.mark.parametrize("density", ["geodesic", "euclid"])
def test_extra_channel_gradients_match_finite_differences(density):
    """Autograd gradients of the curvature and distortion maps (plus the four base
    channels) match central differences of the FP64 forward for the geometric
    parameters of a tiny scene."""
    H = W = 20
    for seed in range(30):
        sc, cam = _tiny_grad_scene(seed)
        rng = np.random.default_rng(200 + seed)
        g = dict(rgb=rng.normal(size=(3, H, W)), alpha=rng.normal(size=(H, W)), depth=rng.normal(size=(H, W)),
                 normal=rng.normal(size=(3, H, W)), curvature=rng.normal(size=(H, W)),
                 distortion=rng.normal(size=(H, W)))
        ref = O.render(sc, cam, grad_images=g, density=density, extras=True)
        if ref["margin"].min() > 1e-4 and ref["n_contrib"].max() > 1:
            break
    else:
        pytest.fail("no seed without near-decision pairs")
    binning = ref["binning"]
    prm = O.Params(sc)
    c64 = O.CamF64(cam)

    def loss_of(pr):
        tot = 0.0
        for tile in range(binning.tiles_x * binning.tiles_y):
            s, e = binning.ranges[tile]
            if e <= s:
                continue
            xs, ys = O._tile_pixels(cam, tile, binning.tiles_x)
            r = O._composite(pr, c64, torch.from_numpy(binning.vals[s:e].astype(np.int64)), t64(xs), t64(ys),
                             density=density, extras=True)
            tot += float((t64(g["rgb"][:, ys, xs].T) * r["rgb"]).sum() + (t64(g["alpha"][ys, xs]) * r["alpha"]).sum()
                         + (t64(g["depth"][ys, xs]) * r["depth"]).sum()
                         + (t64(g["normal"][:, ys, xs].T) * r["normal"]).sum()
                         + (t64(g["curvature"][ys, xs]) * r["curvature"]).sum()
                         + (t64(g["distortion"][ys, xs]) * r["distortion"]).sum())
        return tot

    grads = ref["grads"]
    for name in ("mean", "quat", "scale", "curv", "opacity"):
        leaf = getattr(prm, name)
        flat = leaf.view(-1)
        gref = grads[name].reshape(-1)
        scale = max(np.abs(gref).max(), 1e-12)
        for j in range(flat.numel()):
            v0 = float(flat[j])
            h = 1e-6 * max(1.0, abs(v0))
            with torch.no_grad():
                flat[j] = v0 + h
                lp = loss_of(prm)
                flat[j] = v0 - h
                lm = loss_of(prm)
                flat[j] = v0
            fd = (lp - lm) / (2 * h)
            assert abs(fd - gref[j]) <= 1e-5 * scale + 1e-6 * abs(fd), (name, j, fd, gref[j])
