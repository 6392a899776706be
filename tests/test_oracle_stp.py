"""Pins of the oracle's StopThePop ordering (per-tile hit depth + per-pixel resorting in a
buffer of 8), each against something other than the oracle itself: an FP64 root-finding
of the representative ray, plain per-pixel loops with a sorted list and with a heap, the
list-order compositor, and finite differences."""
import heapq
import math

import numpy as np
import pytest
import torch
from scipy import optimize

import oracle.qgs_oracle as O
from paper_2411_16392_gb300.scenes import Camera, Scene, f32_to_bf16_bits, scene_small

F64 = torch.float64


def t64(x):
    return torch.tensor(np.asarray(x, np.float64), dtype=F64)


def _rot(q):
    q = np.asarray(q, np.float64)
    q = q / np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def test_hit_keys_are_the_representative_rays_depths():
    """The per-tile key is the camera z of the nearest intersection (in front of the near
    plane) of the tile pixel ray closest to the projected centre with the whole paraboloid,
    found here by bracketing and Brent in FP64 world space; the centre depth when the ray
    misses."""
    sc, cam = scene_small(2, 300)
    b = O.bin_fp32(sc, cam, emit=False, order="hit")
    checked = missed = 0
    Rcw = cam.R_cw.astype(np.float64)
    c_w = -Rcw.T @ cam.t_cw.astype(np.float64)
    for tile in range(b.tiles_x * b.tiles_y):
        prims = O.tile_list(b, tile)
        if prims.size == 0:
            continue
        keys = O.hit_keys(b, prims, tile).view(np.float32).astype(np.float64)
        ty, tx = divmod(tile, b.tiles_x)
        for p, key in zip(prims, keys):
            mu = sc.mean[p].astype(np.float64)
            mc = Rcw @ mu + cam.t_cw.astype(np.float64)
            uc = cam.fx * mc[0] / mc[2] + cam.cx
            vc = cam.fy * mc[1] / mc[2] + cam.cy
            px = min(max(math.floor(uc), 16 * tx), min(16 * tx + 15, cam.W - 1))
            py = min(max(math.floor(vc), 16 * ty), min(16 * ty + 15, cam.H - 1))
            if abs(uc - round(uc)) < 1e-4 or abs(vc - round(vc)) < 1e-4:
                continue            # the float32 recipe may pick the neighbouring pixel
            d_cam = np.array([(px + 0.5 - cam.cx) / cam.fx, (py + 0.5 - cam.cy) / cam.fy, 1.0])
            R = _rot(sc.quat[p])
            a, bb = sc.curv[p].astype(np.float64)

            def f(t):
                loc = R.T @ (c_w + t * (Rcw.T @ d_cam) - mu)
                return a * loc[0] ** 2 + bb * loc[1] ** 2 - loc[2]

            ts = np.linspace(cam.near, mc[2] + 60 * max(sc.scale[p]) + 5.0, 6000)
            fv = np.array([f(t) for t in ts])
            idx = np.nonzero(np.sign(fv[:-1]) != np.sign(fv[1:]))[0]
            if idx.size == 0:
                missed += 1
                assert key == np.float32(mc[2]) or abs(key - mc[2]) <= 1e-5 * mc[2], (p, tile, key, mc[2])
                continue
            root = optimize.brentq(f, ts[idx[0]], ts[idx[0] + 1], xtol=1e-14)
            assert abs(key - root) <= 2e-5 * root, (p, tile, key, root)
            checked += 1
    assert checked > 100 and missed > 0


def _pairs(sc, cam, tile, density="geodesic"):
    b = O.bin_fp32(sc, cam, order="hit")
    s, e = b.ranges[tile]
    idx = torch.from_numpy(b.vals[s:e].astype(np.int64))
    xs, ys = O._tile_pixels(cam, tile, b.tiles_x)
    prm, c64 = O.Params(sc), O.CamF64(cam)
    return prm, c64, idx, t64(xs), t64(ys)


def _busiest_tile(sc, cam):
    b = O.bin_fp32(sc, cam, emit=False)
    return int(np.argmax([O.tile_list(b, t).size for t in range(b.tiles_x * b.tiles_y)]))


def _blend_sequence(pe, k, order):
    """Plain loop: blend the contributing pairs of pixel k in the given list order."""
    T, acc, dep = 1.0, np.zeros(3), 0.0
    for j in order:
        al = float(pe["alpha"][k, j])
        if T * (1 - al) < O.T_MIN:
            break
        acc += al * T * pe["rgb"][j].numpy()
        dep += al * T * float(pe["t"][k, j])
        T *= 1 - al
    return T, acc, dep


def _scene_dense():
    sc, _ = scene_small(4, 600)
    sc.opacity[:] = np.float32(0.6)
    return sc, Camera(48, 48, 48.0, 48.0, 24.0, 24.0)


def test_resort_with_a_large_buffer_is_the_exact_per_pixel_sort():
    sc, cam = _scene_dense()
    tile = _busiest_tile(sc, cam)
    prm, c64, idx, px, py = _pairs(sc, cam, tile)
    L = idx.shape[0]
    r = O._composite_resort(prm, c64, idx, px, py, buf=L + 1)
    pe = O._eval_pairs(prm, c64, idx, px, py)
    for k in range(px.shape[0]):
        js = [j for j in range(L) if bool(pe["valid"][k, j])]
        js.sort(key=lambda j: (float(pe["t"][k, j]), j))
        T, acc, dep = _blend_sequence(pe, k, js)
        assert abs(float(r["T_final"][k]) - T) < 1e-13
        assert np.abs(r["rgb"][k].detach().numpy() - acc).max() < 1e-12
        assert abs(float(r["depth"][k]) - dep) < 1e-11


def test_resort_with_a_buffer_of_one_is_list_order():
    sc, cam = _scene_dense()
    tile = _busiest_tile(sc, cam)
    prm, c64, idx, px, py = _pairs(sc, cam, tile)
    a = O._composite_resort(prm, c64, idx, px, py, buf=1)
    b = O._composite(prm, c64, idx, px, py)
    for key in ("rgb", "alpha", "depth", "normal", "T_final"):
        assert torch.abs(a[key] - b[key]).max() < 1e-13, key


def test_resort_buffer_of_eight_matches_a_heap_loop():
    """The window algorithm written independently with a heap per pixel: push every
    contributing pair; when 8 are held pop the nearest and blend it; at the end pop the
    rest in depth order."""
    sc, cam = _scene_dense()
    tile = _busiest_tile(sc, cam)
    prm, c64, idx, px, py = _pairs(sc, cam, tile)
    L = idx.shape[0]
    r = O._composite_resort(prm, c64, idx, px, py, buf=8)
    pe = O._eval_pairs(prm, c64, idx, px, py)
    amb = 0
    for k in range(px.shape[0]):
        heap, order = [], []
        for j in range(L):
            if bool(pe["valid"][k, j]):
                heapq.heappush(heap, (float(pe["t"][k, j]), j))
                if len(heap) == 8:
                    order.append(heapq.heappop(heap)[1])
        while heap:
            order.append(heapq.heappop(heap)[1])
        T, acc, dep = _blend_sequence(pe, k, order)
        if float(r["margin"][k]) < 1e-9:
            amb += 1
            continue
        assert abs(float(r["T_final"][k]) - T) < 1e-13, k
        assert np.abs(r["rgb"][k].detach().numpy() - acc).max() < 1e-12, k
    assert amb <= 2


def test_stp_order_differs_from_centre_order_only_where_hits_reorder():
    """Well separated primitives (depth gaps far above their extent): the hit order is
    the centre order, so both orderings give the same image."""
    rng = np.random.default_rng(3)
    n = 40
    mean = np.stack([rng.uniform(-0.3, 0.3, n), rng.uniform(-0.3, 0.3, n), 2.0 + 0.5 * np.arange(n)], 1)
    q = rng.normal(size=(n, 4))
    sc = Scene(mean.astype(np.float32), (q / np.linalg.norm(q, axis=1, keepdims=True)).astype(np.float32),
               rng.uniform(0.05, 0.1, (n, 2)).astype(np.float32), rng.uniform(-2, 2, (n, 2)).astype(np.float32),
               rng.uniform(0.2, 0.6, n).astype(np.float32),
               f32_to_bf16_bits(rng.normal(0, 0.3, (n, 48)).astype(np.float32)))
    cam = Camera(32, 32, 40.0, 40.0, 16.0, 16.0)
    a = O.render(sc, cam)
    b = O.render(sc, cam, order="stp")
    for key in ("rgb", "alpha", "depth", "normal"):
        assert np.abs(a[key] - b[key]).max() < 1e-12, key


def test_stp_gradients_match_finite_differences():
    rng = np.random.default_rng(5)
    n = 6
    s = rng.uniform(0.12, 0.3, (n, 2))
    q = rng.normal(size=(n, 4))
    sc = Scene(np.stack([rng.uniform(-0.3, 0.3, n), rng.uniform(-0.3, 0.3, n), rng.uniform(1.8, 2.2, n)],
                        1).astype(np.float32),
               (q / np.linalg.norm(q, axis=1, keepdims=True)).astype(np.float32), s.astype(np.float32),
               (rng.uniform(-1.5, 1.5, (n, 2)) / s).astype(np.float32), rng.uniform(0.3, 0.9, n).astype(np.float32),
               f32_to_bf16_bits(rng.normal(0, 0.3, (n, 48)).astype(np.float32)))
    cam = Camera(20, 20, 17.0, 17.0, 10.0, 10.0)
    g = dict(rgb=rng.normal(size=(3, 20, 20)), alpha=rng.normal(size=(20, 20)), depth=rng.normal(size=(20, 20)),
             normal=rng.normal(size=(3, 20, 20)))
    ref = O.render(sc, cam, grad_images=g, order="stp")
    assert ref["margin"].min() > 1e-4 and ref["n_contrib"].max() > 1
    binning = ref["binning"]
    prm = O.Params(sc)
    c64 = O.CamF64(cam)

    def loss_of(pr):
        tot = 0.0
        for tile in range(binning.tiles_x * binning.tiles_y):
            s0, e0 = binning.ranges[tile]
            if e0 <= s0:
                continue
            xs, ys = O._tile_pixels(cam, tile, binning.tiles_x)
            r = O._composite_resort(pr, c64, torch.from_numpy(binning.vals[s0:e0].astype(np.int64)), t64(xs), t64(ys))
            tot += float((t64(g["rgb"][:, ys, xs].T) * r["rgb"]).sum() + (t64(g["alpha"][ys, xs]) * r["alpha"]).sum()
                         + (t64(g["depth"][ys, xs]) * r["depth"]).sum()
                         + (t64(g["normal"][:, ys, xs].T) * r["normal"]).sum())
        return tot

    for name in ("mean", "quat", "scale", "curv", "opacity"):
        leaf = getattr(prm, name)
        flat = leaf.view(-1)
        gref = ref["grads"][name].reshape(-1)
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
