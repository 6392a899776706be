"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Sizes: the 1,000-primitive 128x128 scene in full; the 300k-primitive 1600x1200 object
scene in full on the GPU against oracle crops; the 3M-primitive 1297x840 scene in full on
the GPU against bit-exact tile rectangles for every primitive, bit-exact lists of sampled
tiles, sampled pixels and a gradient crop; sampled pixels of both large scenes against the
oracle's list-free compositing (every primitive that can reach the pixel, no tile lists).
Plus edge cases. Every pixel meets the bars of tests/parity_util.py, against one of its
branches where a decision is within rounding distance of its threshold.
"""
import numpy as np
import pytest
import torch

import oracle.qgs_oracle as O
from paper_2411_16392_gb300.scenes import (Camera, Scene, f32_to_bf16_bits, scene_object, scene_small,
                                           scene_unbounded)
from tests.parity_util import check_grads, check_images, check_pixels, near_pixels

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_16392_gb300 import _lib as L
    L.load()
    return torch.device("cuda", 0)


def _ras(dev, **kw):
    from paper_2411_16392_gb300.render import Rasterizer
    return Rasterizer(dev, **kw)


def _ds(sc, dev):
    from paper_2411_16392_gb300.render import DeviceScene
    return DeviceScene.from_host(sc, dev)


def _np(out):
    return {k: v.detach().cpu().numpy() for k, v in out.items()}


def _grad_images(H, W, seed, mask=None):
    rng = np.random.default_rng(seed)
    g = dict(rgb=rng.normal(size=(3, H, W)), alpha=rng.normal(size=(H, W)), depth=rng.normal(size=(H, W)),
             normal=rng.normal(size=(3, H, W)))
    if mask is not None:
        for k in g:
            g[k] = g[k] * mask
    return {k: v.astype(np.float32).astype(np.float64) for k, v in g.items()}


def _to_dev(g, dev):
    return {k: torch.from_numpy(np.ascontiguousarray(v, np.float32)).to(dev) for k, v in g.items()}


def _check_binning(ras, ref_bin, label):
    keys, vals, ranges, rects = ras.binning()
    vis = ref_bin.count > 0
    want_rect = np.where(vis[:, None], ref_bin.rect, -1)
    assert np.array_equal(rects, want_rect), label + ": tile rectangles differ"
    if ref_bin.keys is not None:
        assert keys.shape == ref_bin.keys.shape, label
        assert np.array_equal(keys, ref_bin.keys), label + ": keys differ"
        assert np.array_equal(vals, ref_bin.vals), label + ": values differ"
        r = ranges.astype(np.int64)
        empty = ref_bin.ranges[:, 1] == ref_bin.ranges[:, 0]
        assert np.array_equal(r[~empty], ref_bin.ranges[~empty]), label + ": tile ranges differ"
        assert np.all(r[empty, 1] == r[empty, 0]), label + ": empty tiles must have empty ranges"
    return keys, vals, ranges, rects


# ----------------------------------------------------------------------------- small scene
@pytest.mark.parametrize("sort_mode", [0, 1])
def test_small_scene_forward(dev, sort_mode):
    sc, cam = scene_small(0, 1000)
    ras = _ras(dev, sort_mode=sort_mode)
    out = _np(ras.forward(_ds(sc, dev), cam))
    ref = O.render(sc, cam)
    _check_binning(ras, ref["binning"], f"small/mode{sort_mode}")
    check_images(out, ref, sc, cam, ref["binning"], label=f"small/mode{sort_mode}")
    T, nc = ras.residue()
    ok = ~near_pixels(ref)
    assert np.array_equal(nc[ok], ref["n_contrib"][ok])
    assert np.abs(T - ref["T_final"])[ok].max() <= 1e-4
    st = ras.stats()
    print("stats", st, "oracle pair evals", int(ref["n_eval"].sum()))
    amb_evals = int(np.abs(ref["n_eval"][~ok]).sum())
    assert abs(st["pair_evals"] - int(ref["n_eval"].sum())) <= amb_evals + 256 * (~ok).sum()
    assert st["n_instances"] == len(ref["binning"].keys)


def test_sort_modes_bit_identical(dev):
    sc, cam = scene_small(1, 1000)
    outs = []
    bins = []
    for m in (0, 1):
        ras = _ras(dev, sort_mode=m)
        outs.append(_np(ras.forward(_ds(sc, dev), cam)))
        bins.append(ras.binning())
    for k in outs[0]:
        assert np.array_equal(outs[0][k], outs[1][k]), k
    for a, b in zip(bins[0], bins[1]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("order", ["centre", "stp"])
def test_tile_mask_store_does_not_change_results(dev, order):
    """The emission replays the tile-count pass's masks; without the store (capacity 0),
    with one too small for the frame (some primitives tested again) and with the default,
    the instances and images are identical (sort modes 0 and 1, both orderings)."""
    sc, cam = scene_small(2, 3000)
    sc.scale *= np.float32(2.0)
    ds = _ds(sc, dev)
    for mode in ((0, 1) if order == "centre" else (0,)):
        res = []
        for cap in (None, 0, 64):
            ras = _ras(dev, sort_mode=mode, order=order)
            if cap is not None:
                ras.set_tile_mask_capacity(cap)
            out = _np(ras.forward(ds, cam))
            res.append((out, ras.binning()))
        for out, b in res[1:]:
            for k in out:
                assert np.array_equal(out[k], res[0][0][k]), (mode, k)
            for x, y in zip(b, res[0][1]):
                assert np.array_equal(x, y), mode
    with pytest.raises(Exception):
        _ras(dev).set_tile_mask_capacity(-1)


def test_pair_counters_switch(dev):
    """Without the per-pair counters the compositing kernels give bit-identical images and
    gradients; the counters then read -1 and come back when re-enabled."""
    sc, cam = scene_small(3, 1500)
    ds = _ds(sc, dev)
    g = _to_dev(_grad_images(cam.H, cam.W, 5), dev)
    res = []
    for on in (True, False):
        ras = _ras(dev)
        ras.set_pair_counters(on)
        out = _np(ras.forward(ds, cam))
        gr = {k: v.cpu().numpy() for k, v in ras.backward(ds, cam, g).items()}
        st = ras.stats()
        res.append((out, gr, st))
        if not on:
            assert st["pair_evals"] == -1 and st["bwd_pairs"] == -1
            ras.set_pair_counters(True)
            ras.forward(ds, cam)
            assert ras.stats()["pair_evals"] == res[0][2]["pair_evals"]
    assert res[0][2]["pair_evals"] > 0
    for k in res[0][0]:
        assert np.array_equal(res[0][0][k], res[1][0][k]), k
    for k in res[0][1]:   # equal up to the order of the floating-point atomic accumulation
        assert np.abs(res[0][1][k] - res[1][1][k]).max() <= 1e-5 * max(np.abs(res[0][1][k]).max(), 1e-30), k


def test_sort_modes_same_gradients(dev):
    """Both key modes give the same gradients: the depth-ordered packed keys (gradient
    records by depth rank) and the primitive-order 64-bit keys (records by index, the
    preprocessing backward over the compacted visible primitives in index order). The tile
    lists are identical, so the gradients agree up to the order of the atomic additions;
    the scene is sparse enough on screen that some primitives are culled."""
    sc, cam = scene_small(4, 2000)
    sc.mean[:, 0] *= np.float32(6.0)   # spread beyond the frame: part of the scene is culled
    ds = _ds(sc, dev)
    g = _to_dev(_grad_images(cam.H, cam.W, 11), dev)
    res = []
    for m in (0, 1):
        ras = _ras(dev, sort_mode=m)
        ras.forward(ds, cam)
        assert 0 < ras.stats()["n_visible"] < sc.n
        res.append({k: v.cpu().numpy() for k, v in ras.backward(ds, cam, g).items()})
    for k in res[0]:
        a, b = res[0][k], res[1][k]
        assert np.abs(a).max() > 0, k
        assert np.abs(a - b).max() <= 1e-5 * np.abs(a).max(), (k, np.abs(a - b).max(), np.abs(a).max())


def test_small_scene_backward(dev):
    sc, cam = scene_small(0, 1000)
    g = _grad_images(cam.H, cam.W, 7)
    ref = O.render(sc, cam, grad_images=g)
    ras = _ras(dev)
    ds = _ds(sc, dev)
    ras.forward(ds, cam)
    gg = ras.backward(ds, cam, _to_dev(g, dev))
    gg = {k: v.cpu().numpy() for k, v in gg.items()}
    check_grads(gg, ref, sc, cam, g, ref["binning"], label="small/bwd")


def test_autograd_function_matches_raw_backward(dev):
    from paper_2411_16392_gb300.render import render
    sc, cam = scene_small(2, 500)
    ds = _ds(sc, dev)
    ras = _ras(dev)
    leaves = [t.clone().requires_grad_(True) for t in (ds.mean, ds.quat, ds.scale, ds.curv, ds.opacity)]
    sh = ds.sh.view(torch.bfloat16).clone().requires_grad_(True)
    rgb, alpha, depth, normal = render(ras, cam, *leaves, sh)
    g = _to_dev(_grad_images(cam.H, cam.W, 3), dev)
    loss = (rgb * g["rgb"]).sum() + (alpha * g["alpha"]).sum() + (depth * g["depth"]).sum() + \
        (normal * g["normal"]).sum()
    loss.backward()
    raw = ras.backward(ds, cam, g) if ras.forward(ds, cam) is not None else None
    for leaf, k in zip(leaves, ("mean", "quat", "scale", "curv", "opacity")):
        assert torch.allclose(leaf.grad, raw[k], rtol=1e-5, atol=1e-7), k
    assert torch.allclose(sh.grad.float(), raw["sh"].to(torch.bfloat16).float())


# ----------------------------------------------------------------------------- edge cases
def test_empty_and_culled_scenes(dev):
    ras = _ras(dev)
    cam = Camera(37, 23, 30.0, 30.0, 18.5, 11.5)
    sc, _ = scene_small(0, 50)
    empty = sc.subset(np.arange(0))
    out = _np(ras.forward(_ds(empty, dev), cam))
    assert all(np.all(v == 0) for v in out.values())
    behind = sc.copy()
    behind.mean[:, 2] = -behind.mean[:, 2]
    out = _np(ras.forward(_ds(behind, dev), cam))
    assert all(np.all(v == 0) for v in out.values())
    assert ras.stats()["n_instances"] == 0


def test_invalid_parameters_are_culled(dev):
    sc, cam = scene_small(3, 300)
    bad = sc.copy()
    bad.mean[0, 0] = np.nan
    bad.quat[1] = 0
    bad.scale[2, 0] = 0
    bad.opacity[3] = np.inf
    ras = _ras(dev)
    out = _np(ras.forward(_ds(bad, dev), cam))
    ref = O.render(bad, cam)
    _check_binning(ras, ref["binning"], "invalid")
    assert not ref["binning"].visible[:4].any()
    check_images(out, ref, bad, cam, ref["binning"], label="invalid")


@pytest.mark.parametrize("W,H", [(1, 1), (17, 33), (129, 70)])
def test_ragged_image_sizes(dev, W, H):
    sc, _ = scene_small(4, 400)
    cam = Camera(W, H, 128.0, 128.0, W / 2, H / 2)
    ras = _ras(dev)
    out = _np(ras.forward(_ds(sc, dev), cam))
    ref = O.render(sc, cam)
    _check_binning(ras, ref["binning"], f"ragged{W}x{H}")
    check_images(out, ref, sc, cam, ref["binning"], label=f"ragged{W}x{H}")


def test_camera_inside_the_cloud_near_plane_clipping(dev):
    sc, cam = scene_small(5, 1000)
    sc.mean[:, 2] -= 3.6
    sc.scale *= 4
    cam = Camera(96, 80, 70.0, 70.0, 48.0, 40.0)
    ras = _ras(dev)
    ds = _ds(sc, dev)
    out = _np(ras.forward(ds, cam))
    ref = O.render(sc, cam)
    _check_binning(ras, ref["binning"], "inside")
    check_images(out, ref, sc, cam, ref["binning"], label="inside")
    g = _grad_images(cam.H, cam.W, 11)
    refg = O.render(sc, cam, ref["binning"], grad_images=g)
    gg = {k: v.cpu().numpy() for k, v in ras.backward(ds, cam, _to_dev(g, dev)).items()}
    check_grads(gg, refg, sc, cam, g, ref["binning"], label="inside/bwd")


def test_planar_primitives(dev):
    """Zero and near-zero curvature (the 2DGS limit, and the near-planar share of the
    unbounded scene)."""
    sc, cam = scene_small(6, 800)
    sc.curv[:400] = 0
    sc.curv[400:] = (np.random.default_rng(0).uniform(-1e-6, 1e-6, (400, 2)) / sc.scale[400:]).astype(np.float32)
    ras = _ras(dev)
    ds = _ds(sc, dev)
    out = _np(ras.forward(ds, cam))
    ref = O.render(sc, cam)
    check_images(out, ref, sc, cam, ref["binning"], label="planar")
    g = _grad_images(cam.H, cam.W, 12)
    refg = O.render(sc, cam, ref["binning"], grad_images=g)
    gg = {k: v.cpu().numpy() for k, v in ras.backward(ds, cam, _to_dev(g, dev)).items()}
    check_grads(gg, refg, sc, cam, g, ref["binning"], label="planar/bwd")


# ----------------------------------------------------------------------------- 300k object scene
@pytest.fixture(scope="module")
def object_scene():
    return scene_object(0)


def test_object_scene_crop_forward_backward(dev, object_scene):
    """Full 1600x1200 render and backward on the GPU; the oracle renders a tile-aligned
    64x64 crop (lists from the full camera) with upstream gradients only there."""
    sc, cam = object_scene
    x0, y0, w = 768, 560, 64
    binning = O.bin_fp32(sc, cam, emit=False)
    TX = binning.tiles_x
    tiles = [(y0 // 16 + j) * TX + (x0 // 16 + i) for j in range(w // 16) for i in range(w // 16)]
    ras = _ras(dev)
    ds = _ds(sc, dev)
    out = _np(ras.forward(ds, cam))
    keys, vals, ranges, rects = _check_binning(ras, binning, "object")
    for t in tiles:
        s, e = ranges[t]
        assert np.array_equal(vals[s:e], O.tile_list(binning, t)), t
    ref = O.render(sc, cam, binning, tiles=tiles)
    crop = np.zeros((cam.H, cam.W), bool)
    crop[y0:y0 + w, x0:x0 + w] = True
    # strongly curved patches (|kappa| up to 20) make grazing silhouettes common
    check_images(out, ref, sc, cam, binning, mask=crop, label="object/crop")
    g = _grad_images(cam.H, cam.W, 21, crop)
    refg = O.render(sc, cam, binning, tiles=tiles, grad_images=g)
    gg = {k: v.cpu().numpy() for k, v in ras.backward(ds, cam, _to_dev(g, dev)).items()}
    touched = np.unique(np.concatenate([O.tile_list(binning, t) for t in tiles])).astype(np.int64)
    check_grads(gg, refg, sc, cam, g, binning, mask=crop, idx=touched, label="object/crop bwd")
    for k, v in gg.items():
        assert np.isfinite(v).all(), k


# ----------------------------------------------------------------------------- 3M unbounded scene
@pytest.fixture(scope="module")
def unbounded():
    sc, cam = scene_unbounded(0)
    return sc, cam, O.bin_fp32(sc, cam, emit=False)


def test_unbounded_scene_full_size(dev, unbounded):
    """3M primitives at 1297x840 (the benchmark workload): bit-exact tile rectangles for
    all primitives, bit-exact sorted lists and keys of sampled tiles, sampled pixels
    against the oracle one by one, and output invariants everywhere."""
    sc, cam, binning = unbounded
    ras = _ras(dev)
    ds = _ds(sc, dev)
    out = _np(ras.forward(ds, cam))
    keys, vals, ranges, rects = _check_binning(ras, binning, "unbounded")
    st = ras.stats()
    assert st["n_instances"] == int(binning.count.sum())
    rng = np.random.default_rng(0)
    TX = binning.tiles_x
    ntiles = TX * binning.tiles_y
    sample_tiles = np.unique(np.concatenate([[0, ntiles - 1, ntiles // 2], rng.integers(0, ntiles, 12)]))
    for t in sample_tiles:
        s, e = ranges[t]
        lst = O.tile_list(binning, t)
        assert np.array_equal(vals[s:e], lst), t
        want = (np.uint64(t) << np.uint64(32)) | binning.zbits[lst].astype(np.uint64)
        assert np.array_equal(keys[s:e], want), t
    pix = [(int(x), int(y)) for x, y in zip(rng.integers(0, cam.W, 40), rng.integers(0, cam.H, 40))]
    pix += [(0, 0), (cam.W - 1, cam.H - 1), (cam.W // 2, cam.H // 2)]
    _, br = check_pixels(out, sc, cam, pix, binning, label="unbounded/sampled")
    T, nc = ras.residue()
    for (x, y), it in zip(pix, br):
        if len(it["leaves"]) == 1:
            assert nc[y, x] == it["n_contrib"][0], (x, y)
    assert np.all((out["alpha"] >= 0) & (out["alpha"] <= 1))
    assert np.allclose(T, 1 - out["alpha"], atol=1e-6)
    assert all(np.isfinite(v).all() for v in out.values())


def test_unbounded_scene_gradient_crop(dev, unbounded):
    """Full-size backward at 3M primitives with upstream gradients on a 32x32 crop,
    against the oracle's gradient of the same crop."""
    sc, cam, binning = unbounded
    x0, y0, w = 640, 416, 32
    TX = binning.tiles_x
    tiles = [(y0 // 16 + j) * TX + (x0 // 16 + i) for j in range(w // 16) for i in range(w // 16)]
    crop = np.zeros((cam.H, cam.W), bool)
    crop[y0:y0 + w, x0:x0 + w] = True
    # ~1000 pairs are visited per pixel here, so more pixels hold a pair near a decision
    g = _grad_images(cam.H, cam.W, 31, crop)
    refg = O.render(sc, cam, binning, tiles=tiles, grad_images=g)
    ras = _ras(dev)
    ds = _ds(sc, dev)
    out = _np(ras.forward(ds, cam))
    check_images(out, refg, sc, cam, binning, mask=crop, label="unbounded/crop")
    gg = {k: v.cpu().numpy() for k, v in ras.backward(ds, cam, _to_dev(g, dev)).items()}
    touched = np.unique(np.concatenate([O.tile_list(binning, t) for t in tiles])).astype(np.int64)
    check_grads(gg, refg, sc, cam, g, binning, mask=crop, idx=touched, label="unbounded/crop bwd")
    untouched = np.setdiff1d(np.arange(sc.n), touched)[:100000]
    for k, v in gg.items():
        assert np.isfinite(v).all(), k
        assert np.all(v[untouched] == 0), k


# ----------------------------------------------------------------------------- list-free check
@pytest.mark.parametrize("which", ["object", "unbounded"])
def test_listfree_sampled_pixels(dev, which, object_scene, unbounded):
    """The tile lists drop no pair with a hit (the bound of the supplementary's bounding-box
    section must be conservative): sampled pixels of the full-size renders against the
    oracle's list-free compositing, which takes every primitive whose centre lies in front
    of the near plane and within 3 max(s_u, s_v) of the pixel's ray (arc >= chord), in
    (FP64 centre depth, index) order, with no FP32 recipe and no tile list."""
    if which == "object":
        sc, cam = object_scene
        rng = np.random.default_rng(5)
        # pixels on the object's silhouette region and inside it
        xs = rng.integers(cam.W // 4, 3 * cam.W // 4, 48)
        ys = rng.integers(cam.H // 4, 3 * cam.H // 4, 48)
    else:
        sc, cam, _ = unbounded
        rng = np.random.default_rng(6)
        xs = rng.integers(0, cam.W, 48)
        ys = rng.integers(0, cam.H, 48)
    pix = [(int(x), int(y)) for x, y in zip(xs, ys)]
    ras = _ras(dev)
    out = _np(ras.forward(_ds(sc, dev), cam))
    st, br = check_pixels(out, sc, cam, pix, None, list_free=True, label=f"{which}/list-free")
    assert sum(len(it["leaves"][0]) > 0 for it in br) == len(pix)
    lit = sum(float(it["leaves"][0]["alpha"][0]) > 1e-3 for it in br)
    print(f"{which}: {lit} of {len(pix)} sampled pixels covered")
    assert lit >= len(pix) // 4
