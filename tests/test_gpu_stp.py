"""Parity of the StopThePop ordering (per-tile hit-depth lists, per-pixel resorting in a
buffer of 8, front-to-back backward) with the oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle.qgs_oracle as O
from paper_2411_16392_gb300.scenes import scene_object, scene_small
from tests.parity_util import check_grads, check_images, near_pixels

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
    return Rasterizer(dev, order="stp", **kw)


def _ds(sc, dev):
    from paper_2411_16392_gb300.render import DeviceScene
    return DeviceScene.from_host(sc, dev)


def _np(out):
    return {k: v.detach().cpu().numpy() for k, v in out.items()}


def _to_dev(g, dev):
    return {k: torch.from_numpy(np.ascontiguousarray(v, np.float32)).to(dev) for k, v in g.items()}


def _grad_images(H, W, seed, mask=1.0, extras=False):
    rng = np.random.default_rng(seed)
    g = dict(rgb=rng.normal(size=(3, H, W)), alpha=rng.normal(size=(H, W)), depth=rng.normal(size=(H, W)),
             normal=rng.normal(size=(3, H, W)))
    if extras:
        g["curvature"] = rng.normal(size=(H, W))
        g["distortion"] = rng.normal(size=(H, W))
    return {k: (v * mask).astype(np.float32).astype(np.float64) for k, v in g.items()}


def test_hit_depth_keys_and_lists_are_bit_exact(dev):
    sc, cam = scene_small(0, 1000)
    ras = _ras(dev)
    ras.forward(_ds(sc, dev), cam)
    keys, vals, ranges, rects = ras.binning()
    ref = O.bin_fp32(sc, cam, order="hit")
    assert np.array_equal(keys, ref.keys)
    assert np.array_equal(vals, ref.vals)
    # the order really differs from the centre-depth one
    assert not np.array_equal(vals, O.bin_fp32(sc, cam).vals)


@pytest.mark.parametrize("density", ["geodesic", "euclid"])
def test_small_scene_forward(dev, density):
    sc, cam = scene_small(0, 1000)
    ras = _ras(dev, density=density)
    out = _np(ras.forward(_ds(sc, dev), cam, extras=True))
    ref = O.render(sc, cam, order="stp", density=density, extras=True)
    check_images(out, ref, sc, cam, ref["binning"], extras=True, label=f"stp/small/{density}", order="stp",
                 density=density)
    T, nb = ras.residue()
    ok = ~near_pixels(ref, extras=True)
    assert np.array_equal(nb[ok], ref["n_contrib"][ok])   # blended pairs per pixel


def test_small_scene_backward(dev):
    sc, cam = scene_small(4, 800)
    g = _grad_images(cam.H, cam.W, 19)
    ref = O.render(sc, cam, order="stp", grad_images=g)
    ras = _ras(dev)
    ds = _ds(sc, dev)
    ras.forward(ds, cam)
    gg = {k: v.cpu().numpy() for k, v in ras.backward(ds, cam, _to_dev(g, dev)).items()}
    check_grads(gg, ref, sc, cam, g, ref["binning"], label="stp/small/bwd", order="stp")


def test_small_scene_backward_with_extra_channels(dev):
    sc, cam = scene_small(6, 700)
    g = _grad_images(cam.H, cam.W, 29, extras=True)
    ref = O.render(sc, cam, order="stp", extras=True, grad_images=g)
    ras = _ras(dev)
    ds = _ds(sc, dev)
    ras.forward(ds, cam, extras=True)
    gg = {k: v.cpu().numpy() for k, v in ras.backward(ds, cam, _to_dev(g, dev)).items()}
    check_grads(gg, ref, sc, cam, g, ref["binning"], extras=True, label="stp/small/bwd+extras", order="stp")


def test_object_scene_crop(dev):
    """Strongly curved primitives, where the hit order and the centre order differ most."""
    sc, cam = scene_object(0)
    x0, y0, w = 768, 560, 48
    binning = O.bin_fp32(sc, cam, emit=False, order="hit")
    TX = binning.tiles_x
    tiles = [(y0 // 16 + j) * TX + (x0 // 16 + i) for j in range(w // 16) for i in range(w // 16)]
    ras = _ras(dev)
    ds = _ds(sc, dev)
    out = _np(ras.forward(ds, cam))
    keys, vals, ranges, rects = ras.binning()
    for t in tiles:
        s, e = ranges[t]
        assert np.array_equal(vals[s:e], O.tile_list(binning, t)), t
    ref = O.render(sc, cam, binning, tiles=tiles, order="stp")
    crop = np.zeros((cam.H, cam.W), bool)
    crop[y0:y0 + w, x0:x0 + w] = True
    check_images(out, ref, sc, cam, binning, mask=crop, label="stp/object/crop", order="stp")
    g = _grad_images(cam.H, cam.W, 31, crop)
    refg = O.render(sc, cam, binning, tiles=tiles, order="stp", grad_images=g)
    gg = {k: v.cpu().numpy() for k, v in ras.backward(ds, cam, _to_dev(g, dev)).items()}
    touched = np.unique(np.concatenate([O.tile_list(binning, t) for t in tiles])).astype(np.int64)
    check_grads(gg, refg, sc, cam, g, binning, mask=crop, idx=touched, label="stp/object/crop bwd", order="stp")


def test_batch_refuses_the_stp_order(dev):
    from paper_2411_16392_gb300 import _lib as L
    sc, cam = scene_small(0, 100)
    ras = _ras(dev)
    with pytest.raises(L.QGSError) as e:
        ras.forward_batch(_ds(sc, dev), [cam])
    assert e.value.status == 1
