"""Parity of the extra channels (curvature map, depth distortion, median depth) and of
the Euclidean-density variant with the FP64 oracle, forward and backward, through the
C ABI."""
import numpy as np
import pytest
import torch

import oracle.qgs_oracle as O
from paper_2411_16392_gb300.scenes import orbit_camera, scene_object, scene_small, serving_scene
from tests.parity_util import check_grads, check_images

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


def _to_dev(g, dev):
    return {k: torch.from_numpy(np.ascontiguousarray(v, np.float32)).to(dev) for k, v in g.items()}


def _grad_images(H, W, seed, mask=1.0, extras=True):
    rng = np.random.default_rng(seed)
    g = dict(rgb=rng.normal(size=(3, H, W)), alpha=rng.normal(size=(H, W)), depth=rng.normal(size=(H, W)),
             normal=rng.normal(size=(3, H, W)))
    if extras:
        g["curvature"] = rng.normal(size=(H, W))
        g["distortion"] = rng.normal(size=(H, W))
    return {k: (v * mask).astype(np.float32).astype(np.float64) for k, v in g.items()}


@pytest.mark.parametrize("density", ["geodesic", "euclid"])
def test_small_scene_all_channels(dev, density):
    sc, cam = scene_small(0, 1000)
    ras = _ras(dev, density=density)
    out = _np(ras.forward(_ds(sc, dev), cam, extras=True))
    ref = O.render(sc, cam, density=density, extras=True)
    check_images(out, ref, sc, cam, ref["binning"], extras=True, label=f"small/{density}", density=density)


def test_euclid_differs_from_geodesic_where_curved(dev):
    """The two densities agree on planar primitives and differ on curved ones (the
    variant is really switched)."""
    sc, cam = scene_small(3, 600)
    ds = _ds(sc, dev)
    a = _np(_ras(dev).forward(ds, cam))
    b = _np(_ras(dev, density="euclid").forward(ds, cam))
    assert np.abs(a["alpha"] - b["alpha"]).max() > 1e-3
    flat = sc.copy()
    flat.curv[:] = 0
    dsf = _ds(flat, dev)
    a = _np(_ras(dev).forward(dsf, cam))
    b = _np(_ras(dev, density="euclid").forward(dsf, cam))
    for k in a:
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("density", ["geodesic", "euclid"])
def test_small_scene_backward_with_extra_channels(dev, density):
    sc, cam = scene_small(4, 800)
    g = _grad_images(cam.H, cam.W, 17)
    ref = O.render(sc, cam, density=density, extras=True, grad_images=g)
    ras = _ras(dev, density=density)
    ds = _ds(sc, dev)
    ras.forward(ds, cam, extras=True)
    gg = {k: v.cpu().numpy() for k, v in ras.backward(ds, cam, _to_dev(g, dev)).items()}
    check_grads(gg, ref, sc, cam, g, ref["binning"], extras=True, label=f"small/{density}/bwd+extras",
                density=density)


def test_curvature_gradient_without_extra_forward(dev):
    """A curvature-only upstream gradient needs no residue: the backward recomputes K per
    pair, so it is accepted after a forward of the base planes and gives the gradient of
    a forward with every plane."""
    sc, cam = scene_small(5, 500)
    rng = np.random.default_rng(3)
    g = {"curvature": rng.normal(size=(cam.H, cam.W)).astype(np.float32)}
    ras = _ras(dev)
    ds = _ds(sc, dev)
    ras.forward(ds, cam)
    g1 = {k: v.cpu().numpy() for k, v in ras.backward(ds, cam, _to_dev(g, dev)).items()}
    ras.forward(ds, cam, extras=True)
    g2 = {k: v.cpu().numpy() for k, v in ras.backward(ds, cam, _to_dev(g, dev)).items()}
    for k in g1:   # equal up to the order of the floating-point atomic accumulation
        assert np.abs(g1[k] - g2[k]).max() <= 1e-5 * max(np.abs(g2[k]).max(), 1e-30), k
    assert np.abs(g1["curv"]).max() > 0


def test_extra_channel_state_errors(dev):
    from paper_2411_16392_gb300 import _lib as L
    sc, cam = scene_small(0, 300)
    ras = _ras(dev)
    ds = _ds(sc, dev)
    o = ras.forward(ds, cam)
    with pytest.raises(L.QGSError) as e:       # the distortion needs the forward's moments
        ras.backward(ds, cam, {"distortion": torch.zeros_like(o["alpha"])})
    assert e.value.status == 8
    ras.forward(ds, cam, extras=True)
    with pytest.raises(L.QGSError) as e:       # the median depth has no gradient
        ras.backward(ds, cam, {"median_depth": torch.zeros_like(o["alpha"])})
    assert e.value.status == 1


def test_object_scene_crop_extra_channels(dev):
    """Strongly curved patches (|kappa| up to 20): full 1600x1200 GPU render with every
    plane against an oracle crop, forward and backward."""
    sc, cam = scene_object(0)
    x0, y0, w = 768, 560, 48
    binning = O.bin_fp32(sc, cam, emit=False)
    TX = binning.tiles_x
    tiles = [(y0 // 16 + j) * TX + (x0 // 16 + i) for j in range(w // 16) for i in range(w // 16)]
    ras = _ras(dev)
    ds = _ds(sc, dev)
    out = _np(ras.forward(ds, cam, extras=True))
    ref = O.render(sc, cam, binning, tiles=tiles, extras=True)
    crop = np.zeros((cam.H, cam.W), bool)
    crop[y0:y0 + w, x0:x0 + w] = True
    check_images(out, ref, sc, cam, binning, mask=crop, extras=True, label="object/extras")
    g = _grad_images(cam.H, cam.W, 23, crop)
    refg = O.render(sc, cam, binning, tiles=tiles, extras=True, grad_images=g)
    gg = {k: v.cpu().numpy() for k, v in ras.backward(ds, cam, _to_dev(g, dev)).items()}
    touched = np.unique(np.concatenate([O.tile_list(binning, t) for t in tiles])).astype(np.int64)
    check_grads(gg, refg, sc, cam, g, binning, mask=crop, idx=touched, extras=True, label="object/extras bwd")


def test_batched_extra_channels_equal_single_renders(dev):
    ds = _ds(serving_scene(2, 100_000), dev)
    rng = np.random.default_rng(9)
    cams = [orbit_camera(rng, res=(256, 256)), orbit_camera(rng, res=(130, 70)), orbit_camera(rng, res=(512, 384))]
    for density in ("geodesic", "euclid"):
        ras = _ras(dev, density=density)
        singles = [{k: v.clone() for k, v in ras.forward(ds, c, extras=True).items()} for c in cams]
        outs = ras.forward_batch(ds, cams, [{k: torch.full_like(v, 3.0) for k, v in s.items()} for s in singles])
        torch.cuda.synchronize()
        for v, (b, s) in enumerate(zip(outs, singles)):
            for k in s:
                assert torch.equal(b[k], s[k]), (density, v, k)
