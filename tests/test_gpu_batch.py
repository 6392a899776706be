"""Batched multi-view forward (render_forward_batch): every view's planes equal a plain
render_forward of that camera bit for bit, at mixed and ragged resolutions (with and
without the tile-mask store), and the batch's counters are the sums of the single
renders' counters."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2411_16392_gb300.scenes import Camera, orbit_camera, scene_small, serving_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_16392_gb300 import _lib as L
    L.load()
    return torch.device("cuda", 0)


def _singles(ras, ds, cams):
    outs, stats = [], []
    for cam in cams:
        o = ras.forward(ds, cam)
        outs.append({k: v.clone() for k, v in o.items()})
        stats.append(ras.stats())
    return outs, stats


def _assert_bit_equal(batch, singles, cams):
    for v, (b, s, cam) in enumerate(zip(batch, singles, cams)):
        for k in s:
            assert b[k].shape == s[k].shape
            diff = (b[k] != s[k]).sum().item()
            assert diff == 0, f"view {v} ({cam.W}x{cam.H}) plane {k}: {diff} values differ"


def test_batch_equals_single_renders_mixed_resolutions(dev):
    from paper_2411_16392_gb300.render import DeviceScene, Rasterizer
    ds = DeviceScene.from_host(serving_scene(1, 200_000), dev)
    rng = np.random.default_rng(5)
    cams = [orbit_camera(rng) for _ in range(6)]
    cams += [orbit_camera(rng, res=(17, 33)), orbit_camera(rng, res=(1, 1)), orbit_camera(rng, res=(129, 70))]
    ras = Rasterizer(dev)
    singles, st1 = _singles(ras, ds, cams)
    outs = [{k: torch.full_like(v, 7.0) for k, v in s.items()} for s in singles]
    ras.forward_batch(ds, cams, outs)
    torch.cuda.synchronize()
    _assert_bit_equal(outs, singles, cams)
    sb = ras.stats()
    # the batch keeps the same tiles of each rectangle as the single renders (tile test
    # against the parallelogram and the conic): the same lists, evaluations and blending
    for key in ("n_tiles", "n_instances", "n_visible", "pair_evals", "pair_isect", "pair_hits", "pair_blended"):
        assert sb[key] == sum(s[key] for s in st1), key
    assert sb["n_primitives"] == len(cams) * ds.n
    # the tile-mask store does not change the batch either: none, too small for the batch
    for cap in (0, 64):
        ras.set_tile_mask_capacity(cap)
        outs2 = [{k: torch.full_like(v, 5.0) for k, v in s.items()} for s in singles]
        ras.forward_batch(ds, cams, outs2)
        torch.cuda.synchronize()
        _assert_bit_equal(outs2, singles, cams)
        assert ras.stats()["n_instances"] == sb["n_instances"]
    # a second batch in another order reuses the buffers and still matches
    perm = [4, 0, 8, 2]
    outs2 = ras.forward_batch(ds, [cams[i] for i in perm])
    torch.cuda.synchronize()
    _assert_bit_equal(outs2, [singles[i] for i in perm], [cams[i] for i in perm])


def test_batch_of_one_and_the_small_scene(dev):
    from paper_2411_16392_gb300.render import DeviceScene, Rasterizer
    sc, cam = scene_small()
    ds = DeviceScene.from_host(sc, dev)
    ras = Rasterizer(dev)
    singles, _ = _singles(ras, ds, [cam])
    outs = ras.forward_batch(ds, [cam])
    torch.cuda.synchronize()
    _assert_bit_equal(outs, singles, [cam])
    # another camera, twice in one batch
    inside = Camera(96, 80, 90.0, 90.0, 48.0, 40.0, np.eye(3, dtype=np.float32), np.zeros(3, np.float32))
    singles, _ = _singles(ras, ds, [inside])
    outs = ras.forward_batch(ds, [inside, inside])
    torch.cuda.synchronize()
    _assert_bit_equal(outs, singles * 2, [inside, inside])


def test_batch_of_an_empty_scene(dev):
    from paper_2411_16392_gb300.render import DeviceScene, Rasterizer
    sc, cam = scene_small()
    ds = DeviceScene.from_host(sc.subset(np.zeros(0, dtype=np.int64)), dev)
    ras = Rasterizer(dev)
    singles, _ = _singles(ras, ds, [cam])
    outs = ras.forward_batch(ds, [cam, cam])
    torch.cuda.synchronize()
    _assert_bit_equal(outs, singles * 2, [cam, cam])


def test_batch_argument_errors(dev):
    from paper_2411_16392_gb300 import _lib as L
    from paper_2411_16392_gb300.render import DeviceScene, Rasterizer, camera_to_c
    sc, cam = scene_small()
    ds = DeviceScene.from_host(sc, dev)
    ras = Rasterizer(dev)
    with pytest.raises(L.QGSError) as e:
        ras.forward_batch(ds, [])
    assert e.value.status == 1
    o = ras.forward_batch(ds, [cam])[0]
    # n_views * n at 2^31: refused before any device work
    s = ds.to_c()
    s.n = 1 << 21
    cc = (L.qgs_camera * 1024)(*([camera_to_c(cam)] * 1024))
    im = (L.qgs_image * 1024)(*([L.qgs_image(o["rgb"].data_ptr(), o["alpha"].data_ptr(), o["depth"].data_ptr(),
                                             o["normal"].data_ptr())] * 1024))
    st = ras.lib.render_forward_batch(ras._ctx, C.byref(s), 1024, cc, im, None)
    assert st == 1
    # a NULL plane in one view
    im2 = (L.qgs_image * 2)(L.qgs_image(o["rgb"].data_ptr(), o["alpha"].data_ptr(), o["depth"].data_ptr(),
                                        o["normal"].data_ptr()), L.qgs_image(o["rgb"].data_ptr(), None, None, None))
    cc2 = (L.qgs_camera * 2)(camera_to_c(cam), camera_to_c(cam))
    assert ras.lib.render_forward_batch(ras._ctx, C.byref(ds.to_c()), 2, cc2, im2, None) == 1
    # no residue is kept: backward after a batch is a state error
    with pytest.raises(L.QGSError) as e:
        ras._last = (ds, cam)
        ras.backward(ds, cam, {"rgb": torch.zeros_like(o["rgb"])})
    assert e.value.status == 8
