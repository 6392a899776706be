"""The allocation-free forward entry point (render_forward_noalloc) against render_forward.

render_forward_noalloc serves callers that cannot allocate device memory while rendering
(a host whose memory manager owns the GPU's memory pool, or a real-time loop that bans
cudaMalloc/cudaFree after warm-up). It runs the same kernels on the same tile lists as
the allocating entry point, so its planes must be the same bit for bit, twice in a row
(the static scratch keeps the previous call's contents), and it must not grow the
device's memory use after its first call. Frames beyond its fixed capacities are refused
with QGS_ECAPACITY, including one whose tile-instance count (known only after the tile
test) exceeds the array's share for instances, and the next call works again.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2411_16392_gb300.scenes import Camera, scene_small

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_16392_gb300 import _lib as L
    L.load()
    return torch.device("cuda", 0)


def _outputs(dev, H, W):
    return dict(rgb=torch.full((3, H, W), 7.0, device=dev), alpha=torch.full((H, W), 7.0, device=dev),
                depth=torch.full((H, W), 7.0, device=dev), normal=torch.full((3, H, W), 7.0, device=dev))


def _noalloc(lib, ds, cam, out, dev):
    from paper_2411_16392_gb300 import _lib as L
    from paper_2411_16392_gb300.render import camera_to_c
    img = L.qgs_image(out["rgb"].data_ptr(), out["alpha"].data_ptr(), out["depth"].data_ptr(),
                      out["normal"].data_ptr())
    sc = ds.to_c()
    cc = camera_to_c(cam)
    st = C.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    return lib.render_forward_noalloc(C.byref(sc), C.byref(cc), C.byref(img), st)


def _cases():
    cases = [scene_small(0, 1000), scene_small(3, 2000), scene_small(5, 20000)]
    cases[1] = (cases[1][0], Camera(200, 120, 150.0, 150.0, 100.0, 60.0))
    cases[2] = (cases[2][0], Camera(333, 257, 260.0, 260.0, 166.5, 128.5))   # ragged tiles
    return cases


def test_noalloc_forward_matches_render_forward_twice(dev):
    from paper_2411_16392_gb300 import _lib as L
    from paper_2411_16392_gb300.render import DeviceScene, Rasterizer
    lib = L.load()
    ras = Rasterizer(dev)
    prepared = []
    for sc, cam in _cases():
        ds = DeviceScene.from_host(sc, dev)
        want = {k: v.clone() for k, v in ras.forward(ds, cam).items()}
        prepared.append((ds, cam, want, [_outputs(dev, cam.H, cam.W) for _ in range(2)]))
    # first call on this device: looks up the scratch array (done before measuring)
    ds, cam, _, outs = prepared[0]
    assert _noalloc(lib, ds, cam, _outputs(dev, cam.H, cam.W), dev) == 0
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info(dev)[0]
    for rep in range(2):
        for ds, cam, want, outs in prepared:
            status = _noalloc(lib, ds, cam, outs[rep], dev)
            assert status == 0, L.STATUS.get(status, status)
        torch.cuda.synchronize()
        for ds, cam, want, outs in prepared:
            for k in want:
                assert torch.equal(outs[rep][k], want[k]), (rep, k, (outs[rep][k] - want[k]).abs().max().item())
    # the calls allocated no device memory (the scratch is static)
    assert torch.cuda.mem_get_info(dev)[0] == free_before


def test_noalloc_rejects_sizes_beyond_its_limits(dev):
    from paper_2411_16392_gb300 import _lib as L
    from paper_2411_16392_gb300.render import DeviceScene, Rasterizer
    lib = L.load()
    sc, cam = scene_small(0, 1000)
    ds = DeviceScene.from_host(sc, dev)
    big = Camera(1024, 1024, 512.0, 512.0, 512.0, 512.0)   # 1M pixels > 262144
    assert _noalloc(lib, ds, big, _outputs(dev, big.H, big.W), dev) == 3            # QGS_ECAPACITY
    many, _ = scene_small(1, 40000)                          # > 32768 primitives
    assert _noalloc(lib, DeviceScene.from_host(many, dev), cam, _outputs(dev, cam.H, cam.W), dev) == 3
    # within the primitive, pixel and tile limits, but more than 1,048,576 tile instances:
    # refused after the tile test
    wide, _ = scene_small(2, 30000)
    wide.scale *= np.float32(20.0)
    cam512 = Camera(512, 512, 512.0, 512.0, 256.0, 256.0)
    dw = DeviceScene.from_host(wide, dev)
    ras = Rasterizer(dev)
    ras.forward(dw, cam512)
    assert ras.stats()["n_instances"] > (1 << 20)
    assert _noalloc(lib, dw, cam512, _outputs(dev, cam512.H, cam512.W), dev) == 3
    # the next call renders correctly again
    want = {k: v.clone() for k, v in ras.forward(ds, cam).items()}
    got = _outputs(dev, cam.H, cam.W)
    assert _noalloc(lib, ds, cam, got, dev) == 0
    torch.cuda.synchronize()
    for k in want:
        assert torch.equal(got[k], want[k]), k
