"""The allocation-free forward entry point (render_forward_noalloc) against render_forward.

render_forward_noalloc serves callers that cannot allocate device memory while rendering
(a host whose memory manager owns the GPU's memory pool, or a real-time loop that bans
cudaMalloc/cudaFree after warm-up). It must produce the same images as the allocating
entry point, twice in a row (the static scratch keeps the previous call's contents), and
must not grow the device's memory use after its first call.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2411_16392_gb300.scenes import Camera, scene_small
from tests.parity_util import TOL_ABS

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


def test_noalloc_forward_matches_render_forward_twice(dev):
    from paper_2411_16392_gb300 import _lib as L
    from paper_2411_16392_gb300.render import DeviceScene, Rasterizer
    lib = L.load()
    cases = [scene_small(0, 1000), scene_small(3, 2000)]
    cases[1] = (cases[1][0], Camera(200, 120, 150.0, 150.0, 100.0, 60.0))
    ras = Rasterizer(dev)
    prepared = []
    for sc, cam in cases:
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
            got = outs[rep]
            status = _noalloc(lib, ds, cam, got, dev)
            assert status == 0, L.STATUS.get(status, status)
        torch.cuda.synchronize()
        for ds, cam, want, outs in prepared:
            for k in want:
                err = (outs[rep][k] - want[k]).abs().max().item()
                assert err <= TOL_ABS, (rep, k, err)
    # the calls allocated no device memory (the scratch is static)
    assert torch.cuda.mem_get_info(dev)[0] == free_before


def test_noalloc_rejects_sizes_beyond_its_limits(dev):
    from paper_2411_16392_gb300 import _lib as L
    from paper_2411_16392_gb300.render import DeviceScene
    lib = L.load()
    sc, cam = scene_small(0, 1000)
    ds = DeviceScene.from_host(sc, dev)
    big = Camera(1024, 1024, 512.0, 512.0, 512.0, 512.0)   # 1M pixels > 262144
    got = _outputs(dev, big.H, big.W)
    assert _noalloc(lib, ds, big, got, dev) == 3            # QGS_ECAPACITY
    many, _ = scene_small(1, 40000)                          # > 32768 primitives
    assert _noalloc(lib, DeviceScene.from_host(many, dev), cam, _outputs(dev, cam.H, cam.W), dev) == 3
