"""Serving on the GPU: each result is the same alone (render_forward) and in the mix
(several requests of mixed resolutions in flight on a 4-slot server, or batched into
shared launches on a 2-slot server)."""
import numpy as np
import pytest
import torch

from paper_2411_16392_gb300.scenes import orbit_camera, serving_scene
from tests.parity_util import TOL_ABS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_16392_gb300 import _lib as L
    L.load()
    return torch.device("cuda", 0)


@pytest.mark.parametrize("slots,batch", [(4, 1), (2, 4)])
def test_results_alone_equal_results_in_the_mix(dev, slots, batch):
    from paper_2411_16392_gb300.render import DeviceScene, Rasterizer
    from paper_2411_16392_gb300.serve import Server
    sc = serving_scene(0, 200_000)
    ds = DeviceScene.from_host(sc, dev)
    rng = np.random.default_rng(0)
    cams = [orbit_camera(rng) for _ in range(12)]
    ras = Rasterizer(dev)
    alone = []
    for cam in cams:
        o = ras.forward(ds, cam)
        alone.append({k: v.clone() for k, v in o.items()})
    srv = Server(dev.index or 0, budget_bytes=16 << 30, slots=slots, batch=batch)
    sid = srv.load_scene(ds)
    del ds
    tickets = [srv.submit(sid, cam) for cam in cams]      # all in flight together
    for i, (t, cam, ref) in enumerate(zip(tickets, cams, alone)):
        out = {k: torch.full_like(v, 9.0) for k, v in ref.items()}
        srv.wait(t, out=out, timeout_ms=60_000)
        torch.cuda.synchronize()
        for k in ref:
            err = (out[k] - ref[k]).abs().max().item()
            if err > TOL_ABS:
                bad = (out[k] - ref[k]).abs().reshape(-1, cam.H, cam.W).amax(0) > TOL_ABS
                ys, xs = torch.nonzero(bad, as_tuple=True)
                tiles = sorted(set(((ys // 16) * ((cam.W + 15) // 16) + xs // 16).tolist()))
                fresh = Rasterizer(dev).forward(DeviceScene.from_host(sc, dev), cam)[k]
                print(f"request {i} {cam.W}x{cam.H} plane {k}: {int(bad.sum())} px in {len(tiles)} tiles "
                      f"{tiles[:8]}; served {out[k].reshape(-1, cam.H, cam.W)[:, ys[0], xs[0]].tolist()} "
                      f"alone {ref[k].reshape(-1, cam.H, cam.W)[:, ys[0], xs[0]].tolist()} "
                      f"fresh {fresh.reshape(-1, cam.H, cam.W)[:, ys[0], xs[0]].tolist()}")
            assert err <= TOL_ABS, (i, k, err)
    st = srv.stats()
    print("serve stats", st)
    assert st["completed"] == len(cams) and st["failed"] == 0
    assert st["max_in_flight"] >= 2
    if batch > 1:
        assert st["max_batch"] >= 2
    srv.close()
