"""Serving on the GPU: each result is the same alone (render_forward) and in the mix
(several requests of mixed resolutions in flight on a 4-slot server, or batched into
shared launches on a 1-slot server)."""
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


@pytest.mark.parametrize("slots,batch", [(4, 1), (1, 4)])
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


def test_served_backward_equals_plain_backward(dev):
    """A backward request (forward + backward with upstream planes given on the host) gives
    the planes and parameter gradients of Rasterizer.forward/backward, up to the order of
    the floating-point atomic accumulation; forward requests queued with it still batch."""
    from paper_2411_16392_gb300.render import DeviceScene, Rasterizer
    from paper_2411_16392_gb300.serve import Server
    sc = serving_scene(3, 100_000)
    ds = DeviceScene.from_host(sc, dev)
    rng = np.random.default_rng(4)
    cam = orbit_camera(rng, res=(320, 240))
    H, W = cam.H, cam.W
    g_host = {"rgb": rng.normal(size=(3, H, W)).astype(np.float32),
              "alpha": rng.normal(size=(H, W)).astype(np.float32),
              "depth": rng.normal(size=(H, W)).astype(np.float32),
              "normal": rng.normal(size=(3, H, W)).astype(np.float32)}
    ras = Rasterizer(dev)
    ref_out = {k: v.clone() for k, v in ras.forward(ds, cam).items()}
    ref_g = {k: v.cpu().numpy() for k, v in
             ras.backward(ds, cam, {k: torch.from_numpy(v).to(dev) for k, v in g_host.items()}).items()}
    srv = Server(dev.index or 0, budget_bytes=16 << 30, slots=1, batch=4)
    sid = srv.load_scene(ds)
    others = [orbit_camera(rng) for _ in range(5)]
    t_fwd = [srv.submit(sid, c) for c in others[:3]]
    t_bwd = srv.submit(sid, cam, backward=True, grad_out=g_host)
    t_fwd += [srv.submit(sid, c) for c in others[3:]]
    n = sc.n
    got_g = {k: np.zeros(s, np.float32) for k, s in (("mean", (n, 3)), ("quat", (n, 4)), ("scale", (n, 2)),
                                                     ("curv", (n, 2)), ("opacity", (n,)), ("sh", (n, 48)))}
    got_out = {k: torch.zeros_like(v) for k, v in ref_out.items()}
    srv.wait(t_bwd, out=got_out, grads=got_g, timeout_ms=60_000)
    for t in t_fwd:
        srv.wait(t, timeout_ms=60_000)
    torch.cuda.synchronize()
    for k in ref_out:
        assert torch.equal(got_out[k], ref_out[k]), k
    for k in ref_g:
        scale = max(np.abs(ref_g[k]).max(), 1e-30)
        assert np.abs(got_g[k] - ref_g[k]).max() <= 1e-5 * scale, k
    assert np.abs(got_g["mean"]).max() > 0
    st = srv.stats()
    assert st["completed"] == 6 and st["failed"] == 0
    srv.close()
