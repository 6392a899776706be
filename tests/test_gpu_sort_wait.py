"""The radix sorts' bounded look-back waits: a wait that runs out is reported, not hung.

The single-kernel radix passes find each chunk's output offsets by waiting for the digit
counts that earlier chunks publish. Each wait is bounded; when it runs out, the sort sets
a failure word, the frame's later kernels do nothing, and the context reports the failure
(QGS_ECUDA) from the next call that waits for the frame. The test hook withholds chunk 0
of the depth sort's first pass, so nothing ever publishes the counts the other chunks
wait for (a flag that nothing sets): the waits give up after a short poll limit, the GPU
keeps answering, and the context renders correctly again afterwards.
"""
import numpy as np
import pytest
import torch

from paper_2411_16392_gb300.scenes import scene_small

pytestmark = pytest.mark.gpu

SPINS = 2000  # polls per wait (about a microsecond each)


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_16392_gb300 import _lib as L
    L.load()
    return torch.device("cuda", 0)


@pytest.fixture(scope="module")
def scene(dev):
    from paper_2411_16392_gb300.render import DeviceScene
    sc, cam = scene_small(7, 12000)   # ~8k visible primitives: a depth sort of several chunks
    return DeviceScene.from_host(sc, dev), cam


def _planes(ras, ds, cam):
    return {k: v.clone() for k, v in ras.forward(ds, cam).items()}


def _status(exc):
    return getattr(exc, "status", None)


def test_withheld_chunk_is_reported_by_check_frame(dev, scene):
    from paper_2411_16392_gb300 import _lib as L
    from paper_2411_16392_gb300.render import Rasterizer
    ds, cam = scene
    want = _planes(Rasterizer(dev), ds, cam)
    ras = Rasterizer(dev)
    ras.forward(ds, cam)                      # a good frame first: warm buffers
    ras.check_frame()
    assert ras.stats()["n_visible"] > 2048, "the depth sort needs at least two chunks"
    ras.debug_withhold_sort_chunk(SPINS)
    ras.forward(ds, cam)                      # returns before its sorts have run
    with pytest.raises(L.QGSError) as ei:
        ras.check_frame()
    assert _status(ei.value) == 4             # QGS_ECUDA
    torch.cuda.synchronize()                  # the GPU still answers
    # the failed frame is discarded: no backward of it
    g = {k: torch.zeros_like(v) for k, v in want.items()}
    with pytest.raises(L.QGSError) as eb:
        ras.backward(ds, cam, g)
    assert _status(eb.value) == 8             # QGS_ESTATE
    got = _planes(ras, ds, cam)               # the hook was one-shot
    ras.check_frame()
    for k in want:
        assert torch.equal(got[k], want[k]), k


def test_withheld_chunk_is_reported_by_backward_and_next_forward(dev, scene):
    from paper_2411_16392_gb300 import _lib as L
    from paper_2411_16392_gb300.render import Rasterizer
    ds, cam = scene
    ras = Rasterizer(dev)
    want = _planes(ras, ds, cam)
    g = {k: torch.ones_like(v) for k, v in want.items()}
    # the backward reports the failure of the frame it would differentiate
    ras.debug_withhold_sort_chunk(SPINS)
    ras.forward(ds, cam)
    with pytest.raises(L.QGSError) as ei:
        ras.backward(ds, cam, g)
    assert _status(ei.value) == 4
    # unchecked, the failure is reported by the next forward (which then renders nothing)
    ras.debug_withhold_sort_chunk(SPINS)
    ras.forward(ds, cam)
    with pytest.raises(L.QGSError) as en:
        ras.forward(ds, cam)
    assert _status(en.value) == 4
    got = _planes(ras, ds, cam)
    grads = ras.backward(ds, cam, g)
    torch.cuda.synchronize()
    for k in want:
        assert torch.equal(got[k], want[k]), k
    assert all(torch.isfinite(v).all() for v in grads.values())
    # a cleared hook does nothing
    ras.debug_withhold_sort_chunk(SPINS)
    ras.debug_withhold_sort_chunk(0)
    got = _planes(ras, ds, cam)
    ras.check_frame()
    for k in want:
        assert torch.equal(got[k], want[k]), k
