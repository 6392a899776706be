"""The bounds-checked build (libqgs_check.so, -DQGS_DEBUG_CHECKS) on the GPU: the binning
kernels check every instance slot, tile id and sort scatter position they compute; on
valid frames no check fails and the images and gradients equal the normal build's bit for
bit (the checks only guard accesses). Run in a child process, which loads the checked
library in place of libqgs.so."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from paper_2411_16392_gb300.scenes import Camera, scene_small

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# renders the cases with whichever library _lib.LIB_PATH names; saves planes and gradients
_CHILD = r"""
import ctypes, json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
import paper_2411_16392_gb300._lib as L
if sys.argv[3] != "-":
    L.LIB_PATH = sys.argv[3]
lib = L.load()
from paper_2411_16392_gb300.render import DeviceScene, Rasterizer
from paper_2411_16392_gb300.scenes import Camera, scene_small
dev = torch.device("cuda", 0)
cases = [(scene_small(0, 1000), 0), (scene_small(0, 1000), 1), (scene_small(5, 20000), 0)]
cases[2] = ((cases[2][0][0], Camera(333, 257, 260.0, 260.0, 166.5, 128.5)), 0)
out = {}
for c, ((sc, cam), mode) in enumerate(cases):
    ras = Rasterizer(dev, sort_mode=mode)
    ds = DeviceScene.from_host(sc, dev)
    img = ras.forward(ds, cam)
    g = {k: torch.ones_like(v) for k, v in img.items()}
    gr = ras.backward(ds, cam, g)
    torch.cuda.synchronize()
    for k, v in list(img.items()) + [("g_" + k, v) for k, v in gr.items()]:
        out[f"{c}_{k}"] = v.cpu().numpy()
ci, w = ctypes.c_int32(0), ctypes.c_uint32(0)
st = lib.qgs_debug_check_word(0, ctypes.byref(ci), ctypes.byref(w))
np.savez(sys.argv[2], **out)
print(json.dumps({"status": st, "compiled_in": ci.value, "word": w.value}))
"""


def _run(lib_path, npz):
    r = subprocess.run([sys.executable, "-c", _CHILD, ROOT, npz, lib_path], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_bounds_checked_build_passes_and_matches(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_16392_gb300 import build as B
    chk = B.OUT_CHECK if os.path.exists(B.OUT_CHECK) else B.build(debug_checks=True)
    a = _run(chk, str(tmp_path / "chk.npz"))
    assert a == {"status": 0, "compiled_in": 1, "word": 0}, a
    b = _run("-", str(tmp_path / "rel.npz"))
    assert b["status"] == 0 and b["compiled_in"] == 0
    x, y = np.load(tmp_path / "chk.npz"), np.load(tmp_path / "rel.npz")
    assert sorted(x.files) == sorted(y.files)
    for k in x.files:
        if k.split("_", 1)[1].startswith("g_"):   # gradients: up to the atomics' order
            assert np.abs(x[k] - y[k]).max() <= 1e-5 * max(np.abs(y[k]).max(), 1e-30), k
        else:
            assert np.array_equal(x[k], y[k]), k
