"""Python wrapper of the serving loop (include/qgs_serve.h): argument marshalling only."""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L
from .render import DeviceScene, camera_to_c


def _ptr(v):
    if v is None:
        return None
    if isinstance(v, torch.Tensor):
        return v.data_ptr()
    return v.ctypes.data


class Server:
    """Continuous-batching server: resident scenes, bounded queue, memory-budget admission,
    `slots` concurrent worker contexts, each rendering up to `batch` queued views of one
    scene in shared launches (slots = batch = 1: plain one-at-a-time)."""

    def __init__(self, device: int = 0, budget_bytes: int = 8 << 30, slots: int = 4, queue: int = 1024,
                 fake_us_per_mpix: float = 0.0, batch: int = 1):
        self.lib = L.load()
        self._srv = C.c_void_p()
        L.check(self.lib.serve_create(C.byref(self._srv), device, int(budget_bytes), slots, batch, queue,
                                      float(fake_us_per_mpix)))
        self.device = device

    def close(self):
        if self._srv:
            self.lib.serve_destroy(self._srv)
            self._srv = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_scene(self, scene: DeviceScene | None = None, n: int | None = None) -> int:
        sid = C.c_int32()
        if scene is None:  # host-only server: only the primitive count matters
            sc = L.qgs_scene(int(n or 0), None, None, None, None, None, None)
        else:
            sc = scene.to_c()
        L.check(self.lib.serve_load_scene(self._srv, C.byref(sc), C.byref(sid)))
        return sid.value

    def submit(self, scene_id: int, cam, backward: bool = False, grad_out: dict | None = None) -> int:
        """Queue a forward render, or with `backward` a forward + backward whose upstream
        gradient planes are `grad_out` (dict of rgb/alpha/depth/normal, host or device;
        missing planes are zero; copied before this returns)."""
        t = C.c_uint64()
        cc = camera_to_c(cam)
        g = None
        if grad_out is not None:
            g = L.qgs_image(*[_ptr(grad_out.get(k)) for k in ("rgb", "alpha", "depth", "normal")])
        st = self.lib.serve_submit(self._srv, scene_id, C.byref(cc), int(bool(backward)),
                                   C.byref(g) if g is not None else None, C.byref(t))
        if st != 0:
            raise L.QGSError(st, "serve_submit")
        return t.value

    def wait(self, ticket: int, cam=None, timeout_ms: int = -1, out: dict | None = None,
             grads: dict | None = None):
        """Wait for a ticket; copy its planes into `out` (dict of tensors/arrays, host or
        device) and, for a backward request, its parameter gradients into `grads` (dict of
        mean/quat/scale/curv/opacity/sh float32 arrays) when given. Returns `out`."""
        img = None
        if out is not None:
            img = L.qgs_image(*[_ptr(out.get(k)) for k in ("rgb", "alpha", "depth", "normal")])
        gr = None
        if grads is not None:
            gr = L.qgs_scene_grad(*[_ptr(grads.get(k)) for k in ("mean", "quat", "scale", "curv", "opacity", "sh")])
        st = self.lib.serve_wait(self._srv, C.c_uint64(ticket), int(timeout_ms),
                                 C.byref(img) if img is not None else None,
                                 C.byref(gr) if gr is not None else None)
        if st != 0:
            raise L.QGSError(st, "serve_wait")
        return out

    def stats(self) -> dict:
        s = L.qgs_serve_stats()
        L.check(self.lib.serve_stats(self._srv, C.byref(s)))
        return {k: getattr(s, k) for k, _ in s._fields_}

    def reset_stats(self):
        L.check(self.lib.serve_reset_stats(self._srv))


def host_planes(cam):
    H, W = int(cam.H), int(cam.W)
    return {"rgb": np.zeros((3, H, W), np.float32), "alpha": np.zeros((H, W), np.float32),
            "depth": np.zeros((H, W), np.float32), "normal": np.zeros((3, H, W), np.float32)}
