"""PyTorch-facing wrapper of libqgs: device tensors in, device tensors out.

PyTorch only supplies device memory and the current CUDA stream; every step of the
rendering path (preprocessing, binning, sorting, compositing, backward) runs in the
library's kernels.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L


@dataclass
class DeviceScene:
    """Scene parameters on a CUDA device (layouts of qgs_scene)."""
    mean: torch.Tensor      # float32 [N, 3]
    quat: torch.Tensor      # float32 [N, 4] (w, x, y, z)
    scale: torch.Tensor     # float32 [N, 2]
    curv: torch.Tensor      # float32 [N, 2]
    opacity: torch.Tensor   # float32 [N]
    sh: torch.Tensor        # int16 [N, 48] holding bfloat16 bits (or torch.bfloat16 [N, 48])

    @property
    def n(self) -> int:
        return int(self.mean.shape[0])

    @staticmethod
    def from_host(scene, device="cuda") -> "DeviceScene":
        def t(x, dt=torch.float32):
            return torch.from_numpy(np.ascontiguousarray(x)).to(device=device, dtype=dt)
        return DeviceScene(t(scene.mean), t(scene.quat), t(scene.scale), t(scene.curv), t(scene.opacity),
                           torch.from_numpy(np.ascontiguousarray(scene.sh).view(np.int16)).to(device))

    def to_c(self) -> L.qgs_scene:
        for k in ("mean", "quat", "scale", "curv", "opacity"):
            v = getattr(self, k)
            if v.dtype != torch.float32 or not v.is_contiguous() or not v.is_cuda:
                raise ValueError(f"scene.{k} must be a contiguous float32 CUDA tensor")
        if self.sh.dtype not in (torch.int16, torch.bfloat16) or not self.sh.is_contiguous():
            raise ValueError("scene.sh must be a contiguous int16/bfloat16 CUDA tensor of bf16 bits")
        return L.qgs_scene(self.n, self.mean.data_ptr(), self.quat.data_ptr(), self.scale.data_ptr(),
                           self.curv.data_ptr(), self.opacity.data_ptr(), self.sh.data_ptr())


def camera_to_c(cam) -> L.qgs_camera:
    c = L.qgs_camera()
    c.W, c.H = int(cam.W), int(cam.H)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.R_cw[:] = [float(v) for v in np.asarray(cam.R_cw, np.float32).reshape(9)]
    c.t_cw[:] = [float(v) for v in np.asarray(cam.t_cw, np.float32).reshape(3)]
    c.near_plane = float(cam.near)
    return c


IMAGE_KEYS = ("rgb", "alpha", "depth", "normal", "curvature", "distortion", "median_depth")
EXTRA_KEYS = IMAGE_KEYS[4:]


def _stream_ptr(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


class Rasterizer:
    """One rendering context (libqgs qgs_ctx) on one CUDA device."""

    DENSITIES = {"geodesic": 0, "euclid": 1}

    ORDERS = {"centre": 0, "stp": 1}

    def __init__(self, device: int | torch.device = 0, sort_mode: int = 0, density: str = "geodesic",
                 order: str = "centre", **consts):
        self.lib = L.load()
        self.device = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
        cfg = L.qgs_config()
        self.lib.qgs_config_default(C.byref(cfg))
        cfg.sort_mode = sort_mode
        cfg.density = self.DENSITIES[density]
        cfg.order = self.ORDERS[order]
        for k, v in consts.items():
            setattr(cfg, k, v)
        self._ctx = C.c_void_p()
        idx = self.device.index if self.device.index is not None else 0
        L.check(self.lib.qgs_create(C.byref(self._ctx), C.byref(cfg), idx))
        self._last = None

    def close(self):
        if self._ctx:
            self.lib.qgs_destroy(self._ctx)
            self._ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ forward
    def forward(self, scene: DeviceScene, cam, out: dict | None = None, extras: bool = False) -> dict:
        """Render; returns dict rgb [3,H,W], alpha [H,W], depth [H,W], normal [3,H,W] and,
        with `extras` (or when `out` holds them), curvature, distortion, median_depth [H,W]."""
        H, W = int(cam.H), int(cam.W)
        if out is None:
            out = dict(rgb=torch.empty(3, H, W, device=self.device), alpha=torch.empty(H, W, device=self.device),
                       depth=torch.empty(H, W, device=self.device), normal=torch.empty(3, H, W, device=self.device))
            if extras:
                for k in EXTRA_KEYS:
                    out[k] = torch.empty(H, W, device=self.device)
        img = L.qgs_image(*[(out[k].data_ptr() if out.get(k) is not None else None) for k in IMAGE_KEYS])
        sc = scene.to_c()
        cc = camera_to_c(cam)
        L.check(self.lib.render_forward(self._ctx, C.byref(sc), C.byref(cc), C.byref(img),
                                        C.c_void_p(_stream_ptr(self.device))), self._ctx)
        self._last = (scene, cam)
        return out

    def forward_batch(self, scene: DeviceScene, cams, outs: list | None = None) -> list:
        """Render several views of one scene in shared launches (render_forward_batch);
        returns one plane dict per camera. Leaves no residue for backward."""
        V = len(cams)
        if outs is None:
            outs = []
            for cam in cams:
                H, W = int(cam.H), int(cam.W)
                outs.append(dict(rgb=torch.empty(3, H, W, device=self.device),
                                 alpha=torch.empty(H, W, device=self.device),
                                 depth=torch.empty(H, W, device=self.device),
                                 normal=torch.empty(3, H, W, device=self.device)))
        cc = (L.qgs_camera * V)(*[camera_to_c(c) for c in cams])
        im = (L.qgs_image * V)(*[L.qgs_image(*[(o[k].data_ptr() if o.get(k) is not None else None)
                                               for k in IMAGE_KEYS]) for o in outs])
        sc = scene.to_c()
        L.check(self.lib.render_forward_batch(self._ctx, C.byref(sc), V, cc, im,
                                              C.c_void_p(_stream_ptr(self.device))), self._ctx)
        self._last = None
        return outs

    # ------------------------------------------------------------------ backward
    def backward(self, scene: DeviceScene, cam, grad_out: dict, grads: dict | None = None) -> dict:
        """Gradients of sum(grad_out * outputs) of the last forward; added into `grads`
        (allocated and zeroed when None). grad_out entries may be None."""
        n = scene.n
        if grads is None:
            z = lambda *s: torch.zeros(*s, device=self.device, dtype=torch.float32)
            grads = dict(mean=z(n, 3), quat=z(n, 4), scale=z(n, 2), curv=z(n, 2), opacity=z(n), sh=z(n, 48))

        def p(k):
            v = grad_out.get(k)
            if v is None:
                return None
            if v.dtype != torch.float32 or not v.is_contiguous():
                raise ValueError(f"grad_out[{k}] must be contiguous float32")
            return v.data_ptr()

        img = L.qgs_image(*[p(k) for k in IMAGE_KEYS])
        g = L.qgs_scene_grad(grads["mean"].data_ptr(), grads["quat"].data_ptr(), grads["scale"].data_ptr(),
                             grads["curv"].data_ptr(), grads["opacity"].data_ptr(), grads["sh"].data_ptr())
        sc = scene.to_c()
        cc = camera_to_c(cam)
        L.check(self.lib.render_backward(self._ctx, C.byref(sc), C.byref(cc), C.byref(img), C.byref(g),
                                         C.c_void_p(_stream_ptr(self.device))), self._ctx)
        return grads

    def set_pair_counters(self, enable: bool):
        """Collect the per-pair counters of stats() (default) or skip them (faster)."""
        L.check(self.lib.qgs_set_pair_counters(self._ctx, 1 if enable else 0), self._ctx)

    def set_tile_mask_capacity(self, words: int):
        """Words of the tile-mask store the emission replays (0: the emission tests every
        tile again). Results never depend on it."""
        L.check(self.lib.qgs_set_tile_mask_capacity(self._ctx, int(words)), self._ctx)

    def check_frame(self):
        """Wait for the last forward's sorts; raises QGSError (QGS_ECUDA) if one of their
        bounded look-back waits ran out (the frame is then discarded)."""
        L.check(self.lib.qgs_check_frame(self._ctx), self._ctx)

    def debug_withhold_sort_chunk(self, spins: int):
        """Test hook: the next forward's first look-back radix sort withholds its first
        chunk, so the waits for it give up after `spins` polls (0 clears the hook)."""
        L.check(self.lib.qgs_debug_withhold_sort_chunk(self._ctx, int(spins)), self._ctx)

    # ------------------------------------------------------------------ inspection
    def stats(self) -> dict:
        s = L.qgs_frame_stats()
        L.check(self.lib.qgs_get_frame_stats(self._ctx, C.byref(s)), self._ctx)
        return {k: getattr(s, k) for k, _ in s._fields_}

    def binning(self):
        n_inst = C.c_int64()
        L.check(self.lib.qgs_copy_binning(self._ctx, None, None, 0, None, None, C.byref(n_inst)), self._ctx)
        I = n_inst.value
        keys = np.zeros(max(I, 1), np.uint64)
        vals = np.zeros(max(I, 1), np.uint32)
        scene, cam = self._last
        TX, TY = (cam.W + 15) // 16, (cam.H + 15) // 16
        ranges = np.zeros((TX * TY, 2), np.uint32)
        rects = np.zeros((scene.n, 4), np.int32)
        L.check(self.lib.qgs_copy_binning(self._ctx, keys.ctypes.data, vals.ctypes.data, max(I, 1),
                                          ranges.ctypes.data, rects.ctypes.data if scene.n else None,
                                          C.byref(n_inst)), self._ctx)
        return keys[:I], vals[:I], ranges, rects

    def residue(self):
        scene, cam = self._last
        T = np.zeros((cam.H, cam.W), np.float32)
        n = np.zeros((cam.H, cam.W), np.uint32)
        L.check(self.lib.qgs_copy_residue(self._ctx, T.ctypes.data, n.ctypes.data), self._ctx)
        return T, n


class QGSRender(torch.autograd.Function):
    """Differentiable render: (mean, quat, scale, curv, opacity, sh) -> (rgb, alpha, depth, normal).

    sh holds bfloat16 values (torch.bfloat16); autograd returns its gradient in that dtype.
    Use Rasterizer.backward directly for float32 SH gradients."""

    @staticmethod
    def forward(ctx, rasterizer: Rasterizer, cam, extras, mean, quat, scale, curv, opacity, sh):
        scene = DeviceScene(mean.detach().contiguous(), quat.detach().contiguous(), scale.detach().contiguous(),
                            curv.detach().contiguous(), opacity.detach().contiguous(),
                            sh.detach().contiguous())
        out = rasterizer.forward(scene, cam, extras=extras)
        ctx.rasterizer = rasterizer
        ctx.cam = cam
        ctx.scene = scene
        ctx.extras = extras
        if extras:
            ctx.mark_non_differentiable(out["median_depth"])
            return tuple(out[k] for k in IMAGE_KEYS)
        return out["rgb"], out["alpha"], out["depth"], out["normal"]

    @staticmethod
    def backward(ctx, *grads):
        keys = IMAGE_KEYS[:len(grads)]
        go = {k: (v.contiguous().float() if v is not None else None) for k, v in zip(keys, grads)}
        go.pop("median_depth", None)          # no gradient flows through the median depth
        r = ctx.rasterizer
        if r._last is None or r._last[0] is not ctx.scene:
            # another forward ran on this rasterizer since: re-render to restore its residue
            r.forward(ctx.scene, ctx.cam, extras=ctx.extras)
        g = r.backward(ctx.scene, ctx.cam, go)
        return None, None, None, g["mean"], g["quat"], g["scale"], g["curv"], g["opacity"], g["sh"]


def render(rasterizer: Rasterizer, cam, mean, quat, scale, curv, opacity, sh, extras: bool = False):
    """Differentiable render through libqgs; returns (rgb, alpha, depth, normal) and, with
    `extras`, also (curvature, distortion, median_depth) (the median depth carries no
    gradient)."""
    return QGSRender.apply(rasterizer, cam, extras, mean, quat, scale, curv, opacity, sh)
