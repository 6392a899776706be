"""FP64 CPU oracle for the quadric Gaussian splatting rasterizer.

TEST INFRASTRUCTURE ONLY. Nothing on the product path may import or call this
module: only the tests, the smoke check in ``__graft_entry__`` and the CPU-baseline
leg of ``bench.py`` use it. It shares no code with the CUDA path.

What it computes, step by step, and where each step is defined in the paper
(arXiv 2411.16392, "Quadratic Gaussian Splatting"):

  * Frame (Sec. 3.2, congruent transform Q = T^-T D T^-1 with T = [R c; 0 1]):
    local coordinates x_hat = R^T (x - mu); the camera centre and the pixel ray
    are taken into that frame.
  * Surface (Sec. 3.2, explicit paraboloid equation): z_hat = a*x_hat^2 + b*y_hat^2,
    with a = sign(s1)*s3/s1^2 and b = sign(s2)*s3/s2^2 (the lambda_1, lambda_2 of the
    curvature paragraph).
  * Ray-splat intersection (supplementary, "Details of Ray-splat Intersection"): the
    quadratic A t^2 + B t + C = 0 and its two roots t_n <= t_f.
  * Hit selection (Sec. 3.2.1): the near root if its geodesic distance is within
    3 sigma(theta), else the far root under the same test, else no hit.
  * Geodesic Gaussian (Sec. 3.2, polar form z = a(theta) rho^2, arc-length Eq.,
    sigma(theta) Eq., G Eq.): l(a(theta), rho) in closed form, G = exp(-l^2/(2 sigma^2)).
  * Normal (Sec. 3.2, normal Eq.): gradient of the implicit function at the hit,
    rotated to camera space and turned to face the camera.
  * Colour (Sec. 3.1): degree-3 real spherical harmonics, as in 3DGS.
  * Alpha blending (Sec. 3.1 blending Eq., Eq. of the normal/curvature maps and the
    supplementary's X_hat = sum alpha_i T_i X_i): front to back, in sorted order.
  * Tile binning (supplementary, per-tile sorting): 16x16 tiles, one 64-bit key
    (tile << 32 | float bits of the view depth) per (tile, primitive) pair, stable sort.
  * Extra channels (render(..., extras=True)): the curvature map sum w_i K_i with the
    Gaussian curvature of Sec. 3.2.1 at each hit; the depth distortion of Sec. 3.3,
    sum_i sum_{j<i} w_i w_j (t_i - t_j)^2, summed as written; the median depth of
    Sec. 4.1, the largest t_i among blended pairs whose transmittance before them
    exceeds 0.5 (0 when none does).
  * StopThePop ordering (render(..., order="stp"), supplementary "Details of Per-tile
    Sorting and Per-pixel Resorting"): tile lists sorted by the depth where the ray of the
    tile pixel closest to the projected vertex meets the paraboloid (an FP32 recipe,
    hit_keys, shared with the kernels as a specification), then per-pixel resorting of
    the contributing pairs in a buffer of 8 (nearest first when full, the rest nearest
    first at the end). Readings: the ray meets the untruncated paraboloid, nearest root
    in front of the near plane, the centre depth when it misses; ties in the buffer go to
    the earlier list entry; the transmittance stop applies when an entry is blended.
  * Density variant (render(..., density="euclid")): the Euclidean-distance Gaussian
    that Sec. 3.2 argues against and Sec. 4.3 ablates, same sigma(theta), distance
    sqrt(rho^2 + z^2) from the vertex.

Readings where the paper is silent (each one is listed with its reason in the
design notes of the repository):
  * alpha = min(0.99, o*G); pairs with alpha < 1/255 are skipped; a pixel stops
    before blending the first pair that would take T below 1e-4 (the 3DGS constants
    of the framework the paper builds on, Sec. 4.1 "Rasterizer").
  * Roots are accepted only in front of the near plane (t > near, near = 0.2);
    primitives whose centre is not in front of the near plane are culled.
  * t is the camera-space z depth of the hit; the depth map is sum w_i t_i
    (unnormalised), the normal map sum w_i n_i (unnormalised), in camera space; the
    distortion uses the same t (the paper's "depth at the ray-splat intersection"); the
    median depth carries no gradient (the paper uses it for mesh extraction only).
  * The roots are the exact roots of the quadratic (evaluated without cancellation);
    the paper's |A| < 1e-6 tangent-plane fallback t = -C/B is the A -> 0 limit of
    the near root and is not used as a separate approximation.
  * Screen bound: the 8 corners of a local box that contains the support, clipped to
    the near plane, projected, and their pixel AABB taken (the supplementary's
    bounding-box section). The box comes from "arc length >= chord" (see bin_fp32).
    A tile of the AABB is listed only if it also meets a screen parallelogram around the
    projected box and the screen conic of the ellipsoid x^2/s_u^2 + y^2/s_v^2 + z^2/m^2
    <= 9 that the same inequality puts around the support (ellipsoid_conic, _tile_pass);
    the AABB is first cut to the conic's bounding box (conic_box). All of it is
    evaluated in FP32 with correctly rounded operations in a fixed order so that tile
    lists and keys can be compared bit for bit; the lists only decide which pairs are
    evaluated, never a pair's value, and they keep every pair with a hit (pinned).

Gradients are exact derivatives of this FP64 forward, taken by PyTorch autograd.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

F64 = torch.float64
TILE = 16
ALPHA_MAX = 0.99
ALPHA_MIN = 1.0 / 255.0
T_MIN = 1e-4
CUTOFF = 3.0          # support radius in sigma(theta) units
TAYLOR_U = 1e-3       # |u| below which l is evaluated from its Taylor series


# =========================================================================== FP32 binning
@dataclass
class Binning:
    visible: np.ndarray     # bool [N]
    zbits: np.ndarray       # uint32 [N] float32 bits of the view depth of the centre
    rect: np.ndarray        # int32 [N, 4] (tx0, tx1, ty0, ty1), inclusive
    count: np.ndarray       # int64 [N] tiles covered
    keys: np.ndarray        # uint64 [I] sorted
    vals: np.ndarray        # uint32 [I] primitive index per sorted key
    ranges: np.ndarray      # int64 [n_tiles, 2] [start, end) into keys
    tiles_x: int
    tiles_y: int
    pix_bbox: np.ndarray    # float32 [N, 4] (xmin, xmax, ymin, ymax) in pixels
    order: str = "centre"   # "centre": key = centre depth; "hit": per-tile hit depth
    geo: dict | None = None  # float32 mu_c, W, a, b, camera (for per-tile hit keys)
    slabs: dict | None = None  # float32 screen parallelogram per primitive (tile test)
    tile_counts: np.ndarray | None = None  # int64 [n_tiles] listed primitives per tile


def _rect_tiles(rect, prims):
    """(primitive, tx, ty) of every tile of the primitives' rectangles, row-major."""
    prims = np.asarray(prims, np.int64)
    w = (rect[prims, 1] - rect[prims, 0] + 1).astype(np.int64)
    h = (rect[prims, 3] - rect[prims, 2] + 1).astype(np.int64)
    n = w * h
    p = np.repeat(prims, n)
    e = np.arange(int(n.sum())) - np.repeat(np.cumsum(n) - n, n)
    ww = np.repeat(w, n)
    return p, rect[p, 0] + e % ww, rect[p, 2] + e // ww


def _tile_pass(sl, p, tx, ty):
    """Whether tile (tx, ty) meets primitive p's screen parallelogram: the two slabs
    |n_k . (x - c)| within [smin_k, smax_k] (spans of the projected support box along the
    normals of the projected local axes, from the projected centre c) against the range
    of n_k . (x - c) over the tile's pixel centres, padded by 2e-3 px + 1e-5 of the span
    ends for rounding. FP32, correctly rounded, in the order written (the kernels follow
    the same specification)."""
    f = np.float32
    half = f(0.5)
    x0 = (16 * tx).astype(f) + half
    x1 = np.minimum(16 * tx + 15, sl["img_w"] - 1).astype(f) + half
    y0 = (16 * ty).astype(f) + half
    y1 = np.minimum(16 * ty + 15, sl["img_h"] - 1).astype(f) + half
    a0, a1 = x0 - sl["uc"][p], x1 - sl["uc"][p]
    b0, b1 = y0 - sl["vc"][p], y1 - sl["vc"][p]
    ok = np.ones(p.shape, bool)
    for k in ("1", "2"):
        nx, ny = sl["n" + k + "x"][p], sl["n" + k + "y"][p]
        smin, smax = sl["s" + k + "min"][p], sl["s" + k + "max"][p]
        e = [nx * a + ny * b for a in (a0, a1) for b in (b0, b1)]
        lo = np.minimum(np.minimum(e[0], e[1]), np.minimum(e[2], e[3]))
        hi = np.maximum(np.maximum(e[0], e[1]), np.maximum(e[2], e[3]))
        pad = f(2e-3) + f(1e-5) * (np.abs(smin) + np.abs(smax))
        ok &= ~(hi < smin - pad) & ~(lo > smax + pad)
    if "qa" in sl:
        ok &= _conic_pass(sl, p, a0, a1, b0, b1)
    return ok


CONIC_KAPPA = 9.02     # squared radius of the padded chord ellipsoid (9 = 3 sigma squared)
CONIC_SHIFT = 4e-6     # diagonal shift of the quadratic form, relative to its trace
CONIC_DELTA = 2e-3     # absolute pad in pixels


def ellipsoid_conic(muc, Wm, su, sv, m, fx, fy):
    """Screen-space conic of the chord ellipsoid that holds the support (FP32 recipe).

    Every point of the support has E + z^2/m^2 <= 9 (the inequality (*) of bin_fp32:
    arc >= chord), i.e. it lies in the ellipsoid |S^-1 x_loc| <= 3 with S = diag(s_u,
    s_v, m). A pixel ray can only meet the support if its line meets that ellipsoid.
    In the scaled frame xi = S^-1 W^T (x - mu_c), with the camera at omega and the ray
    direction delta = S^-1 W^T d, the line meets the ball |xi|^2 <= kappa iff
    |omega x delta|^2 <= kappa |delta|^2. For a pixel at offset p from the projected
    centre, d = mu_c / z + (p_x / f_x, p_y / f_y, 0), and the identity
    (M a) x (M b) = det(M) M^-T (a x b) with M = S^-1 W^T turns the left side into
    |p_x n_x + p_y n_y|^2 with n_x = S W^T (e_x x mu_c) / (f_x s_u s_v m), n_y likewise
    (no cancellation: the camera-distance terms drop out exactly), while the right side
    is kappa |delta_c + p_x h_x + p_y h_y|^2 with h_x = S^-1 W^T e_x / f_x. Hence
        p^T Q p - 2 L.p <= K,   Q = Gram(n) - kappa Gram(h), L = kappa (delta_c.h), K = kappa |delta_c|^2.
    Pads: kappa = 9.02 instead of 9 (FP32 rounding of the kernels' own hit test); Q's
    diagonal lowered by CONIC_SHIFT x its trace (FP32 rounding of Q, which matters along
    the long axis of an elongated ellipse); the normalised threshold raised so that the
    ellipse grows by CONIC_DELTA pixels (the tile test measures offsets from the rounded
    projected centre). The conic is enabled only when the padded Q is positive definite
    (the ellipsoid lies in front of the camera plane); otherwise every pixel passes.
    Returned (normalised so that the test reads F(p) = p^T q p - 2 l.p <= 1):
    qa, qb, qc (q = [[qa, qb], [qb, qc]]), la, lb, the reciprocals iqa = 1/qa and
    iqc = 1/qc used by the tile test, and the enable flag conic_on (all zero when off).
    Correctly rounded FP32 operations in the order written (the kernels follow the same
    specification bit for bit)."""
    f = np.float32
    zero, one, two = f(0.0), f(1.0), f(2.0)
    ifx, ify = one / fx, one / fy
    isu, isv, im = one / su, one / sv, one / m
    rs = (isu, isv, im)                     # 1 / s_c
    ro = (isv * im, isu * im, isu * isv)    # s_c / (s_u s_v m)
    nx = [((Wm[2][c] * muc[1] - Wm[1][c] * muc[2]) * ifx) * ro[c] for c in range(3)]
    ny = [((Wm[0][c] * muc[2] - Wm[2][c] * muc[0]) * ify) * ro[c] for c in range(3)]
    hx = [(Wm[0][c] * ifx) * rs[c] for c in range(3)]
    hy = [(Wm[1][c] * ify) * rs[c] for c in range(3)]
    dcx = muc[0] / muc[2]
    dcy = muc[1] / muc[2]
    dc = [((Wm[0][c] * dcx + Wm[1][c] * dcy) + Wm[2][c]) * rs[c] for c in range(3)]

    def dot(u, v):
        return (u[0] * v[0] + u[1] * v[1]) + u[2] * v[2]

    kap = f(CONIC_KAPPA)
    G00, G01, G11 = dot(nx, nx), dot(nx, ny), dot(ny, ny)
    H00, H01, H11 = dot(hx, hx), dot(hx, hy), dot(hy, hy)
    tau = f(CONIC_SHIFT) * (G00 + G11)
    Q00 = (G00 - kap * H00) - tau
    Q01 = G01 - kap * H01
    Q11 = (G11 - kap * H11) - tau
    L0 = kap * dot(dc, hx)
    L1 = kap * dot(dc, hy)
    K = kap * dot(dc, dc)
    det = Q00 * Q11 - Q01 * Q01
    iK = one / K
    qa, qb, qc, la, lb = Q00 * iK, Q01 * iK, Q11 * iK, L0 * iK, L1 * iK
    dn = qa * qc - qb * qb
    # R = 1 + l^T q^-1 l: (p - p0)^T q (p - p0) <= R is the same ellipse, p0 = q^-1 l
    R0 = one + (((qc * la) * la - (two * (qb * la)) * lb) + (qa * lb) * lb) / dn
    R = np.where(R0 > one, R0, one)
    tr = qa + qc
    dl = f(CONIC_DELTA)
    # growing the ellipse by dl pixels raises F by at most 2 dl sqrt(lmax R) + dl^2 lmax
    T = (one + (f(3.0) * dl) * np.sqrt(tr * R)) + ((two * dl) * dl) * tr
    iT = one / T
    on = (np.isfinite(Q00) & np.isfinite(Q01) & np.isfinite(Q11) & np.isfinite(L0) & np.isfinite(L1)
          & np.isfinite(K) & (K > zero) & (Q00 > zero) & (Q11 > zero) & (det > f(1e-6) * (Q00 * Q11))
          & np.isfinite(T) & (dn > zero) & np.isfinite(R0))
    out = {"qa": qa * iT, "qb": qb * iT, "qc": qc * iT, "la": la * iT, "lb": lb * iT}
    out["iqa"] = one / out["qa"]
    out["iqc"] = one / out["qc"]
    for k in out:
        on &= np.isfinite(out[k])
    on &= (out["qa"] > zero) & (out["qc"] > zero)
    for k in list(out):
        out[k] = np.where(on, out[k], zero).astype(f)
    out["conic_on"] = on
    return out


def conic_box(cn, uc, vc):
    """Tile range (floor(x / 16) bounds, as float32) of the bounding box of the conic
    F(p) <= 1, i.e. of the ellipse (p - p0)^T q (p - p0) <= R with p0 = q^-1 l and
    R = 1 + l.p0, whose half-extents are sqrt(R (q^-1)_00) and sqrt(R (q^-1)_11), placed at
    the projected centre (uc, vc). FP32, correctly rounded, in the order written; entries
    of disabled conics are not used."""
    f = np.float32
    one, sixteenth = f(1.0), f(1.0 / 16.0)
    qa, qb, qc, la, lb = (cn[k] for k in ("qa", "qb", "qc", "la", "lb"))
    with np.errstate(all="ignore"):
        dn = qa * qc - qb * qb
        p0x = (qc * la - qb * lb) / dn
        p0y = (qa * lb - qb * la) / dn
        R = (one + la * p0x) + lb * p0y
        ex = np.sqrt((R * qc) / dn)
        ey = np.sqrt((R * qa) / dn)
        cx = uc + p0x
        cy = vc + p0y
        return (np.floor((cx - ex) * sixteenth), np.floor((cx + ex) * sixteenth),
                np.floor((cy - ey) * sixteenth), np.floor((cy + ey) * sixteenth))


def conic_value(sl, p, u, v):
    """F(u, v) = u (qa u + 2 qb v - 2 la) + v (qc v - 2 lb) in the recipe's FP32 order."""
    two = np.float32(2.0)
    qa, qb, qc, la, lb = (sl[k][p] for k in ("qa", "qb", "qc", "la", "lb"))
    return u * ((qa * u + two * (qb * v)) - two * la) + v * (qc * v - two * lb)


def _conic_pass(sl, p, x0, x1, y0, y1):
    """Whether the rectangle [x0, x1] x [y0, y1] of pixel-centre offsets from the projected
    centre meets the conic F <= 1. F is convex (q positive definite), and F(0) <= 1 (the
    ray through the projected centre meets the ellipsoid's centre), so the rectangle meets
    the ellipse iff it holds the origin or the minimum of F over an edge facing the
    ellipse is <= 1; the edge minima are the clamped stationary points of F along the
    edge (a vertical edge when 0 is left or right of [x0, x1], a horizontal one when it
    is above or below [y0, y1]). FP32, correctly rounded, in the order written."""
    f = np.float32
    zero, one = f(0.0), f(1.0)
    qa, qb, qc, la, lb = (sl[k][p] for k in ("qa", "qb", "qc", "la", "lb"))
    on = sl["conic_on"][p]
    with np.errstate(all="ignore"):
        inside = (x0 <= zero) & (zero <= x1) & (y0 <= zero) & (zero <= y1)
        ue = np.where(x0 > zero, x0, x1)
        has_u = (x0 > zero) | (x1 < zero)
        vs = np.minimum(np.maximum((lb - qb * ue) * sl["iqc"][p], y0), y1)
        fu = conic_value(sl, p, ue, vs)
        ve = np.where(y0 > zero, y0, y1)
        has_v = (y0 > zero) | (y1 < zero)
        us = np.minimum(np.maximum((la - qb * ve) * sl["iqa"][p], x0), x1)
        fv = conic_value(sl, p, us, ve)
        meets = inside | (has_u & (fu <= one)) | (has_v & (fv <= one))
    return ~on | meets


def hit_keys(binning: Binning, prims: np.ndarray, tile: int) -> np.ndarray:
    """Per-tile sort depth of StopThePop's ordering as adopted by the supplementary
    ("Details of Per-tile Sorting and Per-pixel Resorting"): the depth where the ray of
    the tile's pixel closest to the projected vertex meets the paraboloid, shared by all
    pixels of the tile. Returns the float32 depths' bits [len(prims)].

    Specified in FP32 with correctly rounded + - * / sqrt, each rounded, in the order
    written (the kernels follow the same recipe):
      uc = fx*(x/z) + cx, vc likewise (the centre mu_c, from the binning recipe);
      px = min(max(floor(uc), 16 tx), min(16 tx + 15, W - 1)), py likewise;
      dx = ((px + 0.5) - cx)/fx, dy likewise, d = (dx, dy, 1);
      ex = dx*z - x, ey = dy*z - y (offset from the centre at the centre's depth);
      b_k = W[0][k]*ex + W[1][k]*ey, d_k = (W[0][k]*dx + W[1][k]*dy) + W[2][k];
      A = (a*d0)*d0 + (b*d1)*d1;  B' = ((a*b0)*d0 + (b*b1)*d1) - 0.5*d2;
      C = ((a*b0)*b0 + (b*b1)*b1) - b2;  D' = B'*B' - A*C;
      q = -(B' + sgn(B') sqrt(D')) (sgn(0) = +1), s in {C/q, q/A}, t = z + s;
      the smallest finite t > near; the centre depth z when D' < 0 or no root qualifies.
    The ray is taken relative to the point where it crosses the centre's depth, so the
    quadratic's coefficients have the size of the primitive (no cancellation at the
    camera distance)."""
    f = np.float32
    g = binning.geo
    prims = np.asarray(prims, np.int64)
    ty_, tx_ = divmod(int(tile), binning.tiles_x)
    x, y, z = (g["muc"][k][prims] for k in range(3))
    Wm = [[g["Wm"][r][c][prims] for c in range(3)] for r in range(3)]
    a, b = g["a"][prims], g["b"][prims]
    fx, fy, cx, cy, near, Wimg, Himg = (g[k] for k in ("fx", "fy", "cx", "cy", "near", "img_w", "img_h"))
    with np.errstate(all="ignore"):
        uc = fx * (x / z) + cx
        vc = fy * (y / z) + cy
        px = np.minimum(np.maximum(np.floor(uc), f(16 * tx_)), f(min(16 * tx_ + 15, Wimg - 1)))
        py = np.minimum(np.maximum(np.floor(vc), f(16 * ty_)), f(min(16 * ty_ + 15, Himg - 1)))
        half = f(0.5)
        dx = ((px + half) - cx) / fx
        dy = ((py + half) - cy) / fy
        ex = dx * z - x
        ey = dy * z - y
        bk = [Wm[0][k] * ex + Wm[1][k] * ey for k in range(3)]
        dk = [(Wm[0][k] * dx + Wm[1][k] * dy) + Wm[2][k] for k in range(3)]
        A = (a * dk[0]) * dk[0] + (b * dk[1]) * dk[1]
        Bh = ((a * bk[0]) * dk[0] + (b * bk[1]) * dk[1]) - half * dk[2]
        C = ((a * bk[0]) * bk[0] + (b * bk[1]) * bk[1]) - bk[2]
        D = Bh * Bh - A * C
        sq = np.sqrt(np.maximum(D, f(0.0)))
        q = -(Bh + np.where(Bh >= f(0.0), sq, -sq))
        t1 = z + C / q
        t2 = z + q / A
        ok1 = np.isfinite(t1) & (t1 > near) & (D >= f(0.0))
        ok2 = np.isfinite(t2) & (t2 > near) & (D >= f(0.0))
        t = np.where(ok1 & ok2, np.minimum(t1, t2), np.where(ok1, t1, np.where(ok2, t2, z)))
    return t.astype(f).view(np.uint32)


def bin_fp32(scene, cam, emit: bool = True, order: str = "centre") -> Binning:
    """Conservative screen bound, tile rectangle and sort key of every primitive.

    FP32, correctly rounded + - * / sqrt only, each operation rounded separately in
    the order written below (no fused multiply-add). Bounding box of the support in the
    local frame, projected (the supplementary's "Details of Bounding Box Calculation":
    project the 8 vertices of a 3-D box of the patch and take their 2-D AABB).
    The box: a point (x, y, z) of the support has l <= 3 sigma(theta), and the arc is no
    shorter than its chord, so x^2 + y^2 + z^2 <= 9 sigma(theta)^2; dividing by
    sigma(theta)^2 (with (x^2+y^2)/sigma^2 = x^2/s_u^2 + y^2/s_v^2 =: E and
    sigma <= m = max(s_u, s_v)) gives   E + z^2/m^2 <= 9.                          (*)
      z: with X = x^2, Y = y^2 >= 0 and X/s_u^2 + Y/s_v^2 <= 9 - z^2/m^2, z = aX + bY is
         at most (9 - z^2/m^2) c+ with c+ = max(0, a s_u^2, b s_v^2), so z <= z+, the
         positive root of (c+/m^2) z^2 + z - 9 c+ = 0, i.e. 18 c+ / (1 + sqrt(1 + 36 c+^2/m^2));
         likewise z >= -z- with c- = max(0, -a s_u^2, -b s_v^2).
      x: if a and b do not have opposite signs, (a X + b Y)^2 >= (a X)^2, so (*) gives
         X/s_u^2 + a^2 X^2/m^2 <= 9, X <= 18 / (1/s_u^2 + sqrt(1/s_u^4 + 36 a^2/m^2));
         otherwise X <= 9 s_u^2 (E <= 9). Same for y with b, s_v.
    """
    f = np.float32
    N = scene.n
    with np.errstate(all="ignore"):
        mx, my, mz = (scene.mean[:, k].astype(f) for k in range(3))
        Rc = cam.R_cw.astype(f)
        tc = cam.t_cw.astype(f)
        near = f(cam.near)

        def cam_row(i):
            return ((Rc[i, 0] * mx + Rc[i, 1] * my) + Rc[i, 2] * mz) + tc[i]

        muc = [cam_row(0), cam_row(1), cam_row(2)]
        qw, qx, qy, qz = (scene.quat[:, k].astype(f) for k in range(4))
        n2 = ((qw * qw + qx * qx) + qy * qy) + qz * qz
        r = np.sqrt(n2)
        w, x, y, z = qw / r, qx / r, qy / r, qz / r
        one, two = f(1.0), f(2.0)
        R = [[one - two * (y * y + z * z), two * (x * y - w * z), two * (x * z + w * y)],
             [two * (x * y + w * z), one - two * (x * x + z * z), two * (y * z - w * x)],
             [two * (x * z - w * y), two * (y * z + w * x), one - two * (x * x + y * y)]]
        Wm = [[(Rc[i, 0] * R[0][j] + Rc[i, 1] * R[1][j]) + Rc[i, 2] * R[2][j] for j in range(3)]
              for i in range(3)]
        su = scene.scale[:, 0].astype(f)
        sv = scene.scale[:, 1].astype(f)
        a = scene.curv[:, 0].astype(f)
        b = scene.curv[:, 1].astype(f)
        nine, zero = f(9.0), f(0.0)
        c18, c36 = f(18.0), f(36.0)
        m = np.maximum(su, sv)
        su2 = su * su
        sv2 = sv * sv
        ap = a * su2
        bp = b * sv2
        cpos = np.maximum(np.maximum(ap, bp), zero)
        cneg = np.maximum(np.maximum(-ap, -bp), zero)

        def root(num, c):
            # num / (1 + sqrt(1 + 36 (c/m)^2)): the positive roots above, written with
            # the dimensionless c/m so that nothing overflows
            t = c / m
            t = c36 * (t * t)
            return num / (one + np.sqrt(one + t))

        zmax = root(c18 * cpos, cpos)
        zmin = -root(c18 * cneg, cneg)
        same = ~(((a > zero) & (b < zero)) | ((a < zero) & (b > zero)))
        Xs = np.where(same, root(c18 * su2, ap), nine * su2)
        Ys = np.where(same, root(c18 * sv2, bp), nine * sv2)
        X = np.sqrt(Xs)
        Y = np.sqrt(Ys)

        corners = []
        for k in range(8):
            sx = X if (k & 1) else -X
            sy = Y if (k & 2) else -Y
            sz = zmax if (k & 4) else zmin
            corners.append([((muc[i] + Wm[i][0] * sx) + Wm[i][1] * sy) + Wm[i][2] * sz
                            for i in range(3)])
        fx, fy, cx, cy = f(cam.fx), f(cam.fy), f(cam.cx), f(cam.cy)
        inf = f(np.inf)
        xmin = np.full(N, inf, f)
        xmax = np.full(N, -inf, f)
        ymin = np.full(N, inf, f)
        ymax = np.full(N, -inf, f)
        anyp = np.zeros(N, bool)
        # screen parallelogram: spans of the projected points along the normals of the
        # projected local x and y axes, measured from the projected centre (uc, vc)
        uc = fx * (muc[0] / muc[2]) + cx
        vc = fy * (muc[1] / muc[2]) + cy

        def axis_normal(a):
            du = fx * (Wm[0][a] * muc[2] - muc[0] * Wm[2][a])
            dv = fy * (Wm[1][a] * muc[2] - muc[1] * Wm[2][a])
            l2 = du * du + dv * dv
            l = np.sqrt(l2)
            ok = (l2 > zero) & np.isfinite(l2)
            return np.where(ok, -(dv / l), one), np.where(ok, du / l, zero)

        n1x, n1y = axis_normal(0)
        n2x, n2y = axis_normal(1)
        s1min = np.full(N, inf, f)
        s1max = np.full(N, -inf, f)
        s2min = np.full(N, inf, f)
        s2max = np.full(N, -inf, f)

        def add_point(mask, px, py, pz):
            u = fx * (px / pz) + cx
            v = fy * (py / pz) + cy
            xmin[mask] = np.minimum(xmin[mask], u[mask])
            xmax[mask] = np.maximum(xmax[mask], u[mask])
            ymin[mask] = np.minimum(ymin[mask], v[mask])
            ymax[mask] = np.maximum(ymax[mask], v[mask])
            du_, dv_ = u - uc, v - vc
            t1 = n1x * du_ + n1y * dv_
            t2 = n2x * du_ + n2y * dv_
            s1min[mask] = np.minimum(s1min[mask], t1[mask])
            s1max[mask] = np.maximum(s1max[mask], t1[mask])
            s2min[mask] = np.minimum(s2min[mask], t2[mask])
            s2max[mask] = np.maximum(s2max[mask], t2[mask])
            anyp[mask] = True

        inside = [c[2] >= near for c in corners]
        for k in range(8):
            add_point(inside[k], *corners[k])
        for k0 in range(8):
            for bit in (1, 2, 4):
                if k0 & bit:
                    continue
                k1 = k0 | bit
                P0, P1 = corners[k0], corners[k1]
                cross = inside[k0] != inside[k1]
                lam = (near - P0[2]) / (P1[2] - P0[2])
                ex = P0[0] + lam * (P1[0] - P0[0])
                ey = P0[1] + lam * (P1[1] - P0[1])
                add_point(cross, ex, ey, np.full(N, near, f))

        TX = (cam.W + TILE - 1) // TILE
        TY = (cam.H + TILE - 1) // TILE
        finite_in = (np.isfinite(scene.mean).all(1) & np.isfinite(scene.quat).all(1)
                     & np.isfinite(scene.scale).all(1) & np.isfinite(scene.curv).all(1)
                     & np.isfinite(scene.opacity))
        vis = (finite_in & (n2 > zero) & (su > zero) & (sv > zero) & (su2 > zero) & (sv2 > zero)
               & (muc[2] > near) & anyp
               & np.isfinite(xmin) & np.isfinite(xmax) & np.isfinite(ymin) & np.isfinite(ymax))
        vis &= ~((xmax < zero) | (ymax < zero) | (xmin >= f(cam.W)) | (ymin >= f(cam.H)))
        sixteenth = f(1.0 / TILE)
        tx0 = np.maximum(np.floor(xmin * sixteenth), zero)
        tx1 = np.minimum(np.floor(xmax * sixteenth), f(TX - 1))
        ty0 = np.maximum(np.floor(ymin * sixteenth), zero)
        ty1 = np.minimum(np.floor(ymax * sixteenth), f(TY - 1))
        # the rectangle shrunk to the tiles of the conic's bounding box (see conic_box)
        cb = conic_box(slabs_conic := ellipsoid_conic(muc, Wm, su, sv, m, fx, fy), uc, vc)
        con = slabs_conic["conic_on"]
        tx0 = np.where(con, np.maximum(tx0, cb[0]), tx0)
        tx1 = np.where(con, np.minimum(tx1, cb[1]), tx1)
        ty0 = np.where(con, np.maximum(ty0, cb[2]), ty0)
        ty1 = np.where(con, np.minimum(ty1, cb[3]), ty1)
        vis &= ~(tx0 > tx1) & ~(ty0 > ty1)
        rect = np.zeros((N, 4), np.int32)
        rect[vis, 0] = tx0[vis].astype(np.int32)
        rect[vis, 1] = tx1[vis].astype(np.int32)
        rect[vis, 2] = ty0[vis].astype(np.int32)
        rect[vis, 3] = ty1[vis].astype(np.int32)
        slabs = dict(n1x=n1x, n1y=n1y, s1min=s1min, s1max=s1max, n2x=n2x, n2y=n2y, s2min=s2min, s2max=s2max,
                     uc=uc, vc=vc, img_w=cam.W, img_h=cam.H)
        slabs.update(slabs_conic)
        # tiles of the rectangle that meet the parallelogram (row-major), counted in chunks
        count = np.zeros(N, np.int64)
        tile_counts = np.zeros(TX * TY, np.int64)
        vidx = np.nonzero(vis)[0]
        per = ((rect[vidx, 1] - rect[vidx, 0] + 1).astype(np.int64) * (rect[vidx, 3] - rect[vidx, 2] + 1))
        start = 0
        while start < vidx.size:
            stop = start + 1
            tot = per[start]
            while stop < vidx.size and tot + per[stop] <= 4_000_000:
                tot += per[stop]
                stop += 1
            p_, tx_, ty_ = _rect_tiles(rect, vidx[start:stop])
            ok = _tile_pass(slabs, p_, tx_, ty_)
            count += np.bincount(p_[ok], minlength=N)
            tile_counts += np.bincount((ty_[ok] * TX + tx_[ok]).astype(np.int64), minlength=TX * TY)
            start = stop
        vis &= count > 0
        rect[~vis] = 0
        zbits = muc[2].astype(f).view(np.uint32).copy()

    pix_bbox = np.stack([xmin, xmax, ymin, ymax], 1).astype(np.float32)
    geo = None
    if order == "hit":
        geo = dict(muc=[c.astype(f) for c in muc], Wm=Wm, a=a, b=b, fx=fx, fy=fy, cx=cx, cy=cy, near=near,
                   img_w=cam.W, img_h=cam.H)
    elif order != "centre":
        raise ValueError(order)
    bn = Binning(vis, zbits, rect, count, None, None, None, TX, TY, pix_bbox, order, geo, slabs, tile_counts)
    if not emit:
        return bn
    # instances in primitive order, tiles row-major inside each rectangle (those that meet
    # the parallelogram)
    I = int(count.sum())
    keys = np.empty(I, np.uint64)
    vals = np.empty(I, np.uint32)
    pos = 0
    for i in np.nonzero(count)[0]:
        p_, tx_, ty_ = _rect_tiles(rect, np.array([i]))
        ok = _tile_pass(slabs, p_, tx_, ty_)
        tiles = (ty_[ok] * TX + tx_[ok]).astype(np.int64)
        c = tiles.size
        if order == "hit":
            low = np.array([hit_keys(bn, np.array([i]), t)[0] for t in tiles], np.uint64)
        else:
            low = np.uint64(zbits[i])
        keys[pos:pos + c] = (tiles.astype(np.uint64) << np.uint64(32)) | low
        vals[pos:pos + c] = i
        pos += c
    srt = np.argsort(keys, kind="stable")
    keys = keys[srt]
    vals = vals[srt]
    tiles_sorted = (keys >> np.uint64(32)).astype(np.int64)
    ntiles = TX * TY
    starts = np.searchsorted(tiles_sorted, np.arange(ntiles), side="left")
    ends = np.searchsorted(tiles_sorted, np.arange(ntiles), side="right")
    ranges = np.stack([starts, ends], 1).astype(np.int64)
    return Binning(vis, zbits, rect, count, keys, vals, ranges, TX, TY, pix_bbox, order, geo, slabs, tile_counts)


def tile_list(binning: Binning, tile: int) -> np.ndarray:
    """Sorted primitive list of one tile, from the rectangles and depth keys alone
    (the same order as the sorted 64-bit keys: depth bits, then primitive index)."""
    ty, tx = divmod(int(tile), binning.tiles_x)
    r = binning.rect
    sel = np.nonzero((binning.count > 0) & (r[:, 0] <= tx) & (tx <= r[:, 1]) & (r[:, 2] <= ty) & (ty <= r[:, 3]))[0]
    sel = sel[_tile_pass(binning.slabs, sel, np.full(sel.shape, tx), np.full(sel.shape, ty))]
    depth = hit_keys(binning, sel, tile) if binning.order == "hit" else binning.zbits[sel]
    order = np.lexsort((sel, depth))
    return sel[order].astype(np.uint32)


# =========================================================================== FP64 geometry
def quat_to_rot(q: torch.Tensor) -> torch.Tensor:
    """Rotation matrix (local -> world) of the normalised quaternion (w, x, y, z)."""
    q = q / torch.linalg.vector_norm(q, dim=-1, keepdim=True)
    w, x, y, z = q.unbind(-1)
    return torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
    ], -2)


def arc_length(a_theta: torch.Tensor, rho: torch.Tensor) -> torch.Tensor:
    """Arc length of the radial section z = a rho^2 from the vertex to rho (Sec. 3.2,
    geodesic Eq.): l = [ln(sqrt(u^2+1) + u) + u sqrt(u^2+1)] / (4a), u = 2 a rho.
    For |u| < 1e-3 the series rho (1 + u^2/6 - u^4/40) is used (it also covers a = 0,
    where l = rho, the planar limit stated in Sec. 3.2)."""
    u = 2.0 * a_theta * rho
    small = u.abs() < TAYLOR_U
    u_s = torch.where(small, torch.full_like(u, 1.0), u)
    a_s = torch.where(small, torch.full_like(u, 1.0), a_theta)
    r = torch.sqrt(u_s * u_s + 1.0)
    closed = (torch.log(r + u_s) + u_s * r) / (4.0 * a_s)
    u2 = u * u
    series = rho * (1.0 + u2 / 6.0 - u2 * u2 / 40.0)
    return torch.where(small, series, closed)


def sigma_theta(theta: torch.Tensor, s1: torch.Tensor, s2: torch.Tensor) -> torch.Tensor:
    """Directional standard deviation of the in-surface Gaussian (Sec. 3.2, sigma Eq.)."""
    return s1 * s2 / torch.sqrt((s2 * torch.cos(theta)) ** 2 + (s1 * torch.sin(theta)) ** 2)


def geodesic_gaussian(x, y, a, b, s1, s2):
    """Geodesic Gaussian at a surface point with local (x, y) (Sec. 3.2).
    Returns (G, l, sigma). theta is the cylindrical angle of (x, y);
    a(theta) = a cos^2 theta + b sin^2 theta (polar form of the paraboloid)."""
    rho2 = x * x + y * y
    zero = rho2 == 0
    xs = torch.where(zero, torch.ones_like(x), x)
    ys = torch.where(zero, torch.zeros_like(y), y)
    theta = torch.atan2(ys, xs)
    rho = torch.sqrt(torch.where(zero, torch.ones_like(rho2), rho2))
    rho = torch.where(zero, torch.zeros_like(rho), rho)
    a_th = a * torch.cos(theta) ** 2 + b * torch.sin(theta) ** 2
    l = arc_length(a_th, rho)
    sig = sigma_theta(theta, s1, s2)
    G = torch.exp(-(l * l) / (2.0 * sig * sig))
    return G, l, sig


def euclid_gaussian(x, y, a, b, s1, s2):
    """The Euclidean-distance density that the paper contrasts with its geodesic one
    (Sec. 3.2, the disk -> paraboloid deformation argument; ablated as "w/ Euclid" in
    Sec. 4.3): the same sigma(theta), with l the straight-line distance from the vertex to
    the surface point, sqrt(rho^2 + z^2), z = a x^2 + b y^2. Returns (G, l, sigma)."""
    rho2 = x * x + y * y
    zero = rho2 == 0
    xs = torch.where(zero, torch.ones_like(x), x)
    ys = torch.where(zero, torch.zeros_like(y), y)
    theta = torch.atan2(ys, xs)
    z = a * x * x + b * y * y
    l = torch.sqrt(rho2 + z * z)
    sig = sigma_theta(theta, s1, s2)
    G = torch.exp(-(l * l) / (2.0 * sig * sig))
    return G, l, sig


def gaussian_curvature(x, y, a, b):
    """Gaussian curvature of z = a x^2 + b y^2 at local (x, y) (Sec. 3.2.1 curvature Eq.,
    derived in the supplementary's "Details of Curvature"; lambda_1 = a, lambda_2 = b):
    4ab / (1 + 4a^2 x^2 + 4b^2 y^2)^2."""
    S = 1.0 + 4.0 * a * a * x * x + 4.0 * b * b * y * y
    return 4.0 * a * b / (S * S)


def quadratic_roots(A, B, C, flip_real=None, d_shift=None):
    """Both real roots (t1 <= t2) of A t^2 + B t + C = 0 and whether they exist.
    q = -(B + sgn(B) sqrt(D)) / 2 with sgn(0) = +1; the roots are C/q and q/A, each
    missing when its denominator is zero (A = 0 leaves the single root -C/B).
    Bracketing (decisions taken the other way, see bracket_pixels): flip_real inverts the
    decision D >= 0 (a negative D then counts as 0, the double root); d_shift moves the
    discriminant by that much, by solving the quadratic with C - d_shift / (4A) (A != 0)."""
    if d_shift is not None:
        A_s = torch.where(A != 0, A, torch.ones_like(A))
        C = torch.where(A != 0, C - d_shift / (4.0 * A_s), C)
    D = B * B - 4.0 * A * C
    real = D >= 0
    if flip_real is not None:
        real = real ^ flip_real
    Ds = torch.where(real & (D > 0), D, torch.zeros_like(D))
    sgn = torch.where(B >= 0, torch.ones_like(B), -torch.ones_like(B))
    q = -0.5 * (B + sgn * torch.sqrt(Ds))
    ok1 = real & (q != 0)
    ok2 = real & (A != 0)
    q_s = torch.where(q != 0, q, torch.ones_like(q))
    A_s = torch.where(A != 0, A, torch.ones_like(A))
    r1 = C / q_s
    r2 = q / A_s
    ok1 = ok1 & torch.isfinite(r1)
    ok2 = ok2 & torch.isfinite(r2)
    # order: put the smaller existing root first
    swap = ok1 & ok2 & (r2 < r1)
    t1 = torch.where(swap, r2, r1)
    t2 = torch.where(swap, r1, r2)
    e1 = torch.where(swap, ok2, ok1)
    e2 = torch.where(swap, ok1, ok2)
    # a single existing root is the "near" one
    only2 = ~e1 & e2
    t1, t2 = torch.where(only2, t2, t1), torch.where(only2, t1, t2)
    e1, e2 = e1 | e2, e1 & e2
    margin_D = (D.abs() / (B * B + 4.0 * (A * C).abs()).clamp_min(1e-300)).detach()
    return t1, t2, e1, e2, margin_D


# =========================================================================== colour
SH_C0 = 0.5 * math.sqrt(1.0 / math.pi)
SH_C1 = math.sqrt(3.0 / (4.0 * math.pi))
SH_C2 = (0.5 * math.sqrt(15.0 / math.pi), -0.5 * math.sqrt(15.0 / math.pi),
         0.25 * math.sqrt(5.0 / math.pi), -0.5 * math.sqrt(15.0 / math.pi),
         0.25 * math.sqrt(15.0 / math.pi))
SH_C3 = (-0.25 * math.sqrt(35.0 / (2 * math.pi)), 0.5 * math.sqrt(105.0 / math.pi),
         -0.25 * math.sqrt(21.0 / (2 * math.pi)), 0.25 * math.sqrt(7.0 / math.pi),
         -0.25 * math.sqrt(21.0 / (2 * math.pi)), 0.25 * math.sqrt(105.0 / math.pi),
         -0.25 * math.sqrt(35.0 / (2 * math.pi)))


def sh_basis(d: torch.Tensor) -> torch.Tensor:
    """The 16 real spherical-harmonic basis functions of degree <= 3 at unit directions
    d [..., 3], in the order and sign convention of 3DGS (Sec. 3.1 uses its colour model)."""
    x, y, z = d.unbind(-1)
    xx, yy, zz = x * x, y * y, z * z
    one = torch.ones_like(x)
    return torch.stack([
        SH_C0 * one,
        -SH_C1 * y, SH_C1 * z, -SH_C1 * x,
        SH_C2[0] * x * y, SH_C2[1] * y * z, SH_C2[2] * (2 * zz - xx - yy),
        SH_C2[3] * x * z, SH_C2[4] * (xx - yy),
        SH_C3[0] * y * (3 * xx - yy), SH_C3[1] * x * y * z,
        SH_C3[2] * y * (4 * zz - xx - yy), SH_C3[3] * z * (2 * zz - 3 * xx - 3 * yy),
        SH_C3[4] * x * (4 * zz - xx - yy), SH_C3[5] * z * (xx - yy),
        SH_C3[6] * x * (xx - 3 * yy),
    ], -1)


# =========================================================================== params
def bf16_to_f64(bits) -> np.ndarray:
    """Values of bfloat16 bit patterns: a bfloat16 is the upper half of an IEEE binary32,
    so the pattern shifted up by 16 bits is that binary32 exactly (widened to FP64)."""
    b = np.asarray(bits, np.uint16).astype(np.uint32) << np.uint32(16)
    return b.view(np.float32).astype(np.float64)


class Params:
    """FP64 leaf tensors of a scene (SH decoded from its bfloat16 storage)."""

    def __init__(self, scene, requires_grad=False):
        def t(x):
            return torch.tensor(np.asarray(x, np.float64), dtype=F64, requires_grad=requires_grad)

        self.mean = t(scene.mean)
        self.quat = t(scene.quat)
        self.scale = t(scene.scale)
        self.curv = t(scene.curv)
        self.opacity = t(scene.opacity)
        self.sh = t(bf16_to_f64(scene.sh).reshape(-1, 16, 3))

    def leaves(self):
        return dict(mean=self.mean, quat=self.quat, scale=self.scale, curv=self.curv,
                    opacity=self.opacity, sh=self.sh)


class CamF64:
    def __init__(self, cam):
        self.W, self.H = cam.W, cam.H
        self.fx, self.fy = float(np.float32(cam.fx)), float(np.float32(cam.fy))
        self.cx, self.cy = float(np.float32(cam.cx)), float(np.float32(cam.cy))
        self.R = torch.tensor(cam.R_cw.astype(np.float64), dtype=F64)
        self.t = torch.tensor(cam.t_cw.astype(np.float64), dtype=F64)
        self.near = float(np.float32(cam.near))
        self.c_w = -(self.R.T @ self.t)      # camera centre in world coordinates


# =========================================================================== per-pair evaluation
DECISIONS = ("D", "near1", "near2", "in1", "in2", "amin", "amax")


def _eval_pairs(prm: Params, cam: CamF64, idx: torch.Tensor, px: torch.Tensor, py: torch.Tensor,
                density: str = "geodesic", flip: dict | None = None, d_shift=None, root_leaves: bool = False,
                ray_noise=None, coef_noise=None):
    """Evaluate every (pixel, primitive) pair of a pixel set [P] and a primitive list [L].
    Returns per-pair tensors [P, L]: alpha (0 where no contribution), validity, depth t,
    colour [P, L, 3] (broadcast), camera-space unit normal [P, L, 3], Gaussian curvature
    at the hit and decision margins. density: "geodesic" (the paper's) or "euclid".

    The pair's discrete decisions, each with its relative margin (how far the deciding
    quantity is from its threshold; infinite where the decision cannot change the pair's
    contribution) in `margins`:
      D      real roots, D >= 0 (counted only where the double root lies on the support);
      near1  the near root is in front of the near plane (t > near);
      near2  the same for the far root;
      in1    the near root's hit is within 3 sigma(theta) (l <= 3 sigma, Sec. 3.2.1);
      in2    the same for the far root (counted only where the near root is not taken);
      amin   alpha >= 1/255 (blended at all);
      amax   o G < 0.99 (alpha not clamped: the same value either way, another derivative).
    `flip` (bracketing, see bracket_pixels) maps decision names to bool tensors
    broadcastable to [P, L] that take those decisions the other way; `d_shift` [P, L] is
    added to the discriminant (in units of the scale of its rounding, below). With
    root_leaves, the two roots are made leaves of the autograd graph (returned as "roots"),
    so that a backward pass yields the derivative of the outputs with respect to each root
    (see graze_bands). ray_noise [P, L, 6] (see ray_sensitivity) perturbs each pair's local
    ray: its origin where it crosses the centre's depth and its direction, componentwise
    and relatively; coef_noise [P, L, 3] perturbs the quadratic's coefficients in the frame
    re-based at the centre's depth, each relative to the magnitudes of its terms."""
    weight_fn = {"geodesic": geodesic_gaussian, "euclid": euclid_gaussian}[density]
    fl = flip or {}
    mu = prm.mean[idx]
    R = quat_to_rot(prm.quat[idx])                  # [L,3,3] columns = local axes (world)
    su, sv = prm.scale[idx].unbind(-1)
    a, b = prm.curv[idx].unbind(-1)
    o = prm.opacity[idx]

    # Local camera centre and pixel rays (congruent transform, Sec. 3.2).
    o_hat = torch.einsum("lji,lj->li", R, cam.c_w[None, :] - mu)         # R^T (c - mu)
    d_cam = torch.stack([(px + 0.5 - cam.cx) / cam.fx, (py + 0.5 - cam.cy) / cam.fy,
                         torch.ones_like(px)], -1)                         # [P,3], z = 1
    d_w = d_cam @ cam.R                                                    # R_cw^T d_cam
    d_hat = torch.einsum("lji,pj->pli", R, d_w)                            # [P,L,3]
    ox, oy, oz = (o_hat[:, k][None, :] for k in range(3))
    dx, dy, dz = d_hat.unbind(-1)
    if ray_noise is not None:
        t0n = (mu @ cam.R[2] + cam.t[2])[None, :]
        o0 = [(o + t0n * d) * (1.0 + ray_noise[..., k]) for k, (o, d) in enumerate(((ox, dx), (oy, dy), (oz, dz)))]
        dx, dy, dz = (d * (1.0 + ray_noise[..., 3 + k]) for k, d in enumerate((dx, dy, dz)))
        ox, oy, oz = o0[0] - t0n * dx, o0[1] - t0n * dy, o0[2] - t0n * dz
    A_ = a * dx * dx + b * dy * dy
    B_ = 2.0 * (a * ox * dx + b * oy * dy) - dz
    C_ = (a * ox * ox + b * oy * oy - oz).expand_as(A_)
    if coef_noise is not None:
        with torch.no_grad():
            t0c = (mu @ cam.R[2] + cam.t[2])[None, :]
            qx, qy, qz = ox + t0c * dx, oy + t0c * dy, oz + t0c * dz
            sA = a.abs() * dx * dx + b.abs() * dy * dy
            sB = 2.0 * ((a * qx * dx).abs() + (b * qy * dy).abs()) + dz.abs()
            sC = a.abs() * qx * qx + b.abs() * qy * qy + qz.abs()
        A0n = A_ + coef_noise[..., 0] * sA
        B0n = (B_ + 2.0 * A_ * t0c) + coef_noise[..., 1] * sB
        C0n = ((A_ * t0c + B_) * t0c + C_) + coef_noise[..., 2] * sC
        A_, B_, C_ = A0n, B0n - 2.0 * A0n * t0c, (A0n * t0c - B0n) * t0c + C0n
    # Scale of the discriminant's rounding: D is the same for the ray re-parametrised as
    # s = t - t0 around the depth t0 of the centre, where the ray starts at o0 = o + t0 d,
    # of the size of the primitive instead of the camera distance. A, B0 and C0 are sums of
    # terms that cancel on saddles (a b < 0) and near tangency, so an implementation that
    # rounds them knows D to a fraction of the same sums taken over the terms' absolute
    # values, not of |B0|^2 + 4 |A C0|.
    with torch.no_grad():
        t0 = (mu @ cam.R[2] + cam.t[2])[None, :]
        o0x, o0y, o0z = ox + t0 * dx, oy + t0 * dy, oz + t0 * dz
        Aab = a.abs() * dx * dx + b.abs() * dy * dy
        Bab = 2.0 * ((a * o0x * dx).abs() + (b * o0y * dy).abs()) + dz.abs()
        Cab = a.abs() * o0x * o0x + b.abs() * o0y * o0y + o0z.abs()
        d_scale = (Bab * Bab + 4.0 * Aab * Cab).clamp_min(1e-300)
    shift = None if d_shift is None else d_shift * d_scale
    t1, t2, e1, e2, _ = quadratic_roots(A_, B_, C_, fl.get("D"), shift)
    if root_leaves:
        t1 = t1.detach().requires_grad_(True)
        t2 = t2.detach().requires_grad_(True)
    roots = (t1, t2)
    with torch.no_grad():
        D_ = B_ * B_ - 4.0 * A_ * C_ + (0.0 if shift is None else torch.where(A_ != 0, shift, 0.0 * shift))
        m_D = D_.abs() / d_scale
        # Conditioning of a hit's derivative: at a root, d f / d t = +-sqrt(D), so the
        # derivative of the root (and everything downstream of it) scales like 1/sqrt(D);
        # a rounding error e d_scale of D moves it by about e d_scale / (2 D).
        m_cond = m_D.clone()
        # The decision only matters where the double root t* = -B/(2A) lies on the
        # support (x^2/s_u^2 + y^2/s_v^2 <= 9, with slack); elsewhere both outcomes
        # contribute nothing.
        As = torch.where(A_ != 0, A_, torch.ones_like(A_))
        tv = -B_ / (2.0 * As)
        ev = ((ox + tv * dx) / su) ** 2 + ((oy + tv * dy) / sv) ** 2
        m_D = torch.where((A_ != 0) & (ev <= 10.0), m_D, torch.full_like(m_D, np.inf))

    near = cam.near

    def front(t, e, name):
        ok = t > near
        if name in fl:
            ok = ok ^ fl[name]
        m = torch.where(e, (t - near).abs() / near, torch.full_like(t, np.inf)).detach()
        return e & ok, m

    f1, m_near1 = front(t1, e1, "near1")
    f2, m_near2 = front(t2, e2, "near2")

    def at(t, ok, name):
        ts = torch.where(ok, t, torch.zeros_like(t))
        x = ox + ts * dx
        y = oy + ts * dy
        G, l, sig = weight_fn(x, y, a, b, su, sv)
        within = l <= CUTOFF * sig
        if name in fl:
            within = within ^ fl[name]
        margin = torch.where(ok, (l - CUTOFF * sig).abs() / (CUTOFF * sig), torch.full_like(l, np.inf))
        return ts, x, y, G, ok & within, margin.detach()

    # candidates in increasing t: the near root first, then the far one (Sec. 3.2.1)
    tn, xn, yn, Gn, in_n, m_in1 = at(t1, f1, "in1")
    tf, xf, yf, Gf, in_f, m_in2 = at(t2, f2, "in2")
    pick_n = in_n
    pick_f = ~in_n & in_f
    hit = pick_n | pick_f
    t = torch.where(pick_n, tn, tf)
    x = torch.where(pick_n, xn, xf)
    y = torch.where(pick_n, yn, yf)
    G = torch.where(pick_n, Gn, torch.where(pick_f, Gf, torch.zeros_like(Gf)))
    m_in2 = torch.where(in_n, torch.full_like(m_in2, np.inf), m_in2)

    oG = o * G
    clamped = oG > ALPHA_MAX
    if "amax" in fl:
        clamped = clamped ^ fl["amax"]
    alpha = torch.where(clamped, torch.full_like(oG, ALPHA_MAX), oG)
    blend = alpha >= ALPHA_MIN
    if "amin" in fl:
        blend = blend ^ fl["amin"]
    valid = hit & blend
    alpha = torch.where(valid, alpha, torch.zeros_like(alpha))
    m_amin = torch.where(hit, (oG - ALPHA_MIN).abs() / ALPHA_MIN, torch.full_like(oG, np.inf)).detach()
    m_amax = torch.where(valid, (oG - ALPHA_MAX).abs() / ALPHA_MAX, torch.full_like(oG, np.inf)).detach()

    # Normal: gradient of a x^2 + b y^2 - z at the hit (Sec. 3.2 normal Eq.), camera space,
    # facing the camera.
    n_l = torch.stack([2.0 * a * x, 2.0 * b * y, -torch.ones_like(x)], -1)   # [P,L,3]
    n_w = torch.einsum("lij,plj->pli", R, n_l)
    n_c = n_w @ cam.R.T
    n_c = n_c / torch.linalg.vector_norm(n_c, dim=-1, keepdim=True)
    facing = (n_c * d_cam[:, None, :]).sum(-1) > 0
    n_c = torch.where(facing[..., None], -n_c, n_c)

    # View-dependent colour (degree-3 SH, Sec. 3.1) at dir = normalise(mu - c).
    dv = mu - cam.c_w[None, :]
    dv = dv / torch.linalg.vector_norm(dv, dim=-1, keepdim=True)
    rgb = torch.clamp((sh_basis(dv)[:, :, None] * prm.sh[idx]).sum(1) + 0.5, min=0.0)   # [L,3]

    margins = dict(D=m_D, near1=m_near1, near2=m_near2, in1=m_in1, in2=m_in2, amin=m_amin, amax=m_amax)
    margin = m_D
    for k in DECISIONS[1:]:
        margin = torch.minimum(margin, margins[k])
    cond = torch.where(valid, m_cond, torch.full_like(m_cond, np.inf))
    K = gaussian_curvature(x, y, a, b)
    return dict(alpha=alpha, valid=valid, hit=hit, t=t, rgb=rgb, normal=n_c, curvature=K, margin=margin,
                cond=cond, margins=margins, roots=roots, pick_near=pick_n)


MEDIAN_T = 0.5   # median depth: the largest hit depth among blended pairs with T_i > 0.5


def _distortion(w: torch.Tensor, t: torch.Tensor, block: int = 32) -> torch.Tensor:
    """Depth distortion of each pixel (Sec. 3.3, depth distortion Eq.):
    sum_i sum_{j<i} w_i w_j (t_i - t_j)^2 over the pixel's blended pairs in order, summed
    as written (blocks of i only bound the memory)."""
    P, L = w.shape
    out = torch.zeros(P, dtype=F64)
    jj = torch.arange(L)
    for i0 in range(0, L, block):
        i1 = min(i0 + block, L)
        diff = t[:, i0:i1, None] - t[:, None, :i1]                        # [P, B, i1]
        below = (jj[None, :i1] < torch.arange(i0, i1)[:, None]).to(F64)  # j < i
        out = out + (w[:, i0:i1, None] * w[:, None, :i1] * diff * diff * below[None]).sum((1, 2))
    return out


def _composite(prm, cam, idx, px, py, chunk=4096, density="geodesic", extras=False, collect=None, noise=None):
    """Front-to-back alpha blending of a pixel set over one sorted primitive list
    (blending Eq. of Sec. 3.1 and X_hat = sum alpha_i T_i X_i of the supplementary).
    extras: also the curvature map (Sec. 3.2.1, N/K rendering Eq.), the depth distortion
    (Sec. 3.3) and the median depth (Sec. 4.1, max t_i with T_i > 0.5; 0 where no blended
    pair qualifies)."""
    P = px.shape[0]
    dev = dict(dtype=F64)
    T = torch.ones(P, **dev)
    alive = torch.ones(P, dtype=torch.bool)
    rgb = torch.zeros(P, 3, **dev)
    depth = torch.zeros(P, **dev)
    normal = torch.zeros(P, 3, **dev)
    n_eval = torch.zeros(P, dtype=torch.int64)
    n_contrib = torch.zeros(P, dtype=torch.int64)
    margin = torch.full((P,), np.inf, **dev)
    cond = torch.full((P,), np.inf, **dev)
    list_cond = None
    curv = torch.zeros(P, **dev)
    curv_scale = torch.zeros(P, **dev)
    median = torch.zeros(P, **dev)
    m_median = torch.full((P,), np.inf, **dev)
    w_cols, t_cols = [], []
    L = idx.shape[0]
    for c0 in range(0, L, chunk):
        sl = idx[c0:c0 + chunk]
        Lc = sl.shape[0]
        rn, cn = (None, None) if noise is None else noise(P, sl.shape[0], c0)
        pe = _eval_pairs(prm, cam, sl, px, py, density, root_leaves=collect is not None, ray_noise=rn,
                         coef_noise=cn)
        if collect is not None:
            collect.append((c0, pe))
        al, v = pe["alpha"], pe["valid"]
        onem = 1.0 - al
        cp = torch.cumprod(onem, dim=1)
        Tex = T[:, None] * torch.cat([torch.ones(P, 1, **dev), cp[:, :-1]], 1)
        m_T = torch.where(v, (Tex * onem - T_MIN).abs().detach() / T_MIN,
                          torch.full_like(Tex, np.inf))
        term = v & ((Tex * onem) < T_MIN) & alive[:, None]
        has = term.any(1)
        k = torch.where(has, torch.argmax(term.to(torch.int8), 1), torch.full((P,), Lc))
        ar = torch.arange(Lc)[None, :]
        seen = (ar <= k[:, None]) & alive[:, None]
        keep = v & (ar < k[:, None]) & alive[:, None]
        w = torch.where(keep, al * Tex, torch.zeros_like(al))
        rgb = rgb + (w[..., None] * pe["rgb"][None, :, :]).sum(1)
        depth = depth + (w * pe["t"]).sum(1)
        normal = normal + (w[..., None] * pe["normal"]).sum(1)
        if extras:
            curv = curv + (w * pe["curvature"]).sum(1)
            curv_scale = curv_scale + (w * pe["curvature"].abs()).sum(1).detach()
            med_ok = keep & (Tex > MEDIAN_T)
            tm = torch.where(med_ok, pe["t"], torch.zeros_like(pe["t"])).detach()
            median = torch.maximum(median, tm.max(1).values)
            mm_ = torch.where(keep, (Tex - MEDIAN_T).abs().detach() / MEDIAN_T, torch.full_like(Tex, np.inf))
            m_median = torch.minimum(m_median, mm_.min(1).values)
            w_cols.append(w)
            t_cols.append(torch.where(keep, pe["t"], torch.zeros_like(pe["t"])))
        T = T * torch.where(keep, onem, torch.ones_like(onem)).prod(1)
        mm = torch.minimum(pe["margin"], m_T)
        margin = torch.minimum(margin, torch.where(seen, mm, torch.full_like(mm, np.inf)).min(1).values)
        cond = torch.minimum(cond, torch.where(keep, pe["cond"], torch.full_like(mm, np.inf)).min(1).values)
        lc = torch.where(keep, pe["cond"], torch.full_like(mm, np.inf)).min(0).values
        list_cond = lc if list_cond is None else torch.cat([list_cond, lc])
        n_eval = n_eval + torch.where(alive, torch.where(has, k + 1, torch.full_like(k, Lc)),
                                      torch.zeros_like(k))
        last = torch.where(keep, ar.expand(P, Lc) + c0 + 1, torch.zeros_like(keep, dtype=torch.int64))
        n_contrib = torch.maximum(n_contrib, last.max(1).values)
        alive = alive & ~has
        if not bool(alive.any()):
            break
    if list_cond is None or list_cond.shape[0] < L:
        pad = torch.full((L - (0 if list_cond is None else list_cond.shape[0]),), np.inf, **dev)
        list_cond = pad if list_cond is None else torch.cat([list_cond, pad])
    res = dict(rgb=rgb, alpha=1.0 - T, depth=depth, normal=normal, T_final=T,
               n_eval=n_eval, n_contrib=n_contrib, margin=margin, cond=cond, list_cond=list_cond)
    if extras:
        if w_cols:
            dist = _distortion(torch.cat(w_cols, 1), torch.cat(t_cols, 1))
        else:
            dist = torch.zeros(P, **dev)
        res.update(curvature=curv, curvature_scale=curv_scale, distortion=dist, median_depth=median,
                   margin_median=m_median)
    return res


RESORT = 8   # per-pixel resort buffer length of the supplementary's resorting
# The resort decision compares two hit depths t = z + s that an FP32 implementation forms
# to about one ulp (6e-8 relative); its margin is the relative gap scaled so that a gap
# of 1e-6 (16 ulp) meets the common 1e-5 margin threshold.
ORDER_GAP_SCALE = 10.0


def _composite_resort(prm, cam, idx, px, py, density="geodesic", extras=False, buf=RESORT, collect=None,
                      noise=None):
    """Front-to-back blending with StopThePop's per-pixel local resorting as adopted by
    the supplementary ("Details of Per-tile Sorting and Per-pixel Resorting"): each pixel
    walks its tile's list and puts every contributing pair (alpha >= 1/255) into a buffer
    of `buf` entries; whenever the buffer is full, the entry with the smallest hit depth
    (ties: earlier in the list) is blended and removed; at the end of the list the rest
    is blended nearest first. The transmittance rule is unchanged: a pixel stops before
    a pair that would take T below 1e-4. Same outputs as _composite; the order decision
    (smallest depth in the buffer) adds its relative gap to the decision margins."""
    P = px.shape[0]
    L = idx.shape[0]
    dev = dict(dtype=F64)
    rn, cn = (None, None) if noise is None else noise(P, L, 0)
    pe = _eval_pairs(prm, cam, idx, px, py, density, root_leaves=collect is not None, ray_noise=rn,
                     coef_noise=cn)
    if collect is not None:
        collect.append((0, pe))
    al, valid, tt = pe["alpha"], pe["valid"], pe["t"]
    rows = torch.arange(P)
    T = torch.ones(P, **dev)
    alive = torch.ones(P, dtype=torch.bool)
    rgb = torch.zeros(P, 3, **dev)
    depth = torch.zeros(P, **dev)
    normal = torch.zeros(P, 3, **dev)
    curv = torch.zeros(P, **dev)
    curv_scale = torch.zeros(P, **dev)
    median = torch.zeros(P, **dev)
    m_median = torch.full((P,), np.inf, **dev)
    margin = torch.full((P,), np.inf, **dev)
    cond = torch.full((P,), np.inf, **dev)
    n_contrib = torch.zeros(P, dtype=torch.int64)
    stop_at = torch.full((P,), L - 1, dtype=torch.int64)    # last list entry each pixel evaluated
    bt = torch.full((P, buf), np.inf, **dev)                 # buffered depths (decisions only)
    bj = torch.full((P, buf), -1, dtype=torch.int64)         # buffered list positions
    w_cols, t_cols = [], []
    state = dict(T=T, alive=alive, rgb=rgb, depth=depth, normal=normal, curv=curv, curv_scale=curv_scale,
                 median=median, m_median=m_median, margin=margin, cond=cond, n_contrib=n_contrib)

    def pop(mask, j_now):
        st = state
        big = torch.iinfo(torch.int64).max
        mn = bt.min(1).values
        cand = (bt == mn[:, None]) & (bj >= 0)
        jsel = torch.where(cand, bj, torch.full_like(bj, big)).min(1).values
        sel = mask & (jsel != big)
        if not bool(sel.any()):
            return
        slot = (bj == jsel[:, None]).long().argmax(1)
        if buf > 1:
            srt = bt.sort(1).values
            gap = torch.where(torch.isfinite(srt[:, 1]),
                              ORDER_GAP_SCALE * (srt[:, 1] - srt[:, 0]).abs() / srt[:, 0].abs(),
                              torch.full_like(mn, np.inf))
        else:
            gap = torch.full_like(mn, np.inf)
        st["margin"] = torch.minimum(st["margin"], torch.where(sel, gap, torch.full_like(gap, np.inf)))
        js = torch.where(sel, jsel, torch.zeros_like(jsel))
        a = al[rows, js]
        Tn = st["T"] * (1.0 - a)
        m_T = ((Tn - T_MIN).abs() / T_MIN).detach()
        st["margin"] = torch.minimum(st["margin"], torch.where(sel, m_T, torch.full_like(m_T, np.inf)))
        stop = sel & (Tn < T_MIN)
        keep = sel & ~stop
        w = torch.where(keep, a * st["T"], torch.zeros_like(a))
        t_sel = tt[rows, js]
        st["rgb"] = st["rgb"] + w[:, None] * pe["rgb"][js]
        st["depth"] = st["depth"] + w * t_sel
        st["normal"] = st["normal"] + w[:, None] * pe["normal"][rows, js]
        st["cond"] = torch.minimum(st["cond"], torch.where(keep, pe["cond"][rows, js],
                                                           torch.full_like(m_T, np.inf)))
        if extras:
            K = pe["curvature"][rows, js]
            st["curv"] = st["curv"] + w * K
            st["curv_scale"] = st["curv_scale"] + (w * K.abs()).detach()
            med_ok = keep & (st["T"] > MEDIAN_T)
            st["median"] = torch.maximum(st["median"], torch.where(med_ok, t_sel, torch.zeros_like(t_sel)).detach())
            mm_ = torch.where(keep, (st["T"] - MEDIAN_T).abs().detach() / MEDIAN_T, torch.full_like(m_T, np.inf))
            st["m_median"] = torch.minimum(st["m_median"], mm_)
            w_cols.append(w[:, None])
            t_cols.append(torch.where(keep, t_sel, torch.zeros_like(t_sel))[:, None])
        st["T"] = torch.where(keep, Tn, st["T"])
        st["n_contrib"] = st["n_contrib"] + keep.long()
        st["alive"] = st["alive"] & ~stop
        stop_at[stop] = j_now
        bt[rows[sel], slot[sel]] = np.inf
        bj[rows[sel], slot[sel]] = -1

    for j in range(L):
        m = state["alive"] & valid[:, j]
        if bool(m.any()):
            slot = (bj == -1).long().argmax(1)
            r = rows[m]
            bt[r, slot[m]] = tt[m, j].detach()
            bj[r, slot[m]] = j
            full = m & ((bj >= 0).sum(1) == buf)
            if bool(full.any()):
                pop(full, j)
    for _ in range(buf):
        pending = state["alive"] & ((bj >= 0).sum(1) > 0)
        if not bool(pending.any()):
            break
        pop(pending, L - 1)
    # decision margins of every pair each pixel evaluated
    seen = torch.arange(L)[None, :] <= stop_at[:, None]
    pm = torch.where(seen, pe["margin"], torch.full_like(pe["margin"], np.inf)).min(1).values
    st = state
    res = dict(rgb=st["rgb"], alpha=1.0 - st["T"], depth=st["depth"], normal=st["normal"], T_final=st["T"],
               n_eval=stop_at + 1, n_contrib=st["n_contrib"], margin=torch.minimum(st["margin"], pm),
               cond=st["cond"],
               list_cond=torch.where(valid, pe["cond"], torch.full_like(pe["cond"], np.inf)).min(0).values)
    if extras:
        dist = _distortion(torch.cat(w_cols, 1), torch.cat(t_cols, 1)) if w_cols else torch.zeros(P, **dev)
        res.update(curvature=st["curv"], curvature_scale=st["curv_scale"], distortion=dist,
                   median_depth=st["median"], margin_median=st["m_median"])
    return res


# =========================================================================== images
OUT_KEYS = ("rgb", "alpha", "depth", "normal")
EXTRA_KEYS = ("curvature", "distortion", "median_depth")


def _tile_pixels(cam, tile, TX):
    ty, tx = divmod(int(tile), TX)
    ys, xs = np.meshgrid(np.arange(ty * TILE, min(ty * TILE + TILE, cam.H)),
                         np.arange(tx * TILE, min(tx * TILE + TILE, cam.W)), indexing="ij")
    return xs.reshape(-1), ys.reshape(-1)


def render(scene, cam, binning: Binning | None = None, tiles=None, grad_images=None, density="geodesic",
           extras=False, order="centre", ray_noise_seed=None, timings: dict | None = None):
    """Render the full image (or the listed tiles). Returns a dict of numpy arrays:
    rgb [3,H,W], alpha [H,W], depth [H,W], normal [3,H,W], margin [H,W], n_eval [H,W],
    n_contrib [H,W], T_final [H,W]; with `extras` also curvature, distortion,
    median_depth, curvature_scale (sum w |K|) and margin_median [H,W]. With
    `grad_images` (a dict of upstream gradients with the same shapes as the outputs,
    missing ones zero; curvature and distortion may be included, the median depth has
    none), also returns
    `grads`: the exact FP64 gradient of sum(grad * output) with respect to every scene
    parameter. density: "geodesic" (the paper's) or "euclid". order: "centre" (tile lists
    by centre depth) or "stp" (StopThePop: per-tile hit depth, then per-pixel resorting
    in a buffer of RESORT entries). ray_noise_seed: perturb every pair's local ray by
    uniform relative noise of RAY_EPS per component, drawn from a generator seeded by
    (seed, tile, list position), and the quadratic's coefficients by as much of the
    magnitudes of their terms (see ray_sensitivity). timings: if a dict, receives the
    seconds spent on each rendered tile (forward and, with grad_images, backward)."""
    if binning is None:
        binning = bin_fp32(scene, cam, order="hit" if order == "stp" else "centre")
    comp = _composite_resort if order == "stp" else _composite
    want_grad = grad_images is not None
    c64 = CamF64(cam)
    H, W = cam.H, cam.W
    out = dict(rgb=np.zeros((3, H, W)), alpha=np.zeros((H, W)), depth=np.zeros((H, W)),
               normal=np.zeros((3, H, W)), margin=np.full((H, W), np.inf), cond=np.full((H, W), np.inf),
               n_eval=np.zeros((H, W), np.int64), n_contrib=np.zeros((H, W), np.int64),
               T_final=np.ones((H, W)), prim_cond=np.full(scene.n, np.inf))
    if extras:
        for k in ("curvature", "distortion", "median_depth", "curvature_scale"):
            out[k] = np.zeros((H, W))
        out["margin_median"] = np.full((H, W), np.inf)
    TX = binning.tiles_x
    if tiles is None:
        tiles = range(binning.tiles_x * binning.tiles_y)
    tiles = list(tiles)
    # the tiles' lists, and parameters only for the primitives they hold (local indices)
    lists = {}
    for tile in tiles:
        if binning.ranges is not None:
            s_, e_ = binning.ranges[tile]
            lists[tile] = np.asarray(binning.vals[s_:e_], np.int64)
        else:
            lists[tile] = np.asarray(tile_list(binning, tile), np.int64)
    used = np.unique(np.concatenate([np.zeros(0, np.int64)] + list(lists.values())))
    prm = Params(scene.subset(used), requires_grad=want_grad)
    g = None
    if want_grad:
        g = {k: torch.tensor(np.asarray(v, np.float64)) for k, v in grad_images.items()}
    import time as _time
    for tile in tiles:
        t_start = _time.perf_counter()
        lst = lists[tile]
        xs, ys = _tile_pixels(cam, tile, TX)
        if lst.size == 0:
            continue
        idx = torch.from_numpy(np.searchsorted(used, lst))
        px = torch.tensor(xs, dtype=F64)
        py = torch.tensor(ys, dtype=F64)
        noise = None
        if ray_noise_seed is not None:
            def noise(P_, L_, c0, _t=tile):
                gen = torch.Generator().manual_seed(int(ray_noise_seed) * 1_000_003 + _t * 4099 + c0)
                rn = (2.0 * torch.rand(P_, L_, 6, generator=gen, dtype=F64) - 1.0) * RAY_EPS
                cn = (2.0 * torch.rand(P_, L_, 3, generator=gen, dtype=F64) - 1.0) * RAY_EPS
                return rn, cn
        with torch.set_grad_enabled(want_grad):
            r = comp(prm, c64, idx, px, py, density=density, extras=extras, noise=noise)
            if want_grad:
                loss = torch.zeros((), dtype=F64)
                for k in ("rgb", "normal"):
                    if k in g:
                        loss = loss + (g[k][:, ys, xs].T * r[k]).sum()
                for k in ("alpha", "depth", "curvature", "distortion"):
                    if k in g:
                        if k not in r:
                            raise ValueError(f"grad_images[{k!r}] needs extras=True")
                        loss = loss + (g[k][ys, xs] * r[k]).sum()
                if loss.requires_grad:
                    loss.backward()
        if timings is not None:
            timings[int(tile)] = _time.perf_counter() - t_start
        out["rgb"][:, ys, xs] = r["rgb"].detach().numpy().T
        out["alpha"][ys, xs] = r["alpha"].detach().numpy()
        out["depth"][ys, xs] = r["depth"].detach().numpy()
        out["normal"][:, ys, xs] = r["normal"].detach().numpy().T
        out["margin"][ys, xs] = r["margin"].numpy()
        out["cond"][ys, xs] = r["cond"].numpy()
        np.minimum.at(out["prim_cond"], lst, r["list_cond"].numpy())
        out["n_eval"][ys, xs] = r["n_eval"].numpy()
        out["n_contrib"][ys, xs] = r["n_contrib"].numpy()
        out["T_final"][ys, xs] = r["T_final"].detach().numpy()
        if extras:
            for k in ("curvature", "distortion", "median_depth", "curvature_scale", "margin_median"):
                out[k][ys, xs] = r[k].detach().numpy()
    if want_grad:
        grads = {}
        for k, v in prm.leaves().items():
            gr = v.grad if v.grad is not None else torch.zeros_like(v)
            full = np.zeros((scene.n,) + tuple(v.shape[1:]))
            full[used] = gr.numpy()
            grads[k] = full
        grads["sh"] = grads["sh"].reshape(-1, 48)
        out["grads"] = grads
    out["binning"] = binning
    return out


def render_pixels(scene, cam, pixels, binning: Binning | None = None, density="geodesic", extras=False,
                  order="centre"):
    """Render individual pixels [(x, y), ...] one at a time (same lists and order as
    the full image). Returns dict of arrays indexed like `pixels`."""
    if binning is None:
        binning = bin_fp32(scene, cam, order="hit" if order == "stp" else "centre")
    c64 = CamF64(cam)
    TX = binning.tiles_x
    keys = ["rgb", "alpha", "depth", "normal", "margin", "cond", "n_eval", "n_contrib"]
    if extras:
        keys += ["curvature", "distortion", "median_depth", "curvature_scale", "margin_median"]
    res = {k: [] for k in keys}
    lists = {}
    for (x, y) in pixels:
        tile = (y // TILE) * TX + (x // TILE)
        if binning.ranges is not None:
            s, e = binning.ranges[tile]
            lst = binning.vals[s:e]
        else:
            if tile not in lists:
                lists[tile] = tile_list(binning, tile)
            lst = lists[tile]
        prm = Params(scene.subset(np.asarray(lst, np.int64)))
        idx = torch.arange(len(lst))
        with torch.no_grad():
            comp = _composite_resort if order == "stp" else _composite
            r = comp(prm, c64, idx, torch.tensor([float(x)], dtype=F64),
                     torch.tensor([float(y)], dtype=F64), density=density, extras=extras)
        for k in res:
            res[k].append(r[k][0].numpy())
    return {k: np.array(v) for k, v in res.items()}


def pair_count(binning: Binning, cam) -> int:
    """Number of (pixel, listed primitive) pairs before any early termination."""
    TX = binning.tiles_x
    tot = 0
    for tile in range(binning.tiles_x * binning.tiles_y):
        s, e = binning.ranges[tile]
        xs, _ = _tile_pixels(cam, tile, TX)
        tot += int(e - s) * xs.size
    return tot


# =========================================================================== bracketing
# Where an FP32 implementation and this FP64 oracle can take a discrete decision differently
# (a quantity within rounding distance of its threshold), both outcomes are correct
# renderings of the same inputs. bracket_pixels enumerates, per pixel, the outputs of every
# combination of such decisions (each taken both ways); a rendering matches the oracle at
# that pixel if it matches one of them. The same combinations bound the gradients: each
# pixel's gradient contribution lies between those of its branches.
BRACKET_MARGIN = 1e-5     # relative margin below which a decision is taken both ways
BRACKET_LEAVES = 512      # most branches enumerated per pixel (more: the pixel is unresolved)
GRAZE_MARGIN = 1e-2       # blended pairs whose discriminant margin is below this ...
GRAZE_SHIFT = 1e-6        # ... are also evaluated with D moved by this fraction of its scale
GRAZE_FULL = 20 * GRAZE_SHIFT  # below this margin a shifted pair is re-evaluated (above: graze_bands)
ORDER_GAP = 2.0 ** -20    # list-free order: neighbours whose centre depths are this close may swap
# An FP32 implementation forms each pair's local ray (where it crosses the centre's depth,
# and its direction) in a handful of rounded operations from rounded per-primitive state:
# about 8 units in the last place of each component, relative.
RAY_EPS = 8.0 * 2.0 ** -24
OUT_LEN = {"rgb": 3, "alpha": 1, "depth": 1, "normal": 3, "curvature": 1, "distortion": 1, "median_depth": 1}


def listfree_candidates(scene, cam, x: int, y: int):
    """Primitives that can have a hit on the ray of pixel (x, y), without tile lists or any
    FP32 recipe: every valid primitive whose centre lies in front of the near plane and whose
    centre is within 3 max(s_u, s_v) of the ray's line. A support point p has l <= 3 sigma
    (Sec. 3.2.1), the arc from the vertex is no shorter than its chord |p - mu|, and
    sigma(theta) <= max(s_u, s_v) (Sec. 3.2, sigma Eq.), so |p - mu| <= 3 max(s_u, s_v):
    a ray with a hit passes that close to the centre. Returned in (FP64 centre depth, index)
    order, the order of the tile lists' keys, with the depths."""
    mean = np.asarray(scene.mean, np.float64)
    R = np.asarray(cam.R_cw, np.float32).astype(np.float64)
    tc = np.asarray(cam.t_cw, np.float32).astype(np.float64)
    fx, fy, cx, cy = (float(np.float32(v)) for v in (cam.fx, cam.fy, cam.cx, cam.cy))
    c_w = -(R.T @ tc)
    d_cam = np.array([(x + 0.5 - cx) / fx, (y + 0.5 - cy) / fy, 1.0])
    d_w = R.T @ d_cam
    d_w = d_w / np.linalg.norm(d_w)
    z = mean @ R[2] + tc[2]
    rel = mean - c_w
    cr = np.cross(rel, d_w)
    dist2 = (cr * cr).sum(1)
    m = np.max(np.asarray(scene.scale, np.float64), 1)
    q = np.asarray(scene.quat, np.float64)
    ok = (np.isfinite(mean).all(1) & np.isfinite(q).all(1) & np.isfinite(scene.scale).all(1)
          & np.isfinite(scene.curv).all(1) & np.isfinite(scene.opacity) & ((q * q).sum(1) > 0)
          & (np.min(scene.scale, 1) > 0))
    near = float(np.float32(cam.near))
    sel = np.nonzero(ok & (z > near * (1.0 - BRACKET_MARGIN)) & (dist2 <= (3.0 * m) ** 2 * (1.0 + 1e-9)))[0]
    order = np.lexsort((sel, z[sel]))
    return sel[order].astype(np.int64), z[sel[order]]


def _order_outputs(pe, order, extras, margin=BRACKET_MARGIN):
    """Outputs of one branch: the pairs of list positions `order` blended in that order by
    the blending Eq. of Sec. 3.1 (w_k = alpha_k T_k), and the extra channels. The median
    depth's own decision (T_k > 0.5, Sec. 4.1) is bracketed as an interval: median_lo /
    median_hi leave out / take in the pairs whose T_k is within `margin` of 0.5."""
    idx = torch.tensor(order, dtype=torch.long)
    al = pe["alpha"][0, idx]
    t = pe["t"][0, idx]
    onem = 1.0 - al
    Tex = torch.cat([torch.ones(1, dtype=F64), torch.cumprod(onem, 0)[:-1]]) if len(order) else al
    w = al * Tex
    out = {"rgb": (w[:, None] * pe["rgb"][idx]).sum(0), "alpha": 1.0 - torch.prod(onem)[None],
           "depth": (w * t).sum()[None], "normal": (w[:, None] * pe["normal"][0, idx]).sum(0)}
    if extras:
        out["curvature"] = (w * pe["curvature"][0, idx]).sum()[None]
        out["curvature_scale"] = (w * pe["curvature"][0, idx].abs()).sum()[None].detach()
        out["distortion"] = _distortion(w[None], t[None]) if len(order) else torch.zeros(1, dtype=F64)
        zero = torch.zeros(1, dtype=F64)
        for nm, thr in (("median_depth", MEDIAN_T), ("median_lo", MEDIAN_T * (1.0 + margin)),
                        ("median_hi", MEDIAN_T * (1.0 - margin))):
            sel = Tex > thr
            out[nm] = (t[sel].max()[None] if bool(sel.any()) else zero).detach()
    return out


def _list_orders(pe, perm, margin, orig=None):
    """Blend orders of the list order `perm` (the base ordering: front to back in list
    order) for every place where the pixel may stop: the transmittance rule of Sec. 4.1
    (stop before a pair that would take T below 1e-4), taken both ways where T after the
    pair is within `margin` of the threshold. Returns [(order, n_contrib)], the nominal
    branch (every decision taken as computed) first; n_contrib counts positions of the
    original list `orig` (positions of the pairs kept, default the identity)."""
    al = pe["alpha"][0].detach().tolist()
    v = pe["valid"][0].tolist()
    res, order, T = [], [], 1.0
    nominal = None

    def leaf():
        if not order:
            return (list(order), 0)
        return (list(order), (max(orig[k] for k in order) if orig is not None else max(perm.index(k) for k in order)) + 1)

    for j in perm:
        if not v[j]:
            continue
        ta = T * (1.0 - al[j])
        if abs(ta - T_MIN) / T_MIN < margin:
            res.append(leaf())
            if ta < T_MIN and nominal is None:
                nominal = len(res) - 1
        elif ta < T_MIN:
            res.append(leaf())
            if nominal is None:
                nominal = len(res) - 1
            break
        order.append(j)
        T = ta
    else:
        res.append(leaf())
        if nominal is None:
            nominal = len(res) - 1
    return [res[nominal]] + res[:nominal] + res[nominal + 1:]


def _resort_orders(pe, buf, margin, max_branches):
    """Blend orders of StopThePop's per-pixel resorting (supplementary, "Details of Per-tile
    Sorting and Per-pixel Resorting", as in _composite_resort): contributing pairs enter a
    buffer of `buf`; when it is full the nearest hit is blended (ties: earlier in the list),
    the rest nearest first at the end; the transmittance stop applies when an entry is
    blended. Branches where the two nearest buffered depths are within the order margin
    (their relative gap times ORDER_GAP_SCALE below `margin`: either may come first) and
    where the stop rule is within `margin`. Returns [(order, n_blended)], the nominal branch
    first, or None when the branches exceed max_branches."""
    al = pe["alpha"][0].detach().tolist()
    v = pe["valid"][0].tolist()
    tt = pe["t"][0].detach().tolist()
    L = len(v)
    res = []   # (order, n_blended, nominal path?)
    stack = [(0, (), 1.0, (), True)]   # (next list position, buffer of (t, j), T, blended, nominal)
    while stack:
        if len(res) + len(stack) > max_branches:
            return None
        j, bufr, T, order, nom = stack.pop()
        while True:
            if j < L and len(bufr) < buf:
                if v[j]:
                    bufr = bufr + ((tt[j], j),)
                j += 1
                if len(bufr) < buf:
                    continue
            if not bufr:
                res.append((list(order), len(order), nom))
                break
            srt = sorted(bufr)
            cands = [(srt[0], True)]
            if len(srt) > 1 and abs(srt[1][0] - srt[0][0]) * ORDER_GAP_SCALE < margin * abs(srt[0][0]):
                cands.append((srt[1], False))
            outs = []   # ("stop" | "go", order, state, nominal)
            for c, c_nom in cands:
                rest = tuple(e for e in bufr if e != c)
                ta = T * (1.0 - al[c[1]])
                stop_nom = ta < T_MIN
                if abs(ta - T_MIN) / T_MIN < margin:
                    outs.append(("stop", order, None, nom and c_nom and stop_nom))
                    outs.append(("go", order + (c[1],), (rest, ta), nom and c_nom and not stop_nom))
                elif stop_nom:
                    outs.append(("stop", order, None, nom and c_nom))
                else:
                    outs.append(("go", order + (c[1],), (rest, ta), nom and c_nom))
            cont = None
            for kind, od, st, nn in outs:
                if kind == "stop":
                    res.append((list(od), len(od), nn))
                elif cont is None:
                    cont = (od, st, nn)
                else:
                    stack.append((j, st[0], st[1], od, nn))
            if cont is None:
                break
            order, (bufr, T), nom = cont
    k = next(i for i, r in enumerate(res) if r[2])
    res = [res[k]] + res[:k] + res[k + 1:]
    return [(od, nb) for od, nb, _ in res]


def bracket_pixels(scene, cam, pixels, binning: Binning | None = None, list_free: bool = False,
                   density: str = "geodesic", extras: bool = False, grad_images=None, order: str = "centre",
                   margin: float = BRACKET_MARGIN, max_leaves: int = BRACKET_LEAVES, graze: bool = True):
    """Outputs (and gradients) of pixels [(x, y), ...] on every branch of their near-threshold
    decisions. Per pixel, the list is its tile's list (binning, the per-tile sorting of the
    supplementary) or, with list_free, listfree_candidates. A decision is taken both ways
    when its relative margin is below `margin`: the pair decisions of _eval_pairs (real
    roots, the near plane for either root, 3 sigma for either root, alpha >= 1/255, and,
    with gradients, the 0.99 clamp, which changes only the derivative), the transmittance
    stop, the order of two neighbours whose centre depths are within ORDER_GAP of each
    other (list-free), and, with order="stp", which of the two nearest buffered hits is
    blended first (_resort_orders). With `graze`, each blended pair whose discriminant
    margin is below GRAZE_FULL is also evaluated with D moved by +-GRAZE_SHIFT of its
    scale: near a grazing ray the root's derivative goes like 1/sqrt(D), and an FP32
    implementation knows D only to about that much (graze_bands covers the margins from
    GRAZE_FULL to GRAZE_MARGIN to first order). These shifts are small and independent,
    so they are taken one pair at a time (their effects add to first order), on the
    nominal branch of the discrete decisions, which are taken in every combination.
    Returns one dict per pixel: "leaves" (list of output dicts of numpy arrays, the first
    the nominal branch), "groups" per leaf ("d" for a combination of discrete decisions,
    ("g", j) for list position j's shifted discriminant), "n_contrib" per leaf, "resolved"
    (False when the discrete combinations exceed max_leaves: only the nominal one is
    returned), "n_branch_decisions"; with grad_images (dict of upstream planes as in
    render) also "prims" (the list's primitive indices) and "grads" (per leaf, dict of
    gradient arrays [len(prims), ...] of sum(g * outputs) at this pixel)."""
    if order == "stp":
        if list_free:
            raise ValueError("the list-free mode uses the centre order")
        if binning is None or binning.order != "hit":
            binning = bin_fp32(scene, cam, order="hit") if binning is None else binning
    want_grad = grad_images is not None
    c64 = CamF64(cam)
    res = []
    names = DECISIONS if want_grad else tuple(n for n in DECISIONS if n != "amax")
    outkeys = OUT_KEYS + (EXTRA_KEYS + ("median_lo", "median_hi", "curvature_scale") if extras else ())
    g = None
    if want_grad:
        g = {k: torch.tensor(np.asarray(v, np.float64)) for k, v in grad_images.items()}
    for (x, y) in pixels:
        x, y = int(x), int(y)
        if list_free:
            lst, zc = listfree_candidates(scene, cam, x, y)
        else:
            tile = (y // TILE) * binning.tiles_x + (x // TILE)
            if binning.ranges is not None:
                s_, e_ = binning.ranges[tile]
                lst = binning.vals[s_:e_].astype(np.int64)
            else:
                lst = tile_list(binning, tile).astype(np.int64)
            zc = None
        L = int(lst.size)
        item = {"x": x, "y": y, "leaves": [], "groups": [], "n_contrib": [], "resolved": True,
                "n_branch_decisions": 0}
        if want_grad:
            item["prims"] = lst
            item["grads"] = []
        if L == 0:
            item["leaves"].append({k: np.zeros(OUT_LEN.get(k, 1)) for k in outkeys})
            item["groups"].append("d")
            item["n_contrib"].append(0)
            if want_grad:
                item["grads"].append(None)
            res.append(item)
            continue
        px = torch.tensor([float(x)], dtype=F64)
        py = torch.tensor([float(y)], dtype=F64)
        with torch.no_grad():
            pe0 = _eval_pairs(Params(scene.subset(lst)), c64, torch.arange(L), px, py, density)
        # per pair: the decisions within the margin; where a decision can flip, the pair may
        # contribute (or not) on some branch
        per_pair = {}
        for nm in names:
            for j in torch.nonzero(pe0["margins"][nm][0] < margin).flatten().tolist():
                per_pair.setdefault(j, []).append(nm)
        maybe = pe0["valid"][0].clone()
        for j in per_pair:
            maybe[j] = True
        # A pair with no hit and no decision near its threshold contributes nothing on any
        # branch (its own decisions alone decide whether it contributes): keep the others.
        keep = torch.nonzero(maybe).flatten()
        if list_free:
            near = float(np.float32(cam.near))
            keep = torch.unique(torch.cat([keep, torch.from_numpy(np.nonzero(np.abs(zc - near) / near < margin)[0])]))
        remap = {int(j): q for q, j in enumerate(keep.tolist())}
        orig_pos = keep.tolist()
        per_pair = {remap[j]: v for j, v in per_pair.items()}
        lst = lst[keep.numpy()]
        if zc is not None:
            zc = zc[keep.numpy()]
        L = int(lst.size)
        if want_grad:
            item["prims"] = lst
        pe0 = {k: (v[:, keep] if torch.is_tensor(v) and v.dim() == 2 else v) for k, v in pe0.items() if k not in
               ("margins", "rgb", "normal", "roots", "pick_near")}
        maybe = maybe[keep]
        if L == 0:
            item["leaves"].append({k: np.zeros(OUT_LEN.get(k, 1)) for k in outkeys})
            item["groups"].append("d")
            item["n_contrib"].append(0)
            if want_grad:
                item["grads"].append(None)
            res.append(item)
            continue
        prm = Params(scene.subset(lst), requires_grad=want_grad)
        idx = torch.arange(L)
        if list_free:  # a centre at the near plane may be culled or not
            near = float(np.float32(cam.near))
            for j in np.nonzero(np.abs(zc - near) / near < margin)[0].tolist():
                per_pair.setdefault(j, []).append("cull")
            keep_c = torch.from_numpy(zc > near)
        choices = []   # (kind, payload) binary (ternary for graze) choices
        for j, nms in sorted(per_pair.items()):
            for nm in nms:
                choices.append(("flip", (j, nm)))
        grazing = torch.nonzero(pe0["cond"][0] < GRAZE_FULL).flatten().tolist() if graze else []
        if list_free:
            cj = torch.nonzero(maybe).flatten().tolist()
            for a_, b_ in zip(cj[:-1], cj[1:]):
                if abs(zc[b_] - zc[a_]) <= ORDER_GAP * abs(zc[a_]):
                    choices.append(("swap", (a_, b_)))
        item["n_branch_decisions"] = len(choices) + len(grazing)
        if 2 ** len(choices) > max_leaves:
            item["resolved"] = False
            choices = []
        combos = [[]]
        for kind, pl in choices:
            combos = [c + [(kind, pl, o)] for c in combos for o in (False, True)]
        runs = [("d", c) for c in combos]
        runs += [(("g", j), [("graze", j, sg)]) for j in grazing for sg in (-1.0, 1.0)]
        for group, combo in runs:
            flip = {}
            shift = None
            perm = list(range(L))
            culled = []
            for kind, pl, o in combo:
                if kind == "flip" and o:
                    j, nm = pl
                    if nm == "cull":
                        culled.append(j)
                        continue
                    flip.setdefault(nm, torch.zeros(1, L, dtype=torch.bool))[0, j] = True
                elif kind == "graze" and o is not None:
                    if shift is None:
                        shift = torch.zeros(1, L, dtype=F64)
                    shift[0, pl] = o * GRAZE_SHIFT
                elif kind == "swap" and o:
                    a_, b_ = pl
                    ia, ib = perm.index(a_), perm.index(b_)
                    perm[ia], perm[ib] = perm[ib], perm[ia]
            with torch.set_grad_enabled(want_grad):
                pe = _eval_pairs(prm, c64, idx, px, py, density, flip=flip, d_shift=shift)
                if list_free:
                    kc = keep_c.clone()
                    for j in culled:
                        kc[j] = ~kc[j]
                    pe["valid"] = pe["valid"] & kc[None]
                    pe["alpha"] = torch.where(pe["valid"], pe["alpha"], torch.zeros_like(pe["alpha"]))
                if order == "stp":
                    branches = _resort_orders(pe, RESORT, margin, max_leaves)
                    if branches is None:
                        item["resolved"] = False
                        branches = _resort_orders(pe, RESORT, 0.0, 1)
                else:
                    branches = _list_orders(pe, perm, margin, orig_pos)
                if group != "d":
                    branches = branches[:1]
                for od, nc in branches:
                    out = _order_outputs(pe, od, extras, margin)
                    item["leaves"].append({k: v.detach().numpy().copy() for k, v in out.items()})
                    item["groups"].append(group)
                    item["n_contrib"].append(nc)
                    if want_grad:
                        loss = torch.zeros((), dtype=F64)
                        for k in ("rgb", "normal"):
                            if k in g:
                                loss = loss + (g[k][:, y, x] * out[k]).sum()
                        for k in ("alpha", "depth", "curvature", "distortion"):
                            if k in g and k in out:
                                loss = loss + g[k][y, x] * out[k][0]
                        leaves_t = prm.leaves()
                        if loss.requires_grad:
                            gr = torch.autograd.grad(loss, list(leaves_t.values()), retain_graph=True,
                                                     allow_unused=True)
                        else:
                            gr = [None] * len(leaves_t)
                        gd = {}
                        for (k, v), gk in zip(leaves_t.items(), gr):
                            gd[k] = (gk if gk is not None else torch.zeros_like(v)).detach().numpy().copy()
                        gd["sh"] = gd["sh"].reshape(-1, 48)
                        item["grads"].append(gd)
        res.append(item)
    return res


def pixel_vector(out: dict, keys) -> np.ndarray:
    """Concatenated outputs of one pixel (rgb 3, alpha, depth, normal 3, then `keys` extras)."""
    return np.concatenate([np.asarray(out[k], np.float64).reshape(-1) for k in OUT_KEYS + tuple(keys)])



def graze_bands(scene, cam, binning: Binning, tiles, grad_images, density: str = "geodesic", extras: bool = False,
                order: str = "centre", lo: float = GRAZE_FULL, hi: float = GRAZE_MARGIN,
                shift: float = GRAZE_SHIFT):
    """First-order bounds on how far each primitive's gradient moves when the discriminant of
    each of its blended grazing pairs (margin in [lo, hi)) is moved by `shift` of its
    rounding scale. Near a grazing ray the derivative of the root t with respect to the
    primitive's parameters goes like 1/sqrt(D) (at a root, df/dt = +-sqrt(D)), so moving D by
    e scales that derivative by about 1 -+ e / (2 D); the part of a pixel's gradient that
    flows through the root, (dL_p/dt) (dt/dtheta), moves by as much. Per element, the band
    sums |shift / (2 margin)| |dL_p/dt| |dt/dtheta| over the primitive's grazing pairs (one
    pixel's error may have either sign). dL_p/dt comes from one backward pass per tile with
    the roots as leaves; dt/dtheta from the single pair. Returns {parameter: (primitive
    indices, band array)} over the primitives that have such pairs in `tiles`."""
    comp = _composite_resort if order == "stp" else _composite
    c64 = CamF64(cam)
    g = {k: torch.tensor(np.asarray(v, np.float64)) for k, v in grad_images.items()}
    pairs = []   # (primitive, x, y, kappa * |dL/dt|)
    for tile in tiles:
        lst = tile_list(binning, tile) if binning.ranges is None else binning.vals[slice(*binning.ranges[tile])]
        if len(lst) == 0:
            continue
        lst = np.asarray(lst, np.int64)
        prm_nograd = Params(scene.subset(lst))
        xs, ys = _tile_pixels(cam, tile, binning.tiles_x)
        idx = torch.arange(lst.size)
        px = torch.tensor(xs, dtype=F64)
        py = torch.tensor(ys, dtype=F64)
        collect = []
        r = comp(prm_nograd, c64, idx, px, py, density=density, extras=extras, collect=collect)
        loss = torch.zeros((), dtype=F64)
        for k in ("rgb", "normal"):
            if k in g:
                loss = loss + (g[k][:, ys, xs].T * r[k]).sum()
        for k in ("alpha", "depth", "curvature", "distortion"):
            if k in g and k in r:
                loss = loss + (g[k][ys, xs] * r[k]).sum()
        leaves = [t for _, pe in collect for t in pe["roots"]]
        if not loss.requires_grad:
            continue
        grads = torch.autograd.grad(loss, leaves, allow_unused=True)
        for q, (c0, pe) in enumerate(collect):
            g1, g2 = grads[2 * q], grads[2 * q + 1]
            g1 = torch.zeros_like(pe["roots"][0]) if g1 is None else g1
            g2 = torch.zeros_like(pe["roots"][1]) if g2 is None else g2
            dLdt = torch.where(pe["pick_near"], g1, g2)
            cond = pe["cond"]
            sel = (cond >= lo) & (cond < hi) & pe["valid"]
            for pi, jj in torch.nonzero(sel).tolist():
                kap = shift / (2.0 * float(cond[pi, jj]))
                pairs.append((int(lst[c0 + jj]), int(xs[pi]), int(ys[pi]), kap * abs(float(dLdt[pi, jj]))))
    bands = {}
    by_prim = {}
    for i, x, y, c in pairs:
        by_prim.setdefault(i, []).append((x, y, c))
    for i, lst in by_prim.items():
        prm = Params(scene.subset(np.array([i])), requires_grad=True)
        px = torch.tensor([float(x) for x, _, _ in lst], dtype=F64)
        py = torch.tensor([float(y) for _, y, _ in lst], dtype=F64)
        pe = _eval_pairs(prm, c64, torch.tensor([0]), px, py, density)
        acc = None
        for r_, (_, _, c) in enumerate(lst):
            gr = torch.autograd.grad(pe["t"][r_, 0], list(prm.leaves().values()), retain_graph=True, allow_unused=True)
            vec = {k: (v if v is not None else torch.zeros_like(l)).detach().numpy()[0] * c
                   for (k, l), v in zip(prm.leaves().items(), gr)}
            vec = {k: np.abs(v) for k, v in vec.items()}
            acc = vec if acc is None else {k: acc[k] + vec[k] for k in acc}
        bands[i] = acc
    out = {}
    prims = np.array(sorted(bands), np.int64)
    for k in ("mean", "quat", "scale", "curv", "opacity", "sh"):
        if prims.size:
            arr = np.stack([bands[i][k] for i in prims])
            out[k] = (prims, arr.reshape(prims.size, -1) if k == "sh" else arr)
        else:
            out[k] = (prims, None)
    return out


def ray_sensitivity(scene, cam, binning: Binning, tiles, grad_images, ref_grads, samples: int = 3,
                    density: str = "geodesic", extras: bool = False, order: str = "centre"):
    """How far the exact gradients move under the rounding an FP32 implementation incurs in
    forming each pair's local ray and its quadratic: the largest change, over `samples`
    renders whose every (pixel, primitive) pair has its local ray perturbed by independent
    uniform relative noise of RAY_EPS per component (origin and direction) and each
    coefficient of its quadratic (re-based at the centre's depth) by as much of the
    magnitudes of its terms. Near tangency
    (the ray meeting a steep flank of a strongly curved patch, a grazing pair moving a
    thin primitive's hit) and where the pixels' contributions to a parameter cancel, the
    exact gradient itself is defined by FP32 inputs only to this much.
    Returns {parameter: array like ref_grads}."""
    spread = {k: np.zeros_like(v) for k, v in ref_grads.items()}
    for smp in range(samples):
        r = render(scene, cam, binning, tiles=tiles, grad_images=grad_images, density=density, extras=extras,
                   order=order, ray_noise_seed=smp + 1)
        for k in spread:
            spread[k] = np.maximum(spread[k], np.abs(r["grads"][k] - ref_grads[k]))
    return spread


def ray_sensitivity_images(scene, cam, binning: Binning, tiles, ref, samples: int = 3, density: str = "geodesic",
                           extras: bool = False, order: str = "centre"):
    """The forward counterpart of ray_sensitivity: the largest change of each output plane,
    per pixel, over `samples` renders of `tiles` whose every pair's local ray is perturbed
    by FP32-sized rounding (RAY_EPS per component). Near a grazing ray the hit point, its
    depth and its normal move by about e / sqrt(D) under a rounding e of D. Returns a dict
    of planes like ref's."""
    keys = OUT_KEYS + (("curvature", "distortion") if extras else ())
    spread = {k: np.zeros_like(ref[k]) for k in keys}
    for smp in range(samples):
        r = render(scene, cam, binning, tiles=tiles, density=density, extras=extras, order=order,
                   ray_noise_seed=smp + 101)
        for k in keys:
            spread[k] = np.maximum(spread[k], np.abs(r[k] - ref[k]))
    return spread
