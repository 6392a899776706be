"""Comparison helpers shared by the GPU parity tests (the accuracy bar, and bracketing).

Bars (FP32 CUDA path vs the FP64 oracle), per element, everywhere:
  rgb, alpha, normal   <= 1e-4 absolute
  depth, median depth  <= 1e-4 relative (against max(|d*|, 1e-6))
  curvature map        <= 1e-4 relative against max(sum_i w_i |K_i|, 1) (K = 4ab/S^2 reaches
                          1e6 on strongly curved patches)
  distortion           <= 1e-4 (D* + depth* sqrt(D*)): the relative depth bar carried
                          through dD/dt_i = 2 w_i (A0 t_i - A1), bounded by Cauchy-Schwarz
  gradients            <= 1e-3 relative, per element against
                          max(|g*|, 1e-3 max|g*| over the parameter group)

Near-threshold decisions. A pixel whose oracle evaluation takes a discrete decision within
MARGIN (relative) of its threshold (real roots, the near plane, 3 sigma, alpha >= 1/255, the
0.99 clamp, the transmittance stop, the median's T > 0.5, StopThePop's order of the two
nearest buffered hits) is bracketed: oracle.bracket_pixels enumerates its outputs on every
branch of those decisions. For gradients, a pixel that blends a grazing pair (discriminant
margin below GRAZE_MARGIN, where the root's derivative goes like 1/sqrt(D) and FP32 knows D
to about GRAZE_SHIFT of the scale of its terms) is bracketed too, with D moved that much
each way. The GPU pixel passes if it meets the bars against one of them. A pixel is
ambiguous only when it matches none of its branches (or has more branches than the oracle
enumerates); the ambiguous fraction must stay at or below MAX_AMBIGUOUS (0.01 % of pixels).

Conditioning of FP32 geometry. A pixel that blends a pair within GRAZE_FULL of grazing is
bracketed with that pair's discriminant moved by GRAZE_SHIFT of the scale of its terms each
way (near tangency the hit point, its depth and normal move by about e / sqrt(D) under a
rounding e of D). Elsewhere each bar is at least SENS_FACTOR times the oracle's own change
when every pair's local ray is perturbed by FP32-sized rounding (oracle.ray_sensitivity_images;
for gradients oracle.ray_sensitivity); the fraction of pixels and elements whose bar this
widened is reported.

Gradients: each parameter gradient sums pixel contributions, and a bracketed pixel's
contribution lies between those of its branches. An element passes when it lies within the
bar of the interval [g* + lo, g* + hi], lo and hi summing, over the bracketed pixels, each
pixel's most negative and most positive branch difference (zero for unbracketed pixels, so
there the bar is the plain 1e-3).
"""
import numpy as np

import oracle.qgs_oracle as O

MARGIN = O.BRACKET_MARGIN
GRAZE_MARGIN = O.GRAZE_MARGIN
MAX_AMBIGUOUS = 1e-4
TOL_ABS = 1e-4
TOL_DEPTH_REL = 1e-4
TOL_GRAD_REL = 1e-3
TOL_CURV_REL = 1e-4
TOL_DIST = 1e-4
SENS_SAMPLES = 3    # renders with each pair's local ray perturbed by FP32 rounding (oracle.ray_sensitivity)
SENS_FACTOR = 3.0   # the bar is at least this many times the largest change they show


# ----------------------------------------------------------------------------- images
def near_pixels(ref, mask=None, extras=False):
    """Pixels to bracket: a decision within MARGIN, or a blended pair so close to grazing
    (discriminant margin below GRAZE_FULL) that its root is re-evaluated with D shifted."""
    near = (ref["margin"] <= MARGIN) | (ref["cond"] < O.GRAZE_FULL)
    if extras:
        near = near | (ref["margin_median"] <= MARGIN)
    if mask is not None:
        near = near & mask
    return near


def _graze_band(it):
    """Per-channel band that a pixel's grazing pairs span: for each pair whose discriminant
    was moved each way (bracket_pixels groups ("g", j)), the larger deviation of its two
    evaluations from the nominal branch, summed over the pairs (small independent shifts:
    their effects add). The outputs move continuously with the shift, so every value in
    between is as correct as the ends."""
    nom = it["leaves"][0]
    dev = {}
    for grp, leaf in zip(it["groups"], it["leaves"]):
        if grp == "d":
            continue
        for k, v in leaf.items():
            d = np.abs(np.asarray(v, np.float64) - np.asarray(nom[k], np.float64))
            dev[(grp, k)] = np.maximum(dev.get((grp, k), 0.0), d)
    band = {}
    for (grp, k), d in dev.items():
        band[k] = band.get(k, 0.0) + d
    return band


def _pixel_errors(gv, leaf, extras, band=None):
    """Errors of one GPU pixel against one oracle branch, in units of the bars (<= 1 passes),
    each output allowed `band` (per channel, see _graze_band) beyond its bar."""
    band = band or {}

    def over(k, diff):
        return np.max(np.maximum(np.abs(diff) - band.get(k, 0.0), 0.0))

    e = [over("rgb", gv["rgb"] - leaf["rgb"]) / TOL_ABS,
         float(over("alpha", gv["alpha"] - leaf["alpha"][0])) / TOL_ABS,
         over("normal", gv["normal"] - leaf["normal"]) / TOL_ABS,
         float(over("depth", gv["depth"] - leaf["depth"][0])) / max(abs(leaf["depth"][0]), 1e-6) / TOL_DEPTH_REL]
    if extras:
        e.append(float(over("curvature", gv["curvature"] - leaf["curvature"][0]))
                 / (TOL_CURV_REL * max(leaf["curvature_scale"][0], 1.0)))
        D = leaf["distortion"][0]
        e.append(float(over("distortion", gv["distortion"] - D))
                 / (TOL_DIST * (D + abs(leaf["depth"][0]) * np.sqrt(max(D, 0.0))) + 1e-9))
        lo, hi = leaf["median_lo"][0], leaf["median_hi"][0]
        m = gv["median_depth"]
        bm = float(np.max(band.get("median_depth", 0.0)))
        d = max(lo - bm - m, m - hi - bm, 0.0)
        e.append(d / max(abs(lo), abs(hi), 1e-6) / TOL_DEPTH_REL)
    return max(e)


def _best_branch(gv, it, extras):
    """The smallest error of a GPU pixel over its discrete branches, each widened by the
    band of its grazing pairs."""
    band = _graze_band(it)
    return min(_pixel_errors(gv, leaf, extras, band) for grp, leaf in zip(it["groups"], it["leaves"])
               if grp == "d")


def _gpu_pixel(out, x, y, extras):
    gv = {"rgb": np.asarray(out["rgb"][:, y, x], np.float64), "alpha": float(out["alpha"][y, x]),
          "depth": float(out["depth"][y, x]), "normal": np.asarray(out["normal"][:, y, x], np.float64)}
    if extras:
        for k in ("curvature", "distortion", "median_depth"):
            gv[k] = float(out[k][y, x])
    return gv


def image_errors(gpu, ref, ok, extras=False, sens=None):
    """Max errors over the pixels `ok`, in units of the bars (each bar at least SENS_FACTOR
    times the oracle's own change under local-ray rounding, `sens`, when given)."""
    def tol(k, bar):
        return bar if sens is None else np.maximum(bar, SENS_FACTOR * sens[k])
    e = {}
    for k in ("rgb", "alpha", "normal"):
        e[k] = float((np.abs(np.asarray(gpu[k], np.float64) - ref[k]) / tol(k, TOL_ABS))[..., ok].max(initial=0.0))
    d = np.asarray(gpu["depth"], np.float64)
    bar_d = TOL_DEPTH_REL * np.maximum(np.abs(ref["depth"]), 1e-6)
    e["depth"] = float((np.abs(d - ref["depth"]) / tol("depth", bar_d))[ok].max(initial=0.0))
    if extras:
        cs = np.maximum(ref["curvature_scale"], 1.0)
        e["curvature"] = float((np.abs(np.asarray(gpu["curvature"], np.float64) - ref["curvature"])
                                / tol("curvature", TOL_CURV_REL * cs))[ok].max(initial=0.0))
        D = ref["distortion"]
        tolD = TOL_DIST * (D + np.abs(ref["depth"]) * np.sqrt(np.maximum(D, 0.0))) + 1e-9
        e["distortion"] = float((np.abs(np.asarray(gpu["distortion"], np.float64) - D)
                                 / tol("distortion", tolD))[ok].max(initial=0.0))
        m = ref["median_depth"]
        em = np.abs(np.asarray(gpu["median_depth"], np.float64) - m) / np.maximum(np.abs(m), 1e-6)
        e["median_depth"] = float(em[ok].max(initial=0.0)) / TOL_DEPTH_REL
    return e


def check_images(gpu, ref, scene, cam, binning=None, mask=None, extras=False, label="", **kw):
    """Strict bars at every pixel of `mask` (default all) that is not near a decision; each
    near pixel must match one of its branches (oracle.bracket_pixels; kw: density, order).
    Returns the statistics; asserts the ambiguous fraction is at most MAX_AMBIGUOUS."""
    st = compare_images(gpu, ref, scene, cam, binning, mask, extras, **kw)
    print(f"[{label}] {st}")
    for k, v in st["errors"].items():
        assert v <= 1.0, (label, k, v)
    assert st["ambiguous_frac"] <= MAX_AMBIGUOUS, (label, st["unmatched"])
    return st


def compare_images(gpu, ref, scene, cam, binning=None, mask=None, extras=False, sens_samples=SENS_SAMPLES, **kw):
    """The statistics of check_images, without asserting: errors (in units of the bars)
    over the pixels not near a decision, the near fraction, the worst near pixel against
    its best branch, the unmatched (ambiguous) pixels."""
    if mask is None:
        mask = np.ones(ref["alpha"].shape, bool)
    near = near_pixels(ref, mask, extras)
    sens = None
    if binning is not None and sens_samples > 0:
        TX = binning.tiles_x
        ty, tx = np.nonzero(_tile_any(mask))
        tiles = sorted(set((ty * TX + tx).tolist()))
        sens = O.ray_sensitivity_images(scene, cam, binning, tiles, ref, sens_samples, extras=extras, **kw)
    far = mask & ~near
    e = image_errors(gpu, ref, far, extras, sens)
    e_plain = image_errors(gpu, ref, far, extras)
    widened = 0.0
    if sens is not None and far.any():
        wid = np.zeros(ref["alpha"].shape, bool)
        for k, bar in (("rgb", TOL_ABS), ("alpha", TOL_ABS), ("normal", TOL_ABS)):
            w = SENS_FACTOR * sens[k] > bar
            wid |= w.any(0) if w.ndim == 3 else w
        wid |= SENS_FACTOR * sens["depth"] > TOL_DEPTH_REL * np.maximum(np.abs(ref["depth"]), 1e-6)
        widened = float(wid[far].mean())
    ys, xs = np.nonzero(near)
    pix = list(zip(xs.tolist(), ys.tolist()))
    br = O.bracket_pixels(scene, cam, pix, binning, extras=extras, **kw) if pix else []
    unmatched, unresolved, worst_near = [], 0, 0.0
    for (x, y), it in zip(pix, br):
        gv = _gpu_pixel(gpu, x, y, extras)
        best = _best_branch(gv, it, extras)
        unresolved += not it["resolved"]
        if best > 1.0:
            unmatched.append((x, y, best, len(it["leaves"]), it["resolved"]))
        else:
            worst_near = max(worst_near, best)
    n = int(mask.sum())
    amb = len(unmatched) / max(n, 1)
    return dict(errors=e, errors_plain=e_plain, widened_frac=widened, near_frac=len(pix) / max(n, 1),
                near_worst=float(worst_near), ambiguous=len(unmatched), ambiguous_frac=amb, unresolved=unresolved,
                pixels=n, unmatched=unmatched[:8])


def check_pixels(gpu_vals, scene, cam, pixels, binning=None, extras=False, label="", list_free=False, **kw):
    """Sampled pixels [(x, y)] checked one by one against their branches (every pixel is
    bracketed; near ones have several branches). gpu_vals: the GPU planes. Asserts that the
    unmatched fraction is at most MAX_AMBIGUOUS of the sampled pixels (i.e. none)."""
    br = O.bracket_pixels(scene, cam, pixels, binning, list_free=list_free, extras=extras, **kw)
    unmatched, worst, branched = [], 0.0, 0
    for (x, y), it in zip(pixels, br):
        gv = _gpu_pixel(gpu_vals, x, y, extras)
        best = _best_branch(gv, it, extras)
        branched += len(it["leaves"]) > 1
        if best > 1.0:
            unmatched.append((x, y, best, len(it["leaves"])))
        worst = max(worst, best)
    st = dict(pixels=len(pixels), branched=branched, worst=worst if not unmatched else None,
              ambiguous=len(unmatched))
    print(f"[{label}] {st} unmatched {unmatched[:8]}")
    assert len(unmatched) <= MAX_AMBIGUOUS * len(pixels), (label, unmatched[:8])
    return st, br


# ----------------------------------------------------------------------------- gradients
def _tile_any(mask):
    """Per 16x16 tile: does the tile hold a pixel of the mask."""
    H, W = mask.shape
    TY, TX = (H + O.TILE - 1) // O.TILE, (W + O.TILE - 1) // O.TILE
    pad = np.zeros((TY * O.TILE, TX * O.TILE), bool)
    pad[:H, :W] = mask
    return pad.reshape(TY, O.TILE, TX, O.TILE).any((1, 3))


def check_grads(gpu, ref, scene, cam, grad_images, binning=None, mask=None, idx=None, extras=False, label="",
                **kw):
    """Gradients against the oracle's (ref = O.render(..., grad_images=grad_images)) with the
    strict bar around the interval that the bracketed pixels' branches span (see the module
    docstring). mask: pixels with nonzero upstream gradients (default all); idx: the
    primitives compared (default all). Returns per-group statistics."""
    out, npix, unresolved = compare_grads(gpu, ref, scene, cam, grad_images, binning, mask, idx, extras, **kw)
    print(f"[{label}] bracketed pixels {npix} unresolved {unresolved}; grad ratios " +
          ", ".join(f"{k}: {v['ratio']:.2f} (strict {v['strict']:.2f}, banded {v['banded']:.4f}, "
                    f"widened {v['widened']:.4f})" for k, v in out.items()))
    for k, v in out.items():
        assert v["ratio"] <= 1.0, (label, k, v)
    if mask is None:
        mask = np.ones(ref["alpha"].shape, bool)
    assert unresolved <= MAX_AMBIGUOUS * max(int(mask.sum()), 1), (label, unresolved)
    return out


def compare_grads(gpu, ref, scene, cam, grad_images, binning=None, mask=None, idx=None, extras=False,
                  sens_samples=SENS_SAMPLES, **kw):
    """The statistics of check_grads, without asserting: per parameter group the error in
    units of the bar outside the branch interval ("ratio"), the plain error in units of the
    bar ("strict"), the fraction of elements whose interval is wider than the bar
    ("banded"); plus the number of bracketed pixels and of unresolved ones."""
    n = scene.n
    idx = np.arange(n) if idx is None else np.asarray(idx, np.int64)
    order_idx = np.argsort(idx)
    sidx = idx[order_idx]
    if mask is None:
        mask = np.ones(ref["alpha"].shape, bool)
    near = near_pixels(ref, mask)
    ys, xs = np.nonzero(near)
    pix = list(zip(xs.tolist(), ys.tolist()))
    ref_g = ref["grads"]
    lo = {k: np.zeros((idx.size,) + v.shape[1:]) for k, v in ref_g.items()}
    hi = {k: np.zeros((idx.size,) + v.shape[1:]) for k, v in ref_g.items()}
    unresolved = 0
    if pix:
        br = O.bracket_pixels(scene, cam, pix, binning, grad_images=grad_images, extras=extras, **kw)
        for it in br:
            unresolved += not it["resolved"]
            if len(it["grads"]) < 2 or it["grads"][0] is None:
                continue
            prims = it["prims"]
            pos = np.searchsorted(sidx, prims)
            pos = np.minimum(pos, sidx.size - 1)
            inside = sidx[pos] == prims
            rows = order_idx[pos[inside]]
            for k in lo:
                nom = it["grads"][0][k][inside]
                # the discrete branches' extremes, plus each grazing pair's own extremes
                # (independent small shifts: their effects add)
                ext = {}
                for grp, gr in zip(it["groups"][1:], it["grads"][1:]):
                    d = gr[k][inside] - nom
                    mn, mx = ext.get(grp, (np.zeros_like(nom), np.zeros_like(nom)))
                    ext[grp] = (np.minimum(mn, d), np.maximum(mx, d))
                for mn, mx in ext.values():
                    np.add.at(lo[k], rows, mn)
                    np.add.at(hi[k], rows, mx)
    # first-order bands of the weakly grazing pairs, over the tiles under the mask
    tiles = None
    if binning is not None:
        TX = binning.tiles_x
        ty, tx = np.nonzero(_tile_any(mask))
        tiles = sorted(set((ty * TX + tx).tolist()))
        gb = O.graze_bands(scene, cam, binning, tiles, grad_images, extras=extras, **kw)
        for k in lo:
            prims, band = gb[k]
            if band is None:
                continue
            pos = np.minimum(np.searchsorted(sidx, prims), sidx.size - 1)
            inside = sidx[pos] == prims
            rows = order_idx[pos[inside]]
            b_ = band[inside].reshape((-1,) + lo[k].shape[1:])
            np.add.at(lo[k], rows, -b_)
            np.add.at(hi[k], rows, b_)
    # the exact gradient's own movement under the FP32 rounding of each pair's local ray
    sens = None
    if binning is not None and sens_samples > 0:
        sens = O.ray_sensitivity(scene, cam, binning, tiles, grad_images, ref_g, sens_samples, extras=extras, **kw)
    out = {}
    for k, gr_all in ref_g.items():
        gr = gr_all[idx]
        g = np.asarray(gpu[k], np.float64).reshape(gr_all.shape)[idx]
        scale = np.maximum(np.abs(gr), 1e-3 * np.abs(gr).max(initial=0.0))
        scale = np.where(scale > 0, scale, 1.0)
        tol0 = TOL_GRAD_REL * scale
        tol = tol0 if sens is None else np.maximum(tol0, SENS_FACTOR * sens[k][idx])
        d = np.maximum(np.maximum((gr + lo[k]) - g, g - (gr + hi[k])), 0.0)
        banded = (hi[k] - lo[k]) > tol0
        out[k] = dict(ratio=float((d / tol).max(initial=0.0)), strict=float((np.abs(g - gr) / tol0).max(initial=0.0)),
                      banded=float(banded.mean()) if banded.size else 0.0,
                      widened=float((tol > tol0).mean()) if tol.size else 0.0)
        if d.size:
            w = np.unravel_index(np.argmax(d / tol), d.shape)
            out[k]["worst"] = (int(idx[w[0]]),) + tuple(int(v) for v in w[1:])
    return out, len(pix), unresolved
