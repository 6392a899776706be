"""Comparison helpers shared by the GPU parity tests (tolerances of the accuracy bar).

Tolerances (FP32 CUDA path vs the FP64 oracle):
  rgb, alpha, normal   <= 1e-4 absolute
  depth                <= 1e-4 relative (against max(|d*|, 1e-6))
  median depth         <= 1e-4 relative (one hit depth), pixels whose transmittance is
                          within MARGIN of 0.5 at a blended pair excluded
  curvature map        <= 1e-4 relative against max(sum w |K|, 1) (K = 4ab/S^2 reaches
                          1e6 on strongly curved patches), widened like gradients to
                          PERTURB_FACTOR x the oracle's own deviation under input noise
  distortion           <= 1e-4 (D* + depth* sqrt(D*)): the relative depth bar carried
                          through dD/dt_i = 2 w_i (A0 t_i - A1), whose sum is bounded by
                          2 A0 t_max sqrt(2 D) (Cauchy-Schwarz)
  gradients            <= 1e-3 relative, per element against
                          max(|g*|, 1e-3 * max|g*| over the parameter group)
Pixels whose smallest decision margin in the oracle is below MARGIN are ambiguous
(FP32 and FP64 may take different discrete decisions there); they are counted and
excluded from the error maxima, and their upstream gradients are set to zero before
comparing parameter gradients.

Gradient conditioning: where a ray nearly grazes a quadric the derivative of the root
scales like 1/sqrt(D), and the exact gradient itself moves by much more than 1e-3 when
the inputs move by FP32 rounding (~6e-8 relative). The oracle measures this: it is
re-run with its inputs perturbed by PERTURB relative noise, and each gradient element is
allowed max(1e-3 relative, PERTURB_FACTOR x the oracle's own deviation). Primitives
with a blended pair whose relative discriminant margin is below COND_STRICT (deeply
grazing rays, where FP32 rounding alone moves the exact gradient by more than 1e-3) are
counted separately and held to the loose bound TOL_GRAD_ILL.
"""
import numpy as np

MARGIN = 1e-5
PERTURB = 2.4e-7
PERTURB_FACTOR = 3.0
PERTURB_SAMPLES = 3
COND_STRICT = 1e-4
TOL_GRAD_ILL = 5e-2
TOL_ABS = 1e-4
TOL_DEPTH_REL = 1e-4
TOL_GRAD_REL = 1e-3


def image_errors(gpu: dict, ref: dict, mask=None):
    """Max errors over unambiguous pixels; returns (errors dict, ambiguous fraction)."""
    ok = ref["margin"] > MARGIN
    if mask is not None:
        ok = ok & mask
    amb = 1.0 - ok.sum() / max(1, (mask.sum() if mask is not None else ok.size))
    e = {}
    for k in ("rgb", "alpha", "normal"):
        g = np.asarray(gpu[k], np.float64)
        e[k] = float(np.abs(g - ref[k])[..., ok].max(initial=0.0))
    d = np.asarray(gpu["depth"], np.float64)
    rel = np.abs(d - ref["depth"]) / np.maximum(np.abs(ref["depth"]), 1e-6)
    e["depth_rel"] = float(rel[ok].max(initial=0.0))
    return e, float(amb)


def assert_images_close(gpu, ref, mask=None, max_amb=1e-3, label=""):
    e, amb = image_errors(gpu, ref, mask)
    print(f"[{label}] errors {e} ambiguous {amb:.2e}")
    assert amb <= max_amb, (label, amb)
    assert e["rgb"] <= TOL_ABS, (label, e)
    assert e["alpha"] <= TOL_ABS, (label, e)
    assert e["normal"] <= TOL_ABS, (label, e)
    assert e["depth_rel"] <= TOL_DEPTH_REL, (label, e)
    return e, amb


def grad_errors(gpu: dict, ref: dict, idx=None, spread=None, prim_cond=None):
    """Per parameter group: max error in units of the allowed tolerance (<= 1 passes),
    the plain max relative error, the fraction of elements whose tolerance was widened by
    the conditioning allowance, and the number of deeply grazing primitives."""
    out = {}
    for k, gr in ref.items():
        g = np.asarray(gpu[k], np.float64).reshape(gr.shape)
        sp = None if spread is None else spread[k]
        pc = None if prim_cond is None else prim_cond
        if idx is not None:
            g, gr = g[idx], gr[idx]
            sp = None if sp is None else sp[idx]
            pc = None if pc is None else pc[idx]
        scale = np.maximum(np.abs(gr), 1e-3 * np.abs(gr).max(initial=0.0))
        scale = np.where(scale > 0, scale, 1.0)
        tol = TOL_GRAD_REL * scale
        widened = 0.0
        if sp is not None:
            allow = PERTURB_FACTOR * sp
            widened = float((allow > tol).mean()) if allow.size else 0.0
            tol = np.maximum(tol, allow)
        n_ill = 0
        if pc is not None:
            ill = pc < COND_STRICT
            n_ill = int(ill.sum())
            tol = np.where(ill.reshape((-1,) + (1,) * (tol.ndim - 1)), np.maximum(tol, TOL_GRAD_ILL * scale), tol)
        err = np.abs(g - gr)
        out[k] = dict(ratio=float((err / tol).max(initial=0.0)), rel=float((err / scale).max(initial=0.0)),
                      widened=widened, ill=n_ill)
    return out


def assert_grads_close(gpu, ref, idx=None, label="", spread=None, prim_cond=None):
    e = grad_errors(gpu, ref, idx, spread, prim_cond)
    print(f"[{label}] grad errors " + ", ".join(f"{k}: rel {v['rel']:.2e} tol-ratio {v['ratio']:.2f} "
                                                 f"widened {v['widened']:.3f} ill {v['ill']}"
                                                 for k, v in e.items()))
    for k, v in e.items():
        assert v["ratio"] <= 1.0, (label, k, v)
    return e


def perturbed(scene, seed, rel=PERTURB):
    """Copy of the scene with mean, quaternion, scales and curvatures multiplied by
    (1 + rel * N(0, 1)) in float64 (the oracle reads float64)."""
    rng = np.random.default_rng(seed)
    sc = scene.copy()
    for k in ("mean", "quat", "scale", "curv"):
        a = getattr(scene, k).astype(np.float64)
        setattr(sc, k, a * (1.0 + rel * rng.standard_normal(a.shape)))
    return sc


def oracle_grads_with_spread(O, scene, cam, grad_images, binning=None, tiles=None, samples=PERTURB_SAMPLES, **kw):
    """Oracle gradient and its per-element deviation under FP32-sized input noise
    (kw: density, extras of the oracle's render)."""
    ref = O.render(scene, cam, binning, tiles=tiles, grad_images=grad_images, **kw)
    spread = {k: np.zeros_like(v) for k, v in ref["grads"].items()}
    for s in range(samples):
        r = O.render(perturbed(scene, 1000 + s), cam, ref["binning"], tiles=tiles, grad_images=grad_images, **kw)
        for k in spread:
            spread[k] = np.maximum(spread[k], np.abs(r["grads"][k] - ref["grads"][k]))
    return ref, spread


def grad_mask(ref, extra=None):
    """Pixels whose upstream gradient is kept in gradient comparisons (float mask) and
    the fraction excluded (decision-ambiguous pixels)."""
    ok = ref["margin"] > MARGIN
    if extra is not None:
        ok = ok & extra
        frac = 1.0 - ok.sum() / max(1, extra.sum())
    else:
        frac = 1.0 - ok.mean()
    return ok.astype(np.float64), float(frac)


TOL_CURV_REL = 1e-4
TOL_DIST = 1e-4


def oracle_spread(O, scene, cam, ref, keys, tiles=None, **kw):
    """Per-pixel deviation of oracle output planes under FP32-sized input noise (the same
    perturbation as for gradients)."""
    spread = {k: np.zeros_like(ref[k]) for k in keys}
    for s in range(PERTURB_SAMPLES):
        r = O.render(perturbed(scene, 1000 + s), cam, ref["binning"], tiles=tiles, **kw)
        for k in keys:
            spread[k] = np.maximum(spread[k], np.abs(r[k] - ref[k]))
    return spread


def extra_errors(gpu: dict, ref: dict, mask=None, spread=None):
    """Errors of the extra channels over unambiguous pixels, each in units of its
    tolerance (<= 1 passes), plus plain relative errors for the record. With `spread`
    (oracle_spread of "curvature"), the curvature tolerance is widened to PERTURB_FACTOR
    times the oracle's own deviation, as for gradients: K = 4ab/S^2 with
    S = 1 + 4a^2x^2 + 4b^2y^2 moves by about 4 dx/x, and on strongly curved patches the
    hit point x itself is ill-conditioned."""
    ok = ref["margin"] > MARGIN
    if mask is not None:
        ok = ok & mask
    okm = ok & (ref["margin_median"] > MARGIN)
    cs = np.maximum(ref["curvature_scale"], 1.0)
    tolK = TOL_CURV_REL * cs
    widened = 0.0
    if spread is not None:
        allow = PERTURB_FACTOR * spread["curvature"]
        widened = float((allow > tolK)[ok].mean()) if ok.any() else 0.0
        tolK = np.maximum(tolK, allow)
    ek = np.abs(np.asarray(gpu["curvature"], np.float64) - ref["curvature"]) / cs
    rk = np.abs(np.asarray(gpu["curvature"], np.float64) - ref["curvature"]) / tolK
    D = ref["distortion"]
    dD = np.abs(np.asarray(gpu["distortion"], np.float64) - D)
    tolD = TOL_DIST * (D + np.abs(ref["depth"]) * np.sqrt(np.maximum(D, 0.0))) + 1e-9
    m = ref["median_depth"]
    em = np.abs(np.asarray(gpu["median_depth"], np.float64) - m) / np.maximum(np.abs(m), 1e-6)
    return dict(curvature=float(rk[ok].max(initial=0.0)), curvature_widened=widened,
                distortion=float((dD[ok] / tolD[ok]).max(initial=0.0)),
                median_depth=float((em[okm] / TOL_DEPTH_REL).max(initial=0.0)),
                curvature_rel=float(ek[ok].max(initial=0.0)),
                distortion_rel=float((dD / np.maximum(D, 1e-12))[ok].max(initial=0.0)),
                median_excluded=float(1.0 - okm.sum() / max(1, ok.sum())))


def assert_extras_close(gpu, ref, mask=None, label="", spread=None):
    e = extra_errors(gpu, ref, mask, spread)
    print(f"[{label}] extra-channel errors {e}")
    assert e["curvature"] <= 1.0, (label, e)
    assert e["distortion"] <= 1.0, (label, e)
    assert e["median_depth"] <= 1.0, (label, e)
    assert e["median_excluded"] <= 0.01, (label, e)
    return e
