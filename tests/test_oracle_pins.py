"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: numerical
quadrature, brute-force ray marching, the planar-surfel special case, the frame
symmetries of the paraboloid, finite differences, orthonormality of the SH basis,
and brute-force coverage of the screen bound.
"""
import math

import numpy as np
import pytest
import torch
from scipy import integrate, optimize

import oracle.qgs_oracle as O
from paper_2411_16392_gb300.scenes import Camera, Scene, f32_to_bf16_bits, scene_small

F64 = torch.float64


def t64(x):
    return torch.tensor(np.asarray(x, np.float64), dtype=F64)


# --------------------------------------------------------------------------- arc length
def _quad_arc(a, rho):
    val, _ = integrate.quad(lambda t: math.sqrt(1.0 + (2.0 * a * t) ** 2), 0.0, rho,
                            epsabs=0.0, epsrel=5e-14, limit=200)
    return val


def test_arc_length_matches_quadrature():
    """Closed form of the geodesic Eq. (Sec. 3.2) equals the defining integral
    int_0^rho sqrt(1 + (2 a t)^2) dt, on both sides of the Taylor threshold."""
    rng = np.random.default_rng(1)
    cases = [(a, r) for a, r in zip(rng.uniform(-50, 50, 40), rng.uniform(1e-3, 0.5, 40))]
    cases += [(1e-4, 1.0), (-1e-4, 2.0), (0.4999e-3, 1.0), (0.5001e-3, 1.0), (-0.5001e-3, 1.0),
              (1e4, 0.01), (-3e3, 0.02), (1e-12, 0.3), (0.0, 0.7), (2.0, 0.0)]
    a = t64([c[0] for c in cases])
    r = t64([c[1] for c in cases])
    got = O.arc_length(a, r).numpy()
    for (aa, rr), g in zip(cases, got):
        want = _quad_arc(aa, rr)
        assert abs(g - want) <= 1e-12 * max(want, 1e-300), (aa, rr, g, want)


def test_arc_length_high_precision():
    """Against 40-digit quadrature (mpmath) at a few points, including u near 1e-3."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    for aa, rr in [(3.0, 0.2), (-7.5, 0.05), (0.001 / 2 / 0.3, 0.3), (0.00099 / 2, 1.0)]:
        want = mp.quad(lambda t: mp.sqrt(1 + (2 * aa * t) ** 2), [0, rr])
        got = float(O.arc_length(t64([aa]), t64([rr]))[0])
        assert abs(got - float(want)) <= 1e-12 * float(want)


def test_arc_length_planar_limit():
    """a -> 0 gives l -> rho (the 2DGS degenerate case, Sec. 3.2)."""
    r = t64([0.1, 1.0, 3.0])
    for a in (0.0, 1e-14, -1e-10):
        l = O.arc_length(torch.full_like(r, a), r)
        assert torch.allclose(l, r, rtol=1e-15, atol=0)


def test_arc_length_bounds():
    """rho <= l and |a| rho^2 <= l (the two facts the screen bound relies on)."""
    rng = np.random.default_rng(2)
    a = t64(rng.uniform(-1e3, 1e3, 1000))
    r = t64(rng.uniform(0, 0.1, 1000))
    l = O.arc_length(a, r)
    assert bool((l >= r * (1 - 1e-15)).all())
    assert bool((l >= a.abs() * r * r * (1 - 1e-15)).all())


# --------------------------------------------------------------------------- sigma and G
def test_sigma_is_ellipse_radius():
    """sigma(theta) (Sec. 3.2) is the radius of the 1-sigma ellipse along theta."""
    rng = np.random.default_rng(3)
    th = t64(rng.uniform(-math.pi, math.pi, 200))
    s1 = t64(rng.uniform(0.001, 1, 200))
    s2 = t64(rng.uniform(0.001, 1, 200))
    sig = O.sigma_theta(th, s1, s2)
    lhs = (sig * torch.cos(th) / s1) ** 2 + (sig * torch.sin(th) / s2) ** 2
    assert torch.allclose(lhs, torch.ones_like(lhs), rtol=0, atol=1e-13)


def test_geodesic_gaussian_planar_is_2d_gaussian():
    """With a = b = 0 the geodesic Gaussian is the planar 2-D Gaussian of 2DGS."""
    rng = np.random.default_rng(4)
    x = t64(rng.normal(0, 0.1, 500))
    y = t64(rng.normal(0, 0.1, 500))
    s1 = t64(rng.uniform(0.01, 0.2, 500))
    s2 = t64(rng.uniform(0.01, 0.2, 500))
    z = torch.zeros_like(x)
    G, l, sig = O.geodesic_gaussian(x, y, z, z, s1, s2)
    want = torch.exp(-0.5 * (x * x / (s1 * s1) + y * y / (s2 * s2)))
    assert torch.allclose(G, want, rtol=1e-13, atol=0)


def test_geodesic_gaussian_by_quadrature_along_radial_curve():
    """G at a surface point equals exp(-l^2/(2 sigma^2)) with l obtained by integrating
    the length of the radial curve (x, y, a x^2 + b y^2) numerically in 3-D."""
    rng = np.random.default_rng(5)
    for _ in range(30):
        a, b = rng.uniform(-30, 30, 2)
        s1, s2 = rng.uniform(0.01, 0.1, 2)
        x, y = rng.normal(0, 0.05, 2)

        def speed(s):
            # curve c(s) = (s x, s y, a (s x)^2 + b (s y)^2), s in [0, 1]
            dz = 2 * a * s * x * x + 2 * b * s * y * y
            return math.sqrt(x * x + y * y + dz * dz)

        l_num, _ = integrate.quad(speed, 0, 1, epsabs=0, epsrel=1e-13)
        rr = math.hypot(x, y)
        # 1-sigma radius along theta found by root finding on the ellipse equation
        c, s = x / rr, y / rr
        sig_num = optimize.brentq(lambda r: (r * c / s1) ** 2 + (r * s / s2) ** 2 - 1, 0, 10, xtol=1e-15)
        G, l, sig = O.geodesic_gaussian(t64([x]), t64([y]), t64([a]), t64([b]), t64([s1]), t64([s2]))
        assert abs(float(l[0]) - l_num) <= 1e-11 * l_num
        assert abs(float(sig[0]) - sig_num) <= 1e-12 * sig_num
        assert abs(float(G[0]) - math.exp(-l_num ** 2 / (2 * sig_num ** 2))) <= 1e-11


# --------------------------------------------------------------------------- intersection
def _march_roots(f, t_lo, t_hi, n=200001):
    ts = np.linspace(t_lo, t_hi, n)
    v = f(ts)
    roots = []
    for i in np.nonzero(np.sign(v[:-1]) * np.sign(v[1:]) < 0)[0]:
        roots.append(optimize.brentq(f, ts[i], ts[i + 1], xtol=1e-15, rtol=1e-15))
    return roots


def test_quadratic_roots_match_ray_marching():
    """Roots of A t^2 + B t + C (supplementary, intersection Eq.) are the points where a
    marched ray crosses the surface z = a x^2 + b y^2."""
    rng = np.random.default_rng(6)
    checked = 0
    for _ in range(200):
        a, b = rng.uniform(-40, 40, 2)
        o = rng.normal(0, 0.3, 3)
        d = rng.normal(0, 1, 3)
        f = lambda t: a * (o[0] + t * d[0]) ** 2 + b * (o[1] + t * d[1]) ** 2 - (o[2] + t * d[2])
        A = a * d[0] ** 2 + b * d[1] ** 2
        B = 2 * (a * o[0] * d[0] + b * o[1] * d[1]) - d[2]
        C = a * o[0] ** 2 + b * o[1] ** 2 - o[2]
        t1, t2, e1, e2, _ = O.quadratic_roots(t64([A]), t64([B]), t64([C]))
        got = [float(t1[0])] * bool(e1[0]) + [float(t2[0])] * bool(e2[0])
        want = _march_roots(f, -5, 5)
        got_in = [g for g in got if -5 < g < 5]
        if len(want) != len(got_in):
            # a tangent double root can be missed by sign-change marching
            continue
        checked += 1
        for g, w in zip(sorted(got_in), want):
            assert abs(g - w) <= 1e-10 * max(1, abs(w))
    assert checked > 150


def test_linear_limit_is_tangent_plane_depth():
    """For A -> 0 the near root tends to -C/B, the paper's near-flat fallback."""
    B = t64([0.7, -1.3, 2.0])
    C = t64([0.4, 0.5, -3.0])
    for A in (1e-7, 1e-10, 0.0):
        t1, t2, e1, e2, _ = O.quadratic_roots(torch.full_like(B, A), B, C)
        near = torch.where((-C / B - t1).abs() < (-C / B - t2).abs(), t1, t2)
        assert torch.allclose(near, -C / B, rtol=max(1e-15, 10 * A), atol=0)


def _brute_hit(o, d, a, b, s1, s2, near):
    """Independent hit selection: march the ray, and at each crossing with t > near
    measure the radial arc length and sigma numerically; take the first crossing
    within 3 sigma."""
    f = lambda t: a * (o[0] + t * d[0]) ** 2 + b * (o[1] + t * d[1]) ** 2 - (o[2] + t * d[2])
    for t in _march_roots(f, near, 20.0, n=40001):
        x, y = o[0] + t * d[0], o[1] + t * d[1]
        rr = math.hypot(x, y)

        def speed(s):
            dz = 2 * a * s * x * x + 2 * b * s * y * y
            return math.sqrt(x * x + y * y + dz * dz)

        l, _ = integrate.quad(speed, 0, 1, epsabs=0, epsrel=1e-12)
        c, s = x / rr, y / rr
        sig = optimize.brentq(lambda r: (r * c / s1) ** 2 + (r * s / s2) ** 2 - 1, 0, 10, xtol=1e-15)
        if l <= 3 * sig:
            return t, math.exp(-l * l / (2 * sig * sig))
    return None, 0.0


def _one_prim_scene(mu, q, s, ab, o=0.9):
    return Scene(np.array([mu], np.float32), np.array([q], np.float32), np.array([s], np.float32),
                 np.array([ab], np.float32), np.array([o], np.float32),
                 f32_to_bf16_bits(np.zeros((1, 48), np.float32)))


def test_hit_selection_matches_brute_force():
    """Near-then-far selection within 3 sigma (Sec. 3.2.1) on single primitives, against
    marching plus numerical arc length; includes rays whose near hit is outside 3 sigma."""
    rng = np.random.default_rng(7)
    cam = Camera(32, 32, 24.0, 24.0, 16.0, 16.0)
    c64 = O.CamF64(cam)
    n_far = n_hit = 0
    for trial in range(25):
        s = rng.uniform(0.05, 0.2, 2)
        kap = rng.uniform(-6, 6, 2)
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        sc = _one_prim_scene([rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3), rng.uniform(1.5, 3)],
                             q, s, kap / s)
        prm = O.Params(sc)
        px = t64(np.repeat(np.arange(0, 32, 3), 11))
        py = t64(np.tile(np.arange(0, 32, 3), 11))
        pe = O._eval_pairs(prm, c64, torch.tensor([0]), px, py)
        R = O.quat_to_rot(prm.quat)[0].numpy()
        mu = sc.mean[0].astype(np.float64)
        a, b = sc.curv[0].astype(np.float64)
        s1, s2 = sc.scale[0].astype(np.float64)
        for k in range(px.shape[0]):
            d_cam = np.array([(px[k].item() + 0.5 - cam.cx) / cam.fx, (py[k].item() + 0.5 - cam.cy) / cam.fy, 1.0])
            o_l = R.T @ (c64.c_w.numpy() - mu)
            d_l = R.T @ d_cam
            t_b, G_b = _brute_hit(o_l, d_l, a, b, s1, s2, cam.near)
            got_hit = bool(pe["valid"][k, 0]) or False
            if t_b is None:
                assert float(pe["alpha"][k, 0]) == 0.0
                continue
            Gs = float(pe["alpha"][k, 0]) / float(np.float32(0.9)) if got_hit else None
            if got_hit:
                n_hit += 1
                assert abs(float(pe["t"][k, 0]) - t_b) <= 1e-9 * t_b
                assert abs(Gs - G_b) <= 1e-9
                f = lambda t: a * (o_l[0] + t * d_l[0]) ** 2 + b * (o_l[1] + t * d_l[1]) ** 2 - (o_l[2] + t * d_l[2])
                if len([r for r in _march_roots(f, cam.near, t_b - 1e-9)]) > 0:
                    n_far += 1
            else:
                assert float(np.float32(0.9)) * G_b < O.ALPHA_MIN * (1 + 1e-9)
    assert n_hit > 60
    assert n_far > 0


def test_normal_is_implicit_gradient_facing_camera():
    """The normal (Sec. 3.2 normal Eq.) is parallel to the gradient of a x^2 + b y^2 - z
    at the hit (taken by finite differences in world space) and faces the camera."""
    rng = np.random.default_rng(8)
    cam = Camera(32, 32, 24.0, 24.0, 16.0, 16.0)
    c64 = O.CamF64(cam)
    for _ in range(10):
        s = rng.uniform(0.1, 0.3, 2)
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        sc = _one_prim_scene([0.0, 0.0, 2.0], q, s, rng.uniform(-3, 3, 2) / s, 0.99)
        prm = O.Params(sc)
        R = O.quat_to_rot(prm.quat)[0].numpy()
        a, b = sc.curv[0].astype(np.float64)
        mu = sc.mean[0].astype(np.float64)
        px = t64(np.arange(10, 22))
        py = t64(np.arange(10, 22))
        pe = O._eval_pairs(prm, c64, torch.tensor([0]), px, py)
        for k in range(px.shape[0]):
            if not bool(pe["valid"][k, 0]):
                continue
            d_cam = np.array([(px[k].item() + 0.5 - 16) / 24, (py[k].item() + 0.5 - 16) / 24, 1.0])
            p = float(pe["t"][k, 0]) * d_cam      # world == camera here
            fw = lambda X: (lambda l: a * l[0] ** 2 + b * l[1] ** 2 - l[2])(R.T @ (X - mu))
            h = 1e-6
            grad = np.array([(fw(p + h * e) - fw(p - h * e)) / (2 * h) for e in np.eye(3)])
            grad /= np.linalg.norm(grad)
            n = pe["normal"][k, 0].numpy()
            assert abs(abs(n @ grad) - 1) < 1e-8
            assert n @ d_cam < 0


# --------------------------------------------------------------------------- whole renders
def _compose_rot(q, r):
    """Hamilton product q * r, so that R(q * r) = R(q) R(r)."""
    w1, x1, y1, z1 = q.T
    w2, x2, y2, z2 = r
    return np.stack([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                     w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                     w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2], 1).astype(np.float32)


def _small_scene(n=250, W=48, seed=0):
    sc, cam = scene_small(seed, n)
    return sc, Camera(W, W, float(W), float(W), W / 2, W / 2)


@pytest.mark.parametrize("sym", ["rz180", "rz90_swap", "rx180_flip"])
def test_frame_symmetries(sym):
    """The paraboloid and its Gaussian are unchanged by (1) a half turn about the local
    z axis, (2) a quarter turn with (s_u, a) and (s_v, b) exchanged, (3) a half turn about
    the local x axis with the curvatures negated (surface flipped)."""
    sc, cam = _small_scene()
    ref = O.render(sc, cam)
    s2 = sc.copy()
    if sym == "rz180":
        s2.quat = _compose_rot(sc.quat, np.array([0.0, 0, 0, 1]))
    elif sym == "rz90_swap":
        c = math.sqrt(0.5)
        s2.quat = _compose_rot(sc.quat, np.array([c, 0, 0, c]))
        s2.scale = sc.scale[:, ::-1].copy()
        s2.curv = sc.curv[:, ::-1].copy()
    else:
        s2.quat = _compose_rot(sc.quat, np.array([0.0, 1, 0, 0]))
        s2.curv = -sc.curv
    got = O.render(s2, cam)
    ok = (ref["margin"] > 1e-6) & (got["margin"] > 1e-6)
    assert ok.mean() > 0.99
    # the quarter-turn quaternion is rounded to float32, a ~6e-8 rotation perturbation
    tol = 2e-6 if sym == "rz90_swap" else 1e-9
    for k in ("rgb", "alpha", "depth", "normal"):
        diff = np.abs(ref[k] - got[k])
        assert diff[..., ok].max() < tol, k


def _planar_surfel_render(sc, cam):
    """Independent planar 2-D Gaussian surfel compositor (the a = b = 0 case):
    ray-plane intersection in world space, in-plane coordinates, 2-D Gaussian, same
    order and alpha rules."""
    from paper_2411_16392_gb300.scenes import bf16_bits_to_f32
    b = O.bin_fp32(sc, cam)
    H, W = cam.H, cam.W
    Rcw = cam.R_cw.astype(np.float64)
    c_w = -Rcw.T @ cam.t_cw.astype(np.float64)
    sh = bf16_bits_to_f32(sc.sh).astype(np.float64).reshape(-1, 16, 3)
    rgb = np.zeros((3, H, W)); alpha = np.zeros((H, W)); depth = np.zeros((H, W)); normal = np.zeros((3, H, W))
    for y in range(H):
        for x in range(W):
            tile = (y // 16) * b.tiles_x + x // 16
            s, e = b.ranges[tile]
            d_cam = np.array([(x + 0.5 - np.float32(cam.cx)) / np.float32(cam.fx),
                              (y + 0.5 - np.float32(cam.cy)) / np.float32(cam.fy), 1.0])
            d_w = Rcw.T @ d_cam
            T = 1.0
            for i in b.vals[s:e]:
                q = sc.quat[i].astype(np.float64)
                q = q / np.linalg.norm(q)
                w_, qx, qy, qz = q
                ru = np.array([1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy + w_ * qz), 2 * (qx * qz - w_ * qy)])
                rv = np.array([2 * (qx * qy - w_ * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz + w_ * qx)])
                rn = np.cross(ru, rv)
                mu = sc.mean[i].astype(np.float64)
                den = rn @ d_w
                if den == 0:
                    continue
                t = rn @ (mu - c_w) / den
                if not t > cam.near:
                    continue
                p = c_w + t * d_w - mu
                u, v = ru @ p, rv @ p
                su, sv = sc.scale[i].astype(np.float64)
                E = u * u / (su * su) + v * v / (sv * sv)
                if E > 9:
                    continue
                al = min(0.99, float(sc.opacity[i]) * math.exp(-0.5 * E))
                if al < 1 / 255:
                    continue
                if T * (1 - al) < 1e-4:
                    break
                dv = mu - c_w
                dv /= np.linalg.norm(dv)
                basis = O.sh_basis(t64(dv)).numpy()
                col = np.maximum(basis @ sh[i] + 0.5, 0)
                n = Rcw @ rn
                if n @ d_cam > 0:
                    n = -n
                w = al * T
                rgb[:, y, x] += w * col
                depth[y, x] += w * t
                normal[:, y, x] += w * n
                T *= 1 - al
            alpha[y, x] = 1 - T
    return dict(rgb=rgb, alpha=alpha, depth=depth, normal=normal)


def test_planar_limit_equals_surfel_renderer():
    """With zero curvature the whole render equals an independent 2-D surfel compositor
    (Sec. 3.2: 2DGS is the degenerate case of QGS)."""
    sc, cam = _small_scene(n=120, W=32, seed=3)
    sc.curv[:] = 0
    ref = _planar_surfel_render(sc, cam)
    got = O.render(sc, cam)
    ok = got["margin"] > 1e-7
    assert ok.mean() > 0.99
    for k in ref:
        assert np.abs(ref[k] - got[k])[..., ok].max() < 1e-10, k


def test_composite_matches_sequential_loop():
    """The chunked vectorised compositing equals a plain per-pixel loop over the list
    (T_i, the 1/255 skip, the 0.99 clamp and the stop before T < 1e-4)."""
    sc, cam = _small_scene(n=400, W=32, seed=5)
    sc.opacity[:] = np.float32(0.95)
    b = O.bin_fp32(sc, cam)
    prm = O.Params(sc)
    c64 = O.CamF64(cam)
    tile = int(np.argmax(b.ranges[:, 1] - b.ranges[:, 0]))
    s, e = b.ranges[tile]
    idx = torch.from_numpy(b.vals[s:e].astype(np.int64))
    xs, ys = O._tile_pixels(cam, tile, b.tiles_x)
    px, py = t64(xs), t64(ys)
    r = O._composite(prm, c64, idx, px, py, chunk=7)
    pe = O._eval_pairs(prm, c64, idx, px, py)
    for k in range(px.shape[0]):
        T, acc, ne, last = 1.0, np.zeros(3), 0, 0
        for j in range(idx.shape[0]):
            ne += 1
            if not bool(pe["valid"][k, j]):
                continue
            al = float(pe["alpha"][k, j])
            if T * (1 - al) < O.T_MIN:
                break
            acc += al * T * pe["rgb"][j].numpy()
            T *= 1 - al
            last = j + 1
        assert abs(r["T_final"][k].item() - T) < 1e-14
        assert np.abs(r["rgb"][k].numpy() - acc).max() < 1e-13
        assert int(r["n_eval"][k]) == ne and int(r["n_contrib"][k]) == last


def test_back_to_front_and_front_to_back_alpha_gradients():
    """The supplementary's back-to-front and front-to-back forms of dX/d(alpha_i) are equal
    and match the derivative of X = sum alpha_i T_i X_i."""
    rng = np.random.default_rng(9)
    n = 12
    al = torch.tensor(rng.uniform(0.01, 0.9, n), dtype=F64, requires_grad=True)
    X = t64(rng.normal(size=n))
    T = torch.cat([torch.ones(1, dtype=F64), torch.cumprod(1 - al, 0)[:-1]])
    Xh = (al * T * X).sum()
    (g,) = torch.autograd.grad(Xh, al)
    a = al.detach()
    Tn = T.detach()
    Tnext = Tn * (1 - a)
    w = a * Tn * X
    for i in range(n):
        b2f = (X[i] - w[i + 1:].sum() / Tnext[i]) * Tn[i]
        f2b = (X[i] - (Xh.detach() - w[:i + 1].sum()) / Tnext[i]) * Tn[i]
        assert abs(b2f - g[i]) < 1e-13 and abs(f2b - g[i]) < 1e-13


def _tiny_grad_scene(seed):
    rng = np.random.default_rng(seed)
    n = 5
    s = rng.uniform(0.12, 0.3, (n, 2))
    kap = rng.uniform(-1.5, 1.5, (n, 2))
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    # keep the surface normals roughly towards the camera
    sc = Scene(np.stack([rng.uniform(-0.4, 0.4, n), rng.uniform(-0.4, 0.4, n), rng.uniform(1.8, 2.6, n)], 1).astype(np.float32),
               q.astype(np.float32), s.astype(np.float32), (kap / s).astype(np.float32),
               rng.uniform(0.3, 0.9, n).astype(np.float32),
               f32_to_bf16_bits(rng.normal(0, 0.3, (n, 48)).astype(np.float32)))
    cam = Camera(24, 24, 20.0, 20.0, 12.0, 12.0)
    return sc, cam


def test_gradients_match_finite_differences():
    """Autograd gradients of the FP64 forward match central differences for every
    parameter of a tiny scene (seeds with a decision closer than 1e-4 are skipped)."""
    from paper_2411_16392_gb300.scenes import bf16_bits_to_f32
    for seed in range(20):
        sc, cam = _tiny_grad_scene(seed)
        rng = np.random.default_rng(100 + seed)
        g = dict(rgb=rng.normal(size=(3, 24, 24)), alpha=rng.normal(size=(24, 24)),
                 depth=rng.normal(size=(24, 24)), normal=rng.normal(size=(3, 24, 24)))
        ref = O.render(sc, cam, grad_images=g)
        if ref["margin"].min() > 1e-4 and ref["n_contrib"].max() > 0:
            break
    else:
        pytest.fail("no seed without near-decision pairs")
    binning = ref["binning"]
    prm = O.Params(sc)

    def loss_of(pr):
        c64 = O.CamF64(cam)
        tot = 0.0
        for tile in range(binning.tiles_x * binning.tiles_y):
            s, e = binning.ranges[tile]
            if e <= s:
                continue
            xs, ys = O._tile_pixels(cam, tile, binning.tiles_x)
            r = O._composite(pr, c64, torch.from_numpy(binning.vals[s:e].astype(np.int64)), t64(xs), t64(ys))
            tot += float((t64(g["rgb"][:, ys, xs].T) * r["rgb"]).sum() + (t64(g["alpha"][ys, xs]) * r["alpha"]).sum()
                         + (t64(g["depth"][ys, xs]) * r["depth"]).sum() + (t64(g["normal"][:, ys, xs].T) * r["normal"]).sum())
        return tot

    grads = ref["grads"]
    for name in ("mean", "quat", "scale", "curv", "opacity", "sh"):
        leaf = getattr(prm, name)
        flat = leaf.view(-1)
        gref = grads[name].reshape(-1)
        scale = max(np.abs(gref).max(), 1e-12)
        for j in range(flat.numel()):
            v0 = float(flat[j])
            h = 1e-6 * max(1.0, abs(v0))
            with torch.no_grad():
                flat[j] = v0 + h
                lp = loss_of(prm)
                flat[j] = v0 - h
                lm = loss_of(prm)
                flat[j] = v0
            fd = (lp - lm) / (2 * h)
            assert abs(fd - gref[j]) <= 1e-5 * scale + 1e-6 * abs(fd), (name, j, fd, gref[j])


# --------------------------------------------------------------------------- binning
def _brute_support(sc, cam):
    """For every primitive and pixel (no binning), whether the pair has a selected hit."""
    prm = O.Params(sc)
    c64 = O.CamF64(cam)
    ys, xs = np.meshgrid(np.arange(cam.H), np.arange(cam.W), indexing="ij")
    px, py = t64(xs.reshape(-1)), t64(ys.reshape(-1))
    out = []
    for i0 in range(0, sc.n, 64):
        idx = torch.arange(i0, min(i0 + 64, sc.n))
        pe = O._eval_pairs(prm, c64, idx, px, py)
        # hit within 3 sigma, regardless of the 1/255 skip: recompute alpha without it
        out.append(pe["hit"].numpy().T)
    return np.concatenate(out, 0), xs.reshape(-1), ys.reshape(-1)


@pytest.mark.parametrize("inside,kappa", [(False, 1.0), (True, 1.0), (False, 4.0), (False, 0.0)])
def test_screen_bound_is_conservative(inside, kappa):
    """Every pixel where a primitive has a hit within 3 sigma lies inside the primitive's
    tile rectangle, inside its pixel AABB (box of the support, clipped to the near plane)
    and in a tile that the screen-parallelogram test keeps in its list. `inside` puts the camera among the primitives; `kappa` scales the curvatures
    (4: |kappa| up to 20 as in the object scene, 0: planar)."""
    sc, cam = _small_scene(n=300, W=40, seed=11)
    sc.curv *= np.float32(kappa)
    if inside:
        sc.mean[:, 2] -= 3.6   # centres now in [-0.6, 1.4]: many boxes cross z = near
    b = O.bin_fp32(sc, cam)
    sup, xs, ys = _brute_support(sc, cam)
    n_in = 0
    for i in range(sc.n):
        hit = sup[i]
        if not hit.any():
            continue
        if sc.mean[i, 2] <= cam.near:
            continue   # culled by its centre (a reading), not by the bound
        assert b.visible[i], i
        x0, x1, y0, y1 = b.rect[i]
        tx, ty = xs[hit] // 16, ys[hit] // 16
        assert ((tx >= x0) & (tx <= x1) & (ty >= y0) & (ty <= y1)).all(), i
        bb = b.pix_bbox[i]
        assert ((xs[hit] + 0.5 >= bb[0]) & (xs[hit] + 0.5 <= bb[1]) & (ys[hit] + 0.5 >= bb[2])
                & (ys[hit] + 0.5 <= bb[3])).all(), i
        # and inside the screen parallelogram: every tile with a hit pixel is listed
        for t in np.unique(ty * b.tiles_x + tx):
            s, e = b.ranges[t]
            assert i in b.vals[s:e], (i, t)
        n_in += 1
    assert n_in > 50
    # the parallelogram removes tiles the rectangle would list
    full = int(sum((b.rect[i, 1] - b.rect[i, 0] + 1) * (b.rect[i, 3] - b.rect[i, 2] + 1)
                   for i in range(sc.n) if b.visible[i]))
    assert len(b.keys) < full


def test_keys_are_tile_and_depth_bits():
    """Sorted keys are (tile << 32) | float32 bits of the centre's view depth, tiles
    row-major, ties in depth broken by primitive index; ranges delimit each tile."""
    sc, cam = scene_small(0, 1000)
    b = O.bin_fp32(sc, cam)
    z64 = sc.mean.astype(np.float64) @ cam.R_cw.astype(np.float64)[2] + cam.t_cw[2]
    assert np.all(np.abs(b.zbits.view(np.float32) - z64) <= 1e-6 * z64)
    assert np.all(b.keys[1:] >= b.keys[:-1])
    same = b.keys[1:] == b.keys[:-1]
    assert np.all(b.vals[1:][same] > b.vals[:-1][same])
    assert np.all((b.keys & np.uint64(0xFFFFFFFF)).astype(np.uint32) == b.zbits[b.vals])
    tiles = (b.keys >> np.uint64(32)).astype(np.int64)
    for t in range(b.tiles_x * b.tiles_y):
        s, e = b.ranges[t]
        assert np.all(tiles[s:e] == t)
        x0, x1, y0, y1 = b.rect[b.vals[s:e]].T
        ty, tx = divmod(t, b.tiles_x)
        assert np.all((x0 <= tx) & (tx <= x1) & (y0 <= ty) & (ty <= y1))
    assert len(b.keys) == b.count.sum()


def test_fp32_rect_agrees_with_fp64_box():
    """The FP32 recipe's pixel AABB agrees with the same box restated in FP64 (textbook
    quadratic formula instead of the recipe's rationalised roots) to FP32 rounding (a
    transposed rotation, a wrong corner or a wrong root would not)."""
    sc, cam = scene_small(0, 1000)
    b = O.bin_fp32(sc, cam)
    R = O.quat_to_rot(t64(sc.quat)).numpy()
    for i in range(0, 1000, 7):
        if not b.visible[i]:
            continue
        su, sv = sc.scale[i].astype(np.float64)
        a, bb = sc.curv[i].astype(np.float64)
        m = max(su, sv)
        # z range: root of (c/m^2) z^2 + z - 9c = 0 (quadratic formula, FP64)
        cp = max(0.0, a * su * su, bb * sv * sv)
        cn = max(0.0, -a * su * su, -bb * sv * sv)
        root = lambda c: 0.0 if c == 0 else (-1 + math.sqrt(1 + 36 * c * c / (m * m))) / (2 * c / (m * m))
        zhi, zlo = root(cp), -root(cn)
        same = a * bb >= 0
        ext = lambda s_, k: (math.sqrt((-1 / s_ ** 2 + math.sqrt(1 / s_ ** 4 + 36 * k * k / m ** 2)) / (2 * k * k / m ** 2))
                             if (same and k != 0) else 3 * s_)
        X, Y = ext(su, a), ext(sv, bb)
        pts = []
        for sx in (-X, X):
            for sy in (-Y, Y):
                for sz in (zlo, zhi):
                    p = sc.mean[i].astype(np.float64) + R[i] @ np.array([sx, sy, sz])
                    pts.append((cam.fx * p[0] / p[2] + cam.cx, cam.fy * p[1] / p[2] + cam.cy))
        pts = np.array(pts)
        want = [pts[:, 0].min(), pts[:, 0].max(), pts[:, 1].min(), pts[:, 1].max()]
        assert np.allclose(b.pix_bbox[i], want, rtol=0, atol=2e-4), i


# --------------------------------------------------------------------------- colour
def test_sh_basis_orthonormal_and_matches_scipy():
    """The 16 basis functions are orthonormal on the sphere (a wrong constant or a dropped
    term breaks this) and each equals +-1 times scipy's real spherical harmonic."""
    from scipy.special import roots_legendre, sph_harm_y
    xg, wg = roots_legendre(12)
    nph = 24
    ph = (np.arange(nph) + 0.5) * 2 * np.pi / nph
    th = np.arccos(xg)
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    Wt = np.repeat(wg[:, None], nph, 1) * (2 * np.pi / nph)
    d = np.stack([np.sin(TH) * np.cos(PH), np.sin(TH) * np.sin(PH), np.cos(TH)], -1)
    Y = O.sh_basis(t64(d)).numpy()                     # [12, 24, 16]
    G = np.einsum("ijk,ijl,ij->kl", Y, Y, Wt)
    assert np.allclose(G, np.eye(16), atol=1e-12)
    k = 0
    for l in range(4):
        for m in range(-l, l + 1):
            # real SH from the complex ones
            if m < 0:
                ref = np.sqrt(2) * (-1) ** m * sph_harm_y(l, -m, TH, PH).imag
            elif m == 0:
                ref = sph_harm_y(l, 0, TH, PH).real
            else:
                ref = np.sqrt(2) * (-1) ** m * sph_harm_y(l, m, TH, PH).real
            mine = Y[..., k]
            assert np.allclose(mine, ref, atol=1e-12) or np.allclose(mine, -ref, atol=1e-12), (l, m)
            k += 1


# --------------------------------------------------------------------------- chord ellipsoid
def test_support_lies_in_chord_ellipsoid():
    """Every point of the support (geodesic distance <= 3 sigma(theta), Sec. 3.2) satisfies
    x^2/s_u^2 + y^2/s_v^2 + z^2/m^2 <= 9 with m = max(s_u, s_v): the ellipsoid behind the
    screen-space conic of the tile lists. Points sampled on the paraboloid in FP64 up to
    the support's rim, for saddles, cups and elongated scales."""
    rng = np.random.default_rng(4)
    n = 4000
    su, sv = np.exp(rng.uniform(np.log(1e-3), np.log(0.1), (2, n)))
    a = rng.uniform(-10, 10, n) / su
    b = rng.uniform(-10, 10, n) / sv
    th = rng.uniform(0, 2 * np.pi, n)
    c, s = np.cos(th), np.sin(th)
    at = a * c * c + b * s * s
    sig = O.sigma_theta(t64(th), t64(su), t64(sv)).numpy()
    # the rim: l(a(theta), rho) = 3 sigma(theta), by bisection on rho (l increases with rho)
    lo, hi = np.zeros(n), 3 * sig
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        l = O.arc_length(t64(at), t64(mid)).numpy()
        lo, hi = np.where(l <= 3 * sig, mid, lo), np.where(l <= 3 * sig, hi, mid)
    m = np.maximum(su, sv)
    for frac in (1.0, 0.7, 0.3):
        rho = lo * frac
        x, y = rho * c, rho * s
        z = a * x * x + b * y * y
        v = x * x / su ** 2 + y * y / sv ** 2 + z * z / m ** 2
        assert v.max() <= 9.0 * (1 + 1e-9), v.max()
    assert v.max() > 0.5   # the rim is reached for some primitives


def _ellipsoid_line_dist2(sc, cam, i, X, Y):
    """Squared distance, in the frame scaled by (s_u, s_v, m), from the centre of primitive
    i to the line through the camera centre and pixel position (X, Y): FP64, world
    coordinates, by orthogonal projection (no use of the recipe's algebra)."""
    R = O.quat_to_rot(t64(sc.quat[i:i + 1])).numpy()[0]
    su, sv = sc.scale[i].astype(np.float64)
    S = np.diag(1.0 / np.array([su, sv, max(su, sv)]))
    Rcw = cam.R_cw.astype(np.float64)
    c_w = -Rcw.T @ cam.t_cw.astype(np.float64)
    d_cam = np.stack([(X - cam.cx) / cam.fx, (Y - cam.cy) / cam.fy, np.ones_like(X)], -1)
    d = (S @ R.T @ (Rcw.T @ d_cam.T)).T                     # scaled local directions
    o = S @ R.T @ (c_w - sc.mean[i].astype(np.float64))    # scaled local camera centre
    t = -(d @ o) / np.einsum("ij,ij->i", d, d)              # closest point on the line
    p = o[None, :] + t[:, None] * d
    return np.einsum("ij,ij->i", p, p)


@pytest.mark.parametrize("kappa,aspect", [(1.0, False), (4.0, True), (0.0, True)])
def test_conic_is_the_projected_chord_ellipsoid(kappa, aspect):
    """The FP32 conic F(p) <= 1 holds every pixel whose ray line meets the chord ellipsoid
    (squared scaled distance <= 9) and is no looser than the recipe's pads (9.02 radius
    squared, a 2e-3 px rim and the diagonal shift, which grows with the ellipse's
    elongation): pixels with F <= 1 have squared distance <= 9.1 (9.3 with scale ratios up
    to 50) where the projected ellipse covers a dozen pixel centres or more."""
    sc, cam = _small_scene(n=300, W=64, seed=5)
    sc.curv *= np.float32(kappa)
    if aspect:   # elongated primitives: ratio of scales up to 50
        sc.scale[:, 1] = (sc.scale[:, 0] * np.exp(np.random.default_rng(2).uniform(-np.log(50), np.log(50), sc.n))
                          ).astype(np.float32)
    b = O.bin_fp32(sc, cam, emit=False)
    sl = b.slabs
    ys, xs = np.meshgrid(np.arange(-8, cam.H + 8), np.arange(-8, cam.W + 8), indexing="ij")
    X, Y = xs.reshape(-1) + 0.5, ys.reshape(-1) + 0.5
    n_on = n_tight = 0
    for i in np.nonzero(b.visible)[0]:
        d2 = _ellipsoid_line_dist2(sc, cam, i, X, Y)
        if not sl["conic_on"][i]:
            continue
        n_on += 1
        p = np.full(X.shape, i)
        u = (X.astype(np.float32) - sl["uc"][i]).astype(np.float32)
        v = (Y.astype(np.float32) - sl["vc"][i]).astype(np.float32)
        F = O.conic_value(sl, p, u, v).astype(np.float64)
        assert np.all(F[d2 <= 9.0] <= 1.0), i
        if (d2 <= 9.0).sum() >= 12:
            assert d2[F <= 1.0].max() <= (9.3 if aspect else 9.1), (i, d2[F <= 1.0].max())
            n_tight += 1
    assert n_on >= 0.9 * b.visible.sum() and n_tight > 20


def test_conic_tile_test_against_the_rectangle():
    """The conic part of the tile test (edges of the rectangle of pixel-centre offsets,
    clamped stationary points) against a direct minimisation of F over the rectangle:
    a fine grid refined by a bounded quasi-Newton search (FP64). Tiles whose minimum is
    below 1 - 1e-6 pass, tiles whose minimum is above 1 + 1e-6 fail."""
    sc, cam = _small_scene(n=200, W=96, seed=6)
    sc.scale *= np.float32(4.0)     # primitives spanning several tiles
    sc.curv /= np.float32(4.0)
    b = O.bin_fp32(sc, cam, emit=False)
    sl = b.slabs
    f = np.float32
    checked = rejected = 0
    for i in np.nonzero(b.visible & sl["conic_on"])[0][:60]:
        x0r, x1r, y0r, y1r = b.rect[i]   # the rectangle and one ring of tiles around it
        for ty in range(max(y0r - 1, 0), min(y1r + 1, b.tiles_y - 1) + 1):
            for tx in range(max(x0r - 1, 0), min(x1r + 1, b.tiles_x - 1) + 1):
                x0 = f(16 * tx) + f(0.5) - sl["uc"][i]
                x1 = f(min(16 * tx + 15, cam.W - 1)) + f(0.5) - sl["uc"][i]
                y0 = f(16 * ty) + f(0.5) - sl["vc"][i]
                y1 = f(min(16 * ty + 15, cam.H - 1)) + f(0.5) - sl["vc"][i]
                got = bool(O._conic_pass(sl, np.array([i]), np.array([x0]), np.array([x1]), np.array([y0]),
                                         np.array([y1]))[0])
                q = [float(sl[k][i]) for k in ("qa", "qb", "qc", "la", "lb")]

                def F(pt):
                    u, v = pt
                    return q[0] * u * u + 2 * q[1] * u * v + q[2] * v * v - 2 * q[3] * u - 2 * q[4] * v

                gu, gv = np.meshgrid(np.linspace(x0, x1, 41), np.linspace(y0, y1, 41))
                vals = F((gu, gv))
                k = np.argmin(vals)
                r = optimize.minimize(F, [gu.flat[k], gv.flat[k]], method="L-BFGS-B",
                                      bounds=[(float(x0), float(x1)), (float(y0), float(y1))],
                                      options=dict(ftol=1e-15, gtol=1e-12))
                fmin = min(float(r.fun), float(vals.flat[k]))
                if fmin < 1 - 1e-6:
                    assert got, (i, tx, ty, fmin)
                elif fmin > 1 + 1e-6:
                    assert not got, (i, tx, ty, fmin)
                    rejected += 1
                checked += 1
    assert checked > 200 and rejected > 20


def test_conic_box_holds_the_conic():
    """The conic's bounding box (the tiles the rectangle is cut to) holds every pixel
    offset with F <= 1: brute force over a fine grid around each projected centre (FP64
    evaluation of the recipe's coefficients), and the box is no wider than the ellipse's
    exact half-extents sqrt(R (q^-1)_ii) plus one tile."""
    sc, cam = _small_scene(n=300, W=96, seed=8)
    sc.scale *= np.float32(3.0)
    sc.curv /= np.float32(3.0)
    b = O.bin_fp32(sc, cam, emit=False)
    sl = b.slabs
    on = np.nonzero(b.visible & sl["conic_on"])[0]
    assert on.size > 50
    cb = O.conic_box({k: sl[k][on] for k in ("qa", "qb", "qc", "la", "lb")}, sl["uc"][on], sl["vc"][on])
    checked = 0
    for j, i in enumerate(on[:80]):
        qa, qb, qc, la, lb = (float(sl[k][i]) for k in ("qa", "qb", "qc", "la", "lb"))
        q = np.array([[qa, qb], [qb, qc]])
        p0 = np.linalg.solve(q, np.array([la, lb]))
        R = 1.0 + la * p0[0] + lb * p0[1]
        ext = np.sqrt(R * np.diag(np.linalg.inv(q)))
        u = np.linspace(p0[0] - 1.2 * ext[0], p0[0] + 1.2 * ext[0], 121)
        v = np.linspace(p0[1] - 1.2 * ext[1], p0[1] + 1.2 * ext[1], 121)
        U, Vv = np.meshgrid(u, v)
        F = qa * U * U + 2 * qb * U * Vv + qc * Vv * Vv - 2 * la * U - 2 * lb * Vv
        inside = F <= 1.0
        X = float(sl["uc"][i]) + U[inside]
        Y = float(sl["vc"][i]) + Vv[inside]
        assert (np.floor(X / 16) >= cb[0][j]).all() and (np.floor(X / 16) <= cb[1][j]).all(), i
        assert (np.floor(Y / 16) >= cb[2][j]).all() and (np.floor(Y / 16) <= cb[3][j]).all(), i
        cx, cy = float(sl["uc"][i]) + p0[0], float(sl["vc"][i]) + p0[1]
        assert cb[0][j] >= np.floor((cx - ext[0]) / 16) - 1 and cb[1][j] <= np.floor((cx + ext[0]) / 16) + 1, i
        assert cb[2][j] >= np.floor((cy - ext[1]) / 16) - 1 and cb[3][j] <= np.floor((cy + ext[1]) / 16) + 1, i
        checked += 1
    assert checked >= 50
