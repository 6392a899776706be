"""Pins of the oracle's bracketing of near-threshold decisions and of its list-free mode.

bracket_pixels takes each discrete decision of a pixel that lies within rounding distance
of its threshold both ways; these tests build pixels whose decision sits a known distance
from its threshold (planar primitives, where G = exp(-E/2) is known in closed form) and
check the branches it returns against values worked out here. The list-free candidates are
checked against brute force over every primitive.
"""
import math
import struct

import numpy as np
import pytest
import torch

import oracle.qgs_oracle as O
from paper_2411_16392_gb300.scenes import Camera, Scene, f32_to_bf16_bits, scene_small

F64 = torch.float64


def test_bf16_decoder_known_patterns():
    """bfloat16 is the upper half of an IEEE binary32."""
    known = {0x3F80: 1.0, 0xC000: -2.0, 0x0000: 0.0, 0x3E80: 0.25, 0x4049: 3.140625, 0x7F80: math.inf,
             0xFF80: -math.inf, 0x0001: 2.0 ** -133}
    got = O.bf16_to_f64(np.array(list(known), np.uint16))
    for (b, want), g in zip(known.items(), got):
        assert g == want, (hex(b), g, want)
    rng = np.random.default_rng(0)
    bits = rng.integers(0, 0x7F80, 200).astype(np.uint16)
    for b, g in zip(bits, O.bf16_to_f64(bits)):
        assert g == struct.unpack(">f", bytes([int(b) >> 8, int(b) & 255, 0, 0]))[0]


def _planar_scene(means, scales, opac, dc=None):
    """Planar primitives (a = b = 0) facing the camera (identity rotation: the local z
    axis is the camera's); `dc` sets the degree-0 SH coefficients (exact in bfloat16),
    giving the constant colour 0.5 + dc / (2 sqrt(pi))."""
    n = len(means)
    sh = np.zeros((n, 48), np.float32)
    if dc is not None:
        sh[:, :3] = np.asarray(dc, np.float32)
    return Scene(np.asarray(means, np.float32), np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)),
                 np.asarray(scales, np.float32), np.zeros((n, 2), np.float32), np.asarray(opac, np.float32),
                 f32_to_bf16_bits(sh))


CAM = Camera(16, 16, 16.0, 16.0, 8.0, 8.0)


def _hit_E(mean, scale, x, y):
    """E = x^2/s_u^2 + y^2/s_v^2 of the pixel ray's hit on a camera-facing plane, in FP64
    from the float32 inputs."""
    mx, my, mz = (float(np.float32(v)) for v in mean)
    dx, dy = (x + 0.5 - 8.0) / 16.0, (y + 0.5 - 8.0) / 16.0
    hx, hy = dx * mz - mx, dy * mz - my
    su, sv = (float(np.float32(v)) for v in scale)
    return (hx / su) ** 2 + (hy / sv) ** 2


def test_alpha_threshold_is_taken_both_ways():
    """o G within 3e-6 (relative) above 1/255: the pair blends, and its other branch drops
    it (alpha 0)."""
    mean, scale = (0.03, -0.02, 2.0), (0.05, 0.04)
    G = math.exp(-0.5 * _hit_E(mean, scale, 8, 8))
    o = np.float32(O.ALPHA_MIN * (1 + 3e-6) / G)
    sc = _planar_scene([mean], [scale], [o])
    oG = float(o) * G
    assert 0 < oG / O.ALPHA_MIN - 1 < 1e-5
    (it,) = O.bracket_pixels(sc, CAM, [(8, 8)], O.bin_fp32(sc, CAM))
    alphas = sorted(float(l["alpha"][0]) for l in it["leaves"])
    assert it["n_branch_decisions"] == 1 and len(alphas) == 2
    assert alphas[0] == 0.0 and abs(alphas[1] - oG) < 1e-15
    assert abs(it["leaves"][0]["alpha"][0] - oG) < 1e-15   # the nominal branch blends it
    ref = O.render(sc, CAM)
    assert abs(ref["alpha"][8, 8] - oG) < 1e-15


def test_three_sigma_edge_is_taken_both_ways():
    """A hit at E = 9 (1 - 2e-6), just inside 3 sigma: blended with G = exp(-E/2), and its
    other branch leaves the support (no hit)."""
    scale = (0.05, 0.05)
    dx = (8 + 0.5 - 8.0) / 16.0
    # centre offset so that the pixel's hit is 3 sigma (1 - 1e-6) from it along x
    mx = dx * 2.0 - 3.0 * 0.05 * (1 - 1e-6)
    mean = (mx, (8.5 - 8.0) / 16.0 * 2.0, 2.0)
    E = _hit_E(mean, scale, 8, 8)
    assert 0 < 1 - E / 9 < 1e-5
    sc = _planar_scene([mean], [scale], [0.9])
    (it,) = O.bracket_pixels(sc, CAM, [(8, 8)], O.bin_fp32(sc, CAM))
    want = float(np.float32(0.9)) * math.exp(-0.5 * E)
    alphas = sorted(float(l["alpha"][0]) for l in it["leaves"])
    assert len(alphas) == 2 and alphas[0] == 0.0 and abs(alphas[1] - want) < 1e-14


def test_transmittance_stop_is_taken_both_ways():
    """Three stacked planes whose third takes T to 1e-4 (1 + 2e-6): blended (T stays just
    above the threshold), and the other branch stops before it."""
    x = y = 8
    d = (0.5 / 16.0)
    means = [(d * z, d * z, z) for z in (2.0, 3.0, 4.0)]   # centres on the pixel's ray
    scales = [(0.05, 0.05)] * 3
    Gs = [math.exp(-0.5 * _hit_E(m, s, x, y)) for m, s in zip(means, scales)]
    a1 = a2 = 0.95
    T2 = (1 - a1) * (1 - a2)
    a3 = 1 - 1e-4 * (1 + 2e-6) / T2
    ops = [np.float32(a / G) for a, G in zip((a1, a2, a3), Gs)]
    al = [float(o) * G for o, G in zip(ops, Gs)]
    T2 = (1 - al[0]) * (1 - al[1])
    T3 = T2 * (1 - al[2])
    assert 0 < T3 / O.T_MIN - 1 < 1e-5
    sc = _planar_scene(means, scales, ops)
    (it,) = O.bracket_pixels(sc, CAM, [(x, y)], O.bin_fp32(sc, CAM))
    got = sorted(float(l["alpha"][0]) for l in it["leaves"])
    assert len(got) == 2
    assert abs(got[0] - (1 - T2)) < 1e-14 and abs(got[1] - (1 - T3)) < 1e-14
    assert abs(it["leaves"][0]["alpha"][0] - (1 - T3)) < 1e-14      # nominal: blended
    assert sorted(it["n_contrib"]) == [2, 3]


def test_resort_order_tie_is_taken_both_ways():
    """StopThePop resorting: two coplanar primitives at one depth (a tie of their hit
    depths) of different colours; both blend orders are branches."""
    x = y = 8
    d = 0.5 / 16.0
    means = [(d * 2.0 + 0.01, d * 2.0, 2.0), (d * 2.0 - 0.01, d * 2.0, 2.0)]
    scales = [(0.05, 0.05)] * 2
    sc = _planar_scene(means, scales, [0.6, 0.7], dc=[(1.0, -1.0, 0.0), (-1.0, 1.0, 0.0)])
    b = O.bin_fp32(sc, CAM, order="hit")
    (it,) = O.bracket_pixels(sc, CAM, [(x, y)], b, order="stp")
    Gs = [math.exp(-0.5 * _hit_E(m, s, x, y)) for m, s in zip(means, scales)]
    a = [float(np.float32(o)) * G for o, G in zip((0.6, 0.7), Gs)]
    hi, lo = 0.5 + 0.5 / math.sqrt(math.pi), 0.5 - 0.5 / math.sqrt(math.pi)
    c0, c1 = np.array([hi, lo]), np.array([lo, hi])      # (red, green) of each primitive
    first0 = a[0] * c0 + (1 - a[0]) * a[1] * c1
    first1 = a[1] * c1 + (1 - a[1]) * a[0] * c0
    got = sorted(tuple(np.round(l["rgb"][:2], 12)) for l in it["leaves"])
    want = sorted(tuple(np.round(v, 12)) for v in (first0, first1))
    assert got == want


def test_discriminant_shift():
    """quadratic_roots(A, B, C, d_shift=s) solves the quadratic whose discriminant is
    D + s (i.e. C - s / (4A))."""
    A = torch.tensor([2.0, -1.5, 0.7], dtype=F64)
    B = torch.tensor([3.0, 0.4, -5.0], dtype=F64)
    C = torch.tensor([0.5, 2.0, 1.0], dtype=F64)
    s = torch.tensor([1e-3, -2e-2, 0.3], dtype=F64)
    t1, t2, e1, e2, _ = O.quadratic_roots(A, B, C, d_shift=s)
    Cs = C - s / (4 * A)
    for r in (t1, t2):
        assert torch.allclose(A * r * r + B * r + Cs, torch.zeros_like(r), atol=1e-12)
    assert bool(e1.all() and e2.all())


def test_listfree_candidates_hold_every_hit():
    """Every primitive whose pair with the pixel has a hit (brute force over all of them)
    is among the list-free candidates, which come in (centre depth, index) order."""
    sc, _ = scene_small(8, 400)
    sc.scale *= np.float32(3.0)
    cam = Camera(40, 40, 40.0, 40.0, 20.0, 20.0)
    prm = O.Params(sc)
    c64 = O.CamF64(cam)
    idx = torch.arange(sc.n)
    rng = np.random.default_rng(2)
    for x, y in rng.integers(0, 40, (12, 2)):
        cand, z = O.listfree_candidates(sc, cam, int(x), int(y))
        pe = O._eval_pairs(prm, c64, idx, torch.tensor([float(x)], dtype=F64), torch.tensor([float(y)], dtype=F64))
        hits = set(torch.nonzero(pe["hit"][0]).flatten().tolist())
        assert hits <= set(cand.tolist()), (x, y)
        assert np.all(np.diff(z) >= 0)
        assert len(cand) < sc.n


def test_listfree_matches_tile_lists_on_small_scene():
    """On the 1k scene, the list-free compositing equals the tile-list compositing at
    every sampled pixel (the tile lists lose nothing), up to its own branches."""
    sc, cam = scene_small(0, 1000)
    ref = O.render(sc, cam)
    rng = np.random.default_rng(3)
    pix = [(int(x), int(y)) for x, y in rng.integers(32, 96, (60, 2))]
    br = O.bracket_pixels(sc, cam, pix, list_free=True)
    covered = 0
    for (x, y), it in zip(pix, br):
        want = np.concatenate([ref["rgb"][:, y, x], [ref["alpha"][y, x], ref["depth"][y, x]], ref["normal"][:, y, x]])
        best = min(np.abs(O.pixel_vector(l, ()) - want).max() for l in it["leaves"])
        assert best < 1e-12, (x, y, best)
        covered += ref["alpha"][y, x] > 1e-3
    assert covered > 20
