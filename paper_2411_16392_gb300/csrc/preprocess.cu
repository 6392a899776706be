// Per-primitive preprocessing (forward and backward) of the quadric rasterizer.
//
// Forward (2048 primitives per CTA: an early exit for all of them, then the full recipe
// for the survivors, one thread each):
//   - camera-space centre, rotation R from the normalised quaternion and the
//     camera-from-local rotation W = R_cw R (the congruent transform of Sec. 3.2);
//   - the conservative screen bounds of the curved patch (supplementary, "Details of
//     Bounding Box Calculation", read with arc >= chord): a local support box clipped to
//     the near plane and projected, a screen parallelogram around it, and the screen
//     conic of the chord ellipsoid; the 16x16 tile rectangle and the 32-bit depth key
//     (supplementary, per-tile sorting);
//   - degree-3 SH colour (Sec. 3.1) from bfloat16 coefficients, evaluated in FP32;
//   - the 128-byte projected-state record read by the compositing kernels.
// The centre depth, the box, the screen bounds and the tile rectangle are computed with
// correctly rounded FP32 operations only (__fmul_rn, __fadd_rn, __fdiv_rn, __frcp_rn,
// __fsqrt_rn), each in a fixed order, so that the tile lists and keys are reproducible bit
// for bit by an independent implementation of the same recipe. The tile-count pass
// (k_count_tiles) keeps the tiles of each rectangle that meet both screen bounds.
//
// Backward (one thread per primitive): chain rule from the per-primitive gradient
// record accumulated by the compositing backward to mean, quaternion, scales,
// curvatures, opacity and SH coefficients.
#include "qgs_internal.cuh"

namespace qgs {

namespace {

__device__ __forceinline__ float bf16_to_f32(uint16_t b) {
  return __uint_as_float(((uint32_t)b) << 16);
}

// Real SH normalisation constants (degree <= 3) in the 3DGS sign convention.
__device__ __constant__ float kSH0 = 0.28209479177387814f;
__device__ __constant__ float kSH1 = 0.4886025119029199f;
__device__ __constant__ float kSH2[5] = {1.0925484305920792f, -1.0925484305920792f, 0.31539156525252005f,
                                        -1.0925484305920792f, 0.5462742152960396f};
__device__ __constant__ float kSH3[7] = {-0.5900435899266435f, 2.890611442640554f, -0.4570457994644658f,
                                        0.3731763325901154f, -0.4570457994644658f, 1.445305721320277f,
                                        -0.5900435899266435f};

__device__ __forceinline__ void sh_basis16(float x, float y, float z, float Y[16]) {
  float xx = x * x, yy = y * y, zz = z * z;
  Y[0] = kSH0;
  Y[1] = -kSH1 * y;
  Y[2] = kSH1 * z;
  Y[3] = -kSH1 * x;
  Y[4] = kSH2[0] * x * y;
  Y[5] = kSH2[1] * y * z;
  Y[6] = kSH2[2] * (2.f * zz - xx - yy);
  Y[7] = kSH2[3] * x * z;
  Y[8] = kSH2[4] * (xx - yy);
  Y[9] = kSH3[0] * y * (3.f * xx - yy);
  Y[10] = kSH3[1] * x * y * z;
  Y[11] = kSH3[2] * y * (4.f * zz - xx - yy);
  Y[12] = kSH3[3] * z * (2.f * zz - 3.f * xx - 3.f * yy);
  Y[13] = kSH3[4] * x * (4.f * zz - xx - yy);
  Y[14] = kSH3[5] * z * (xx - yy);
  Y[15] = kSH3[6] * x * (xx - 3.f * yy);
}

// Gradient of each basis function with respect to the (unnormalised-use) direction
// components, written out from the polynomials above.
__device__ __forceinline__ void sh_basis16_grad(float x, float y, float z, float gx[16], float gy[16],
                                                float gz[16]) {
  float xx = x * x, yy = y * y, zz = z * z;
  gx[0] = gy[0] = gz[0] = 0.f;
  gx[1] = 0.f; gy[1] = -kSH1; gz[1] = 0.f;
  gx[2] = 0.f; gy[2] = 0.f; gz[2] = kSH1;
  gx[3] = -kSH1; gy[3] = 0.f; gz[3] = 0.f;
  gx[4] = kSH2[0] * y; gy[4] = kSH2[0] * x; gz[4] = 0.f;
  gx[5] = 0.f; gy[5] = kSH2[1] * z; gz[5] = kSH2[1] * y;
  gx[6] = -2.f * kSH2[2] * x; gy[6] = -2.f * kSH2[2] * y; gz[6] = 4.f * kSH2[2] * z;
  gx[7] = kSH2[3] * z; gy[7] = 0.f; gz[7] = kSH2[3] * x;
  gx[8] = 2.f * kSH2[4] * x; gy[8] = -2.f * kSH2[4] * y; gz[8] = 0.f;
  gx[9] = 6.f * kSH3[0] * x * y; gy[9] = kSH3[0] * (3.f * xx - 3.f * yy); gz[9] = 0.f;
  gx[10] = kSH3[1] * y * z; gy[10] = kSH3[1] * x * z; gz[10] = kSH3[1] * x * y;
  gx[11] = -2.f * kSH3[2] * x * y; gy[11] = kSH3[2] * (4.f * zz - xx - 3.f * yy); gz[11] = 8.f * kSH3[2] * y * z;
  gx[12] = -6.f * kSH3[3] * x * z; gy[12] = -6.f * kSH3[3] * y * z; gz[12] = kSH3[3] * (6.f * zz - 3.f * xx - 3.f * yy);
  gx[13] = kSH3[4] * (4.f * zz - 3.f * xx - yy); gy[13] = -2.f * kSH3[4] * x * y; gz[13] = 8.f * kSH3[4] * x * z;
  gx[14] = 2.f * kSH3[5] * x * z; gy[14] = -2.f * kSH3[5] * y * z; gz[14] = kSH3[5] * (xx - yy);
  gx[15] = kSH3[6] * (3.f * xx - 3.f * yy); gy[15] = -6.f * kSH3[6] * x * y; gz[15] = 0.f;
}

// Rotation matrix (local -> world, row-major R[3*i + j]) of the normalised quaternion,
// correctly rounded FP32 in a fixed order (the bit-exact recipe).
__device__ __forceinline__ bool quat_rot_exact(float qw, float qx, float qy, float qz, float R[9]) {
  float n2 = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(qw, qw), __fmul_rn(qx, qx)), __fmul_rn(qy, qy)),
                       __fmul_rn(qz, qz));
  if (!(n2 > 0.f)) return false;
  float r = __fsqrt_rn(n2);
  float w = __fdiv_rn(qw, r), x = __fdiv_rn(qx, r), y = __fdiv_rn(qy, r), z = __fdiv_rn(qz, r);
  R[0] = __fsub_rn(1.f, __fmul_rn(2.f, __fadd_rn(__fmul_rn(y, y), __fmul_rn(z, z))));
  R[1] = __fmul_rn(2.f, __fsub_rn(__fmul_rn(x, y), __fmul_rn(w, z)));
  R[2] = __fmul_rn(2.f, __fadd_rn(__fmul_rn(x, z), __fmul_rn(w, y)));
  R[3] = __fmul_rn(2.f, __fadd_rn(__fmul_rn(x, y), __fmul_rn(w, z)));
  R[4] = __fsub_rn(1.f, __fmul_rn(2.f, __fadd_rn(__fmul_rn(x, x), __fmul_rn(z, z))));
  R[5] = __fmul_rn(2.f, __fsub_rn(__fmul_rn(y, z), __fmul_rn(w, x)));
  R[6] = __fmul_rn(2.f, __fsub_rn(__fmul_rn(x, z), __fmul_rn(w, y)));
  R[7] = __fmul_rn(2.f, __fadd_rn(__fmul_rn(y, z), __fmul_rn(w, x)));
  R[8] = __fsub_rn(1.f, __fmul_rn(2.f, __fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y))));
  return true;
}

// Projected points of the support box: their pixel AABB and their spans along the two
// directions of a screen-space parallelogram.
struct Box2 {
  float xmin, xmax, ymin, ymax;
  bool any;
  float n1x, n1y, n2x, n2y, pcx, pcy;   // parallelogram directions, projected centre
  float s1min, s1max, s2min, s2max;
};

// Pixel AABB and parallelogram spans of the projected points (all bit-exact: the tile
// lists depend on them).
__device__ __forceinline__ void box_add(Box2& b, const CamParams& cp, float px, float py, float pz) {
  float u = __fadd_rn(__fmul_rn(cp.fx, __fdiv_rn(px, pz)), cp.cx);
  float v = __fadd_rn(__fmul_rn(cp.fy, __fdiv_rn(py, pz)), cp.cy);
  b.xmin = fminf(b.xmin, u);
  b.xmax = fmaxf(b.xmax, u);
  b.ymin = fminf(b.ymin, v);
  b.ymax = fmaxf(b.ymax, v);
  b.any = true;
  const float du = __fsub_rn(u, b.pcx), dv = __fsub_rn(v, b.pcy);
  const float t1 = __fadd_rn(__fmul_rn(b.n1x, du), __fmul_rn(b.n1y, dv));
  const float t2 = __fadd_rn(__fmul_rn(b.n2x, du), __fmul_rn(b.n2y, dv));
  b.s1min = fminf(b.s1min, t1);
  b.s1max = fmaxf(b.s1max, t1);
  b.s2min = fminf(b.s2min, t2);
  b.s2max = fmaxf(b.s2max, t2);
}

// Unit normal (in pixels) of the projection of the camera-space direction r at the
// centre mu: the screen direction of a local axis, turned by 90 degrees (bit-exact).
__device__ __forceinline__ void screen_normal(const CamParams& cp, const float* muc, float rx, float ry, float rz,
                                              float& nx, float& ny) {
  const float z = muc[2];
  const float du = __fmul_rn(cp.fx, __fsub_rn(__fmul_rn(rx, z), __fmul_rn(muc[0], rz)));
  const float dv = __fmul_rn(cp.fy, __fsub_rn(__fmul_rn(ry, z), __fmul_rn(muc[1], rz)));
  const float l2 = __fadd_rn(__fmul_rn(du, du), __fmul_rn(dv, dv));
  if (l2 > 0.f && isfinite(l2)) {
    const float l = __fsqrt_rn(l2);
    nx = -__fdiv_rn(dv, l);
    ny = __fdiv_rn(du, l);
  } else {
    nx = 1.f;
    ny = 0.f;
  }
}

// Screen-space conic of the chord ellipsoid x^2/s_u^2 + y^2/s_v^2 + z^2/m^2 <= 9 that holds
// the support (arc >= chord): the pixels whose ray line meets it, as
// F(p) = p^T q p - 2 l.p <= 1 for the offset p from the projected centre. With the frame
// scaled by S = diag(s_u, s_v, m), the line meets the ball iff |omega x delta|^2 <=
// kappa |delta|^2 (omega: camera, delta: direction); the cross product is formed as
// S W^T (e x mu_c) / (s_u s_v m), free of the camera distance. Pads: kappa = 9.02, the
// diagonal of q lowered by 4e-6 of its trace, the threshold raised for a 2e-3 px rim.
// Disabled (every pixel passes) unless the padded form is positive definite. Correctly
// rounded FP32 in a fixed order: the tile test built on it is reproduced bit for bit by
// the oracle's recipe.
struct Conic {
  float qa, qb, qc, la, lb, iqa, iqc;
  bool on;
};
__device__ __forceinline__ float dot3_rn(const float* u, const float* v) {
  return __fadd_rn(__fadd_rn(__fmul_rn(u[0], v[0]), __fmul_rn(u[1], v[1])), __fmul_rn(u[2], v[2]));
}
__device__ __forceinline__ Conic ellipsoid_conic(const float* muc, const float* W, float su, float sv, float m,
                                                 float fx, float fy) {
  const float ifx = __frcp_rn(fx), ify = __frcp_rn(fy);
  const float isu = __frcp_rn(su), isv = __frcp_rn(sv), im = __frcp_rn(m);
  const float rs[3] = {isu, isv, im};                                                // 1 / s_c
  const float ro[3] = {__fmul_rn(isv, im), __fmul_rn(isu, im), __fmul_rn(isu, isv)};  // s_c / (s_u s_v m)
  const float dcx = __fdiv_rn(muc[0], muc[2]), dcy = __fdiv_rn(muc[1], muc[2]);
  float nx[3], ny[3], hx[3], hy[3], dc[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    nx[c] = __fmul_rn(__fmul_rn(__fsub_rn(__fmul_rn(W[6 + c], muc[1]), __fmul_rn(W[3 + c], muc[2])), ifx), ro[c]);
    ny[c] = __fmul_rn(__fmul_rn(__fsub_rn(__fmul_rn(W[c], muc[2]), __fmul_rn(W[6 + c], muc[0])), ify), ro[c]);
    hx[c] = __fmul_rn(__fmul_rn(W[c], ifx), rs[c]);
    hy[c] = __fmul_rn(__fmul_rn(W[3 + c], ify), rs[c]);
    dc[c] = __fmul_rn(__fadd_rn(__fadd_rn(__fmul_rn(W[c], dcx), __fmul_rn(W[3 + c], dcy)), W[6 + c]), rs[c]);
  }
  const float kap = 9.02f;
  const float G00 = dot3_rn(nx, nx), G01 = dot3_rn(nx, ny), G11 = dot3_rn(ny, ny);
  const float H00 = dot3_rn(hx, hx), H01 = dot3_rn(hx, hy), H11 = dot3_rn(hy, hy);
  const float tau = __fmul_rn(4e-6f, __fadd_rn(G00, G11));
  const float Q00 = __fsub_rn(__fsub_rn(G00, __fmul_rn(kap, H00)), tau);
  const float Q01 = __fsub_rn(G01, __fmul_rn(kap, H01));
  const float Q11 = __fsub_rn(__fsub_rn(G11, __fmul_rn(kap, H11)), tau);
  const float L0 = __fmul_rn(kap, dot3_rn(dc, hx)), L1 = __fmul_rn(kap, dot3_rn(dc, hy));
  const float K = __fmul_rn(kap, dot3_rn(dc, dc));
  const float det = __fsub_rn(__fmul_rn(Q00, Q11), __fmul_rn(Q01, Q01));
  const float iK = __frcp_rn(K);
  const float qa = __fmul_rn(Q00, iK), qb = __fmul_rn(Q01, iK), qc = __fmul_rn(Q11, iK);
  const float la = __fmul_rn(L0, iK), lb = __fmul_rn(L1, iK);
  const float dn = __fsub_rn(__fmul_rn(qa, qc), __fmul_rn(qb, qb));
  // R = 1 + l^T q^-1 l (the ellipse is (p - p0)^T q (p - p0) <= R); growing it by dl
  // pixels raises F by at most 2 dl sqrt(lmax R) + dl^2 lmax, lmax <= qa + qc
  const float num = __fadd_rn(__fsub_rn(__fmul_rn(__fmul_rn(qc, la), la), __fmul_rn(__fmul_rn(2.f, __fmul_rn(qb, la)), lb)),
                              __fmul_rn(__fmul_rn(qa, lb), lb));
  const float R0 = __fadd_rn(1.f, __fdiv_rn(num, dn));
  const float R = R0 > 1.f ? R0 : 1.f;
  const float tr = __fadd_rn(qa, qc);
  const float dl = 2e-3f;
  const float T = __fadd_rn(__fadd_rn(1.f, __fmul_rn(__fmul_rn(3.f, dl), __fsqrt_rn(__fmul_rn(tr, R)))),
                            __fmul_rn(__fmul_rn(__fmul_rn(2.f, dl), dl), tr));
  const float iT = __frcp_rn(T);
  bool on = isfinite(Q00) && isfinite(Q01) && isfinite(Q11) && isfinite(L0) && isfinite(L1) && isfinite(K) &&
            K > 0.f && Q00 > 0.f && Q11 > 0.f && det > __fmul_rn(1e-6f, __fmul_rn(Q00, Q11)) && isfinite(T) &&
            dn > 0.f && isfinite(R0);
  Conic o;
  o.qa = __fmul_rn(qa, iT); o.qb = __fmul_rn(qb, iT); o.qc = __fmul_rn(qc, iT);
  o.la = __fmul_rn(la, iT); o.lb = __fmul_rn(lb, iT);
  o.iqa = __frcp_rn(o.qa); o.iqc = __frcp_rn(o.qc);
  on = on && isfinite(o.qa) && isfinite(o.qb) && isfinite(o.qc) && isfinite(o.la) && isfinite(o.lb) &&
       isfinite(o.iqa) && isfinite(o.iqc) && o.qa > 0.f && o.qc > 0.f;
  if (!on) o.qa = o.qb = o.qc = o.la = o.lb = o.iqa = o.iqc = 0.f;
  o.on = on;
  return o;
}

// Tile range (floor(x / 16) bounds) of the bounding box of the conic F(p) <= 1, i.e. of
// the ellipse (p - p0)^T q (p - p0) <= R with p0 = q^-1 l, R = 1 + l.p0 and half-extents
// sqrt(R (q^-1)_00), sqrt(R (q^-1)_11), around the projected centre (uc, vc). Correctly
// rounded FP32 in a fixed order (bit-exact with the oracle's recipe).
__device__ __forceinline__ float4 conic_box(const Conic& c, float uc, float vc) {
  const float dn = __fsub_rn(__fmul_rn(c.qa, c.qc), __fmul_rn(c.qb, c.qb));
  const float p0x = __fdiv_rn(__fsub_rn(__fmul_rn(c.qc, c.la), __fmul_rn(c.qb, c.lb)), dn);
  const float p0y = __fdiv_rn(__fsub_rn(__fmul_rn(c.qa, c.lb), __fmul_rn(c.qb, c.la)), dn);
  const float R = __fadd_rn(__fadd_rn(1.f, __fmul_rn(c.la, p0x)), __fmul_rn(c.lb, p0y));
  const float ex = __fsqrt_rn(__fdiv_rn(__fmul_rn(R, c.qc), dn));
  const float ey = __fsqrt_rn(__fdiv_rn(__fmul_rn(R, c.qa), dn));
  const float cx = __fadd_rn(uc, p0x), cy = __fadd_rn(vc, p0y);
  return make_float4(floorf(__fmul_rn(__fsub_rn(cx, ex), 0.0625f)), floorf(__fmul_rn(__fadd_rn(cx, ex), 0.0625f)),
                     floorf(__fmul_rn(__fsub_rn(cy, ey), 0.0625f)), floorf(__fmul_rn(__fadd_rn(cy, ey), 0.0625f)));
}

// s + e = a + b exactly (Knuth's two-sum), each operation rounded as written.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Row r of the camera-space centre R_cw mu + t_cw as an unevaluated sum hi + lo (about 44
// significant bits): the products' rounding errors by fma, the sums' by two-sum. The
// bit-exact FP32 centre of the binning recipe is rounded at every step (an error of a few
// units in the last place of |mu_c|, which is 1e-4 of a small primitive's size at the
// workloads' distances); the compositing measures pixel offsets from this one instead.
__device__ __forceinline__ void centre_cam_df(float mx, float my, float mz, const CamParams& cp, int r, float& hi,
                                              float& lo) {
  const float a = cp.Rc[3 * r], b = cp.Rc[3 * r + 1], c = cp.Rc[3 * r + 2];
  const float p0 = __fmul_rn(a, mx), e0 = __fmaf_rn(a, mx, -p0);
  const float p1 = __fmul_rn(b, my), e1 = __fmaf_rn(b, my, -p1);
  const float p2 = __fmul_rn(c, mz), e2 = __fmaf_rn(c, mz, -p2);
  float s1, w1, s2, w2, s3, w3;
  two_sum(p0, p1, s1, w1);
  two_sum(s1, p2, s2, w2);
  two_sum(s2, cp.tc[r], s3, w3);
  const float err = __fadd_rn(__fadd_rn(__fadd_rn(e0, e1), __fadd_rn(e2, w1)), __fadd_rn(w2, w3));
  hi = __fadd_rn(s3, err);
  lo = __fsub_rn(err, __fsub_rn(hi, s3));
}

// Projected centre f (x / z) + c as an unevaluated sum hi + lo of floats (about 44
// significant bits) from the double-float centre (x, z) = (xh + xl, zh + zl), by
// error-free transformations: the division's remainder by fma, the product's rounding
// error by fma, and a two-sum with the principal point.
__device__ __forceinline__ void centre_df(float xh, float xl, float zh, float zl, float f, float c, float& hi,
                                          float& lo) {
  const float qh = __fdiv_rn(xh, zh);
  // x/z - qh = ((xh - qh zh) + (xl - qh zl)) / z
  const float ql = __fdiv_rn(__fadd_rn(__fmaf_rn(-qh, zh, xh), __fsub_rn(xl, __fmul_rn(qh, zl))), zh);
  const float ph = f * qh;
  const float pl = fmaf(f, qh, -ph) + f * ql;    // f (qh + ql) = ph + pl
  const float sh = ph + c;                       // two-sum of ph and c
  const float bb = sh - ph;
  const float sl = ((ph - (sh - bb)) + (c - bb)) + pl;
  hi = sh + sl;
  lo = sl - (hi - sh);
}


}  // namespace

// Returns the primitive's tile count (0: culled).
__device__ __forceinline__ uint32_t preprocess_one(int64_t i, const SceneView& sc, const CamParams& cp,
                                                   PrimState* __restrict__ state, uint32_t* __restrict__ count,
                                                   uint32_t* __restrict__ zkey, uint32_t* __restrict__ idx,
                                                   short4* __restrict__ rect, uint32_t idx_base = 0,
                                                   TileSlab* __restrict__ tslab = nullptr);

// Camera-space centre of a primitive (bit-exact: correctly rounded, fixed order).
__device__ __forceinline__ void centre_cam(float mx, float my, float mz, const CamParams& cp, float muc[3]) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
    muc[r] = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(cp.Rc[3 * r], mx), __fmul_rn(cp.Rc[3 * r + 1], my)),
                                 __fmul_rn(cp.Rc[3 * r + 2], mz)),
                       cp.tc[r]);
}

// Early exit for primitives the full recipe culls anyway: centre not in front of the
// near plane, or the sphere that holds the support box (every corner lies within
// 3 sqrt(3) max(s_u, s_v) of the centre) entirely beyond one side plane of the image
// (then every projected box point, near-plane points included, falls outside it). The
// sphere is enlarged by 1 % + 1e-6 |mu_c| against rounding, so no primitive the exact
// recipe keeps is dropped.
__device__ __forceinline__ bool may_survive(const float muc[3], float2 s, const CamParams& cp) {
  const float rad = 5.1961524f * fmaxf(s.x, s.y) * 1.01f + 1e-6f * (fabsf(muc[0]) + fabsf(muc[1]) + fabsf(muc[2]));
  const float x = muc[0], y = muc[1], z = muc[2];
  const float rx = (float)cp.W - cp.cx, ry = (float)cp.H - cp.cy;
  const bool outside = !(z > cp.near) || -(cp.fx * x + cp.cx * z) > rad * sqrtf(cp.fx * cp.fx + cp.cx * cp.cx) ||
                       (cp.fx * x - rx * z) > rad * sqrtf(cp.fx * cp.fx + rx * rx) ||
                       -(cp.fy * y + cp.cy * z) > rad * sqrtf(cp.fy * cp.fy + cp.cy * cp.cy) ||
                       (cp.fy * y - ry * z) > rad * sqrtf(cp.fy * cp.fy + ry * ry);
  return !outside;
}

// One CTA preprocesses kPreChunks x 256 consecutive primitives in two phases: the early
// exit for all of them (culled ones get their empty entries), then the full recipe for
// the survivors gathered in shared memory, so that the expensive phase runs on full warps
// although only a small fraction of a large scene survives. Returns, for the calling
// thread, the visible count and tile total of the survivors it handled.
__device__ __forceinline__ void preprocess_block(int64_t n, const SceneView& sc, const CamParams& cp,
                                                 PrimState* __restrict__ state, uint32_t* __restrict__ count,
                                                 uint32_t* __restrict__ zkey, uint32_t* __restrict__ idx,
                                                 short4* __restrict__ rect, uint32_t idx_base,
                                                 TileSlab* __restrict__ tslab, uint32_t* __restrict__ vflag,
                                                 uint32_t& vis, uint32_t& tot) {
  __shared__ uint32_t list[kPreChunks * 256];
  __shared__ uint32_t nlist;
  if (threadIdx.x == 0) nlist = 0;
  __syncthreads();
  const int64_t first = (int64_t)blockIdx.x * (kPreChunks * 256);
  const int lane = threadIdx.x & 31;
  // every chunk's centre and scales in flight at once, then the tests
  float cm[kPreChunks][3];
  float2 cs[kPreChunks];
#pragma unroll
  for (int c = 0; c < kPreChunks; ++c) {
    const int64_t i = first + c * 256 + threadIdx.x;
    if (i < n) {
      cm[c][0] = __ldg(sc.mean + 3 * i);
      cm[c][1] = __ldg(sc.mean + 3 * i + 1);
      cm[c][2] = __ldg(sc.mean + 3 * i + 2);
      cs[c] = __ldg(reinterpret_cast<const float2*>(sc.scale) + i);
    }
  }
#pragma unroll
  for (int c = 0; c < kPreChunks; ++c) {
    const int64_t i = first + c * 256 + threadIdx.x;
    bool keep = false;
    if (i < n) {
      float muc[3];
      centre_cam(cm[c][0], cm[c][1], cm[c][2], cp, muc);
      keep = may_survive(muc, cs[c], cp);
      if (!keep) {
        if (idx) idx[i] = idx_base + (uint32_t)i;
        count[i] = 0u;
        zkey[i] = 0xFFFFFFFFu;
        rect[i] = make_short4(-1, -1, -1, -1);
        if (vflag) vflag[i] = 0u;
      }
    }
    const uint32_t m = __ballot_sync(0xffffffffu, keep);
    uint32_t slot = 0;
    if (lane == 0 && m) slot = atomicAdd(&nlist, (uint32_t)__popc(m));
    slot = __shfl_sync(0xffffffffu, slot, 0);
    if (keep) list[slot + __popc(m & ((1u << lane) - 1u))] = (uint32_t)(i - first);
  }
  __syncthreads();
  const uint32_t nl = nlist;
  vis = tot = 0;
  for (uint32_t t = threadIdx.x; t < nl; t += 256) {
    const int64_t i = first + list[t];
    const uint32_t cnt = preprocess_one(i, sc, cp, state, count, zkey, idx, rect, idx_base, tslab);
    if (vflag) vflag[i] = cnt ? 1u : 0u;
    vis += cnt ? 1u : 0u;
    tot += cnt;
  }
}

__global__ void __launch_bounds__(256) k_preprocess(int64_t n, SceneView sc, CamParams cp, PrimState* __restrict__ state,
                                                    uint32_t* __restrict__ count, uint32_t* __restrict__ zkey,
                                                    uint32_t* __restrict__ idx, short4* __restrict__ rect,
                                                    uint32_t* __restrict__ counters, uint32_t* __restrict__ vflag,
                                                    TileSlab* __restrict__ tslab) {
  uint32_t vis, tot;
  preprocess_block(n, sc, cp, state, count, zkey, idx, rect, 0, tslab, vflag, vis, tot);
  if (!counters) return;
  // one atomic per CTA and counter (per-warp atomics on two addresses serialise)
  __shared__ uint32_t red[2][8];
  vis = __reduce_add_sync(0xffffffffu, vis);
  tot = __reduce_add_sync(0xffffffffu, tot);
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = vis;
    red[1][threadIdx.x >> 5] = tot;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    uint32_t t = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += red[threadIdx.x][w];
    if (t) atomicAdd(&counters[threadIdx.x], t);
  }
}

// Several views (blockIdx.y) of one scene: entry v*n + i of every per-primitive array.
__global__ void __launch_bounds__(256) k_preprocess_views(int64_t n, SceneView sc, const CamParams* __restrict__ cps,
                                                          PrimState* __restrict__ state, uint32_t* __restrict__ count,
                                                          uint32_t* __restrict__ zkey, uint32_t* __restrict__ idx,
                                                          short4* __restrict__ rect, uint32_t* __restrict__ n_visible,
                                                          TileSlab* __restrict__ tslab) {
  const int64_t off = (int64_t)blockIdx.y * n;
  const CamParams cp = cps[blockIdx.y];
  uint32_t vis, tot;
  preprocess_block(n, sc, cp, state + off, count + off, zkey + off, idx + off, rect + off, (uint32_t)off,
                   tslab ? tslab + off : nullptr, nullptr, vis, tot);
  if (!n_visible) return;
  vis = __reduce_add_sync(0xffffffffu, vis);
  __shared__ uint32_t red[8];  // one atomic per CTA
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = vis;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += red[w];
    if (t) atomicAdd(n_visible, t);
  }
}

__device__ __forceinline__ uint32_t preprocess_one(int64_t i, const SceneView& sc, const CamParams& cp,
                                                   PrimState* __restrict__ state, uint32_t* __restrict__ count,
                                                   uint32_t* __restrict__ zkey, uint32_t* __restrict__ idx,
                                                   short4* __restrict__ rect, uint32_t idx_base,
                                                   TileSlab* __restrict__ tslab) {
  if (idx) idx[i] = idx_base + (uint32_t)i;
  const float mx = sc.mean[3 * i], my = sc.mean[3 * i + 1], mz = sc.mean[3 * i + 2];
  const float2 s = reinterpret_cast<const float2*>(sc.scale)[i];

  uint32_t cnt = 0;
  short4 rc = make_short4(-1, -1, -1, -1);
  uint32_t key = 0xFFFFFFFFu;

  // --- bit-exact part: centre depth, box, tile rectangle -------------------------
  float muc[3];
  centre_cam(mx, my, mz, cp, muc);
  if (!may_survive(muc, s, cp)) {
    count[i] = 0u;
    zkey[i] = 0xFFFFFFFFu;
    rect[i] = rc;
    return 0u;
  }
  const float4 q = reinterpret_cast<const float4*>(sc.quat)[i];
  const float2 ab = reinterpret_cast<const float2*>(sc.curv)[i];
  const float op = sc.opacity[i];
  float R[9], W[9];
  bool finite_in = isfinite(mx) && isfinite(my) && isfinite(mz) && isfinite(q.x) && isfinite(q.y) && isfinite(q.z) &&
                   isfinite(q.w) && isfinite(s.x) && isfinite(s.y) && isfinite(ab.x) && isfinite(ab.y) && isfinite(op);
  const float su2 = __fmul_rn(s.x, s.x), sv2 = __fmul_rn(s.y, s.y);
  bool ok = finite_in && quat_rot_exact(q.x, q.y, q.z, q.w, R) && s.x > 0.f && s.y > 0.f && su2 > 0.f &&
            sv2 > 0.f && muc[2] > cp.near;
  Box2 bx;
  Conic con{};
  bx.xmin = INFINITY; bx.xmax = -INFINITY; bx.ymin = INFINITY; bx.ymax = -INFINITY; bx.any = false;
  bx.s1min = INFINITY; bx.s1max = -INFINITY; bx.s2min = INFINITY; bx.s2max = -INFINITY;
  if (ok) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        W[3 * r + c] = __fadd_rn(__fadd_rn(__fmul_rn(cp.Rc[3 * r], R[c]), __fmul_rn(cp.Rc[3 * r + 1], R[3 + c])),
                                 __fmul_rn(cp.Rc[3 * r + 2], R[6 + c]));
    // box of the support from "arc >= chord": E + z^2/m^2 <= 9 (derivation in the oracle)
    const float su = s.x, sv = s.y, a = ab.x, b = ab.y;
    const float m = fmaxf(su, sv);
    const float ap = __fmul_rn(a, su2), bp = __fmul_rn(b, sv2);
    const float cpos = fmaxf(fmaxf(ap, bp), 0.f), cneg = fmaxf(fmaxf(-ap, -bp), 0.f);
    auto root = [&](float num, float c) {
      float t = __fdiv_rn(c, m);
      t = __fmul_rn(36.f, __fmul_rn(t, t));
      return __fdiv_rn(num, __fadd_rn(1.f, __fsqrt_rn(__fadd_rn(1.f, t))));
    };
    const float zmax = root(__fmul_rn(18.f, cpos), cpos);
    const float zmin = -root(__fmul_rn(18.f, cneg), cneg);
    const bool same = !((a > 0.f && b < 0.f) || (a < 0.f && b > 0.f));
    const float Xs = same ? root(__fmul_rn(18.f, su2), ap) : __fmul_rn(9.f, su2);
    const float Ys = same ? root(__fmul_rn(18.f, sv2), bp) : __fmul_rn(9.f, sv2);
    const float X = __fsqrt_rn(Xs), Y = __fsqrt_rn(Ys);
    // parallelogram directions: normals of the projected local x and y axes
    screen_normal(cp, muc, W[0], W[3], W[6], bx.n1x, bx.n1y);
    screen_normal(cp, muc, W[1], W[4], W[7], bx.n2x, bx.n2y);
    // reference point of the spans: the projected centre (bit-exact)
    bx.pcx = __fadd_rn(__fmul_rn(cp.fx, __fdiv_rn(muc[0], muc[2])), cp.cx);
    bx.pcy = __fadd_rn(__fmul_rn(cp.fy, __fdiv_rn(muc[1], muc[2])), cp.cy);
    con = ellipsoid_conic(muc, W, su, sv, m, cp.fx, cp.fy);
    float P[8][3];
    bool in[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float sx = (k & 1) ? X : -X, sy = (k & 2) ? Y : -Y, sz = (k & 4) ? zmax : zmin;
#pragma unroll
      for (int r = 0; r < 3; ++r)
        P[k][r] = __fadd_rn(__fadd_rn(__fadd_rn(muc[r], __fmul_rn(W[3 * r], sx)), __fmul_rn(W[3 * r + 1], sy)),
                            __fmul_rn(W[3 * r + 2], sz));
      in[k] = P[k][2] >= cp.near;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (in[k]) box_add(bx, cp, P[k][0], P[k][1], P[k][2]);
#pragma unroll
    for (int k0 = 0; k0 < 8; ++k0) {
#pragma unroll
      for (int bit = 1; bit <= 4; bit <<= 1) {
        if (k0 & bit) continue;
        const int k1 = k0 | bit;
        if (in[k0] != in[k1]) {
          const float lam = __fdiv_rn(__fsub_rn(cp.near, P[k0][2]), __fsub_rn(P[k1][2], P[k0][2]));
          const float ex = __fadd_rn(P[k0][0], __fmul_rn(lam, __fsub_rn(P[k1][0], P[k0][0])));
          const float ey = __fadd_rn(P[k0][1], __fmul_rn(lam, __fsub_rn(P[k1][1], P[k0][1])));
          box_add(bx, cp, ex, ey, cp.near);
        }
      }
    }
    ok = bx.any && isfinite(bx.xmin) && isfinite(bx.xmax) && isfinite(bx.ymin) && isfinite(bx.ymax) &&
         !(bx.xmax < 0.f || bx.ymax < 0.f || bx.xmin >= (float)cp.W || bx.ymin >= (float)cp.H);
    if (ok) {
      float tx0 = fmaxf(floorf(__fmul_rn(bx.xmin, 0.0625f)), 0.f);
      float tx1 = fminf(floorf(__fmul_rn(bx.xmax, 0.0625f)), (float)(cp.tiles_x - 1));
      float ty0 = fmaxf(floorf(__fmul_rn(bx.ymin, 0.0625f)), 0.f);
      float ty1 = fminf(floorf(__fmul_rn(bx.ymax, 0.0625f)), (float)(cp.tiles_y - 1));
      if (con.on) {  // only the tiles of the conic's bounding box can pass the conic test
        float4 cb = conic_box(con, bx.pcx, bx.pcy);
        tx0 = fmaxf(tx0, cb.x); tx1 = fminf(tx1, cb.y);
        ty0 = fmaxf(ty0, cb.z); ty1 = fminf(ty1, cb.w);
      }
      if (!(tx0 > tx1) && !(ty0 > ty1)) {
        rc = make_short4((short)tx0, (short)tx1, (short)ty0, (short)ty1);
        cnt = (uint32_t)((rc.y - rc.x + 1) * (rc.w - rc.z + 1));
        key = __float_as_uint(muc[2]);
      }
    }
  }
  count[i] = cnt;
  zkey[i] = key;
  rect[i] = rc;
  if (!cnt) return 0u;
  if (tslab) {
    TileSlab t;
    t.a = make_float4(bx.n1x, bx.n1y, bx.s1min, bx.s1max);
    t.b = make_float4(bx.n2x, bx.n2y, bx.s2min, bx.s2max);
    t.c = make_float4(bx.pcx, bx.pcy, con.qa, con.qb);
    t.d = make_float4(con.qc, con.la, con.lb, con.iqa);
    t.e = make_float4(con.iqc, 0.f, 0.f, 0.f);
    tslab[i] = t;
  }

  // --- projected state (ordinary FP32 arithmetic; FP64 is slow on this GPU) -------
  const float zmu = muc[2];
  const float iz = 1.f / zmu;
  float pcx_hi, pcx_lo, pcy_hi, pcy_lo, ch[3], cl[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) centre_cam_df(mx, my, mz, cp, r, ch[r], cl[r]);
  centre_df(ch[0], cl[0], ch[2], cl[2], cp.fx, cp.cx, pcx_hi, pcx_lo);
  centre_df(ch[1], cl[1], ch[2], cl[2], cp.fy, cp.cy, pcy_hi, pcy_lo);
  float g[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) g[c] = fmaf(W[c], muc[0], fmaf(W[3 + c], muc[1], W[6 + c] * zmu)) * iz;

  // colour: degree-3 SH at the direction from the camera centre to the primitive
  float dx = mx - cp.cw[0], dy = my - cp.cw[1], dz = mz - cp.cw[2];
  const float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
  dx *= inv; dy *= inv; dz *= inv;
  float Yb[16];
  sh_basis16(dx, dy, dz, Yb);
  float col[3] = {0.5f, 0.5f, 0.5f};
  const uint4* shp = reinterpret_cast<const uint4*>(sc.sh + 48 * i);
#pragma unroll
  for (int v = 0; v < 6; ++v) {
    const uint4 w4 = shp[v];
    const uint32_t wd[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
    for (int h = 0; h < 8; ++h) {
      const int e = 8 * v + h;  // element index k*3 + c
      const float cval = bf16_to_f32((uint16_t)((h & 1) ? (wd[h >> 1] >> 16) : (wd[h >> 1] & 0xFFFFu)));
      col[e % 3] = fmaf(Yb[e / 3], cval, col[e % 3]);
    }
  }
  PrimState ps;
  ps.f[0] = make_float4(con.qa, 2.f * con.qb, con.qc, 2.f * con.la);
  ps.f[1] = make_float4(pcx_hi, pcx_lo, pcy_hi, pcy_lo);
  ps.f[2] = make_float4(2.f * con.lb, 0.f, iz, zmu);
  ps.f[3] = make_float4(W[0], W[3], W[1], W[4]);
  ps.f[4] = make_float4(W[2], W[5], g[0], g[1]);
  ps.f[5] = make_float4(g[2], ab.x, ab.y, op);
  ps.f[6] = make_float4(1.f / (s.x * s.x), 1.f / (s.y * s.y), W[6], W[7]);
  ps.f[7] = make_float4(W[8], fmaxf(col[0], 0.f), fmaxf(col[1], 0.f), fmaxf(col[2], 0.f));
  state[i] = ps;
  return cnt;
}

__global__ void __launch_bounds__(128, 4) k_preprocess_bwd(int64_t n, const uint32_t* __restrict__ list, SceneView sc,
                                                        CamParams cp, const uint32_t* __restrict__ count,
                                                        const float* __restrict__ pgrad, bool pgrad_by_pos,
                                                        GradView gd) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int64_t i = list ? (int64_t)list[j] : j;
  if (count[i] == 0) return;
  const float* pg = pgrad + (size_t)NGRAD_PAD * (pgrad_by_pos ? j : i);
  float P[9], Hh[3];
#pragma unroll
  for (int k = 0; k < 9; ++k) P[k] = pg[k];
  Hh[0] = pg[9]; Hh[1] = pg[10]; Hh[2] = pg[11];
  const float d_a = pg[12], d_b = pg[13], d_iu = pg[14], d_iv = pg[15], d_o = pg[16];
  const float d_col[3] = {pg[17], pg[18], pg[19]};

  const float mx = sc.mean[3 * i], my = sc.mean[3 * i + 1], mz = sc.mean[3 * i + 2];
  const float4 q = reinterpret_cast<const float4*>(sc.quat)[i];
  const float2 s = reinterpret_cast<const float2*>(sc.scale)[i];
  const float qn = sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
  const float w = q.x / qn, x = q.y / qn, y = q.z / qn, z = q.w / qn;
  float R[9];
  R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z); R[2] = 2.f * (x * z + w * y);
  R[3] = 2.f * (x * y + w * z); R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
  R[6] = 2.f * (x * z - w * y); R[7] = 2.f * (y * z + w * x); R[8] = 1.f - 2.f * (x * x + y * y);
  float W[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      W[3 * r + c] = cp.Rc[3 * r] * R[c] + cp.Rc[3 * r + 1] * R[3 + c] + cp.Rc[3 * r + 2] * R[6 + c];
  // dL/dW = W P ; dL/dmu_cam = -W H
  float dW[9], dmuc[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
#pragma unroll
    for (int c = 0; c < 3; ++c) dW[3 * r + c] = W[3 * r] * P[c] + W[3 * r + 1] * P[3 + c] + W[3 * r + 2] * P[6 + c];
    dmuc[r] = -(W[3 * r] * Hh[0] + W[3 * r + 1] * Hh[1] + W[3 * r + 2] * Hh[2]);
  }
  // to world: dR = R_cw^T dW, dmu = R_cw^T dmu_cam
  float dR[9], dmu[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
#pragma unroll
    for (int c = 0; c < 3; ++c) dR[3 * r + c] = cp.Rc[r] * dW[c] + cp.Rc[3 + r] * dW[3 + c] + cp.Rc[6 + r] * dW[6 + c];
    dmu[r] = cp.Rc[r] * dmuc[0] + cp.Rc[3 + r] * dmuc[1] + cp.Rc[6 + r] * dmuc[2];
  }
  // rotation matrix -> normalised quaternion
  const float gw = 2.f * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
  const float gx = 2.f * (y * dR[1] + z * dR[2] + y * dR[3] - 2.f * x * dR[4] - w * dR[5] + z * dR[6] + w * dR[7] -
                          2.f * x * dR[8]);
  const float gy = 2.f * (-2.f * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] + z * dR[7] -
                          2.f * y * dR[8]);
  const float gz = 2.f * (-2.f * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.f * z * dR[4] + y * dR[5] +
                          x * dR[6] + y * dR[7]);
  // normalisation q_hat = q / |q|
  const float dotq = w * gw + x * gx + y * gy + z * gz;
  const float iqn = 1.f / qn;

  // colour: SH backward through the clamp at 0 and the view direction
  float ddx = mx - cp.cw[0], ddy = my - cp.cw[1], ddz = mz - cp.cw[2];
  const float dn = sqrtf(ddx * ddx + ddy * ddy + ddz * ddz);
  const float idn = 1.f / dn;
  const float vx = ddx * idn, vy = ddy * idn, vz = ddz * idn;
  float Yb[16];
  sh_basis16(vx, vy, vz, Yb);
  float shv[48];
  const uint4* shp = reinterpret_cast<const uint4*>(sc.sh + 48 * i);
#pragma unroll
  for (int v = 0; v < 6; ++v) {
    const uint4 w4 = shp[v];
    const uint32_t wd[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
    for (int h = 0; h < 8; ++h)
      shv[8 * v + h] = bf16_to_f32((uint16_t)((h & 1) ? (wd[h >> 1] >> 16) : (wd[h >> 1] & 0xFFFFu)));
  }
  float dc[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float v = 0.5f;
#pragma unroll
    for (int k = 0; k < 16; ++k) v = fmaf(Yb[k], shv[3 * k + c], v);
    dc[c] = v < 0.f ? 0.f : d_col[c];
  }
  float4* gsh = reinterpret_cast<float4*>(gd.sh + 48 * i);
#pragma unroll
  for (int v = 0; v < 12; ++v) {
    float4 g4 = gsh[v];
    float* gg = reinterpret_cast<float*>(&g4);
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const int e = 4 * v + h;
      gg[h] += Yb[e / 3] * dc[e % 3];
    }
    gsh[v] = g4;
  }
  float Gx[16], Gy[16], Gz[16];
  sh_basis16_grad(vx, vy, vz, Gx, Gy, Gz);
  float gvx = 0.f, gvy = 0.f, gvz = 0.f;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const float t = dc[0] * shv[3 * k] + dc[1] * shv[3 * k + 1] + dc[2] * shv[3 * k + 2];
    gvx = fmaf(t, Gx[k], gvx);
    gvy = fmaf(t, Gy[k], gvy);
    gvz = fmaf(t, Gz[k], gvz);
  }
  const float vd = vx * gvx + vy * gvy + vz * gvz;
  dmu[0] += (gvx - vx * vd) * idn;
  dmu[1] += (gvy - vy * vd) * idn;
  dmu[2] += (gvz - vz * vd) * idn;

  gd.mean[3 * i] += dmu[0];
  gd.mean[3 * i + 1] += dmu[1];
  gd.mean[3 * i + 2] += dmu[2];
  float4 gq = reinterpret_cast<float4*>(gd.quat)[i];
  gq.x += (gw - w * dotq) * iqn;
  gq.y += (gx - x * dotq) * iqn;
  gq.z += (gy - y * dotq) * iqn;
  gq.w += (gz - z * dotq) * iqn;
  reinterpret_cast<float4*>(gd.quat)[i] = gq;
  float2 gs = reinterpret_cast<float2*>(gd.scale)[i];
  gs.x += d_iu * (-2.f / (s.x * s.x * s.x));
  gs.y += d_iv * (-2.f / (s.y * s.y * s.y));
  reinterpret_cast<float2*>(gd.scale)[i] = gs;
  float2 gc = reinterpret_cast<float2*>(gd.curv)[i];
  gc.x += d_a;
  gc.y += d_b;
  reinterpret_cast<float2*>(gd.curv)[i] = gc;
  gd.opacity[i] += d_o;
}

// ---------------------------------------------------------------------------------------
// StopThePop ordering (supplementary, "Details of Per-tile Sorting and Per-pixel
// Resorting"): one key per (tile, primitive) instance, (tile << 32) | float bits of the
// depth where the ray of the tile pixel closest to the projected vertex meets the
// paraboloid. Correctly rounded FP32 in the order below (the same specification as the
// oracle's FP32 key recipe); the ray is re-based at the centre's depth so the quadratic's
// coefficients have the size of the primitive. Instances in primitive order, tiles
// row-major, values = primitive (a stable sort of the keys then orders each tile's list
// by that depth, ties by primitive index).
namespace {

__device__ __forceinline__ void frame_exact(int64_t i, const SceneView& sc, const CamParams& cp, float muc[3],
                                            float W[9]) {
  const float mx = sc.mean[3 * i], my = sc.mean[3 * i + 1], mz = sc.mean[3 * i + 2];
  const float4 q = reinterpret_cast<const float4*>(sc.quat)[i];
#pragma unroll
  for (int r = 0; r < 3; ++r)
    muc[r] = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(cp.Rc[3 * r], mx), __fmul_rn(cp.Rc[3 * r + 1], my)),
                                 __fmul_rn(cp.Rc[3 * r + 2], mz)),
                       cp.tc[r]);
  float R[9];
  quat_rot_exact(q.x, q.y, q.z, q.w, R);  // visible primitives only: the norm is positive
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      W[3 * r + c] = __fadd_rn(__fadd_rn(__fmul_rn(cp.Rc[3 * r], R[c]), __fmul_rn(cp.Rc[3 * r + 1], R[3 + c])),
                               __fmul_rn(cp.Rc[3 * r + 2], R[6 + c]));
}

__device__ __forceinline__ uint32_t hit_key_bits(const float muc[3], const float W[9], float a, float b, float uc,
                                                 float vc, int tx, int ty, const CamParams& cp) {
  const float x = muc[0], y = muc[1], z = muc[2];
  const float px = fminf(fmaxf(floorf(uc), (float)(16 * tx)), (float)min(16 * tx + 15, cp.W - 1));
  const float py = fminf(fmaxf(floorf(vc), (float)(16 * ty)), (float)min(16 * ty + 15, cp.H - 1));
  const float dx = __fdiv_rn(__fsub_rn(__fadd_rn(px, 0.5f), cp.cx), cp.fx);
  const float dy = __fdiv_rn(__fsub_rn(__fadd_rn(py, 0.5f), cp.cy), cp.fy);
  const float ex = __fsub_rn(__fmul_rn(dx, z), x);
  const float ey = __fsub_rn(__fmul_rn(dy, z), y);
  float bk[3], dk[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    bk[k] = __fadd_rn(__fmul_rn(W[k], ex), __fmul_rn(W[3 + k], ey));
    dk[k] = __fadd_rn(__fadd_rn(__fmul_rn(W[k], dx), __fmul_rn(W[3 + k], dy)), W[6 + k]);
  }
  const float A = __fadd_rn(__fmul_rn(__fmul_rn(a, dk[0]), dk[0]), __fmul_rn(__fmul_rn(b, dk[1]), dk[1]));
  const float Bh = __fsub_rn(__fadd_rn(__fmul_rn(__fmul_rn(a, bk[0]), dk[0]), __fmul_rn(__fmul_rn(b, bk[1]), dk[1])),
                             __fmul_rn(0.5f, dk[2]));
  const float C = __fsub_rn(__fadd_rn(__fmul_rn(__fmul_rn(a, bk[0]), bk[0]), __fmul_rn(__fmul_rn(b, bk[1]), bk[1])),
                            bk[2]);
  const float D = __fsub_rn(__fmul_rn(Bh, Bh), __fmul_rn(A, C));
  const float sq = __fsqrt_rn(fmaxf(D, 0.f));
  const float q = -__fadd_rn(Bh, Bh >= 0.f ? sq : -sq);
  const float t1 = __fadd_rn(z, __fdiv_rn(C, q));
  const float t2 = __fadd_rn(z, __fdiv_rn(q, A));
  const bool ok1 = D >= 0.f && isfinite(t1) && t1 > cp.near;
  const bool ok2 = D >= 0.f && isfinite(t2) && t2 > cp.near;
  const float t = (ok1 && ok2) ? fminf(t1, t2) : (ok1 ? t1 : (ok2 ? t2 : z));
  return __float_as_uint(t);
}

}  // namespace

__global__ void __launch_bounds__(256, 4) k_emit_hit(int64_t n, SceneView sc, CamParams cp,
                                                  const uint32_t* __restrict__ count,
                                                  const short4* __restrict__ rect,
                                                  const TileSlab* __restrict__ tslab,
                                                  const uint32_t* __restrict__ offs, uint64_t* __restrict__ keys,
                                                  uint32_t* __restrict__ vals, const uint32_t* __restrict__ tbits,
                                                  const uint32_t* __restrict__ tbits_off) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t wbase = i - lane;
  const uint32_t c = i < n ? count[i] : 0u;
  for (int k = 0; k < 32; ++k) {
    const uint32_t cc = __shfl_sync(0xffffffffu, c, k);
    if (!cc) continue;
    const int64_t p = wbase + k;  // every lane recomputes the primitive's frame (broadcast loads)
    float muc[3], W[9];
    frame_exact(p, sc, cp, muc, W);
    const float2 ab = reinterpret_cast<const float2*>(sc.curv)[p];
    const float uc = __fadd_rn(__fmul_rn(cp.fx, __fdiv_rn(muc[0], muc[2])), cp.cx);
    const float vc = __fadd_rn(__fmul_rn(cp.fy, __fdiv_rn(muc[1], muc[2])), cp.cy);
    const uint32_t off = offs[p];
    const uint32_t wo = tbits ? tbits_off[p] : kNoTileBits;
    warp_tiles(rect[p], tslab ? tslab + p : nullptr, cp.W, cp.H, [&](uint32_t e, int tx, int ty) {
      const uint32_t tile = (uint32_t)ty * (uint32_t)cp.tiles_x + (uint32_t)tx;
      keys[(size_t)off + e] = ((uint64_t)tile << 32) | hit_key_bits(muc, W, ab.x, ab.y, uc, vc, tx, ty, cp);
      vals[(size_t)off + e] = (uint32_t)p;
    }, nullptr, wo != kNoTileBits ? tbits + wo : nullptr);
  }
}

__global__ void __launch_bounds__(kCountBlock) k_count_tiles(int64_t n, const TileSlab* __restrict__ tslab, int W, int H,
                                                     uint32_t* __restrict__ count, short4* __restrict__ rect,
                                                     uint32_t* __restrict__ zkey, uint32_t* __restrict__ vflag,
                                                     uint32_t* __restrict__ counters, uint32_t* __restrict__ tbits,
                                                     uint32_t* __restrict__ tbits_off, uint32_t cap_words,
                                                     const CamParams* __restrict__ cps) {
  if (cps) {  // several views (blockIdx.y): entries v * n + i, the view's image size
    const int64_t off = (int64_t)blockIdx.y * n;
    tslab += off; count += off; rect += off; zkey += off;
    if (vflag) vflag += off;
    if (tbits_off) tbits_off += off;
    W = cps[blockIdx.y].W;
    H = cps[blockIdx.y].H;
  }
  __shared__ uint32_t bsum[2], bdone;
  if (threadIdx.x == 0) {
    bsum[0] = bsum[1] = 0u;
    bdone = 0u;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t c0 = i < n ? count[i] : 0u;
  // words of pass masks for the warp's 32 primitives: one atomic per warp
  uint32_t woff = kNoTileBits;
  if (tbits) {
    const uint32_t words = (c0 + 31u) >> 5;
    uint32_t incl = words;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += y;
    }
    const uint32_t wtot = __shfl_sync(0xffffffffu, incl, 31);
    uint32_t wbase_words = 0;
    if (lane == 31 && wtot) wbase_words = atomicAdd(&counters[2], wtot);
    wbase_words = __shfl_sync(0xffffffffu, wbase_words, 31);
    const uint64_t end = (uint64_t)wbase_words + incl;
    if (words && end <= (uint64_t)cap_words) woff = (uint32_t)(end - words);
    if (i < n) tbits_off[i] = woff;
  }
  // the warp's rectangles and screen bounds, loaded up front (independent loads) and
  // handed out per primitive from registers and shared memory
  __shared__ TileSlab sts[kCountBlock];
  __shared__ float4 hoist[kCountBlock / 32][6 * kHoistMax];  // per warp: column and row terms
  short4 rc0 = make_short4(0, 0, 0, 0);
  if (c0) {
    rc0 = rect[i];
    const float4* src = reinterpret_cast<const float4*>(tslab + i);
    float4* dst = reinterpret_cast<float4*>(&sts[threadIdx.x]);
#pragma unroll
    for (int q = 0; q < (int)(sizeof(TileSlab) / 16); ++q) dst[q] = __ldg(src + q);
  }
  __syncwarp();
  const int rxy = (int)(((uint32_t)(uint16_t)rc0.y << 16) | (uint16_t)rc0.x);
  const int rzw = (int)(((uint32_t)(uint16_t)rc0.w << 16) | (uint16_t)rc0.z);
  uint32_t mine = 0;
  for (int k = 0; k < 32; ++k) {
    const uint32_t cc = __shfl_sync(0xffffffffu, c0, k);
    if (!cc) continue;
    const int a = __shfl_sync(0xffffffffu, rxy, k), b = __shfl_sync(0xffffffffu, rzw, k);
    const short4 rk = make_short4((short)(a & 0xFFFF), (short)(a >> 16), (short)(b & 0xFFFF), (short)(b >> 16));
    const uint32_t wo = __shfl_sync(0xffffffffu, woff, k);
    const uint32_t c = warp_tiles(rk, &sts[(threadIdx.x & ~31) + k], W, H, [](uint32_t, int, int) {},
                                  wo != kNoTileBits ? tbits + wo : nullptr, nullptr, hoist[threadIdx.x >> 5]);
    if (lane == k) mine = c;
  }
  if (i < n) {
    if (c0 && !mine) {  // the rectangle's tiles all miss the screen bounds
      rect[i] = make_short4(-1, -1, -1, -1);
      zkey[i] = 0xFFFFFFFFu;
    }
    count[i] = mine;
    if (vflag) vflag[i] = mine ? 1u : 0u;
  }
  // totals: summed per CTA in shared memory; the CTA's last warp to finish adds them to
  // global memory (no barrier: warps of a CTA finish at very different times here)
  const uint32_t vis = __reduce_add_sync(0xffffffffu, mine ? 1u : 0u);
  const uint32_t tot = __reduce_add_sync(0xffffffffu, mine);
  if (lane == 0) {
    if (vis) atomicAdd(&bsum[0], vis);
    if (tot) atomicAdd(&bsum[1], tot);
    __threadfence_block();
    if (atomicAdd(&bdone, 1u) == (blockDim.x >> 5) - 1) {
      const uint32_t v = atomicAdd(&bsum[0], 0u), t = atomicAdd(&bsum[1], 0u);
      if (v) atomicAdd(&counters[0], v);
      if (t) atomicAdd(&counters[1], t);
    }
  }
}

}  // namespace qgs
