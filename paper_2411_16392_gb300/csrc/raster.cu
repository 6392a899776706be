// Per-tile compositing of quadric Gaussian primitives: forward and backward.
//
// One CTA per 16x16 tile; the forward takes one thread per pixel (warps cover 8x4 pixel
// blocks), the backward two (warps cover 8x8 blocks, see k_raster_bwd). The
// tile's sorted primitive list is walked in batches of projected-state records staged in
// shared memory (256 in the forward, 64 in the two-pixel backward; one 128-byte line per
// primitive, gathered by 8 threads per record). Per (pixel, primitive) pair:
//   - the pixel's offset from the projected centre (double-float) is tested against the
//     screen conic of the chord ellipsoid x^2/s_u^2 + y^2/s_v^2 + z^2/m^2 <= 9 that holds
//     the support (arc >= chord): a pixel whose ray line misses it cannot have a hit;
//   - the pixel ray is expressed in the primitive's local frame relative to the point
//     where it crosses the depth of the primitive's centre (a translation of the ray
//     parameter t = z_mu + s); the pixel offset from the projected centre is formed in
//     double-float, so the local ray origin and the quadratic's coefficients stay of the
//     size of the primitive instead of the camera distance;
//   - ray-quadric intersection with z = a x^2 + b y^2 (supplementary, intersection Eq.),
//     roots from the cancellation-free form q = -(B' + sgn(B') sqrt(D')), s = C/q, q/A
//     (B' = B/2, D' = D/4), and an FP64 re-solve when |D| <= grazing_eps * B^2;
//   - near-then-far selection within 3 sigma(theta) (Sec. 3.2.1) via the trig-free form
//     l^2 / sigma(theta)^2 = F(u)^2 E, E = x^2/s_u^2 + y^2/s_v^2, u = 2 a(theta) rho,
//     F(u) = l / rho = (asinh(u)/u + sqrt(1 + u^2)) / 2 (geodesic Eq. and sigma Eq. of
//     Sec. 3.2); F >= sqrt(1 + u^2/4) >= 1, so E > 9 and then E (1 + u^2/4) > 9 reject a
//     candidate before F is evaluated; F uses its Taylor series for |u| < 0.25;
//   - G = exp(-F^2 E / 2), alpha = min(alpha_max, o G), skip below alpha_min, stop before
//     the transmittance would fall below T_min (Sec. 3.1 blending Eq.);
//   - normal = gradient of the implicit function (Sec. 3.2 normal Eq.) in camera space,
//     facing the camera.
// The backward walks each pixel's list in reverse from its last blended primitive,
// recomputing T_i = T_{i+1} / (1 - alpha_i) (supplementary, back-to-front dX/d(alpha)),
// and differentiates through the implicit root, the geodesic weight and the normal.
// Per-primitive gradients are reduced across each warp with a butterfly reduce-scatter
// (21 shuffles for the 20 components), accumulated per batch in shared memory, and added
// to global memory once per (tile, primitive). The per-pair statistics counters are a
// template parameter (compiled out unless requested).
//
// Every operation that decides whether a pair contributes is written with explicitly
// rounded intrinsics, so the forward and the backward (which recomputes the pairs)
// take identical decisions.
#include "qgs_internal.cuh"

namespace qgs {

namespace {

constexpr unsigned FULL = 0xffffffffu;

struct Hit {
  float s;            // root offset: t = z_mu + s
  float x, y, zs;     // local hit point (zs = a x^2 + b y^2)
  float dx, dy, dz;   // local ray direction (camera-space ray with z component 1)
  float rho2, u, F2, E, G;  // F2 = F(u)^2: l^2 / sigma(theta)^2 = F2 * E
};

__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// F(u) = l(a, rho) / rho with u = 2 a rho: the arc-length closed form of Sec. 3.2 divided
// by rho, (asinh(u)/u + sqrt(1 + u^2)) / 2. For |u| < 0.25 its Taylor series
// 1 + u^2/6 - u^4/40 + u^6/112 - 5u^8/1152 + 7u^10/2816 (truncation < 1e-10 there; for
// |u| < 1e-3 only the first three terms matter in FP32); above, the closed form with
// asinh(|u|) = log(|u| + sqrt(1 + u^2)), well conditioned for |u| >= 0.25. Both are
// formed and one selected (no divergent branch where a warp's lanes fall on both sides).
__device__ __forceinline__ float arc_ratio(float u) {
  const float au = fabsf(u);
  const float u2 = __fmul_rn(u, u);
  float p = 7.f / 2816.f;
  p = __fmaf_rn(p, u2, -5.f / 1152.f);
  p = __fmaf_rn(p, u2, 1.f / 112.f);
  p = __fmaf_rn(p, u2, -0.025f);
  p = __fmaf_rn(p, u2, 1.f / 6.f);
  const float ft = __fmaf_rn(p, u2, 1.f);
  const float r = sqrt_approx(__fmaf_rn(au, au, 1.f));
  const float fl = __fmul_rn(0.5f, __fadd_rn(__fdividef(__logf(__fadd_rn(au, r)), au), r));
  return au < 0.25f ? ft : fl;
}

// dF/du. Series u (1/3 - u^2/10 + 3u^4/56 - 5u^6/144 + 35u^8/1408 - 63u^10/3328) for
// |u| < 0.25; otherwise from (u F)' = sqrt(1 + u^2), i.e. F' = (sqrt(1 + u^2) - F) / u.
__device__ __forceinline__ float arc_ratio_prime(float u, float F) {
  if (fabsf(u) < 0.25f) {
    const float u2 = u * u;
    float p = -63.f / 3328.f;
    p = fmaf(p, u2, 35.f / 1408.f);
    p = fmaf(p, u2, -5.f / 144.f);
    p = fmaf(p, u2, 3.f / 56.f);
    p = fmaf(p, u2, -0.1f);
    p = fmaf(p, u2, 1.f / 3.f);
    return u * p;
  }
  return __fdividef(sqrt_approx(fmaf(u, u, 1.f)) - F, u);
}

// d(F^2)/du: geodesic 2 F F'(u); Euclidean (F^2 = 1 + u^2/4) u/2.
template <bool EUCLID>
__device__ __forceinline__ float f2_prime(float u, float F2) {
  if constexpr (EUCLID) {
    return 0.5f * u;
  } else {
    const float F = sqrt_approx(F2);
    return 2.f * F * arc_ratio_prime(u, F);
  }
}

// Evaluate one (pixel, primitive) pair. Returns true when a root in front of the near
// plane lies within 3 sigma(theta) (the selected hit is in h, G included). EUCLID: the
// Euclidean-distance density (straight-line distance sqrt(rho^2 + z^2) instead of the
// arc length), for which F(u)^2 = 1 + u^2/4 exactly.
template <bool EUCLID>
__device__ __forceinline__ bool eval_pair(const PrimState& P, float X, float Y, const RasterParams& rp, Hit& h,
                                          bool& grazed, uint32_t& isect) {
  const float4 f0 = P.f[0], f1 = P.f[1], f2 = P.f[2];
  // pixel offset from the projected centre (double-float centre); the pixel's ray line
  // must meet the chord ellipsoid that holds the support: conic F(p) <= 1
  const float dxp = __fsub_rn(__fsub_rn(X, f1.x), f1.y);
  const float dyp = __fsub_rn(__fsub_rn(Y, f1.z), f1.w);
  const float Fc = __fmaf_rn(dxp, __fmaf_rn(f0.x, dxp, __fmaf_rn(f0.y, dyp, -f0.w)),
                             __fmul_rn(dyp, __fmaf_rn(f0.z, dyp, -f2.x)));
  if (!(Fc <= 1.f)) return false;
  ++isect;
  const float4 f3 = P.f[3], f4 = P.f[4], f5 = P.f[5], f6 = P.f[6];
  // camera-plane offset at the centre's depth, then the local frame (W^T e, e_z = 0)
  const float ex = __fmul_rn(__fmul_rn(dxp, f2.w), rp.inv_fx);
  const float ey = __fmul_rn(__fmul_rn(dyp, f2.w), rp.inv_fy);
  const float bx = __fmaf_rn(f3.x, ex, __fmul_rn(f3.y, ey));
  const float by = __fmaf_rn(f3.z, ex, __fmul_rn(f3.w, ey));
  const float bz = __fmaf_rn(f4.x, ex, __fmul_rn(f4.y, ey));
  const float dx = __fmaf_rn(bx, f2.z, f4.z);
  const float dy = __fmaf_rn(by, f2.z, f4.w);
  const float dz = __fmaf_rn(bz, f2.z, f5.x);
  const float a = f5.y, b = f5.z;
  const float adx = __fmul_rn(a, dx), bdy = __fmul_rn(b, dy);
  const float A = __fmaf_rn(adx, dx, __fmul_rn(bdy, dy));
  const float Bh = __fmaf_rn(adx, bx, __fmaf_rn(bdy, by, __fmul_rn(-0.5f, dz)));
  const float C = __fmaf_rn(__fmul_rn(a, bx), bx, __fmaf_rn(__fmul_rn(b, by), by, -bz));
  const float Dq = __fmaf_rn(Bh, Bh, -__fmul_rn(A, C));
  const float smin = __fsub_rn(rp.near_plane, f2.w);  // t > near  <=>  s > near - z_mu
  const float iu = f6.x, iv = f6.y;
  // candidate test: within 3 sigma(theta) <=> F(u)^2 E <= 9 (F >= sqrt(1 + u^2/4) >= 1)
  auto accept = [&](float s) -> bool {
    if (!(s > smin)) return false;
    const float x = __fmaf_rn(s, dx, bx), y = __fmaf_rn(s, dy, by);
    const float x2 = __fmul_rn(x, x), y2 = __fmul_rn(y, y);
    const float E = __fmaf_rn(iu, x2, __fmul_rn(iv, y2));
    if (!(E <= 9.f)) return false;
    const float rho2 = __fadd_rn(x2, y2);
    const float zs = __fmaf_rn(a, x2, __fmul_rn(b, y2));
    const float v = rho2 > 0.f ? __fmul_rn(zs, rsqrtf(rho2)) : 0.f;  // u / 2
    const float F2c = __fmaf_rn(v, v, 1.f);                           // chord: 1 + u^2/4
    const float Qc = __fmul_rn(E, F2c);
    if (!(Qc <= 9.f)) return false;  // geodesic: F^2 >= 1 + u^2/4; Euclidean: equality
    const float u = __fmul_rn(2.f, v);
    float F2, Q;
    if constexpr (EUCLID) {
      F2 = F2c;
      Q = Qc;
    } else {
      const float F = arc_ratio(u);
      F2 = __fmul_rn(F, F);
      Q = __fmul_rn(F2, E);
      if (!(Q <= 9.f)) return false;
    }
    h.s = s; h.x = x; h.y = y; h.zs = zs;
    h.dx = dx; h.dy = dy; h.dz = dz;
    h.rho2 = rho2; h.u = u; h.F2 = F2; h.E = E;
    h.G = __expf(__fmul_rn(-0.5f, Q));
    return true;
  };
  if (fabsf(Dq) <= __fmul_rn(rp.grazing_eps, __fmul_rn(Bh, Bh))) {
    // grazing ray: re-solve in FP64 from the FP32 local ray
    grazed = true;
    const double ad = a, bd = b, dxd = dx, dyd = dy, bxd = bx, byd = by;
    const double Ad = ad * dxd * dxd + bd * dyd * dyd;
    const double Bd = ad * bxd * dxd + bd * byd * dyd - 0.5 * (double)dz;
    const double Cd = ad * bxd * bxd + bd * byd * byd - (double)bz;
    const double Dd = Bd * Bd - Ad * Cd;
    if (Dd < 0.0) return false;
    const double sq = sqrt(Dd);
    const double qd = -(Bd + (Bd >= 0.0 ? sq : -sq));
    const float r1 = qd != 0.0 ? (float)(Cd / qd) : __int_as_float(0x7fc00000);
    const float r2 = Ad != 0.0 ? (float)(qd / Ad) : __int_as_float(0x7fc00000);
    const bool e1 = isfinite(r1), e2 = isfinite(r2);
    const float s0 = (e1 && e2) ? fminf(r1, r2) : (e1 ? r1 : r2);
    const float s1 = (e1 && e2) ? fmaxf(r1, r2) : __int_as_float(0x7fc00000);
    if (isfinite(s0) && accept(s0)) return true;
    return isfinite(s1) && accept(s1);
  }
  if (Dq < 0.f) return false;
  const float sq = sqrt_approx(Dq);
  const float q = -__fadd_rn(Bh, Bh >= 0.f ? sq : -sq);
  // q/A is the smaller root iff sign(B') and sign(A) agree (A = 0: the single root C/q)
  const bool qa_first = (Bh >= 0.f) == (A > 0.f);
  const float s0 = qa_first ? __fdividef(q, A) : __fdividef(C, q);
  const bool e0 = isfinite(s0);
  if (e0 && accept(s0)) return true;
  const float s1 = qa_first ? __fdividef(C, q) : __fdividef(q, A);
  return isfinite(s1) && accept(s1);
}

__device__ __forceinline__ void pixel_of(int tile, int tiles_x, int& px, int& py) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  px = (tile % tiles_x) * TILE + (warp & 1) * 8 + (lane & 7);
  py = (tile / tiles_x) * TILE + (warp >> 1) * 4 + (lane >> 3);
}

template <int NT = BLOCK>
__device__ __forceinline__ void stage_batch(PrimState* sm, const uint32_t* ids, int id_stride, uint32_t id_mask,
                                            const PrimState* state, uint32_t first, int cnt) {
  for (int e = threadIdx.x; e < cnt * 8; e += NT) {
    const int r = e >> 3, c = e & 7;
    const uint32_t pid = __ldg(ids + (size_t)(first + r) * id_stride) & id_mask;
    reinterpret_cast<float4*>(sm)[r * 8 + c] = __ldg(reinterpret_cast<const float4*>(state + pid) + c);
  }
}

}  // namespace

// Gaussian curvature of z = a x^2 + b y^2 at local (x, y) (Sec. 3.2.1 curvature Eq.) and
// its partial derivatives with respect to a, b, x, y.
struct Curv {
  float K, dKda, dKdb, dKdx, dKdy;
};
__device__ __forceinline__ float curvature(float a, float b, float x, float y) {
  const float S = fmaf(4.f * a * a, x * x, fmaf(4.f * b * b, y * y, 1.f));
  return __fdividef(4.f * a * b, S * S);
}
__device__ __forceinline__ Curv curvature_grad(float a, float b, float x, float y) {
  const float S = fmaf(4.f * a * a, x * x, fmaf(4.f * b * b, y * y, 1.f));
  const float iS = __fdividef(1.f, S), iS2 = iS * iS;
  Curv c;
  c.K = 4.f * a * b * iS2;
  const float c3 = 2.f * c.K * iS;  // 8ab / S^3
  c.dKda = 4.f * b * iS2 - c3 * 8.f * a * x * x;
  c.dKdb = 4.f * a * iS2 - c3 * 8.f * b * y * y;
  c.dKdx = -c3 * 8.f * a * a * x;
  c.dKdy = -c3 * 8.f * b * b * y;
  return c;
}

// Composite one tile: `tile` indexes the sorted instance ranges, `local_tile` the tile
// grid of the view (they differ when several views share one launch). EXTRA adds the
// curvature map (Sec. 3.2.1), the depth distortion (Sec. 3.3) and the median depth
// (Sec. 4.1). The distortion sum_i sum_{j<i} w_i w_j (t_i - t_j)^2 equals
// A0 A2 - A1^2 with A_k = sum_i w_i tau_i^k for any shift tau = t - c; c is the pixel's
// first blended depth, which keeps the two terms small (no cancellation at the camera
// distance). The per-pixel residue (c, A1, A2) serves its backward.
template <bool EUCLID, bool EXTRA, bool STATS>
__device__ __forceinline__ void raster_fwd_tile(PrimState* sm, uint8_t* used, int tile, int local_tile,
                                                const uint2* __restrict__ ranges, const uint32_t* __restrict__ ids,
                                                int id_stride, const PrimState* __restrict__ state,
                                                const RasterParams& rp, float* __restrict__ out_rgb,
                                                float* __restrict__ out_alpha, float* __restrict__ out_depth,
                                                float* __restrict__ out_normal, float* __restrict__ T_final,
                                                uint32_t* __restrict__ n_contrib, const ExtraPlanes& ex,
                                                RasterStats* __restrict__ stats, uint8_t* __restrict__ inst_used) {
  int px, py;
  pixel_of(local_tile, rp.tiles_x, px, py);
  const bool inside = px < rp.W && py < rp.H;
  const uint2 rg = ranges[tile];
  const int n = (int)(rg.y - rg.x);
  const float X = (float)px + 0.5f, Y = (float)py + 0.5f;
  const float xn = (X - rp.cx) * rp.inv_fx, yn = (Y - rp.cy) * rp.inv_fy;
  float T = 1.f, cr = 0.f, cg = 0.f, cb = 0.f, dep = 0.f, nx = 0.f, ny = 0.f, nz = 0.f;
  float kc = 0.f, tref = 0.f, A1 = 0.f, A2 = 0.f, med = 0.f;  // EXTRA channels
  uint32_t last = 0, evals = 0, grazes = 0, isect = 0, hits = 0, blended = 0;
  bool done = !inside;
  for (int b0 = 0; b0 < n; b0 += BLOCK) {
    if (__syncthreads_count(done) == BLOCK) break;
    const int cnt = min(BLOCK, n - b0);
    stage_batch(sm, ids, id_stride, rp.id_mask, state, rg.x + b0, cnt);
    used[threadIdx.x] = 0;
    __syncthreads();
    if (!done) {
      for (int j = 0; j < cnt; ++j) {
        ++evals;
        Hit h;
        bool gz = false;
        const bool hit = eval_pair<EUCLID>(sm[j], X, Y, rp, h, gz, isect);
        grazes += gz;
        if (!hit) continue;
        ++hits;
        const float4 f5 = sm[j].f[5];
        const float al = fminf(rp.alpha_max, __fmul_rn(f5.w, h.G));
        if (al < rp.alpha_min) continue;
        const float Tn = __fmul_rn(T, __fsub_rn(1.f, al));
        if (Tn < rp.T_min) {
          done = true;
          break;
        }
        const float w = al * T;
        const float4 f2 = sm[j].f[2], f3 = sm[j].f[3], f4 = sm[j].f[4], f6 = sm[j].f[6], f7 = sm[j].f[7];
        cr = fmaf(w, f7.y, cr);
        cg = fmaf(w, f7.z, cg);
        cb = fmaf(w, f7.w, cb);
        dep = fmaf(w, f2.w + h.s, dep);
        const float nlx = 2.f * f5.y * h.x, nly = 2.f * f5.z * h.y;
        const float ncx = fmaf(f3.x, nlx, fmaf(f3.z, nly, -f4.x));
        const float ncy = fmaf(f3.y, nlx, fmaf(f3.w, nly, -f4.y));
        const float ncz = fmaf(f6.z, nlx, fmaf(f6.w, nly, -f7.x));
        float inn = rsqrtf(fmaf(ncx, ncx, fmaf(ncy, ncy, ncz * ncz)));
        if (fmaf(ncx, xn, fmaf(ncy, yn, ncz)) > 0.f) inn = -inn;
        const float wn = w * inn;
        nx = fmaf(wn, ncx, nx);
        ny = fmaf(wn, ncy, ny);
        nz = fmaf(wn, ncz, nz);
        if constexpr (EXTRA) {
          const float t = f2.w + h.s;
          kc = fmaf(w, curvature(f5.y, f5.z, h.x, h.y), kc);
          if (blended == 0) tref = t;
          const float tau = t - tref;
          A1 = fmaf(w, tau, A1);
          A2 = fmaf(w * tau, tau, A2);
          if (T > 0.5f) med = fmaxf(med, t);
        }
        T = Tn;
        ++blended;
        used[j] = 1;
        last = (uint32_t)(b0 + j + 1);
      }
    }
    // one flag per instance: did any pixel of the tile blend it (read by the backward)
    __syncthreads();
    if (inst_used && threadIdx.x < cnt) inst_used[rg.x + b0 + threadIdx.x] = used[threadIdx.x];
  }
  if (inside && out_rgb) {
    const size_t P = (size_t)rp.W * rp.H, pix = (size_t)py * rp.W + px;
    out_rgb[pix] = cr;
    out_rgb[P + pix] = cg;
    out_rgb[2 * P + pix] = cb;
    out_alpha[pix] = 1.f - T;
    out_depth[pix] = dep;
    out_normal[pix] = nx;
    out_normal[P + pix] = ny;
    out_normal[2 * P + pix] = nz;
    if (T_final) T_final[pix] = T;
    if (n_contrib) n_contrib[pix] = last;
    if constexpr (EXTRA) {
      if (ex.curvature) ex.curvature[pix] = kc;
      if (ex.distortion) ex.distortion[pix] = fmaf(1.f - T, A2, -A1 * A1);
      if (ex.median_depth) ex.median_depth[pix] = med;
      if (ex.resid) {
        ex.resid[pix] = tref;
        ex.resid[P + pix] = A1;
        ex.resid[2 * P + pix] = A2;
      }
    }
  }
  // counters: one atomic per warp and counter (without STATS the counts are dead code)
  if (STATS && stats) {
    const unsigned ev = __reduce_add_sync(FULL, evals), is = __reduce_add_sync(FULL, isect);
    const unsigned hi = __reduce_add_sync(FULL, hits), bl = __reduce_add_sync(FULL, blended);
    const unsigned gzz = __reduce_add_sync(FULL, grazes);
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&stats->pair_evals, (unsigned long long)ev);
      atomicAdd(&stats->pair_isect, (unsigned long long)is);
      atomicAdd(&stats->pair_hits, (unsigned long long)hi);
      atomicAdd(&stats->pair_blended, (unsigned long long)bl);
      if (gzz) atomicAdd(&stats->grazing, (unsigned long long)gzz);
    }
  }
}

template <bool EUCLID, bool EXTRA, bool STATS>
__global__ void __launch_bounds__(BLOCK, 4)
    k_raster_fwd(const uint2* __restrict__ ranges, const uint32_t* __restrict__ ids, int id_stride,
                 const PrimState* __restrict__ state, RasterParams rp, float* __restrict__ out_rgb,
                 float* __restrict__ out_alpha, float* __restrict__ out_depth, float* __restrict__ out_normal,
                 float* __restrict__ T_final, uint32_t* __restrict__ n_contrib, ExtraPlanes ex,
                 RasterStats* __restrict__ stats, const uint32_t* __restrict__ tile_order,
                 uint8_t* __restrict__ inst_used) {
  __shared__ PrimState sm[BLOCK];
  __shared__ uint8_t used[BLOCK];
  const int tile = tile_order ? (int)tile_order[blockIdx.x] : (int)blockIdx.x;
  raster_fwd_tile<EUCLID, EXTRA, STATS>(sm, used, tile, tile, ranges, ids, id_stride, state, rp, out_rgb, out_alpha,
                                 out_depth, out_normal, T_final, n_contrib, ex, stats, inst_used);
}

// Several views of one scene in one launch: global tile t belongs to the view v with
// tile_base[v] <= t < tile_base[v + 1].
template <bool EUCLID, bool EXTRA>
__global__ void __launch_bounds__(BLOCK, 3)
    k_raster_fwd_views(const uint2* __restrict__ ranges, const uint32_t* __restrict__ ids, int id_stride,
                       uint32_t id_mask, const PrimState* __restrict__ state, const ViewDesc* __restrict__ views,
                       int n_views,
                       const uint32_t* __restrict__ tile_base, RasterStats* __restrict__ stats,
                       const uint32_t* __restrict__ tile_order) {
  __shared__ PrimState sm[BLOCK];
  __shared__ uint8_t used[BLOCK];
  const int tile = tile_order ? (int)tile_order[blockIdx.x] : (int)blockIdx.x;
  int lo = 0, hi = n_views;  // largest v with tile_base[v] <= tile
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (tile_base[mid] <= (uint32_t)tile) lo = mid; else hi = mid;
  }
  const ViewDesc& vd = views[lo];
  RasterParams rp = vd.rp;
  rp.id_mask = id_mask;
  raster_fwd_tile<EUCLID, EXTRA, true>(sm, used, tile, tile - (int)tile_base[lo], ranges, ids, id_stride, state, rp,
                                 vd.rgb, vd.alpha, vd.depth, vd.normal, vd.T_final, vd.n_contrib, vd.ex, stats,
                                 nullptr);
}

namespace {

// Per-pixel upstream gradients (and the forward's residue) of the backward.
struct PixGrads {
  float gR, gG, gB, gA, gD, gNx, gNy, gNz;
  float gK, tref, g_tau, g_tau2;  // extra channels
  float Tfin;
};

// The pixel's upstream gradients; with EXTRA, the distortion's per-pixel constants from
// the forward's residue (c, A1, A2): dL/dA0 = g A2 joins the alpha gradient, tau and tau^2
// carry -2 g A1 and g A0 (A0 = 1 - T_final).
template <bool EXTRA>
__device__ __forceinline__ PixGrads load_pix_grads(bool inside, size_t pix, size_t P, float Tfin,
                                                   const float* __restrict__ g_rgb, const float* __restrict__ g_alpha,
                                                   const float* __restrict__ g_depth,
                                                   const float* __restrict__ g_normal, const ExtraGrads& eg) {
  PixGrads pg{};
  pg.Tfin = Tfin;
  if (inside) {
    if (g_rgb) { pg.gR = g_rgb[pix]; pg.gG = g_rgb[P + pix]; pg.gB = g_rgb[2 * P + pix]; }
    if (g_alpha) pg.gA = g_alpha[pix];
    if (g_depth) pg.gD = g_depth[pix];
    if (g_normal) { pg.gNx = g_normal[pix]; pg.gNy = g_normal[P + pix]; pg.gNz = g_normal[2 * P + pix]; }
    if constexpr (EXTRA) {
      if (eg.g_curvature) pg.gK = eg.g_curvature[pix];
      const float gDist = eg.g_distortion ? eg.g_distortion[pix] : 0.f;
      if (gDist != 0.f) {
        pg.tref = eg.resid[pix];
        const float A1 = eg.resid[P + pix], A2 = eg.resid[2 * P + pix];
        pg.gA += gDist * A2;
        pg.g_tau = -2.f * gDist * A1;
        pg.g_tau2 = gDist * (1.f - Tfin);
      }
    }
  }
  return pg;
}

// Gradient record of one blended pair (entries 0..NGRAD-1 of v): the back-to-front (or,
// FWD_ORDER, front-to-back) dX/d(alpha) of the supplementary, then the chain rule through
// the alpha clamp, G, F(u), E, the normal and the implicit root. T is the transmittance
// before the pair; S_ref is the sum of w_j (g . X_j) over the pixel's later blended
// pairs, or (FWD_ORDER) over all of them, S_prefix then being that sum over the pairs up
// to and excluding this one. Returns the pair's own term w (g . X).
template <bool EUCLID, bool EXTRA, bool FWD_ORDER, bool ACC = false>
__device__ __forceinline__ float pair_grad(const PrimState& P, const Hit& h, float oG, float al, float T, float xn,
                                           float yn, const RasterParams& rp, const PixGrads& pg, float S_ref,
                                           float S_prefix, float v[32]) {
  // ACC: add the record to v (several pixels of one thread) instead of writing it
  auto put = [&](int k, float x) {
    if constexpr (ACC) v[k] += x;
    else v[k] = x;
  };
  const float4 f2 = P.f[2], f3 = P.f[3], f4 = P.f[4], f5 = P.f[5], f6 = P.f[6], f7 = P.f[7];
  const float a = f5.y, b = f5.z, o = f5.w;
  const float onem = 1.f - al;
  const float w = al * T;
  const float W00 = f3.x, W10 = f3.y, W01 = f3.z, W11 = f3.w, W02 = f4.x, W12 = f4.y, W20 = f6.z,
              W21 = f6.w, W22 = f7.x;
  const float x = h.x, y = h.y;
  const float nlx = 2.f * a * x, nly = 2.f * b * y;
  const float ncx = fmaf(W00, nlx, fmaf(W01, nly, -W02));
  const float ncy = fmaf(W10, nlx, fmaf(W11, nly, -W12));
  const float ncz = fmaf(W20, nlx, fmaf(W21, nly, -W22));
  const float inn = rsqrtf(fmaf(ncx, ncx, fmaf(ncy, ncy, ncz * ncz)));
  const float sg_ = fmaf(ncx, xn, fmaf(ncy, yn, ncz)) > 0.f ? -1.f : 1.f;
  const float hx = ncx * inn, hy = ncy * inn, hz = ncz * inn;  // unsigned unit normal
  const float nox = sg_ * hx, noy = sg_ * hy, noz = sg_ * hz;
  const float t = f2.w + h.s;
  float gX = pg.gR * f7.y + pg.gG * f7.z + pg.gB * f7.w + pg.gD * t + pg.gNx * nox + pg.gNy * noy + pg.gNz * noz;
  float d_t = w * pg.gD;
  Curv kv{};
  if constexpr (EXTRA) {
    kv = curvature_grad(a, b, x, y);
    const float tau = t - pg.tref;
    gX += pg.gK * kv.K + tau * fmaf(pg.g_tau2, tau, pg.g_tau);
    d_t += w * fmaf(2.f * pg.g_tau2, tau, pg.g_tau);
  }
  const float wgx = w * gX;
  const float after = FWD_ORDER ? S_ref - (S_prefix + wgx) : S_ref;  // sum of w_j g.X_j, j after i
  const float dal = T * gX - __fdividef(after - pg.gA * pg.Tfin, onem);
  put(17, w * pg.gR);
  put(18, w * pg.gG);
  put(19, w * pg.gB);
  // alpha = min(alpha_max, o G)
  float dG = 0.f;
  float g_o = 0.f;
  if (oG < rp.alpha_max) {
    g_o = dal * h.G;
    dG = dal * o;
  }
  put(16, g_o);
  const float dQ = -0.5f * h.G * dG;
  const float dE = dQ * h.F2;
  put(14, dE * x * x);
  put(15, dE * y * y);
  float gx = dE * 2.f * f6.x * x, gy = dE * 2.f * f6.y * y;
  float da = 0.f, db = 0.f;
  if constexpr (EXTRA) {
    const float dK = w * pg.gK;
    da += dK * kv.dKda;
    db += dK * kv.dKdb;
    gx += dK * kv.dKdx;
    gy += dK * kv.dKdy;
  }
  if (h.rho2 > 0.f) {
    const float irho = rsqrtf(h.rho2);
    const float du = dQ * h.E * f2_prime<EUCLID>(h.u, h.F2);
    const float ur = h.u * irho * irho;
    gx += du * (4.f * a * x * irho - ur * x);
    gy += du * (4.f * b * y * irho - ur * y);
    da += du * 2.f * x * x * irho;
    db += du * 2.f * y * y * irho;
  }
  // normal: n_out = sg * n_c / |n_c|, n_c = W n_l
  const float dnx = w * pg.gNx, dny = w * pg.gNy, dnz = w * pg.gNz;
  const float dd = hx * dnx + hy * dny + hz * dnz;
  const float sc_ = sg_ * inn;
  const float dcx = sc_ * (dnx - hx * dd), dcy = sc_ * (dny - hy * dd), dcz = sc_ * (dnz - hz * dd);
  const float gmx = W00 * dcx + W10 * dcy + W20 * dcz;
  const float gmy = W01 * dcx + W11 * dcy + W21 * dcz;
  const float gmz = W02 * dcx + W12 * dcy + W22 * dcz;
  gx += 2.f * a * gmx;
  gy += 2.f * b * gmy;
  da += 2.f * x * gmx;
  db += 2.f * y * gmy;
  // the root moves with the parameters: t(theta) from f(p_hat(t)) = 0
  const float den = nlx * h.dx + nly * h.dy - h.dz;
  const float kk = den != 0.f ? __fdividef(gx * h.dx + gy * h.dy + d_t, den) : 0.f;
  const float hhx = gx - kk * nlx, hhy = gy - kk * nly, hhz = kk;
  da -= kk * x * x;
  db -= kk * y * y;
  put(12, da);
  put(13, db);
  put(9, hhx);
  put(10, hhy);
  put(11, hhz);
  // P = p_hat h^T + gamma n_l^T, p_hat = (x, y, zs), n_l = (nlx, nly, -1)
  const float pz = h.zs;
  put(0, x * hhx + gmx * nlx);
  put(1, x * hhy + gmx * nly);
  put(2, x * hhz - gmx);
  put(3, y * hhx + gmy * nlx);
  put(4, y * hhy + gmy * nly);
  put(5, y * hhz - gmy);
  put(6, pz * hhx + gmz * nlx);
  put(7, pz * hhy + gmz * nly);
  put(8, pz * hhz - gmz);
  return wgx;
}

// Reduce-scatter of the 20 gradient components across the warp in 21 shuffles (halving
// the number of partial sums a lane holds at each butterfly stage: 20, 10, 5, 3|2, 2|1,
// 1): afterwards 20 of the lanes each hold the warp-wide sum of one component, k, and the
// others return k = -1.
__device__ __forceinline__ float warp_reduce_scatter20(const float v[32], int& k) {
  const int lane = threadIdx.x & 31;
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2, b0 = lane & 1;
  float r[10], s[5], t[3];
#pragma unroll
  for (int i = 0; i < 10; ++i) {  // 20 -> 10: lanes with bit 4 keep components 10..19
    const float recv = __shfl_xor_sync(FULL, b4 ? v[i] : v[i + 10], 16);
    r[i] = (b4 ? v[i + 10] : v[i]) + recv;
  }
#pragma unroll
  for (int i = 0; i < 5; ++i) {  // 10 -> 5
    const float recv = __shfl_xor_sync(FULL, b3 ? r[i] : r[5 + i], 8);
    s[i] = (b3 ? r[5 + i] : r[i]) + recv;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {  // 5 -> 3 (bit 2 clear) or 2 (bit 2 set)
    const float send = b2 ? s[i] : (i < 2 ? s[3 + i] : 0.f);
    const float recv = __shfl_xor_sync(FULL, send, 4);
    t[i] = b2 ? (i < 2 ? s[3 + i] + recv : 0.f) : s[i] + recv;
  }
  const bool c3 = !b2;  // three partial sums held, else two
  // 3 -> 2|1, 2 -> 1|1
  const float recv1 = __shfl_xor_sync(FULL, b1 ? t[0] : (c3 ? t[2] : t[1]), 2);
  const float recv2 = __shfl_xor_sync(FULL, (b1 && c3) ? t[1] : 0.f, 2);
  const float u0 = (b1 ? (c3 ? t[2] : t[1]) : t[0]) + recv1;
  const float u1 = (!b1 && c3) ? t[1] + recv2 : 0.f;
  const bool two = !b1 && c3;  // two partial sums held, else one
  // 2 -> 1|1, or the pair adds its single partial sums (the lane with bit 0 clear owns it)
  const float recv = __shfl_xor_sync(FULL, two ? (b0 ? u0 : u1) : u0, 1);
  const float out = two ? (b0 ? u1 + recv : u0 + recv) : u0 + recv;
  const int base = (b4 ? 10 : 0) + (b3 ? 5 : 0) + (b2 ? 3 : 0) + (b1 ? (c3 ? 2 : 1) : 0);
  k = two ? base + (b0 ? 1 : 0) : (b0 ? -1 : base);
  return out;
}


}  // namespace

// Backward tile layout: PPT pixels per thread, BLOCK / PPT threads per tile; warp w covers
// 8 columns and 4 PPT rows of the tile, and a lane's pixel p lies 4 p rows below its first.
// The pair's state record is read from shared memory once per thread and evaluated for
// each of its pixels, and the thread's pixels add their gradient records before the warp
// reduces them, so the staging, the loop and the reduction are paid once per PPT pixels.
// Records are staged kBwdBatch<PPT> at a time (the shared memory of the smaller CTAs is
// sized for more CTAs per SM). Each pixel's upstream gradients and residue constants sit
// in shared memory ([field][thread]), read by the pairs that produce a gradient: the
// registers they would hold let the two-pixel CTAs fit 7 per SM without spilling
// (measured 2 % faster than 6 per SM with them in registers and batches of 128).
#ifndef QGS_BWD_BATCH2
#define QGS_BWD_BATCH2 64
#endif
#ifndef QGS_BWD_CTAS2
#define QGS_BWD_CTAS2 7
#endif
template <int PPT>
constexpr int kBwdBatch = PPT == 1 ? BLOCK : QGS_BWD_BATCH2;
template <bool EXTRA>
constexpr int kPixFields = EXTRA ? 13 : 9;
// Two pixels per thread when the frame has at least this many tiles per SM: measured 2 %
// faster than one at 3M / 1297x840 (4346 tiles; the staging, loop and reduction halve per
// pixel; 95 registers, 5 CTAs of 4 warps per SM instead of 3 of 8), while small frames keep
// one pixel per thread for the warps it gives them (64 tiles: 0.16 ms against 0.10).
// Adding the records of pairs with at most two contributing lanes by shared atomics instead
// of the reduce-scatter measured 3 % slower. Two-pixel CTAs take QGS_BWD_CTAS2 per SM except
// with the extra channels, whose larger state keeps 5.
constexpr int kBwdTwoPixelTilesPerSM = 8;
template <int PPT>
constexpr size_t raster_bwd_smem() {
  return (sizeof(PrimState) + sizeof(float) * NGRAD + sizeof(int)) * (size_t)kBwdBatch<PPT>;
}

namespace {
template <int PPT>
__device__ __forceinline__ void pixel_of_bwd(int tile, int tiles_x, int p, int& px, int& py) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  px = (tile % tiles_x) * TILE + (warp & 1) * 8 + (lane & 7);
  py = (tile / tiles_x) * TILE + (warp >> 1) * (4 * PPT) + (lane >> 3) + 4 * p;
}

// A pixel's PixGrads in shared memory: field f of this thread's pixel p at
// s[(p * kPixFields + f) * NT + threadIdx.x] (consecutive threads in consecutive banks).
template <bool EXTRA, int NT>
__device__ __forceinline__ void store_pix(float* s, int p, const PixGrads& g) {
  float* b = s + (size_t)p * kPixFields<EXTRA> * NT + threadIdx.x;
  b[0 * NT] = g.gR; b[1 * NT] = g.gG; b[2 * NT] = g.gB; b[3 * NT] = g.gA;
  b[4 * NT] = g.gD; b[5 * NT] = g.gNx; b[6 * NT] = g.gNy; b[7 * NT] = g.gNz; b[8 * NT] = g.Tfin;
  if constexpr (EXTRA) {
    b[9 * NT] = g.gK; b[10 * NT] = g.tref; b[11 * NT] = g.g_tau; b[12 * NT] = g.g_tau2;
  }
}
template <bool EXTRA, int NT>
__device__ __forceinline__ PixGrads load_pix(const float* s, int p) {
  const float* b = s + (size_t)p * kPixFields<EXTRA> * NT + threadIdx.x;
  PixGrads g{};
  g.gR = b[0 * NT]; g.gG = b[1 * NT]; g.gB = b[2 * NT]; g.gA = b[3 * NT];
  g.gD = b[4 * NT]; g.gNx = b[5 * NT]; g.gNy = b[6 * NT]; g.gNz = b[7 * NT]; g.Tfin = b[8 * NT];
  if constexpr (EXTRA) {
    g.gK = b[9 * NT]; g.tref = b[10 * NT]; g.g_tau = b[11 * NT]; g.g_tau2 = b[12 * NT];
  }
  return g;
}
}  // namespace

// EXTRA: also the gradients of the curvature map and of the depth distortion. With
// D = A0 A2 - A1^2 (A0 = 1 - T_final, A1, A2 the forward's shifted moments), dL/dA0 =
// g_D A2 joins the alpha gradient, and tau = t - c and tau^2 act as two more blended
// channels with upstream gradients -2 g_D A1 and g_D A0.
template <bool EUCLID, bool EXTRA, bool STATS, int PPT>
__global__ void __launch_bounds__(BLOCK / PPT, PPT == 1 ? 3 : (EXTRA ? 5 : QGS_BWD_CTAS2))
    k_raster_bwd(const uint2* __restrict__ ranges, const uint32_t* __restrict__ ids, int id_stride,
                 const PrimState* __restrict__ state, RasterParams rp, const float* __restrict__ g_rgb,
                 const float* __restrict__ g_alpha, const float* __restrict__ g_depth,
                 const float* __restrict__ g_normal, const float* __restrict__ T_final,
                 const uint32_t* __restrict__ n_contrib, ExtraGrads eg, float* __restrict__ pgrad,
                 RasterStats* __restrict__ stats, const uint32_t* __restrict__ tile_order,
                 const uint8_t* __restrict__ inst_used) {
  constexpr int NT = BLOCK / PPT, BATCH = kBwdBatch<PPT>;
  // dynamic shared memory: BATCH records, then BATCH x NGRAD accumulators, then flags
  extern __shared__ float4 dyn_smem[];
  PrimState* sm = reinterpret_cast<PrimState*>(dyn_smem);
  float(*sg)[NGRAD] = reinterpret_cast<float(*)[NGRAD]>(sm + BATCH);
  int* sflag = reinterpret_cast<int*>(&sg[BATCH][0]);
  __shared__ int smax;
  __shared__ uint8_t suse[BATCH];
  const int tile = tile_order ? (int)tile_order[blockIdx.x] : (int)blockIdx.x;
  const uint2 rg = ranges[tile];
  const size_t P = (size_t)rp.W * rp.H;
  float X[PPT], Y[PPT], xn[PPT], yn[PPT], T[PPT], Sdot[PPT];  // Sdot: sum over later pairs of w (g . X)
  uint32_t last[PPT], mlast = 0;
  __shared__ float spg[PPT * kPixFields<EXTRA> * NT];
#pragma unroll
  for (int p = 0; p < PPT; ++p) {
    int px, py;
    pixel_of_bwd<PPT>(tile, rp.tiles_x, p, px, py);
    const bool inside = px < rp.W && py < rp.H;
    X[p] = (float)px + 0.5f;
    Y[p] = (float)py + 0.5f;
    xn[p] = (X[p] - rp.cx) * rp.inv_fx;
    yn[p] = (Y[p] - rp.cy) * rp.inv_fy;
    const size_t pix = inside ? (size_t)py * rp.W + px : 0;
    T[p] = inside ? T_final[pix] : 1.f;
    last[p] = inside ? n_contrib[pix] : 0u;
    store_pix<EXTRA, NT>(spg, p, load_pix_grads<EXTRA>(inside, pix, P, T[p], g_rgb, g_alpha, g_depth, g_normal, eg));
    Sdot[p] = 0.f;
    mlast = max(mlast, last[p]);
  }
  if (threadIdx.x == 0) smax = 0;
  __syncthreads();
  {
    const unsigned m = __reduce_max_sync(FULL, mlast);
    if ((threadIdx.x & 31) == 0) atomicMax(&smax, (int)m);
  }
  __syncthreads();
  const int maxlast = smax;
  uint32_t n_pairs = 0, n_contrib_pairs = 0, isect = 0;
  for (int b0 = ((maxlast - 1) / BATCH) * BATCH; maxlast > 0 && b0 >= 0; b0 -= BATCH) {
    const int cnt = min(BATCH, maxlast - b0);
    __syncthreads();
    stage_batch<NT>(sm, ids, id_stride, rp.id_mask, state, rg.x + b0, cnt);
    for (int e = threadIdx.x; e < BATCH * NGRAD; e += NT) (&sg[0][0])[e] = 0.f;
    for (int e = threadIdx.x; e < BATCH; e += NT) {
      sflag[e] = 0;
      suse[e] = (e < cnt && inst_used) ? inst_used[rg.x + b0 + e] : 1;
    }
    __syncthreads();
    for (int j = cnt - 1; j >= 0; --j) {
      if (!suse[j]) continue;  // no pixel of this tile blended the instance in the forward
      // gradient record of this thread's pairs (entries 0..NGRAD-1; with one pixel per
      // thread written by a contributing lane and zeroed for the others only when the
      // warp reduces, with several pixels summed from zero)
      float v[32];
#pragma unroll
      for (int k = (PPT > 1 ? 0 : NGRAD); k < 32; ++k) v[k] = 0.f;
      bool contrib = false;
#pragma unroll
      for (int p = 0; p < PPT; ++p) {
        if ((uint32_t)(b0 + j) < last[p]) {
          Hit h;
          bool gz = false;
          ++n_pairs;
          if (eval_pair<EUCLID>(sm[j], X[p], Y[p], rp, h, gz, isect)) {
            const float oG = __fmul_rn(sm[j].f[5].w, h.G);
            const float al = fminf(rp.alpha_max, oG);
            if (al >= rp.alpha_min) {
              contrib = true;
              ++n_contrib_pairs;
              T[p] = __fdividef(T[p], 1.f - al);  // T_i from T_{i+1}
              const PixGrads pgp = load_pix<EXTRA, NT>(spg, p);
              Sdot[p] += pair_grad<EUCLID, EXTRA, false, (PPT > 1)>(sm[j], h, oG, al, T[p], xn[p], yn[p], rp,
                                                                    pgp, Sdot[p], 0.f, v);
            }
          }
        }
      }
      if (__any_sync(FULL, contrib)) {
        if (PPT == 1 && !contrib) {
#pragma unroll
          for (int k = 0; k < NGRAD; ++k) v[k] = 0.f;
        }
        int kc;
        const float r = warp_reduce_scatter20(v, kc);
        if (kc >= 0 && r != 0.f) atomicAdd(&sg[j][kc], r);
        if ((threadIdx.x & 31) == 0) sflag[j] = 1;
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < cnt * NGRAD; e += NT) {
      const int r = e / NGRAD, c = e - r * NGRAD;
      if (sflag[r]) {
        const float val = sg[r][c];
        if (val != 0.f) {
          const uint32_t pid = __ldg(ids + (size_t)(rg.x + b0 + r) * id_stride) & rp.id_mask;
          atomicAdd(pgrad + (size_t)pid * NGRAD_PAD + c, val);
        }
      }
    }
  }
  if (STATS && stats) {
    const unsigned np = __reduce_add_sync(FULL, n_pairs), nc = __reduce_add_sync(FULL, n_contrib_pairs);
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&stats->bwd_pairs, (unsigned long long)np);
      atomicAdd(&stats->bwd_contrib, (unsigned long long)nc);
    }
  }
}

// ---------------------------------------------------------------------------------------
// StopThePop ordering (supplementary, "Details of Per-tile Sorting and Per-pixel
// Resorting"): the tile lists are sorted by each primitive's hit depth on the tile's
// representative ray; each pixel keeps its contributing pairs in a buffer of 8 (hit depth,
// list position) entries and blends the nearest one whenever the buffer is full, the rest
// nearest first at the end of the list. The forward keeps each buffered entry's blend data
// (alpha and the normal, formed at its push) in shared memory, so blending it needs only
// its colour. The backward replays the same sequence front to back with the
// supplementary's front-to-back dX/d(alpha), re-evaluating an entry when it is blended
// (from its state record in shared memory: the staged batch, or a per-thread slot filled
// from global memory when the entry was staged in an earlier batch; the gradient needs the
// whole hit, too much to buffer), and adds each pair's gradient record to global memory
// per pixel.
namespace {

constexpr int RESORT = 8;

struct ResortBuf {
  float t[RESORT];
  uint32_t pos[RESORT];
  int n = 0;
  __device__ __forceinline__ void push(float tt, uint32_t p) {
#pragma unroll
    for (int k = 0; k < RESORT; ++k)
      if (k == n) { t[k] = tt; pos[k] = p; }
    ++n;
  }
  // remove and return the entry with the smallest (depth, list position)
  __device__ __forceinline__ uint32_t pop() {
    float bt = INFINITY;
    uint32_t bp = 0xFFFFFFFFu;
    int bk = 0;
#pragma unroll
    for (int k = 0; k < RESORT; ++k)
      if (k < n && (t[k] < bt || (t[k] == bt && pos[k] < bp))) { bt = t[k]; bp = pos[k]; bk = k; }
    float lt = 0.f;
    uint32_t lp = 0;
#pragma unroll
    for (int k = 0; k < RESORT; ++k)
      if (k == n - 1) { lt = t[k]; lp = pos[k]; }
#pragma unroll
    for (int k = 0; k < RESORT; ++k)
      if (k == bk) { t[k] = lt; pos[k] = lp; }
    --n;
    return bp;
  }
};


}  // namespace

// Shared memory of the StopThePop backward: the staged batch, then one record slot per
// thread (a blended entry outside the current batch is copied there from global memory, so
// that its evaluation reads the record from shared memory like a staged one instead of
// holding all 32 floats in registers). Records sit at a 144-byte stride (the 128-byte
// record and 16 bytes of padding): the lanes of a warp blend different entries, and at 128
// bytes their 16-byte reads of one field would all fall in the same four banks.
constexpr int kStpStride = 9;  // float4 per shared record
// The backward stages 128 records per batch and keeps each pixel's upstream gradients in
// shared memory: with the registers and shared memory that frees, 3 CTAs fit per SM
// instead of 2 (measured 5.28 -> 4.65 ms at 3M / 1297x840).
constexpr int kStpBwdBatch = 128;
constexpr size_t RASTER_STP_BWD_SMEM = sizeof(float4) * kStpStride * (kStpBwdBatch + BLOCK);

namespace {
struct StpRecs {
  float4* base;
  __device__ __forceinline__ const PrimState& operator[](int r) const {
    return *reinterpret_cast<const PrimState*>(base + (size_t)r * kStpStride);
  }
  __device__ __forceinline__ PrimState* ptr(int r) const {
    return reinterpret_cast<PrimState*>(base + (size_t)r * kStpStride);
  }
};

__device__ __forceinline__ void stage_batch_stp(StpRecs sm, const uint32_t* ids, uint32_t id_mask,
                                                const PrimState* state, uint32_t first, int cnt) {
  for (int e = threadIdx.x; e < cnt * 8; e += BLOCK) {
    const int r = e >> 3, c = e & 7;
    const uint32_t pid = __ldg(ids + first + r) & id_mask;
    sm.base[r * kStpStride + c] = __ldg(reinterpret_cast<const float4*>(state + pid) + c);
  }
}

// The state record of list position pos: the staged copy when it is in the current batch
// [cur0, cur1), else the thread's slot filled from global memory.
__device__ __forceinline__ const PrimState* stp_record(StpRecs sm, PrimState* slot,
                                                      const PrimState* __restrict__ state,
                                                      const uint32_t* __restrict__ ids, uint32_t id_mask,
                                                      uint32_t pos, uint32_t cur0, uint32_t cur1) {
  if (pos >= cur0 && pos < cur1) return &sm[(int)(pos - cur0)];
  const float4* src = reinterpret_cast<const float4*>(state + (__ldg(ids + pos) & id_mask));
  float4* dst = reinterpret_cast<float4*>(slot);
#pragma unroll
  for (int c = 0; c < 8; ++c) dst[c] = __ldg(src + c);
  return slot;
}

// The forward's resort buffer with the blend data of each buffered entry: (hit depth, list
// position) in registers for the selection, and what blending the entry needs, formed
// when it is pushed (alpha, the normal's signed 1/|n_c| and n_c, with the extra channels
// the Gaussian curvature), in shared memory: field f of entry k at
// ent[(k * NF + f) * BLOCK + threadIdx.x]. Popping moves the last entry into the freed one.
template <int NF>
struct StpEntries {
  float t[RESORT];
  uint32_t pos[RESORT];
  int n = 0;
  float* ent;
  __device__ __forceinline__ void push(float tt, uint32_t p, const float (&d)[NF]) {
#pragma unroll
    for (int k = 0; k < RESORT; ++k)
      if (k == n) { t[k] = tt; pos[k] = p; }
    float* b = ent + (size_t)n * NF * BLOCK + threadIdx.x;
#pragma unroll
    for (int f = 0; f < NF; ++f) b[f * BLOCK] = d[f];
    ++n;
  }
  // remove the entry with the smallest (depth, list position): its depth in tt, its data in d
  __device__ __forceinline__ uint32_t pop(float& tt, float (&d)[NF]) {
    float bt = INFINITY;
    uint32_t bp = 0xFFFFFFFFu;
    int bk = 0;
#pragma unroll
    for (int k = 0; k < RESORT; ++k)
      if (k < n && (t[k] < bt || (t[k] == bt && pos[k] < bp))) { bt = t[k]; bp = pos[k]; bk = k; }
    float* b = ent + (size_t)bk * NF * BLOCK + threadIdx.x;
    const float* l = ent + (size_t)(n - 1) * NF * BLOCK + threadIdx.x;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      d[f] = b[f * BLOCK];
      b[f * BLOCK] = l[f * BLOCK];
    }
    float lt = 0.f;
    uint32_t lp = 0;
#pragma unroll
    for (int k = 0; k < RESORT; ++k)
      if (k == n - 1) { lt = t[k]; lp = pos[k]; }
#pragma unroll
    for (int k = 0; k < RESORT; ++k)
      if (k == bk) { t[k] = lt; pos[k] = lp; }
    --n;
    tt = bt;
    return bp;
  }
};
template <bool EXTRA>
constexpr int kStpEntFields = EXTRA ? 6 : 5;
}  // namespace

// The forward stages kStpFwdBatch records per batch, then holds the entries' blend data
// (measured 3.28 -> 2.67 ms at 3M / 1297x840 against re-evaluating each blended entry;
// 96 records at 4 CTAs per SM spill and take 2.83 ms).
constexpr int kStpFwdBatch = 128;
template <bool EXTRA>
constexpr size_t raster_stp_fwd_smem() {
  return sizeof(float4) * kStpStride * kStpFwdBatch + sizeof(float) * RESORT * kStpEntFields<EXTRA> * BLOCK;
}

template <bool EUCLID, bool EXTRA, bool STATS>
__global__ void __launch_bounds__(BLOCK, 3)
    k_raster_fwd_stp(const uint2* __restrict__ ranges, const uint32_t* __restrict__ ids,
                     const PrimState* __restrict__ state, RasterParams rp, float* __restrict__ out_rgb,
                     float* __restrict__ out_alpha, float* __restrict__ out_depth, float* __restrict__ out_normal,
                     float* __restrict__ T_final, uint32_t* __restrict__ n_blended, float* __restrict__ xres,
                     ExtraPlanes ex, RasterStats* __restrict__ stats, const uint32_t* __restrict__ tile_order) {
  constexpr int NF = kStpEntFields<EXTRA>;
  extern __shared__ float4 dyn_smem[];
  const StpRecs sm{dyn_smem};
  const int tile = tile_order ? (int)tile_order[blockIdx.x] : (int)blockIdx.x;
  int px, py;
  pixel_of(tile, rp.tiles_x, px, py);
  const bool inside = px < rp.W && py < rp.H;
  const uint2 rg = ranges[tile];
  const int n = (int)(rg.y - rg.x);
  const float X = (float)px + 0.5f, Y = (float)py + 0.5f;
  const float xn = (X - rp.cx) * rp.inv_fx, yn = (Y - rp.cy) * rp.inv_fy;
  float T = 1.f, cr = 0.f, cg = 0.f, cb = 0.f, dep = 0.f, nx = 0.f, ny = 0.f, nz = 0.f;
  float kc = 0.f, tref = 0.f, A1 = 0.f, A2 = 0.f, med = 0.f;
  uint32_t evals = 0, grazes = 0, isect = 0, hits = 0, blended = 0;
  bool done = !inside;
  StpEntries<NF> buf;
  buf.ent = reinterpret_cast<float*>(dyn_smem + (size_t)kStpStride * kStpFwdBatch);
  uint32_t cur0 = 0, cur1 = 0;  // list positions [cur0, cur1) staged in sm
  // blend the buffered entry with the smallest hit depth, from the data kept at its push
  // (its colour from the staged record when it is in the current batch, else global memory)
  auto blend = [&]() {
    float t;
    float d[NF];
    const uint32_t pos = buf.pop(t, d);
    const float al = d[0];
    const float Tn = __fmul_rn(T, __fsub_rn(1.f, al));
    if (Tn < rp.T_min) {
      done = true;
      return;
    }
    const float4 f7 = (pos >= cur0 && pos < cur1)
                          ? sm[(int)(pos - cur0)].f[7]
                          : __ldg(reinterpret_cast<const float4*>(state + (__ldg(ids + pos) & rp.id_mask)) + 7);
    const float w = al * T;
    cr = fmaf(w, f7.y, cr);
    cg = fmaf(w, f7.z, cg);
    cb = fmaf(w, f7.w, cb);
    dep = fmaf(w, t, dep);
    const float wn = w * d[1];
    nx = fmaf(wn, d[2], nx);
    ny = fmaf(wn, d[3], ny);
    nz = fmaf(wn, d[4], nz);
    if constexpr (EXTRA) {
      kc = fmaf(w, d[5], kc);
      if (blended == 0) tref = t;
      const float tau = t - tref;
      A1 = fmaf(w, tau, A1);
      A2 = fmaf(w * tau, tau, A2);
      if (T > 0.5f) med = fmaxf(med, t);
    }
    T = Tn;
    ++blended;
  };
  for (int b0 = 0; b0 < n; b0 += kStpFwdBatch) {
    if (__syncthreads_count(done) == BLOCK) break;
    const int cnt = min(kStpFwdBatch, n - b0);
    stage_batch_stp(sm, ids, rp.id_mask, state, rg.x + b0, cnt);
    cur0 = rg.x + (uint32_t)b0;
    cur1 = cur0 + (uint32_t)cnt;
    __syncthreads();
    if (!done) {
      for (int j = 0; j < cnt; ++j) {
        ++evals;
        Hit h;
        bool gz = false;
        const PrimState& P = sm[j];
        const bool hit = eval_pair<EUCLID>(P, X, Y, rp, h, gz, isect);
        grazes += gz;
        if (!hit) continue;
        ++hits;
        const float4 f5 = P.f[5];
        const float al = fminf(rp.alpha_max, __fmul_rn(f5.w, h.G));
        if (al < rp.alpha_min) continue;
        // the blend data: alpha and the camera-space normal n_c = W n_l, facing the camera
        const float4 f3 = P.f[3], f4 = P.f[4], f6 = P.f[6], f7 = P.f[7];
        const float nlx = 2.f * f5.y * h.x, nly = 2.f * f5.z * h.y;
        const float ncx = fmaf(f3.x, nlx, fmaf(f3.z, nly, -f4.x));
        const float ncy = fmaf(f3.y, nlx, fmaf(f3.w, nly, -f4.y));
        const float ncz = fmaf(f6.z, nlx, fmaf(f6.w, nly, -f7.x));
        float inn = rsqrtf(fmaf(ncx, ncx, fmaf(ncy, ncy, ncz * ncz)));
        if (fmaf(ncx, xn, fmaf(ncy, yn, ncz)) > 0.f) inn = -inn;
        float d[NF];
        d[0] = al;
        d[1] = inn;
        d[2] = ncx;
        d[3] = ncy;
        d[4] = ncz;
        if constexpr (EXTRA) d[NF - 1] = curvature(f5.y, f5.z, h.x, h.y);
        buf.push(P.f[2].w + h.s, rg.x + (uint32_t)(b0 + j), d);
        if (buf.n == RESORT) {
          blend();
          if (done) break;
        }
      }
    }
  }
  while (!done && buf.n > 0) blend();
  if (inside) {
    const size_t P = (size_t)rp.W * rp.H, pix = (size_t)py * rp.W + px;
    out_rgb[pix] = cr;
    out_rgb[P + pix] = cg;
    out_rgb[2 * P + pix] = cb;
    out_alpha[pix] = 1.f - T;
    out_depth[pix] = dep;
    out_normal[pix] = nx;
    out_normal[P + pix] = ny;
    out_normal[2 * P + pix] = nz;
    T_final[pix] = T;
    n_blended[pix] = blended;
    // the outputs again, for the front-to-back backward (the caller may reuse its planes)
    xres[pix] = cr;
    xres[P + pix] = cg;
    xres[2 * P + pix] = cb;
    xres[3 * P + pix] = dep;
    xres[4 * P + pix] = nx;
    xres[5 * P + pix] = ny;
    xres[6 * P + pix] = nz;
    xres[7 * P + pix] = kc;
    if constexpr (EXTRA) {
      if (ex.curvature) ex.curvature[pix] = kc;
      if (ex.distortion) ex.distortion[pix] = fmaf(1.f - T, A2, -A1 * A1);
      if (ex.median_depth) ex.median_depth[pix] = med;
      if (ex.resid) {
        ex.resid[pix] = tref;
        ex.resid[P + pix] = A1;
        ex.resid[2 * P + pix] = A2;
      }
    }
  }
  if (STATS && stats) {
    const unsigned ev = __reduce_add_sync(FULL, evals), is = __reduce_add_sync(FULL, isect);
    const unsigned hi = __reduce_add_sync(FULL, hits), bl = __reduce_add_sync(FULL, blended);
    const unsigned gzz = __reduce_add_sync(FULL, grazes);
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&stats->pair_evals, (unsigned long long)ev);
      atomicAdd(&stats->pair_isect, (unsigned long long)is);
      atomicAdd(&stats->pair_hits, (unsigned long long)hi);
      atomicAdd(&stats->pair_blended, (unsigned long long)bl);
      if (gzz) atomicAdd(&stats->grazing, (unsigned long long)gzz);
    }
  }
}

// Each pixel adds the gradient record of each blended pair to global memory: the pixels of
// a tile pop their own sequences, so in general the lanes of a warp blend different pairs
// at the same step and each adds its record with 16-byte vector atomics (per-tile shared
// accumulators would serialise on the many pixels that blend the same near primitive).
// A warp that is converged at the blend and blends one primitive in every lane sums the
// records with the list-order backward's reduce-scatter instead.
template <bool EUCLID, bool EXTRA, bool STATS>
__global__ void __launch_bounds__(BLOCK, 3)
    k_raster_bwd_stp(const uint2* __restrict__ ranges, const uint32_t* __restrict__ ids,
                     const PrimState* __restrict__ state, RasterParams rp, const float* __restrict__ g_rgb,
                     const float* __restrict__ g_alpha, const float* __restrict__ g_depth,
                     const float* __restrict__ g_normal, const float* __restrict__ T_final,
                     const float* __restrict__ xres, ExtraGrads eg, float* __restrict__ pgrad,
                     RasterStats* __restrict__ stats, const uint32_t* __restrict__ tile_order) {
  extern __shared__ float4 dyn_smem[];
  const StpRecs sm{dyn_smem};
  PrimState* slot = sm.ptr(kStpBwdBatch + threadIdx.x);
  __shared__ float spg[kPixFields<EXTRA> * BLOCK];
  const int tile = tile_order ? (int)tile_order[blockIdx.x] : (int)blockIdx.x;
  int px, py;
  pixel_of(tile, rp.tiles_x, px, py);
  const bool inside = px < rp.W && py < rp.H;
  const uint2 rg = ranges[tile];
  const int n = (int)(rg.y - rg.x);
  const float X = (float)px + 0.5f, Y = (float)py + 0.5f;
  const float xn = (X - rp.cx) * rp.inv_fx, yn = (Y - rp.cy) * rp.inv_fy;
  const size_t P = (size_t)rp.W * rp.H, pix = inside ? (size_t)py * rp.W + px : 0;
  const float Tfin = inside ? T_final[pix] : 1.f;
  const PixGrads pg = load_pix_grads<EXTRA>(inside, pix, P, Tfin, g_rgb, g_alpha, g_depth, g_normal, eg);
  store_pix<EXTRA, BLOCK>(spg, 0, pg);
  // sum over all blended pairs of w (g . X): from the forward's outputs
  float S_total = 0.f;
  if (inside) {
    S_total = pg.gR * xres[pix] + pg.gG * xres[P + pix] + pg.gB * xres[2 * P + pix] + pg.gD * xres[3 * P + pix] +
              pg.gNx * xres[4 * P + pix] + pg.gNy * xres[5 * P + pix] + pg.gNz * xres[6 * P + pix];
    if constexpr (EXTRA) {
      S_total += pg.gK * xres[7 * P + pix];
      if (pg.g_tau != 0.f || pg.g_tau2 != 0.f) S_total += pg.g_tau * eg.resid[P + pix] + pg.g_tau2 * eg.resid[2 * P + pix];
    }
  }
  float T = 1.f, S_prefix = 0.f;
  uint32_t n_pairs = 0, n_contrib_pairs = 0, dummy = 0;
  bool done = !inside;
  ResortBuf buf;
  uint32_t cur0 = 0, cur1 = 0;  // list positions [cur0, cur1) staged in sm
  auto blend = [&](uint32_t pos) {
    const uint32_t pid = __ldg(ids + pos) & rp.id_mask;
    const PrimState& Ps = *stp_record(sm, slot, state, ids, rp.id_mask, pos, cur0, cur1);
    Hit h;
    bool gz = false;
    if (!eval_pair<EUCLID>(Ps, X, Y, rp, h, gz, dummy)) return;
    const float oG = __fmul_rn(Ps.f[5].w, h.G);
    const float al = fminf(rp.alpha_max, oG);
    const float Tn = __fmul_rn(T, __fsub_rn(1.f, al));
    if (Tn < rp.T_min) {
      done = true;
      return;
    }
    float v[32];
    const PixGrads pgl = load_pix<EXTRA, BLOCK>(spg, 0);
    S_prefix += pair_grad<EUCLID, EXTRA, true>(Ps, h, oG, al, T, xn, yn, rp, pgl, S_total, S_prefix, v);
    ++n_contrib_pairs;
    // a whole warp that blends the same primitive at this point (pixels with the same hit
    // order so far) sums its records with the reduce-scatter; otherwise each lane adds its
    // record with vector atomics
    bool reduced = false;
    if (__activemask() == FULL && __all_sync(FULL, pid == __shfl_sync(FULL, pid, 0))) {
#pragma unroll
      for (int k = NGRAD; k < 32; ++k) v[k] = 0.f;
      int kc;
      const float r = warp_reduce_scatter20(v, kc);
      if (kc >= 0 && r != 0.f) atomicAdd(pgrad + (size_t)pid * NGRAD_PAD + kc, r);
      reduced = true;
    }
    if (!reduced) {
      float4* dst = reinterpret_cast<float4*>(pgrad + (size_t)pid * NGRAD_PAD);  // 80-byte records
#pragma unroll
      for (int k = 0; k < NGRAD / 4; ++k) {
        const float4 q = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
        if (q.x != 0.f || q.y != 0.f || q.z != 0.f || q.w != 0.f) atomicAdd(dst + k, q);
      }
    }
    T = Tn;
  };
  for (int b0 = 0; b0 < n; b0 += kStpBwdBatch) {
    if (__syncthreads_count(done) == BLOCK) break;
    const int cnt = min(kStpBwdBatch, n - b0);
    stage_batch_stp(sm, ids, rp.id_mask, state, rg.x + b0, cnt);
    cur0 = rg.x + (uint32_t)b0;
    cur1 = cur0 + (uint32_t)cnt;
    __syncthreads();
    if (!done) {
      for (int j = 0; j < cnt; ++j) {
        ++n_pairs;
        Hit h;
        bool gz = false;
        if (!eval_pair<EUCLID>(sm[j], X, Y, rp, h, gz, dummy)) continue;
        const float al = fminf(rp.alpha_max, __fmul_rn(sm[j].f[5].w, h.G));
        if (al < rp.alpha_min) continue;
        buf.push(sm[j].f[2].w + h.s, rg.x + (uint32_t)(b0 + j));
        if (buf.n == RESORT) {
          blend(buf.pop());
          if (done) break;
        }
      }
    }
  }
  while (!done && buf.n > 0) blend(buf.pop());
  if (STATS && stats) {
    const unsigned np = __reduce_add_sync(FULL, n_pairs), nc = __reduce_add_sync(FULL, n_contrib_pairs);
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&stats->bwd_pairs, (unsigned long long)np);
      atomicAdd(&stats->bwd_contrib, (unsigned long long)nc);
    }
  }
}

// Host-side selection of the instantiation: runs the statement(s) with the constants
// E_ (EUCLID) and X_ (EXTRA) set.
#define QGS_RASTER_DISPATCH(euclid, extra, ...)                          \
  do {                                                                   \
    if (euclid) {                                                        \
      if (extra) { constexpr bool E_ = true, X_ = true; __VA_ARGS__; }   \
      else { constexpr bool E_ = true, X_ = false; __VA_ARGS__; }        \
    } else {                                                             \
      if (extra) { constexpr bool E_ = false, X_ = true; __VA_ARGS__; }  \
      else { constexpr bool E_ = false, X_ = false; __VA_ARGS__; }       \
    }                                                                    \
  } while (0)

// The same with the pair counters (S_) compiled in or out.
#define QGS_RASTER_DISPATCH_S(euclid, extra, stats, ...)                        \
  do {                                                                          \
    if (stats) { constexpr bool S_ = true; QGS_RASTER_DISPATCH(euclid, extra, __VA_ARGS__); }  \
    else { constexpr bool S_ = false; QGS_RASTER_DISPATCH(euclid, extra, __VA_ARGS__); }       \
  } while (0)

cudaError_t launch_raster_fwd(bool euclid, bool extra, unsigned grid, cudaStream_t st, const uint2* ranges,
                              const uint32_t* ids, int id_stride, const PrimState* state, const RasterParams& rp,
                              float* out_rgb, float* out_alpha, float* out_depth, float* out_normal, float* T_final,
                              uint32_t* n_contrib, const ExtraPlanes& ex, RasterStats* stats,
                              const uint32_t* tile_order, uint8_t* inst_used) {
  QGS_RASTER_DISPATCH_S(euclid, extra, stats != nullptr,
                        k_raster_fwd<E_, X_, S_><<<grid, BLOCK, 0, st>>>(ranges, ids, id_stride, state, rp, out_rgb,
                                                                         out_alpha, out_depth, out_normal, T_final,
                                                                         n_contrib, ex, stats, tile_order, inst_used));
  return cudaGetLastError();
}

cudaError_t launch_raster_fwd_views(bool euclid, bool extra, unsigned grid, cudaStream_t st, const uint2* ranges,
                                    const uint32_t* ids, int id_stride, uint32_t id_mask, const PrimState* state,
                                    const ViewDesc* views, int n_views, const uint32_t* tile_base,
                                    RasterStats* stats, const uint32_t* tile_order) {
  QGS_RASTER_DISPATCH(euclid, extra,
                      k_raster_fwd_views<E_, X_><<<grid, BLOCK, 0, st>>>(ranges, ids, id_stride, id_mask, state,
                                                                         views, n_views, tile_base, stats,
                                                                         tile_order));
  return cudaGetLastError();
}

cudaError_t launch_raster_bwd(bool euclid, bool extra, unsigned grid, cudaStream_t st, const uint2* ranges,
                              const uint32_t* ids, int id_stride, const PrimState* state, const RasterParams& rp,
                              const float* g_rgb, const float* g_alpha, const float* g_depth, const float* g_normal,
                              const float* T_final, const uint32_t* n_contrib, const ExtraGrads& eg, float* pgrad,
                              RasterStats* stats, const uint32_t* tile_order, const uint8_t* inst_used) {
  cudaError_t e = cudaSuccess;
  int dev = 0, n_sm = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  auto go = [&](auto kern, int nt, size_t smem) {
    // the records, accumulators and flags exceed the 48 KB static limit (one pixel per
    // thread); set for every instantiation alike
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      kern<<<grid, nt, smem, st>>>(ranges, ids, id_stride, state, rp, g_rgb, g_alpha, g_depth, g_normal, T_final,
                                   n_contrib, eg, pgrad, stats, tile_order, inst_used);
  };
  const bool two = (int64_t)grid >= (int64_t)kBwdTwoPixelTilesPerSM * n_sm;
  QGS_RASTER_DISPATCH_S(euclid, extra, stats != nullptr, {
    if (two) go(k_raster_bwd<E_, X_, S_, 2>, BLOCK / 2, raster_bwd_smem<2>());
    else go(k_raster_bwd<E_, X_, S_, 1>, BLOCK, raster_bwd_smem<1>());
  });
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}
cudaError_t launch_raster_fwd_stp(bool euclid, bool extra, unsigned grid, cudaStream_t st, const uint2* ranges,
                                  const uint32_t* ids, const PrimState* state, const RasterParams& rp,
                                  float* out_rgb, float* out_alpha, float* out_depth, float* out_normal,
                                  float* T_final, uint32_t* n_blended, float* xres, const ExtraPlanes& ex,
                                  RasterStats* stats, const uint32_t* tile_order) {
  cudaError_t e = cudaSuccess;
  QGS_RASTER_DISPATCH_S(euclid, extra, stats != nullptr, {
    e = cudaFuncSetAttribute(k_raster_fwd_stp<E_, X_, S_>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)raster_stp_fwd_smem<X_>());
    if (e == cudaSuccess)
      k_raster_fwd_stp<E_, X_, S_><<<grid, BLOCK, raster_stp_fwd_smem<X_>(), st>>>(ranges, ids, state, rp, out_rgb, out_alpha,
                                                                        out_depth, out_normal, T_final, n_blended,
                                                                        xres, ex, stats, tile_order);
  });
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_raster_bwd_stp(bool euclid, bool extra, unsigned grid, cudaStream_t st, const uint2* ranges,
                                  const uint32_t* ids, const PrimState* state, const RasterParams& rp,
                                  const float* g_rgb, const float* g_alpha, const float* g_depth,
                                  const float* g_normal, const float* T_final, const float* xres,
                                  const ExtraGrads& eg, float* pgrad, RasterStats* stats,
                                  const uint32_t* tile_order) {
  cudaError_t e = cudaSuccess;
  QGS_RASTER_DISPATCH_S(euclid, extra, stats != nullptr, {
    e = cudaFuncSetAttribute(k_raster_bwd_stp<E_, X_, S_>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)RASTER_STP_BWD_SMEM);
    if (e == cudaSuccess)
      k_raster_bwd_stp<E_, X_, S_><<<grid, BLOCK, RASTER_STP_BWD_SMEM, st>>>(ranges, ids, state, rp, g_rgb, g_alpha,
                                                                        g_depth, g_normal, T_final, xres, eg,
                                                                        pgrad, stats, tile_order);
  });
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}
#undef QGS_RASTER_DISPATCH_S
#undef QGS_RASTER_DISPATCH

}  // namespace qgs
