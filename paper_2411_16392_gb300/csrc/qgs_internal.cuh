// Internal declarations shared by the translation units of libqgs (not part of the ABI).
#pragma once

#include "qgs_common.cuh"

namespace qgs {

struct SceneView {
  const float* mean;
  const float* quat;
  const float* scale;
  const float* curv;
  const float* opacity;
  const uint16_t* sh;
};

struct GradView {
  float* mean;
  float* quat;
  float* scale;
  float* curv;
  float* opacity;
  float* sh;
};

struct CamParams {
  float Rc[9];   // world -> camera rotation, row-major
  float tc[3];
  float cw[3];   // camera centre in world coordinates
  float fx, fy, cx, cy, near;
  int W, H, tiles_x, tiles_y;
};

// ---------------------------------------------------------------- tile culling
// A primitive's screen bounds for the tile test, measured from the projected centre
// (uc, vc): the parallelogram (normals of the projected local x and y axes with the spans
// of the projected support box along them) and the conic of the chord ellipsoid
// (F(p) = p^T q p - 2 l.p <= 1, q = [[qa, qb], [qb, qc]], l = (la, lb)). All bit-exact
// (correctly rounded FP32 in a fixed order).
struct TileSlab {
  float4 a;  // (n1x, n1y, s1min, s1max)
  float4 b;  // (n2x, n2y, s2min, s2max)
  float4 c;  // (uc, vc, qa, qb)
  float4 d;  // (qc, la, lb, 1/qa)
  float4 e;  // (1/qc, -, -, -); qa = 0: conic disabled (every tile passes)
};

// Does a tile meet the parallelogram? Range of n . (x - c) over the tile's pixel centres
// against each span, padded by 2e-3 px + 1e-5 of the span ends (the same FP32
// specification as the oracle's tile test: the minimum and maximum over the four corner
// sums n_x (x - u_c) + n_y (y - v_c), each rounded). Correctly rounded addition is monotone
// in each operand, so the minimum of the four rounded sums is the rounded sum of the
// column term's minimum and the row term's minimum (likewise for the maximum): the terms'
// extremes are formed once per column and per row, and a tile costs one addition per bound.
struct TileRow {  // per row: offsets of its first and last pixel centre, extremes of n_y (y - v_c)
  float y0, y1, bmin[2], bmax[2];
};
struct TileCol {  // per column: offsets of its first and last pixel centre, extremes of n_x (x - u_c)
  float x0, x1, amin[2], amax[2];
};
__device__ __forceinline__ TileRow tile_row(const TileSlab& t, int ty, int H) {
  TileRow r;
  r.y0 = __fsub_rn(__fadd_rn((float)(16 * ty), 0.5f), t.c.y);
  r.y1 = __fsub_rn(__fadd_rn((float)min(16 * ty + 15, H - 1), 0.5f), t.c.y);
  const float p0 = __fmul_rn(t.a.y, r.y0), p1 = __fmul_rn(t.a.y, r.y1);
  const float q0 = __fmul_rn(t.b.y, r.y0), q1 = __fmul_rn(t.b.y, r.y1);
  r.bmin[0] = fminf(p0, p1); r.bmax[0] = fmaxf(p0, p1);
  r.bmin[1] = fminf(q0, q1); r.bmax[1] = fmaxf(q0, q1);
  return r;
}
__device__ __forceinline__ TileCol tile_col(const TileSlab& t, int tx, int W) {
  TileCol c;
  c.x0 = __fsub_rn(__fadd_rn((float)(16 * tx), 0.5f), t.c.x);
  c.x1 = __fsub_rn(__fadd_rn((float)min(16 * tx + 15, W - 1), 0.5f), t.c.x);
  const float p0 = __fmul_rn(t.a.x, c.x0), p1 = __fmul_rn(t.a.x, c.x1);
  const float q0 = __fmul_rn(t.b.x, c.x0), q1 = __fmul_rn(t.b.x, c.x1);
  c.amin[0] = fminf(p0, p1); c.amax[0] = fmaxf(p0, p1);
  c.amin[1] = fminf(q0, q1); c.amax[1] = fmaxf(q0, q1);
  return c;
}
// The padded spans of a primitive's two slabs (s_min - pad, s_max + pad), formed once.
struct TileSpans {
  float lo[2], hi[2];
};
__device__ __forceinline__ TileSpans tile_spans(const TileSlab& t) {
  TileSpans sp;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float4 s = k == 0 ? t.a : t.b;
    const float pad = __fadd_rn(2e-3f, __fmul_rn(1e-5f, __fadd_rn(fabsf(s.z), fabsf(s.w))));
    sp.lo[k] = __fsub_rn(s.z, pad);
    sp.hi[k] = __fadd_rn(s.w, pad);
  }
  return sp;
}

// F(u, v) = u (qa u + 2 qb v - 2 la) + v (qc v - 2 lb): the conic of the chord ellipsoid at
// the pixel offset (u, v) from the projected centre (F <= 1 inside), FP32 in this order.
__device__ __forceinline__ float conic_value(const TileSlab& t, float u, float v) {
  const float inner = __fsub_rn(__fadd_rn(__fmul_rn(t.c.z, u), __fmul_rn(2.f, __fmul_rn(t.c.w, v))),
                                __fmul_rn(2.f, t.d.y));
  return __fadd_rn(__fmul_rn(u, inner), __fmul_rn(v, __fsub_rn(__fmul_rn(t.d.x, v), __fmul_rn(2.f, t.d.z))));
}

// Does the rectangle of the tile's pixel-centre offsets meet the conic F <= 1? F is convex
// and F(0) <= 1, so: the rectangle holds the origin, or the minimum of F along an edge
// facing the origin (its stationary point, clamped to the edge) is <= 1.
__device__ __forceinline__ bool conic_meets(const TileSlab& t, const TileCol& c, const TileRow& r) {
  if (!(t.c.z > 0.f)) return true;
  if (c.x0 <= 0.f && 0.f <= c.x1 && r.y0 <= 0.f && 0.f <= r.y1) return true;
  if (c.x0 > 0.f || c.x1 < 0.f) {
    const float ue = c.x0 > 0.f ? c.x0 : c.x1;
    const float vs = fminf(fmaxf(__fmul_rn(__fsub_rn(t.d.z, __fmul_rn(t.c.w, ue)), t.e.x), r.y0), r.y1);
    if (conic_value(t, ue, vs) <= 1.f) return true;
  }
  if (r.y0 > 0.f || r.y1 < 0.f) {
    const float ve = r.y0 > 0.f ? r.y0 : r.y1;
    const float us = fminf(fmaxf(__fmul_rn(__fsub_rn(t.d.y, __fmul_rn(t.c.w, ve)), t.d.w), c.x0), c.x1);
    if (conic_value(t, us, ve) <= 1.f) return true;
  }
  return false;
}

__device__ __forceinline__ bool tile_meets(const TileSlab& t, const TileSpans& sp, const TileCol& c,
                                           const TileRow& r) {
  bool ok = true;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float lo = __fadd_rn(c.amin[k], r.bmin[k]);
    const float hi = __fadd_rn(c.amax[k], r.bmax[k]);
    ok = ok && !(hi < sp.lo[k]) && !(lo > sp.hi[k]);
  }
  return ok && conic_meets(t, c, r);
}

// The tile test with its per-column and per-row terms hoisted: tile_col, tile_row and the
// parts of conic_meets that depend on the column or the row alone (the edge facing the
// origin, the unclamped stationary point along it, and the products of the conic's value
// that involve only that coordinate) are formed once per column or row of a rectangle; a
// tile then costs the additions, clamps and products that involve both. Every operation is
// the same correctly rounded one, on the same operands, as in tile_meets, so the result
// is identical bit for bit.
struct ColTerms {
  float4 a;  // x0, x1, ue (edge facing the origin), vs (unclamped stationary v on it)
  float4 b;  // amin[0], amax[0], amin[1], amax[1]
  float4 c;  // qa ue, -, -, -
};
struct RowTerms {
  float4 a;  // y0, y1, ve (edge facing the origin), us (unclamped stationary u on it)
  float4 b;  // bmin[0], bmax[0], bmin[1], bmax[1]
  float4 c;  // 2 (qb ve), ve (qc ve - 2 lb), -, -
};
constexpr int kHoistMax = 48;  // rectangles up to this many columns and rows take the hoisted test
__device__ __forceinline__ ColTerms col_terms(const TileSlab& t, int tx, int W) {
  const TileCol c = tile_col(t, tx, W);
  const float ue = c.x0 > 0.f ? c.x0 : c.x1;
  ColTerms o;
  o.a = make_float4(c.x0, c.x1, ue, __fmul_rn(__fsub_rn(t.d.z, __fmul_rn(t.c.w, ue)), t.e.x));
  o.b = make_float4(c.amin[0], c.amax[0], c.amin[1], c.amax[1]);
  o.c = make_float4(__fmul_rn(t.c.z, ue), 0.f, 0.f, 0.f);
  return o;
}
__device__ __forceinline__ RowTerms row_terms(const TileSlab& t, int ty, int H) {
  const TileRow r = tile_row(t, ty, H);
  const float ve = r.y0 > 0.f ? r.y0 : r.y1;
  RowTerms o;
  o.a = make_float4(r.y0, r.y1, ve, __fmul_rn(__fsub_rn(t.d.y, __fmul_rn(t.c.w, ve)), t.d.w));
  o.b = make_float4(r.bmin[0], r.bmax[0], r.bmin[1], r.bmax[1]);
  o.c = make_float4(__fmul_rn(2.f, __fmul_rn(t.c.w, ve)),
                    __fmul_rn(ve, __fsub_rn(__fmul_rn(t.d.x, ve), __fmul_rn(2.f, t.d.z))), 0.f, 0.f);
  return o;
}
// tile_meets from the hoisted terms (two_la = 2 la, two_lb = 2 lb, formed once per primitive)
__device__ __forceinline__ bool tile_meets_hoisted(const TileSlab& t, const TileSpans& sp, const ColTerms& C,
                                                   const RowTerms& R, float two_la, float two_lb) {
  bool ok = !(__fadd_rn(C.b.y, R.b.y) < sp.lo[0]) && !(__fadd_rn(C.b.x, R.b.x) > sp.hi[0]) &&
            !(__fadd_rn(C.b.w, R.b.w) < sp.lo[1]) && !(__fadd_rn(C.b.z, R.b.z) > sp.hi[1]);
  if (!(t.c.z > 0.f)) return ok;  // conic disabled
  const bool xin = C.a.x <= 0.f && 0.f <= C.a.y, yin = R.a.x <= 0.f && 0.f <= R.a.y;
  // edge x = ue, v clamped to the row: F(ue, vs)
  const float vs = fminf(fmaxf(C.a.w, R.a.x), R.a.y);
  const float inx = __fsub_rn(__fadd_rn(C.c.x, __fmul_rn(2.f, __fmul_rn(t.c.w, vs))), two_la);
  const float fx = __fadd_rn(__fmul_rn(C.a.z, inx), __fmul_rn(vs, __fsub_rn(__fmul_rn(t.d.x, vs), two_lb)));
  // edge y = ve, u clamped to the column: F(us, ve)
  const float us = fminf(fmaxf(R.a.w, C.a.x), C.a.y);
  const float iny = __fsub_rn(__fadd_rn(__fmul_rn(t.c.z, us), R.c.x), two_la);
  const float fy = __fadd_rn(__fmul_rn(us, iny), R.c.y);
  return ok && ((xin && yin) || (!xin && fx <= 1.f) || (!yin && fy <= 1.f));
}

// The whole warp enumerates one primitive's rectangle r in row-major order, 32 tiles at a
// time (lane l takes tile e = e0 + l, its (tx, ty) advanced without divisions); f(k, tx,
// ty) runs for every tile that meets the parallelogram and the conic (every tile when t
// is null), k counting them in row-major order. Returns their number. bits_out (when
// given) receives the pass mask of each group of 32 tiles; bits_in (when given) replays
// such masks instead of testing. Call with the same arguments on every lane.
constexpr uint32_t kNoTileBits = 0xFFFFFFFFu;  // primitive without cached tile masks

template <typename F>
__device__ __forceinline__ uint32_t warp_tiles(short4 r, const TileSlab* t, int W, int H, F&& f,
                                               uint32_t* bits_out = nullptr, const uint32_t* bits_in = nullptr,
                                               float4* hoist = nullptr) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  const int w = r.y - r.x + 1;
  const int h = r.w - r.z + 1;
  const uint32_t total = (uint32_t)w * (uint32_t)h;
  TileSlab ts;
  TileSpans sp{};
  if (t && !bits_in) {
    ts = *t;
    sp = tile_spans(ts);
  }
  // hoisted test: the rectangle's column and row terms in the warp's scratch (hoist holds
  // 3 float4 per entry, kHoistMax columns then kHoistMax rows)
  const bool hoisted = t && !bits_in && hoist && w <= kHoistMax && h <= kHoistMax;
  float two_la = 0.f, two_lb = 0.f;
  if (hoisted) {
    two_la = __fmul_rn(2.f, ts.d.y);
    two_lb = __fmul_rn(2.f, ts.d.z);
    __syncwarp();  // the previous primitive's terms are no longer read
    for (int c = lane; c < w; c += 32) {
      const ColTerms ct = col_terms(ts, r.x + c, W);
      hoist[3 * c] = ct.a;
      hoist[3 * c + 1] = ct.b;
      hoist[3 * c + 2] = ct.c;
    }
    for (int q = lane; q < h; q += 32) {
      const RowTerms rt = row_terms(ts, r.z + q, H);
      hoist[3 * (kHoistMax + q)] = rt.a;
      hoist[3 * (kHoistMax + q) + 1] = rt.b;
      hoist[3 * (kHoistMax + q) + 2] = rt.c;
    }
    __syncwarp();
  }
  int ty = r.z + lane / w, tx = r.x + lane % w;  // tile e = lane
  const int sy = 32 / w, sx = 32 - sy * w;          // tile e + 32: sy rows and sx columns on
  int row_y = -1;
  TileRow row{};
  uint32_t base = 0;
  uint32_t words = 0;  // bits_in: lane l holds mask word 32 g + l of the current group g
  for (uint32_t e0 = 0; e0 < total; e0 += 32) {
    uint32_t m;
    bool pass;
    if (bits_in) {
      const uint32_t wi = e0 >> 5;
      if ((wi & 31u) == 0) {
        const uint32_t wl = wi + (uint32_t)lane;
        words = wl < ((total + 31u) >> 5) ? bits_in[wl] : 0u;
      }
      m = __shfl_sync(0xffffffffu, words, (int)(wi & 31u));
      pass = (m >> lane) & 1u;
    } else {
      pass = e0 + (uint32_t)lane < total;
      if (pass && hoisted) {
        const float4* cp = hoist + 3 * (tx - r.x);
        const float4* rp = hoist + 3 * (kHoistMax + ty - r.z);
        const ColTerms ct{cp[0], cp[1], cp[2]};
        const RowTerms rt{rp[0], rp[1], rp[2]};
        pass = tile_meets_hoisted(ts, sp, ct, rt, two_la, two_lb);
      } else if (pass && t) {
        if (ty != row_y) {
          row = tile_row(ts, ty, H);
          row_y = ty;
        }
        pass = tile_meets(ts, sp, tile_col(ts, tx, W), row);
      }
      m = __ballot_sync(0xffffffffu, pass);
      if (bits_out && lane == 0) bits_out[e0 >> 5] = m;
    }
    if (pass) f(base + __popc(m & lt), tx, ty);
    base += __popc(m);
    tx += sx;  // tile e + 32
    ty += sy;
    if (tx > r.y) {
      tx -= w;
      ++ty;
    }
  }
  return base;
}

// Per primitive with a nonempty rectangle: count its tiles that meet its screen bounds;
// primitives left with none are culled (count 0, rectangle -1s, depth key 0xFFFFFFFF).
// Writes the visibility flags (when given) and adds the visible and instance totals
// to counters[0], counters[1]. With tbits: each primitive's pass masks (one word per 32
// rectangle tiles) go to tbits + tbits_off[i], words taken from counters[2] (the total
// requested, even beyond cap_words); a primitive that does not fit gets kNoTileBits.
// Launched with kCountBlock threads per CTA (small CTAs: the warps' work varies widely and
// a CTA's slot is held until its slowest warp ends).
constexpr int kCountBlock = 64;
// With cps (several views of one scene, blockIdx.y = view): the arrays hold entries
// v * n + i and each view's image size comes from cps[v].
__global__ void k_count_tiles(int64_t n, const TileSlab* tslab, int W, int H, uint32_t* count, short4* rect,
                              uint32_t* zkey, uint32_t* vflag, uint32_t* counters, uint32_t* tbits,
                              uint32_t* tbits_off, uint32_t cap_words, const CamParams* cps = nullptr);

// ---------------------------------------------------------------- preprocessing
// k_preprocess / k_preprocess_views: 256 threads per CTA, kPreChunks x 256 primitives per
// CTA (the grid is pre_blocks(n) wide).
constexpr int kPreChunks = 8;
inline unsigned pre_blocks(int64_t n) { return (unsigned)((n + kPreChunks * 256 - 1) / (kPreChunks * 256)); }
// Per primitive i: projected state (visible ones only), tile count of the rectangle,
// depth key, tile rectangle; idx[i] = i, vflag[i] = (count > 0) and the screen bounds
// (tslab) when given; counters[0] += visible, counters[1] += tile instances when given.
__global__ void k_preprocess(int64_t n, SceneView sc, CamParams cp, PrimState* state, uint32_t* count,
                             uint32_t* zkey, uint32_t* idx, short4* rect, uint32_t* counters, uint32_t* vflag,
                             TileSlab* tslab);
__global__ void k_preprocess_views(int64_t n, SceneView sc, const CamParams* cps, PrimState* state, uint32_t* count,
                                   uint32_t* zkey, uint32_t* idx, short4* rect, uint32_t* n_visible,
                                   TileSlab* tslab);
// StopThePop ordering: per (tile, primitive) instance, in primitive order,
// key = (tile << 32) | bits of the depth where the ray of the tile pixel closest to the
// projected vertex meets the paraboloid; value = primitive.
__global__ void k_emit_hit(int64_t n, SceneView sc, CamParams cp, const uint32_t* count, const short4* rect,
                           const TileSlab* tslab, const uint32_t* offs, uint64_t* keys, uint32_t* vals,
                           const uint32_t* tbits, const uint32_t* tbits_off);
// list == nullptr: threads 0..n-1 are primitives 0..n-1; else primitive list[j].
// pgrad_by_pos: the gradient record of thread j is pgrad[j] (state gathered in list
// order), else pgrad[primitive].
__global__ void k_preprocess_bwd(int64_t n, const uint32_t* list, SceneView sc, CamParams cp, const uint32_t* count,
                                 const float* pgrad, bool pgrad_by_pos, GradView gd);

// ---------------------------------------------------------------- debug bounds checks
// Checks of computed indices in the binning kernels: the emission's instance slots, the
// range pass's tile ids, the radix sort's scatter positions. Built with -DQGS_DEBUG_CHECKS,
// a failed check sets its bit in its translation unit's check word (a static __device__
// word per .cu file) and the guarded access is skipped: the kernel never traps and never
// writes out of range. Without the flag QGS_CHECK is the constant true and compiles away.
#ifdef QGS_DEBUG_CHECKS
#define QGS_CHECK(word, cond, bit) ((cond) || (atomicOr(&(word), (uint32_t)(bit)), false))
constexpr bool kDebugChecks = true;
#else
#define QGS_CHECK(word, cond, bit) true
constexpr bool kDebugChecks = false;
#endif
constexpr uint32_t kChkInstance = 1u;  // an emitted instance's slot beyond the instance count
constexpr uint32_t kChkTile = 2u;      // a tile id beyond the tile grid
constexpr uint32_t kChkScatter = 4u;   // a radix-sort scatter position beyond the chunk or the keys
// Reads and clears sort.cu's check word on the current device (0 without the checks).
cudaError_t sort_check_word(uint32_t* word);

// ---------------------------------------------------------------- sorting / scan
// Keys per CTA of the radix sort (histogram sizes depend on it).
constexpr int kRadixChunk = 2048;

// Polls a look-back chunk makes for a predecessor's digit counts before it gives up.
constexpr int kLookbackSpins = 1 << 22;

// Temporary storage of the device-wide scan and radix sort.
struct SortTemp {
  uint32_t* hist = nullptr;   // radix_hist_elems(n): count matrix, or the single-pass status words
  uint32_t* scan_tmp = nullptr;
  size_t hist_cap = 0, scan_cap = 0;
  // Device word set to nonzero when a look-back wait gave up (optional). Once it is set,
  // the following look-back passes (and the kernels of the pipeline that read a sort's
  // output) do nothing, so an abandoned sort never leads to an out-of-range access.
  uint32_t* err = nullptr;
  int spins = kLookbackSpins;  // poll limit of each look-back wait
  // Test hook (0 in normal use): the first look-back pass starts its chunk tickets at this
  // value and launches that many fewer CTAs, so chunk 0 never publishes its digit counts
  // and the waits for it run out.
  int withhold_chunks = 0;
};

// Exclusive prefix sum of n u32 values; out[n] receives the total (out has n + 1 slots).
cudaError_t scan_exclusive_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* tmp, size_t tmp_cap,
                               cudaStream_t st);
size_t scan_tmp_elems(int64_t n);

// Stable LSD radix sort of u32 keys with u32 values over bits [begin_bit, end_bit).
// Ping-pongs between (k0, v0) and (k1, v1); returns true if the result ends in (k1, v1).
bool radix_sort_u32_pairs(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, int64_t n, int begin_bit,
                          int end_bit, SortTemp& tmp, cudaStream_t st, cudaError_t* err);
// Stable LSD radix sort of u32 keys (no values) over bits [begin_bit, end_bit).
bool radix_sort_u32_keys(uint32_t* k0, uint32_t* k1, int64_t n, int begin_bit, int end_bit, SortTemp& tmp,
                         cudaStream_t st, cudaError_t* err);
// Stable LSD radix sort of u64 keys (no values) over bits [begin_bit, end_bit).
bool radix_sort_u64_keys(uint64_t* k0, uint64_t* k1, int64_t n, int begin_bit, int end_bit, SortTemp& tmp,
                         cudaStream_t st, cudaError_t* err);
// Stable LSD radix sort of u64 keys with u32 values over bits [begin_bit, end_bit).
bool radix_sort_u64_pairs(uint64_t* k0, uint32_t* v0, uint64_t* k1, uint32_t* v1, int64_t n, int begin_bit,
                          int end_bit, SortTemp& tmp, cudaStream_t st, cudaError_t* err);
size_t radix_hist_elems(int64_t n);

// ---------------------------------------------------------------- compositing
struct RasterStats {
  unsigned long long pair_evals, pair_isect, pair_hits, pair_blended, grazing;
  unsigned long long bwd_pairs, bwd_contrib;
};

// Kernel launches issued by the calling host thread (the library's launch sites
// increment it; the API reports per-call differences).
inline int64_t& launch_counter() {
  static thread_local int64_t n = 0;
  return n;
}

// Optional extra output planes of the forward (device, any may be null): curvature map,
// depth distortion, median depth, and the per-pixel residue (c, A1, A2) [3P] that the
// distortion's backward reads.
struct ExtraPlanes {
  float *curvature, *distortion, *median_depth, *resid;
};
// Upstream gradients of the extra planes (null: zero) and the forward's residue.
struct ExtraGrads {
  const float *g_curvature, *g_distortion, *resid;
};

// One view of a batched forward: its raster constants and output planes (device).
struct ViewDesc {
  RasterParams rp;
  float *rgb, *alpha, *depth, *normal;
  float* T_final;        // may be null (no residue kept)
  uint32_t* n_contrib;   // may be null
  ExtraPlanes ex;        // extra planes (EXTRA instantiation only)
};

// Compositing launches (defined with the kernels). euclid: Euclidean-distance density
// instead of the geodesic one; extra: the curvature, distortion and median-depth
// channels. Each returns the launch's error status.
cudaError_t launch_raster_fwd(bool euclid, bool extra, unsigned grid, cudaStream_t st, const uint2* ranges,
                              const uint32_t* ids, int id_stride, const PrimState* state, const RasterParams& rp,
                              float* out_rgb, float* out_alpha, float* out_depth, float* out_normal, float* T_final,
                              uint32_t* n_contrib, const ExtraPlanes& ex, RasterStats* stats,
                              const uint32_t* tile_order, uint8_t* inst_used);
// ids[k * id_stride] & id_mask indexes state (every view's rp.id_mask is replaced).
cudaError_t launch_raster_fwd_views(bool euclid, bool extra, unsigned grid, cudaStream_t st, const uint2* ranges,
                                    const uint32_t* ids, int id_stride, uint32_t id_mask, const PrimState* state,
                                    const ViewDesc* views, int n_views, const uint32_t* tile_base,
                                    RasterStats* stats, const uint32_t* tile_order);
// StopThePop ordering (per-tile hit-depth lists, per-pixel resorting in a buffer of 8):
// forward keeps T_final, the blended count and the outputs (xres, 8 planes: rgb, depth,
// normal, curvature) for the front-to-back backward, which adds per-pixel gradient
// records to pgrad (indexed by the sorted ids).
cudaError_t launch_raster_fwd_stp(bool euclid, bool extra, unsigned grid, cudaStream_t st, const uint2* ranges,
                                  const uint32_t* ids, const PrimState* state, const RasterParams& rp,
                                  float* out_rgb, float* out_alpha, float* out_depth, float* out_normal,
                                  float* T_final, uint32_t* n_blended, float* xres, const ExtraPlanes& ex,
                                  RasterStats* stats, const uint32_t* tile_order);
cudaError_t launch_raster_bwd_stp(bool euclid, bool extra, unsigned grid, cudaStream_t st, const uint2* ranges,
                                  const uint32_t* ids, const PrimState* state, const RasterParams& rp,
                                  const float* g_rgb, const float* g_alpha, const float* g_depth,
                                  const float* g_normal, const float* T_final, const float* xres,
                                  const ExtraGrads& eg, float* pgrad, RasterStats* stats,
                                  const uint32_t* tile_order);
cudaError_t launch_raster_bwd(bool euclid, bool extra, unsigned grid, cudaStream_t st, const uint2* ranges,
                              const uint32_t* ids, int id_stride, const PrimState* state, const RasterParams& rp,
                              const float* g_rgb, const float* g_alpha, const float* g_depth, const float* g_normal,
                              const float* T_final, const uint32_t* n_contrib, const ExtraGrads& eg, float* pgrad,
                              RasterStats* stats, const uint32_t* tile_order, const uint8_t* inst_used);

}  // namespace qgs
