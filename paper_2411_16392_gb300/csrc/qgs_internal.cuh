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

// ---------------------------------------------------------------- preprocessing
// Per primitive i: projected state (visible ones only), tile count, depth key, tile
// rectangle; idx[i] = i and vflag[i] = (count > 0) when given. counters[0] += visible,
// counters[1] += tile instances.
__global__ void k_preprocess(int64_t n, SceneView sc, CamParams cp, PrimState* state, uint32_t* count,
                             uint32_t* zkey, uint32_t* idx, short4* rect, uint32_t* counters, uint32_t* vflag);
__global__ void k_preprocess_views(int64_t n, SceneView sc, const CamParams* cps, PrimState* state, uint32_t* count,
                                   uint32_t* zkey, uint32_t* idx, short4* rect, uint32_t* n_visible);
// StopThePop ordering: per (tile, primitive) instance, in primitive order,
// key = (tile << 32) | bits of the depth where the ray of the tile pixel closest to the
// projected vertex meets the paraboloid; value = primitive.
__global__ void k_emit_hit(int64_t n, SceneView sc, CamParams cp, const uint32_t* count, const short4* rect,
                           const uint32_t* offs, uint64_t* keys, uint32_t* vals);
// list == nullptr: threads 0..n-1 are primitives 0..n-1; else primitive list[j].
// pgrad_by_pos: the gradient record of thread j is pgrad[j] (state gathered in list
// order), else pgrad[primitive].
__global__ void k_preprocess_bwd(int64_t n, const uint32_t* list, SceneView sc, CamParams cp, const uint32_t* count,
                                 const float* pgrad, bool pgrad_by_pos, GradView gd);

// ---------------------------------------------------------------- sorting / scan
// Keys per CTA of the radix sort (histogram sizes depend on it).
constexpr int kRadixChunk = 2048;

// Temporary storage of the device-wide scan and radix sort.
struct SortTemp {
  uint32_t* hist = nullptr;   // [256 * max_blocks]
  uint32_t* scan_tmp = nullptr;
  size_t hist_cap = 0, scan_cap = 0;
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
cudaError_t launch_raster_fwd_views(bool euclid, bool extra, unsigned grid, cudaStream_t st, const uint2* ranges,
                                    const uint32_t* ids, int id_stride, const PrimState* state,
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
constexpr size_t RASTER_BWD_SMEM = sizeof(PrimState) * BLOCK + sizeof(float) * BLOCK * NGRAD + sizeof(int) * BLOCK;
cudaError_t launch_raster_bwd(bool euclid, bool extra, unsigned grid, cudaStream_t st, const uint2* ranges,
                              const uint32_t* ids, int id_stride, const PrimState* state, const RasterParams& rp,
                              const float* g_rgb, const float* g_alpha, const float* g_depth, const float* g_normal,
                              const float* T_final, const uint32_t* n_contrib, const ExtraGrads& eg, float* pgrad,
                              RasterStats* stats, const uint32_t* tile_order, const uint8_t* inst_used);

}  // namespace qgs
