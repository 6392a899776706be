// C ABI of libqgs: rendering context, tile binning and the forward/backward pipelines.
//
// Forward pipeline on the caller's stream (supplementary, per-tile sorting; Sec. 3.1-3.2):
//   k_preprocess            per primitive: projected state, tile rectangle, depth key
//   depth sort              radix sort of the visible primitives by depth (u32 keys)
//   count gather + scan     instance offsets in depth order
//   (one host read of the instance total, to size the instance buffers)
//   k_emit_sorted           (tile << 32 | primitive) per covered tile, in depth order
//   tile sort               stable radix sort of the instances on the tile bits only
//   k_tile_ranges           [start, end) of every tile's list
//   k_raster_fwd            per-tile compositing
// Because the instances are emitted in depth order and the tile sort is stable, the
// final order equals the order of the 64-bit keys (tile << 32 | depth bits) with ties
// broken by primitive index. sort_mode 1 instead emits the 64-bit keys in primitive
// order and radix-sorts all of their significant bits.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "qgs_internal.cuh"

using namespace qgs;

namespace {

template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t cap = 0;
  cudaError_t reserve(size_t n) {
    if (n <= cap) return cudaSuccess;
    size_t want = n + n / 4 + 64;
    if (p) {
      // work already enqueued may still use the old buffer (the forward enqueues kernels
      // before it waits for its totals): let it finish before freeing
      cudaDeviceSynchronize();
      cudaFree(p);
    }
    p = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc((void**)&p, want * sizeof(T));
    if (e != cudaSuccess) {
      p = nullptr;
      return e;
    }
    cap = want;
    return cudaSuccess;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
};

// Kernels that read a radix sort's output (an index permutation or sorted tile keys)
// return at once when the sort's error word is set: an abandoned sort leaves indices that
// are not a permutation, and using them could read or write out of range.
__device__ __forceinline__ bool sort_failed(const uint32_t* err) { return err && *(volatile const uint32_t*)err; }

#ifdef QGS_DEBUG_CHECKS
__device__ uint32_t g_check_api;  // QGS_CHECK bits of this file's kernels
#endif

__global__ void k_gather_u32(int64_t n, const uint32_t* __restrict__ idx, const uint32_t* __restrict__ src,
                             uint32_t* __restrict__ dst, const uint32_t* err) {
  if (sort_failed(err)) return;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[idx[i]];
}

// Write the tile instances of 32 consecutive primitives per warp (coalesced): the tiles
// of each rectangle that meet the primitive's screen bounds (all of them when tslab is
// null), replayed from the tile-count pass's masks where it stored them (tbits). sidx == nullptr: primitive order (full-key mode, keys carry the depth bits,
// values the primitive); otherwise depth order (keys carry the primitive in their low half).
__global__ void k_emit(int64_t n, const uint32_t* __restrict__ sidx, const uint32_t* __restrict__ count,
                       const short4* __restrict__ rect, const TileSlab* __restrict__ tslab, int W, int H,
                       const uint32_t* __restrict__ offs, const uint32_t* __restrict__ zkey, int tiles_x,
                       uint64_t* __restrict__ keys, uint32_t* __restrict__ vals, const uint32_t* __restrict__ tbits,
                       const uint32_t* __restrict__ tbits_off, const uint32_t* err) {
  if (sort_failed(err)) return;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t pid = 0, c = 0, off = 0, lowv = 0;
  short4 r = make_short4(0, 0, 0, 0);
  if (j < n) {
    pid = sidx ? sidx[j] : (uint32_t)j;
    c = count[pid];
    if (c) {
      off = offs[j];
      r = rect[pid];
      lowv = sidx ? pid : zkey[pid];
    }
  }
  for (int k = 0; k < 32; ++k) {
    const uint32_t cc = __shfl_sync(0xffffffffu, c, k);
    if (!cc) continue;
    const uint32_t pp = __shfl_sync(0xffffffffu, pid, k);
    const uint32_t oo = __shfl_sync(0xffffffffu, off, k);
    const uint32_t lv = __shfl_sync(0xffffffffu, lowv, k);
    const short4 rk = make_short4((short)__shfl_sync(0xffffffffu, (int)r.x, k),
                                  (short)__shfl_sync(0xffffffffu, (int)r.y, k),
                                  (short)__shfl_sync(0xffffffffu, (int)r.z, k),
                                  (short)__shfl_sync(0xffffffffu, (int)r.w, k));
    const uint32_t wo = tbits ? tbits_off[pp] : kNoTileBits;
    warp_tiles(rk, tslab ? tslab + pp : nullptr, W, H, [&](uint32_t e, int tx, int ty) {
      const uint32_t tile = (uint32_t)ty * (uint32_t)tiles_x + (uint32_t)tx;
      keys[(size_t)oo + e] = ((uint64_t)tile << 32) | lv;
      if (vals) vals[(size_t)oo + e] = pp;
    }, nullptr, wo != kNoTileBits ? tbits + wo : nullptr);
  }
}

constexpr int kEmitPerWarp = 8;  // primitives per warp in the emission kernels

// Visible primitives in index order: position vpos[i] (exclusive scan of the visibility
// flags) receives the depth key and the index.
__global__ void k_compact(int64_t n, const uint32_t* __restrict__ count, const uint32_t* __restrict__ zkey,
                          const uint32_t* __restrict__ vpos, uint32_t* __restrict__ ckey, uint32_t* __restrict__ cidx) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || count[i] == 0) return;
  const uint32_t p = vpos[i];
  ckey[p] = zkey[i];
  cidx[p] = (uint32_t)i;
}

// Depth order r = 0..V-1 (sidx[r] = primitive): the projected state and the tile count
// gathered into that order (8 threads per 128-byte record).
__global__ void k_gather_state(int64_t V, const uint32_t* __restrict__ sidx, const PrimState* __restrict__ state,
                               const uint32_t* __restrict__ count, PrimState* __restrict__ dstate,
                               uint32_t* __restrict__ cnt_sorted, const uint32_t* err) {
  if (sort_failed(err)) return;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= V * 8) return;
  const int64_t r = e >> 3;
  const int c = (int)(e & 7);
  const uint32_t pid = sidx[r];
  reinterpret_cast<float4*>(dstate + r)[c] = __ldg(reinterpret_cast<const float4*>(state + pid) + c);
  if (c == 0) cnt_sorted[r] = count[pid];
}

// Tile instances of the depth-ordered visible primitives, packed as (tile << rb) | r with
// r the depth rank (rb bits); K = uint32_t when tile and rank bits fit in 32, else
// uint64_t with rb = 32. One warp writes kEmitPerWarp consecutive primitives' tiles
// (coalesced); few primitives per warp keep enough warps in flight, as the visible
// primitives are a small fraction of a large scene.
template <typename K>
__global__ void k_emit_packed(int64_t V, const uint32_t* __restrict__ sidx, const uint32_t* __restrict__ cnt_sorted,
                              const short4* __restrict__ rect, const TileSlab* __restrict__ tslab, int W, int H,
                              const uint32_t* __restrict__ offs, int tiles_x, int rb, K* __restrict__ keys,
                              const uint32_t* __restrict__ tbits, const uint32_t* __restrict__ tbits_off,
                              const uint32_t* err, int64_t n_inst) {
  if (sort_failed(err)) return;
  const int lane = threadIdx.x & 31;
  const int64_t r0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * kEmitPerWarp;
  const int64_t r = r0 + lane;
  uint32_t c = 0, off = 0, pid = 0, wo = kNoTileBits;
  int rxy = 0, rzw = 0;
  if (lane < kEmitPerWarp && r < V) {  // lane k fetches primitive k's entries up front
    c = cnt_sorted[r];
    off = offs[r];
    pid = sidx[r];
    const short4 rc = rect[pid];
    rxy = (int)(((uint32_t)(uint16_t)rc.y << 16) | (uint16_t)rc.x);
    rzw = (int)(((uint32_t)(uint16_t)rc.w << 16) | (uint16_t)rc.z);
    if (tbits) wo = tbits_off[pid];
  }
  for (int k = 0; k < kEmitPerWarp; ++k) {
    const uint32_t cc = __shfl_sync(0xffffffffu, c, k);
    if (!cc) continue;
    const uint32_t rr = (uint32_t)(r0 + k);
    const uint32_t oo = __shfl_sync(0xffffffffu, off, k);
    const uint32_t pp = __shfl_sync(0xffffffffu, pid, k);
    const uint32_t wk = __shfl_sync(0xffffffffu, wo, k);
    const int a = __shfl_sync(0xffffffffu, rxy, k), b = __shfl_sync(0xffffffffu, rzw, k);
    const short4 rk = make_short4((short)(a & 0xFFFF), (short)(a >> 16), (short)(b & 0xFFFF), (short)(b >> 16));
    warp_tiles(rk, tslab ? tslab + pp : nullptr, W, H, [&](uint32_t e, int tx, int ty) {
      const uint32_t tile = (uint32_t)ty * (uint32_t)tiles_x + (uint32_t)tx;
      if (QGS_CHECK(g_check_api, (int64_t)oo + e < n_inst, kChkInstance)) keys[(size_t)oo + e] = ((K)tile << rb) | (K)rr;
    }, nullptr, wk != kNoTileBits ? tbits + wk : nullptr);
  }
}

// Several views of one scene (render_forward_batch): the tile instances of the visible
// (view, primitive) entries in depth order, packed as (global tile << rb) | depth rank like
// k_emit_packed; entry pid = v * n_per_view + i is of view v, whose tiles are numbered from
// its base (vt[v] = (tiles_x, tile base)) and whose image size is in cps[v].
template <typename K>
__global__ void k_emit_packed_views(int64_t V, const uint32_t* __restrict__ sidx,
                                    const uint32_t* __restrict__ cnt_sorted, const short4* __restrict__ rect,
                                    const uint32_t* __restrict__ offs, uint32_t n_per_view,
                                    const int2* __restrict__ vt, const CamParams* __restrict__ cps,
                                    const TileSlab* __restrict__ tslab, const uint32_t* __restrict__ tbits,
                                    const uint32_t* __restrict__ tbits_off, int rb, K* __restrict__ keys,
                                    const uint32_t* err) {
  if (sort_failed(err)) return;
  const int lane = threadIdx.x & 31;
  const int64_t r0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * kEmitPerWarp;
  const int64_t r = r0 + lane;
  uint32_t c = 0, off = 0, pid = 0, wo = kNoTileBits;
  int view = 0, rxy = 0, rzw = 0;
  if (lane < kEmitPerWarp && r < V) {  // lane k fetches entry k's data up front
    c = cnt_sorted[r];
    off = offs[r];
    pid = sidx[r];
    const short4 rc = rect[pid];
    rxy = (int)(((uint32_t)(uint16_t)rc.y << 16) | (uint16_t)rc.x);
    rzw = (int)(((uint32_t)(uint16_t)rc.w << 16) | (uint16_t)rc.z);
    view = (int)(pid / n_per_view);
    if (tbits) wo = tbits_off[pid];
  }
  for (int k = 0; k < kEmitPerWarp; ++k) {
    const uint32_t cc = __shfl_sync(0xffffffffu, c, k);
    if (!cc) continue;
    const uint32_t rr = (uint32_t)(r0 + k);
    const uint32_t oo = __shfl_sync(0xffffffffu, off, k);
    const uint32_t pp = __shfl_sync(0xffffffffu, pid, k);
    const uint32_t wk = __shfl_sync(0xffffffffu, wo, k);
    const int vk = __shfl_sync(0xffffffffu, view, k);
    const int a = __shfl_sync(0xffffffffu, rxy, k), b = __shfl_sync(0xffffffffu, rzw, k);
    const short4 rk = make_short4((short)(a & 0xFFFF), (short)(a >> 16), (short)(b & 0xFFFF), (short)(b >> 16));
    const int2 t = vt[vk];
    warp_tiles(rk, tslab ? tslab + pp : nullptr, cps[vk].W, cps[vk].H, [&](uint32_t e, int tx, int ty) {
      const uint32_t tile = (uint32_t)t.y + (uint32_t)ty * (uint32_t)t.x + (uint32_t)tx;
      keys[(size_t)oo + e] = ((K)tile << rb) | (K)rr;
    }, nullptr, wk != kNoTileBits ? tbits + wk : nullptr);
  }
}

// The same for u32 keys, four per thread (one vector load; the neighbours of the four
// are the thread's own keys except at its ends).
__global__ void k_tile_ranges_x4(int64_t n, const uint32_t* __restrict__ keys, int shift, uint2* __restrict__ ranges,
                                 const uint32_t* err, uint32_t ntiles) {
  if (sort_failed(err)) return;
  const int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (i0 >= n) return;
  uint32_t k[6];  // k[0] = keys[i0 - 1], k[1..4] = keys[i0 .. i0 + 3], k[5] = keys[i0 + 4]
  if (i0 + 4 <= n) {
    const uint4 v = *reinterpret_cast<const uint4*>(keys + i0);
    k[1] = v.x; k[2] = v.y; k[3] = v.z; k[4] = v.w;
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) k[1 + q] = i0 + q < n ? keys[i0 + q] : 0u;
  }
  k[0] = i0 > 0 ? keys[i0 - 1] : 0u;
  k[5] = i0 + 4 < n ? keys[i0 + 4] : 0u;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int64_t i = i0 + q;
    if (i >= n) break;
    const uint32_t t = k[1 + q] >> shift;
    if (!QGS_CHECK(g_check_api, t < ntiles, kChkTile)) continue;
    if (i == 0 || (k[q] >> shift) != t) ranges[t].x = (uint32_t)i;
    if (i == n - 1 || (k[2 + q] >> shift) != t) ranges[t].y = (uint32_t)(i + 1);
  }
}

unsigned emit_blocks(int64_t V) { return (unsigned)((V + 8 * kEmitPerWarp - 1) / (8 * kEmitPerWarp)); }

// [start, end) of every tile's run in keys sorted by tile = key >> shift.
template <typename K>
__global__ void k_tile_ranges_t(int64_t n, const K* __restrict__ keys, int shift, uint2* __restrict__ ranges,
                                const uint32_t* err) {
  if (sort_failed(err)) return;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t t = (uint32_t)(keys[i] >> shift);
  if (i == 0 || (uint32_t)(keys[i - 1] >> shift) != t) ranges[t].x = (uint32_t)i;
  if (i == n - 1 || (uint32_t)(keys[i + 1] >> shift) != t) ranges[t].y = (uint32_t)(i + 1);
}

// Host copy of packed-key binning: keys (tile << 32 | depth bits), values = primitive.
template <typename K>
__global__ void k_debug_packed(int64_t n, const K* __restrict__ inst, int rb, const uint32_t* __restrict__ sidx,
                               const PrimState* __restrict__ dstate, uint64_t* __restrict__ keys,
                               uint32_t* __restrict__ vals) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const K v = inst[i];
  const uint32_t tile = (uint32_t)(v >> rb);
  const uint32_t r = (uint32_t)(v & (((K)1 << rb) - 1));
  keys[i] = ((uint64_t)tile << 32) | __float_as_uint(dstate[r].f[2].w);  // z_mu: the depth key's float
  vals[i] = sidx[r];
}

__global__ void k_tile_ranges(int64_t n, const uint64_t* __restrict__ keys, uint2* __restrict__ ranges,
                              const uint32_t* err) {
  if (sort_failed(err)) return;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t t = (uint32_t)(keys[i] >> 32);
  if (i == 0 || (uint32_t)(keys[i - 1] >> 32) != t) ranges[t].x = (uint32_t)i;
  if (i == n - 1 || (uint32_t)(keys[i + 1] >> 32) != t) ranges[t].y = (uint32_t)(i + 1);
}

// Tile schedule: heaviest tiles (most listed instances) first, by buckets of
// floor(log2(count + 1)), ties in tile order. One CTA of 1024 threads: warp w takes a
// contiguous run of tiles, per-warp bucket counts (lanes of one bucket found with
// __match_any_sync) are scanned bucket-major, and the same walk writes each tile to its
// place (stable, so the schedule does not change from run to run).
__device__ __forceinline__ uint32_t sched_bucket(const uint2* __restrict__ ranges, int t) {
  const uint2 r = ranges[t];
  return (uint32_t)__clz(r.y - r.x + 1u);  // 31 - floor(log2(count + 1)): heaviest first
}
__global__ void __launch_bounds__(1024) k_tile_schedule(int ntiles, const uint2* __restrict__ ranges,
                                                        uint32_t* __restrict__ order) {
  __shared__ uint32_t cnt[32][33];  // [warp][bucket]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  const int per = (ntiles + 31) / 32;
  const int t0 = warp * per, t1 = min(t0 + per, ntiles);
  cnt[warp][lane] = 0u;
  __syncwarp();
  for (int tb = t0; tb < t1; tb += 32) {
    const int t = tb + lane;
    const bool valid = t < t1;
    const uint32_t b = valid ? sched_bucket(ranges, t) : 32u + (uint32_t)lane;
    const uint32_t peers = __match_any_sync(0xffffffffu, b);
    if (valid && (peers & lt) == 0) cnt[warp][b] += (uint32_t)__popc(peers);
    __syncwarp();
  }
  __syncthreads();
  if (warp == 0) {  // bucket-major exclusive scan: bucket b of warp w starts after all of
                    // buckets < b and after bucket b of warps < w
    uint32_t tot = 0;
    for (int w = 0; w < 32; ++w) tot += cnt[w][lane];
    uint32_t inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    uint32_t base = inc - tot;
    for (int w = 0; w < 32; ++w) {
      const uint32_t c = cnt[w][lane];
      cnt[w][lane] = base;
      base += c;
    }
  }
  __syncthreads();
  for (int tb = t0; tb < t1; tb += 32) {
    const int t = tb + lane;
    const bool valid = t < t1;
    const uint32_t b = valid ? sched_bucket(ranges, t) : 32u + (uint32_t)lane;
    const uint32_t peers = __match_any_sync(0xffffffffu, b);
    if (valid) order[cnt[warp][b] + (uint32_t)__popc(peers & lt)] = (uint32_t)t;
    __syncwarp();
    if (valid && (peers & lt) == 0) cnt[warp][b] += (uint32_t)__popc(peers);
    __syncwarp();
  }
}


inline unsigned nblk(int64_t n, int b = 256) { return (unsigned)((n + b - 1) / b); }

}  // namespace

struct qgs_ctx {
  int device = 0;
  qgs_config cfg{};
  std::string err;
  // per-primitive
  DevBuf<PrimState> state;
  DevBuf<uint32_t> count, zkey, idx, zkey2, idx2, cnt_sorted, offs;
  DevBuf<short4> rect;
  // per-instance
  DevBuf<uint64_t> inst, inst2;
  DevBuf<uint32_t> vals, vals2;
  // per-tile / per-pixel
  DevBuf<uint2> ranges;
  DevBuf<uint32_t> torder;                        // heaviest-first tile schedule
  const uint32_t* tile_order = nullptr;
  DevBuf<uint8_t> inst_used;                      // per instance: blended by some pixel
  DevBuf<float> T_final;
  DevBuf<uint32_t> n_contrib;
  // backward
  DevBuf<float> pgrad;
  // scratch
  DevBuf<uint32_t> hist, scan_tmp;
  DevBuf<RasterStats> stats;
  DevBuf<uint32_t> dcount;      // [0] visible primitives, [1] instances, [2] tile-mask words,
                                // [3] radix look-back failure (kept until reported)
  uint32_t* h_total = nullptr;  // pinned: [0..3] the frame's counters read back, [4] the
                                // look-back failure word read back after the frame's sorts
  cudaEvent_t sorts_done = nullptr;  // recorded after that read-back
  bool sorts_pending = false;        // the last forward's sort status has not been checked
  int test_withhold = 0;             // test hook: chunks the next forward's first sort withholds
  int test_spins = kLookbackSpins;   // poll limit of the look-back waits
  int64_t n_visible = 0;
  const uint32_t* vis_list = nullptr;
  // last frame
  bool have_frame = false;
  int64_t n = 0, n_inst = 0;
  int W = 0, H = 0, tiles_x = 0, tiles_y = 0;
  const float* scene_mean = nullptr;
  const uint32_t* ids = nullptr;  // sorted primitive ids of the last frame
  int id_stride = 1;
  const void* sorted_keys = nullptr;
  cudaStream_t last_stream = nullptr;
  DevBuf<float> xres;             // StopThePop order: the forward's outputs for its backward
  bool stp = false;               // the last forward used the StopThePop order
  DevBuf<uint32_t> vpos;          // visibility flags, then their exclusive scan
  DevBuf<TileSlab> tslab;         // per primitive: parallelogram and conic for the tile test
  DevBuf<uint32_t> tbits;         // tile-count pass masks (one word per 32 rectangle tiles)
  DevBuf<uint32_t> tbits_off;     // per primitive: word offset into tbits, or kNoTileBits
  size_t tbits_want = size_t(1) << 22;  // words to provide (grown from the last frame's demand)
  bool tbits_fixed = false;             // capacity set by the caller: provide exactly tbits_want
  DevBuf<PrimState> dstate;       // projected state of the visible primitives in depth order
  const PrimState* raster_state = nullptr;  // state the sorted ids index (dstate or state)
  bool pgrad_by_pos = false;      // gradient records indexed like raster_state's depth order
  bool packed32 = false;          // instances are u32 (tile << rank_bits | depth rank)
  int rank_bits = 32;
  DevBuf<float> resid;            // extra-channel residue (c, A1, A2) [3P] of the last forward
  bool have_resid = false;        // the last forward rendered the extra channels
  // profiling: events at stage boundaries (forward 0..6, backward 7..9)
  bool profiling = false;
  bool have_fwd_times = false, have_bwd_times = false;
  bool pair_counters = true;                   // compile the per-pair counters into the compositing
  bool counted_fwd = true, counted_bwd = true;  // the last forward / backward collected them
  cudaEvent_t ev[10] = {};
  bool nvtx_open = false;  // an NVTX stage range of this context is open
  int64_t launches_fwd = 0, launches_bwd = 0;
  CamParams cp{};
  RasterParams rp{};
  // counters of the last forward (single or batched)
  bool have_stats = false;
  int64_t n_tiles_total = 0;
  // batched forward: view descriptors (device) and their pinned host staging
  DevBuf<uint8_t> vdesc;
  uint8_t* h_vdesc = nullptr;
  size_t h_vdesc_cap = 0;
  cudaEvent_t vdesc_done = nullptr;  // the staging buffer's last upload has completed
  cudaEvent_t totals_ready = nullptr;  // the frame's totals have reached h_total
};

namespace {

qgs_status fail(qgs_ctx* c, qgs_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

qgs_status cuda_fail(qgs_ctx* c, cudaError_t e, const char* where) {
  return fail(c, e == cudaErrorMemoryAllocation ? QGS_ENOMEM : QGS_ECUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}

#define QGS_CU(call, where)                          \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
  } while (0)

bool finite_cam(const qgs_camera* c) {
  bool ok = std::isfinite(c->fx) && std::isfinite(c->fy) && std::isfinite(c->cx) && std::isfinite(c->cy) &&
            std::isfinite(c->near_plane) && c->fx > 0 && c->fy > 0 && c->near_plane > 0;
  for (int i = 0; i < 9; ++i) ok = ok && std::isfinite(c->R_cw[i]);
  for (int i = 0; i < 3; ++i) ok = ok && std::isfinite(c->t_cw[i]);
  return ok;
}

qgs_status check_scene(qgs_ctx* ctx, const qgs_scene* s) {
  if (!s) return fail(ctx, QGS_EINVAL, "scene is NULL");
  if (s->n < 0 || s->n > (int64_t)0x7FFFFFFF) return fail(ctx, QGS_EINVAL, "scene n out of range [0, 2^31)");
  if (s->n > 0 && (!s->mean || !s->quat || !s->scale || !s->curv || !s->opacity || !s->sh))
    return fail(ctx, QGS_EINVAL, "scene has a NULL parameter pointer");
  if (s->n > 0 && ((((uintptr_t)s->quat) & 15) || (((uintptr_t)s->sh) & 15) || (((uintptr_t)s->scale) & 7) ||
                   (((uintptr_t)s->curv) & 7)))
    return fail(ctx, QGS_EINVAL, "quat/sh must be 16-byte aligned, scale/curv 8-byte aligned");
  return QGS_OK;
}

void make_params(const qgs_ctx* ctx, const qgs_camera* cam, CamParams& cp, RasterParams& rp) {
  for (int i = 0; i < 9; ++i) cp.Rc[i] = cam->R_cw[i];
  for (int i = 0; i < 3; ++i) cp.tc[i] = cam->t_cw[i];
  for (int i = 0; i < 3; ++i) {
    double s = 0;
    for (int k = 0; k < 3; ++k) s -= (double)cam->R_cw[3 * k + i] * cam->t_cw[k];
    cp.cw[i] = (float)s;
  }
  cp.fx = cam->fx; cp.fy = cam->fy; cp.cx = cam->cx; cp.cy = cam->cy; cp.near = cam->near_plane;
  cp.W = cam->W; cp.H = cam->H;
  cp.tiles_x = (cam->W + TILE - 1) / TILE;
  cp.tiles_y = (cam->H + TILE - 1) / TILE;
  rp.W = cam->W; rp.H = cam->H; rp.tiles_x = cp.tiles_x; rp.tiles_y = cp.tiles_y;
  rp.cx = cam->cx; rp.cy = cam->cy;
  rp.inv_fx = 1.f / cam->fx; rp.inv_fy = 1.f / cam->fy;
  rp.near_plane = cam->near_plane;
  rp.alpha_max = ctx->cfg.alpha_max; rp.alpha_min = ctx->cfg.alpha_min;
  rp.T_min = ctx->cfg.T_min; rp.grazing_eps = ctx->cfg.grazing_eps;
  rp.id_mask = 0xFFFFFFFFu;
}

// Stage boundaries: CUDA events when profiling is on, and NVTX ranges (host-side, the
// interval in which each stage is enqueued; free unless a tool is attached) named after
// the stage that starts at boundary i (boundaries 6 and 9 end the forward and backward).
inline void mark(qgs_ctx* c, int i, cudaStream_t st) {
  static const char* const names[10] = {"qgs preprocess + tile count",
                                        "qgs totals, compaction, depth sort, gather, offsets",
                                        "qgs key packing",
                                        "qgs key emission",
                                        "qgs tile sort, ranges, schedule",
                                        "qgs raster forward",
                                        nullptr,
                                        "qgs raster backward",
                                        "qgs preprocess backward",
                                        nullptr};
  if (c->profiling) cudaEventRecord(c->ev[i], st);
  if (c->nvtx_open) nvtxRangePop();
  c->nvtx_open = names[i] != nullptr;
  if (c->nvtx_open) nvtxRangePushA(names[i]);
}

int bits_for(int64_t v) {
  int b = 1;
  while (b < 62 && ((int64_t)1 << b) < v) ++b;
  return b;
}

// Sort temporaries of a forward: the context's buffers, its failure word and poll limit,
// and the test hook (consumed by the first sort that reads it).
SortTemp sort_temp(qgs_ctx* ctx) {
  SortTemp tmp;
  tmp.hist = ctx->hist.p;
  tmp.hist_cap = ctx->hist.cap;
  tmp.scan_tmp = ctx->scan_tmp.p;
  tmp.scan_cap = ctx->scan_tmp.cap;
  tmp.err = ctx->dcount.p + 3;
  tmp.spins = ctx->test_spins;
  tmp.withhold_chunks = ctx->test_withhold;
  ctx->test_withhold = 0;
  ctx->test_spins = kLookbackSpins;
  return tmp;
}

// After the frame's last sort: read its failure word back and mark the point.
qgs_status enqueue_sort_check(qgs_ctx* ctx, cudaStream_t st) {
  QGS_CU(cudaMemcpyAsync(ctx->h_total + 4, ctx->dcount.p + 3, sizeof(uint32_t), cudaMemcpyDeviceToHost, st),
         "sort status");
  QGS_CU(cudaEventRecord(ctx->sorts_done, st), "event");
  ctx->sorts_pending = true;
  return QGS_OK;
}

// Wait for the last forward's sorts and report a look-back wait that ran out: the frame is
// then discarded (its lists and images are invalid) and the failure word cleared.
qgs_status check_sorts(qgs_ctx* ctx) {
  if (!ctx->sorts_pending) return QGS_OK;
  ctx->sorts_pending = false;
  const cudaError_t e = cudaEventSynchronize(ctx->sorts_done);
  if (e != cudaSuccess) {
    ctx->have_frame = false;
    return cuda_fail(ctx, e, "waiting for the frame's sorts");
  }
  if (ctx->h_total[4]) {
    ctx->h_total[4] = 0;
    ctx->have_frame = false;
    cudaMemsetAsync(ctx->dcount.p + 3, 0, sizeof(uint32_t), ctx->last_stream);
    cudaStreamSynchronize(ctx->last_stream);
    return fail(ctx, QGS_ECUDA,
                "a radix sort pass of the last forward gave up waiting for an earlier chunk's digit counts; "
                "the frame's tile lists and images are invalid");
  }
  return QGS_OK;
}

}  // namespace

namespace qgs {
int64_t last_instance_count(const qgs_ctx* ctx) { return ctx ? ctx->n_inst : 0; }
}  // namespace qgs

extern "C" {

void qgs_config_default(qgs_config* cfg) {
  if (!cfg) return;
  cfg->alpha_max = 0.99f;
  cfg->alpha_min = 1.0f / 255.0f;
  cfg->T_min = 1e-4f;
  cfg->grazing_eps = 1e-5f;
  cfg->sort_mode = 0;
  cfg->density = 0;
  cfg->order = 0;
}

qgs_status qgs_create(qgs_ctx** out, const qgs_config* cfg, int32_t device) {
  if (!out) return QGS_EINVAL;
  *out = nullptr;
  qgs_ctx* c = new (std::nothrow) qgs_ctx();
  if (!c) return QGS_ENOMEM;
  qgs_config_default(&c->cfg);
  if (cfg) {
    if (!(cfg->alpha_max > 0 && cfg->alpha_max < 1 && cfg->alpha_min >= 0 && cfg->alpha_min < cfg->alpha_max &&
          cfg->T_min > 0 && cfg->T_min < 1 && cfg->grazing_eps >= 0 && (cfg->sort_mode == 0 || cfg->sort_mode == 1) &&
          (cfg->density == 0 || cfg->density == 1) && (cfg->order == 0 || cfg->order == 1))) {
      delete c;
      return QGS_EINVAL;
    }
    c->cfg = *cfg;
  }
  c->device = device;
  if (cudaSetDevice(device) != cudaSuccess) {
    delete c;
    return QGS_ECUDA;
  }
  if (cudaHostAlloc((void**)&c->h_total, 32, cudaHostAllocDefault) != cudaSuccess) {
    delete c;
    return QGS_ENOMEM;
  }
  memset(c->h_total, 0, 32);
  if (c->stats.reserve(1) != cudaSuccess || c->dcount.reserve(4) != cudaSuccess ||
      cudaMemset(c->dcount.p, 0, 4 * sizeof(uint32_t)) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->sorts_done, cudaEventDisableTiming) != cudaSuccess) {
    cudaFreeHost(c->h_total);
    delete c;
    return QGS_ENOMEM;
  }
  *out = c;
  return QGS_OK;
}

void qgs_destroy(qgs_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  c->state.release(); c->count.release(); c->zkey.release(); c->idx.release(); c->zkey2.release();
  c->idx2.release(); c->cnt_sorted.release(); c->offs.release(); c->rect.release(); c->inst.release();
  c->inst2.release(); c->vals.release(); c->vals2.release(); c->ranges.release(); c->T_final.release();
  c->n_contrib.release(); c->pgrad.release(); c->hist.release(); c->scan_tmp.release(); c->stats.release();
  c->dcount.release(); c->torder.release();
  c->inst_used.release();
  c->vdesc.release();
  c->resid.release();
  c->vpos.release();
  c->tslab.release();
  c->tbits.release();
  c->tbits_off.release();
  c->xres.release();
  c->dstate.release();
  if (c->h_vdesc) cudaFreeHost(c->h_vdesc);
  if (c->vdesc_done) cudaEventDestroy(c->vdesc_done);
  if (c->totals_ready) cudaEventDestroy(c->totals_ready);
  if (c->sorts_done) cudaEventDestroy(c->sorts_done);
  if (c->h_total) cudaFreeHost(c->h_total);
  for (int i = 0; i < 10; ++i)
    if (c->ev[i]) cudaEventDestroy(c->ev[i]);
  delete c;
}

const char* qgs_last_error(const qgs_ctx* c) { return c ? c->err.c_str() : "null context"; }

qgs_status render_forward(qgs_ctx* ctx, const qgs_scene* scene, const qgs_camera* cam, const qgs_image* out,
                          qgs_stream stream) {
  if (!ctx) return QGS_EINVAL;
  ctx->err.clear();
  qgs_status s = check_scene(ctx, scene);
  if (s != QGS_OK) return s;
  if (!cam || !out) return fail(ctx, QGS_EINVAL, "camera/output is NULL");
  if (cam->W <= 0 || cam->H <= 0 || cam->W > 32768 || cam->H > 32768)
    return fail(ctx, QGS_EINVAL, "image size must be in [1, 32768]");
  if (!finite_cam(cam)) return fail(ctx, QGS_EINVAL, "camera has non-finite or non-positive intrinsics");
  if (!out->rgb || !out->alpha || !out->depth || !out->normal) return fail(ctx, QGS_EINVAL, "output plane is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  QGS_CU(cudaSetDevice(ctx->device), "cudaSetDevice");
  s = check_sorts(ctx);  // an unreported failure of the previous frame
  if (s != QGS_OK) return s;
  ctx->have_frame = false;
  const int64_t N = scene->n;
  CamParams cp;
  RasterParams rp;
  make_params(ctx, cam, cp, rp);
  const int64_t ntiles = (int64_t)cp.tiles_x * cp.tiles_y;
  const int64_t P = (int64_t)cam->W * cam->H;
  const bool stp = ctx->cfg.order == 1;
  const int sm = stp ? 1 : ctx->cfg.sort_mode;  // the StopThePop keys take the 64-bit key path

  const size_t n1 = (size_t)(N > 0 ? N : 1);
  QGS_CU(ctx->state.reserve(n1), "alloc state");
  QGS_CU(ctx->count.reserve(n1), "alloc count");
  QGS_CU(ctx->zkey.reserve(n1), "alloc zkey");
  QGS_CU(ctx->idx.reserve(n1), "alloc idx");
  QGS_CU(ctx->zkey2.reserve(n1), "alloc zkey2");
  QGS_CU(ctx->idx2.reserve(n1), "alloc idx2");
  QGS_CU(ctx->cnt_sorted.reserve(n1), "alloc cnt");
  QGS_CU(ctx->offs.reserve(n1 + 1), "alloc offs");
  QGS_CU(ctx->rect.reserve(n1), "alloc rect");
  QGS_CU(ctx->vpos.reserve(n1 + 1), "alloc visibility scan");
  QGS_CU(ctx->tslab.reserve(n1), "alloc tile slabs");
  QGS_CU(ctx->tbits_off.reserve(n1), "alloc tile mask offsets");
  if (ctx->tbits_want) QGS_CU(ctx->tbits.reserve(ctx->tbits_want), "alloc tile masks");
  // words the tile-count pass may fill this frame (0: no masks, the emission tests)
  const uint32_t cap_words =
      ctx->tbits_want ? (uint32_t)std::min<size_t>(std::min(ctx->tbits.cap, ctx->tbits_want), 0xFFFFFFF0u) : 0u;
  const bool tb_on = N > 0 && cap_words > 0;
  QGS_CU(ctx->ranges.reserve((size_t)ntiles), "alloc ranges");
  QGS_CU(ctx->torder.reserve((size_t)ntiles), "alloc tile order");
  QGS_CU(ctx->T_final.reserve((size_t)P), "alloc T_final");
  QGS_CU(ctx->n_contrib.reserve((size_t)P), "alloc n_contrib");
  const bool extra = out->curvature || out->distortion || out->median_depth;
  if (extra) QGS_CU(ctx->resid.reserve((size_t)P * 3), "alloc residue");
  if (stp) QGS_CU(ctx->xres.reserve((size_t)P * 8), "alloc output residue");
  QGS_CU(ctx->hist.reserve(radix_hist_elems((int64_t)n1)), "alloc hist");
  QGS_CU(ctx->scan_tmp.reserve(scan_tmp_elems((int64_t)radix_hist_elems((int64_t)n1) + (int64_t)n1)), "alloc scan");
  SortTemp tmp = sort_temp(ctx);

  const int64_t launches0 = launch_counter();
  ctx->have_fwd_times = false;
  ctx->have_stats = false;
  QGS_CU(cudaMemsetAsync(ctx->dcount.p, 0, sizeof(uint32_t) * 3, st), "memset counters");
  mark(ctx, 0, st);
  SceneView sv{scene->mean, scene->quat, scene->scale, scene->curv, scene->opacity, scene->sh};
  if (N > 0) {
    k_preprocess<<<pre_blocks(N), 256, 0, st>>>(N, sv, cp, ctx->state.p, ctx->count.p, ctx->zkey.p,
                                          sm == 0 ? nullptr : ctx->idx.p, ctx->rect.p, nullptr, nullptr,
                                          ctx->tslab.p);
    ++launch_counter();
    QGS_CU(cudaGetLastError(), "k_preprocess");
    // keep the rectangle's tiles that meet the parallelogram and the conic; totals and visibility
    k_count_tiles<<<(unsigned)((N + kCountBlock - 1) / kCountBlock), kCountBlock, 0, st>>>(N, ctx->tslab.p, cam->W, cam->H, ctx->count.p, ctx->rect.p,
                                           ctx->zkey.p, ctx->vpos.p, ctx->dcount.p,
                                           tb_on ? ctx->tbits.p : nullptr, ctx->tbits_off.p, cap_words);
    ++launch_counter();
    QGS_CU(cudaGetLastError(), "k_count_tiles");
  }
  mark(ctx, 1, st);
  // the frame's one synchronisation: visible and instance totals size what follows; the
  // compaction of the visible primitives (index order), which needs no total, is enqueued
  // before the host waits, so it runs during the read-back
  QGS_CU(cudaMemcpyAsync(ctx->h_total, ctx->dcount.p, 4 * sizeof(uint32_t), cudaMemcpyDeviceToHost, st), "totals");
  if (!ctx->totals_ready) QGS_CU(cudaEventCreateWithFlags(&ctx->totals_ready, cudaEventDisableTiming), "event");
  QGS_CU(cudaEventRecord(ctx->totals_ready, st), "event");
  // (both key modes: the list also drives the preprocessing backward)
  if (N > 0) {
    QGS_CU(scan_exclusive_u32(ctx->vpos.p, ctx->vpos.p, N, ctx->scan_tmp.p, ctx->scan_tmp.cap, st), "scan");
    k_compact<<<nblk(N), 256, 0, st>>>(N, ctx->count.p, ctx->zkey.p, ctx->vpos.p, ctx->zkey2.p, ctx->idx2.p);
    ++launch_counter();
    QGS_CU(cudaGetLastError(), "compact");
  }
  QGS_CU(cudaEventSynchronize(ctx->totals_ready), "sync");
  if (ctx->h_total[3]) {  // a radix sort of an earlier call gave up waiting for a chunk
    cudaMemsetAsync(ctx->dcount.p + 3, 0, sizeof(uint32_t), st);
    return fail(ctx, QGS_ECUDA, "a radix sort pass of an earlier call timed out in its look-back");
  }
  const int64_t V = (int64_t)ctx->h_total[0];
  const int64_t I = (int64_t)ctx->h_total[1];
  // primitives whose masks did not fit are tested again by the emission; provide more next frame
  if (tb_on && !ctx->tbits_fixed && (size_t)ctx->h_total[2] > cap_words)
    ctx->tbits_want = (size_t)ctx->h_total[2] + ctx->h_total[2] / 4;
  ctx->n_visible = V;

  const size_t i1 = (size_t)(I > 0 ? I : 1);
  QGS_CU(ctx->inst_used.reserve(i1), "alloc inst flags");
  QGS_CU(ctx->inst.reserve(i1), "alloc inst");
  QGS_CU(ctx->inst2.reserve(i1), "alloc inst2");
  if (sm == 1) {
    QGS_CU(ctx->vals.reserve(i1), "alloc vals");
    QGS_CU(ctx->vals2.reserve(i1), "alloc vals2");
  }
  if (sm == 0) QGS_CU(ctx->dstate.reserve((size_t)(V > 0 ? V : 1)), "alloc ordered state");
  QGS_CU(ctx->hist.reserve(radix_hist_elems((int64_t)i1)), "alloc hist");
  QGS_CU(ctx->scan_tmp.reserve(scan_tmp_elems((int64_t)radix_hist_elems((int64_t)i1))), "alloc scan");
  tmp.hist = ctx->hist.p;
  tmp.hist_cap = ctx->hist.cap;
  tmp.scan_tmp = ctx->scan_tmp.p;
  tmp.scan_cap = ctx->scan_tmp.cap;

  const int tb = bits_for(ntiles);
  cudaError_t e = cudaSuccess;
  const void* sorted = ctx->inst.p;
  int shift = 32;
  if (sm == 0) {
    // visible primitives (index order) -> depth sort -> state, counts and offsets in
    // depth order -> instances (tile << rb | depth rank) -> stable sort on the tile bits
    const bool fl = radix_sort_u32_pairs(ctx->zkey2.p, ctx->idx2.p, ctx->zkey.p, ctx->idx.p, V, 0, 32, tmp, st, &e);
    QGS_CU(e, "depth sort");
    const uint32_t* sidx = fl ? ctx->idx.p : ctx->idx2.p;
    ctx->vis_list = sidx;
    if (V > 0) {
      k_gather_state<<<nblk(V * 8), 256, 0, st>>>(V, sidx, ctx->state.p, ctx->count.p, ctx->dstate.p,
                                                  ctx->cnt_sorted.p, tmp.err);
      ++launch_counter();
      QGS_CU(cudaGetLastError(), "gather state");
    }
    QGS_CU(scan_exclusive_u32(ctx->cnt_sorted.p, ctx->offs.p, V, ctx->scan_tmp.p, ctx->scan_tmp.cap, st), "scan");
    mark(ctx, 2, st);
    const int rb = bits_for(V > 1 ? V : 2);
    ctx->packed32 = rb + tb <= 32;
    ctx->rank_bits = ctx->packed32 ? rb : 32;
    mark(ctx, 3, st);
    if (V > 0 && I > 0) {
      if (ctx->packed32) {
        uint32_t* k0 = reinterpret_cast<uint32_t*>(ctx->inst.p);
        uint32_t* k1 = reinterpret_cast<uint32_t*>(ctx->inst2.p);
        k_emit_packed<uint32_t><<<emit_blocks(V), 256, 0, st>>>(V, sidx, ctx->cnt_sorted.p, ctx->rect.p, ctx->tslab.p,
                                                         cam->W, cam->H, ctx->offs.p, cp.tiles_x, rb, k0,
                                                         tb_on ? ctx->tbits.p : nullptr, ctx->tbits_off.p, tmp.err, I);
        ++launch_counter();
        QGS_CU(cudaGetLastError(), "emit");
        mark(ctx, 4, st);
        const bool f2 = radix_sort_u32_keys(k0, k1, I, rb, rb + tb, tmp, st, &e);
        QGS_CU(e, "tile sort");
        sorted = f2 ? (const void*)k1 : (const void*)k0;
      } else {
        k_emit_packed<uint64_t><<<emit_blocks(V), 256, 0, st>>>(V, sidx, ctx->cnt_sorted.p, ctx->rect.p, ctx->tslab.p,
                                                         cam->W, cam->H, ctx->offs.p, cp.tiles_x, 32, ctx->inst.p,
                                                         tb_on ? ctx->tbits.p : nullptr, ctx->tbits_off.p, tmp.err, I);
        ++launch_counter();
        QGS_CU(cudaGetLastError(), "emit");
        mark(ctx, 4, st);
        const bool f2 = radix_sort_u64_keys(ctx->inst.p, ctx->inst2.p, I, 32, 32 + tb, tmp, st, &e);
        QGS_CU(e, "tile sort");
        sorted = f2 ? (const void*)ctx->inst2.p : (const void*)ctx->inst.p;
      }
    } else {
      mark(ctx, 4, st);
    }
    shift = ctx->rank_bits;
    ctx->ids = reinterpret_cast<const uint32_t*>(sorted);
    ctx->id_stride = ctx->packed32 ? 1 : 2;
    rp.id_mask = ctx->packed32 ? (uint32_t)((1ull << rb) - 1ull) : 0xFFFFFFFFu;
    ctx->raster_state = ctx->dstate.p;
    ctx->pgrad_by_pos = true;
  } else {
    // sort_mode 1: 64-bit (tile << 32 | depth bits) keys in primitive order, one sort
    QGS_CU(scan_exclusive_u32(ctx->count.p, ctx->offs.p, N, ctx->scan_tmp.p, ctx->scan_tmp.cap, st), "scan");
    mark(ctx, 2, st);
    mark(ctx, 3, st);
    ctx->packed32 = false;
    ctx->rank_bits = 32;
    if (N > 0 && I > 0) {
      if (stp)
        k_emit_hit<<<nblk(N), 256, 0, st>>>(N, sv, cp, ctx->count.p, ctx->rect.p, ctx->tslab.p, ctx->offs.p,
                                            ctx->inst.p, ctx->vals.p, tb_on ? ctx->tbits.p : nullptr, ctx->tbits_off.p);
      else
        k_emit<<<nblk(N), 256, 0, st>>>(N, nullptr, ctx->count.p, ctx->rect.p, ctx->tslab.p, cam->W, cam->H,
                                        ctx->offs.p, ctx->zkey.p, cp.tiles_x, ctx->inst.p, ctx->vals.p,
                                        tb_on ? ctx->tbits.p : nullptr, ctx->tbits_off.p, nullptr);
      ++launch_counter();
      QGS_CU(cudaGetLastError(), "emit");
      mark(ctx, 4, st);
      const bool fl =
          radix_sort_u64_pairs(ctx->inst.p, ctx->vals.p, ctx->inst2.p, ctx->vals2.p, I, 0, 32 + tb, tmp, st, &e);
      QGS_CU(e, "key sort");
      sorted = fl ? ctx->inst2.p : ctx->inst.p;
      ctx->ids = fl ? ctx->vals2.p : ctx->vals.p;
    } else {
      ctx->ids = ctx->vals.p;
      mark(ctx, 4, st);
    }
    ctx->id_stride = 1;
    rp.id_mask = 0xFFFFFFFFu;
    ctx->raster_state = ctx->state.p;
    ctx->pgrad_by_pos = false;
    ctx->vis_list = ctx->idx2.p;  // visible primitives in index order (gradient records by index)
  }
  ctx->sorted_keys = sorted;
  QGS_CU(cudaMemsetAsync(ctx->ranges.p, 0, sizeof(uint2) * (size_t)ntiles, st), "memset ranges");
  if (I > 0) {
    if (ctx->packed32)
      k_tile_ranges_x4<<<nblk((I + 3) / 4), 256, 0, st>>>(I, reinterpret_cast<const uint32_t*>(sorted), shift,
                                                           ctx->ranges.p, tmp.err, (uint32_t)ntiles);
    else
      k_tile_ranges_t<uint64_t><<<nblk(I), 256, 0, st>>>(I, reinterpret_cast<const uint64_t*>(sorted), shift,
                                                         ctx->ranges.p, tmp.err);
    ++launch_counter();
    QGS_CU(cudaGetLastError(), "ranges");
  }
  // heaviest-first tile schedule
  k_tile_schedule<<<1, 1024, 0, st>>>((int)ntiles, ctx->ranges.p, ctx->torder.p);
  ++launch_counter();
  QGS_CU(cudaGetLastError(), "tile schedule");
  s = enqueue_sort_check(ctx, st);
  if (s != QGS_OK) return s;
  ctx->tile_order = ctx->torder.p;
  QGS_CU(cudaMemsetAsync(ctx->stats.p, 0, sizeof(RasterStats), st), "memset stats");
  mark(ctx, 5, st);
  const ExtraPlanes ex{out->curvature, out->distortion, out->median_depth, extra ? ctx->resid.p : nullptr};
  if (stp)
    QGS_CU(launch_raster_fwd_stp(ctx->cfg.density == 1, extra, (unsigned)ntiles, st, ctx->ranges.p, ctx->ids,
                                 ctx->raster_state, rp, out->rgb, out->alpha, out->depth, out->normal,
                                 ctx->T_final.p, ctx->n_contrib.p, ctx->xres.p, ex,
                                 ctx->pair_counters ? ctx->stats.p : nullptr, ctx->tile_order),
           "k_raster_fwd_stp");
  else
    QGS_CU(launch_raster_fwd(ctx->cfg.density == 1, extra, (unsigned)ntiles, st, ctx->ranges.p, ctx->ids,
                             ctx->id_stride, ctx->raster_state, rp, out->rgb, out->alpha, out->depth, out->normal,
                             ctx->T_final.p, ctx->n_contrib.p, ex, ctx->pair_counters ? ctx->stats.p : nullptr,
                             ctx->tile_order, ctx->inst_used.p),
           "k_raster_fwd");
  ctx->counted_fwd = ctx->pair_counters;
  ctx->counted_bwd = false;
  ctx->stp = stp;
  ++launch_counter();
  mark(ctx, 6, st);
  ctx->have_fwd_times = ctx->profiling;
  ctx->have_bwd_times = false;
  ctx->launches_fwd = launch_counter() - launches0;
  ctx->launches_bwd = 0;
  ctx->have_frame = true;
  ctx->have_resid = extra;
  ctx->have_stats = true;
  ctx->n_tiles_total = ntiles;
  ctx->n = N;
  ctx->n_inst = I;
  ctx->W = cam->W;
  ctx->H = cam->H;
  ctx->tiles_x = cp.tiles_x;
  ctx->tiles_y = cp.tiles_y;
  ctx->scene_mean = scene->mean;
  ctx->last_stream = st;
  ctx->cp = cp;
  ctx->rp = rp;
  return QGS_OK;
}

qgs_status render_forward_batch(qgs_ctx* ctx, const qgs_scene* scene, int32_t n_views, const qgs_camera* cams,
                                const qgs_image* outs, qgs_stream stream) {
  if (!ctx) return QGS_EINVAL;
  ctx->err.clear();
  qgs_status s = check_scene(ctx, scene);
  if (s != QGS_OK) return s;
  if (n_views < 1 || n_views > 1024) return fail(ctx, QGS_EINVAL, "n_views must be in [1, 1024]");
  if (ctx->cfg.order != 0) return fail(ctx, QGS_EINVAL, "the batched forward uses the centre-depth order only");
  if (!cams || !outs) return fail(ctx, QGS_EINVAL, "camera/output array is NULL");
  const int64_t N = scene->n;
  const int V = n_views;
  const int64_t VN = (int64_t)V * N;
  if (VN > (int64_t)0x7FFFFFFF) return fail(ctx, QGS_EINVAL, "n_views * n must be below 2^31");
  std::vector<CamParams> cps((size_t)V);
  std::vector<RasterParams> rps((size_t)V);
  std::vector<uint32_t> base((size_t)V);
  int64_t T_all = 0;
  for (int v = 0; v < V; ++v) {
    const qgs_camera* cam = &cams[v];
    const qgs_image* o = &outs[v];
    if (cam->W <= 0 || cam->H <= 0 || cam->W > 32768 || cam->H > 32768)
      return fail(ctx, QGS_EINVAL, "view " + std::to_string(v) + ": image size must be in [1, 32768]");
    if (!finite_cam(cam))
      return fail(ctx, QGS_EINVAL, "view " + std::to_string(v) + ": non-finite or non-positive intrinsics");
    if (!o->rgb || !o->alpha || !o->depth || !o->normal)
      return fail(ctx, QGS_EINVAL, "view " + std::to_string(v) + ": output plane is NULL");
    make_params(ctx, cam, cps[v], rps[v]);
    base[v] = (uint32_t)T_all;
    T_all += (int64_t)cps[v].tiles_x * cps[v].tiles_y;
    if (T_all > (int64_t)0x7FFFFFFF) return fail(ctx, QGS_EINVAL, "too many tiles in the batch (2^31)");
  }
  cudaStream_t st = (cudaStream_t)stream;
  QGS_CU(cudaSetDevice(ctx->device), "cudaSetDevice");
  s = check_sorts(ctx);  // an unreported failure of the previous frame
  if (s != QGS_OK) return s;
  ctx->have_frame = false;
  ctx->have_resid = false;
  ctx->have_stats = false;
  ctx->have_fwd_times = false;
  ctx->have_bwd_times = false;

  // view descriptors: CamParams[V] | ViewDesc[V] | tile base u32[V] | (tiles_x, base) int2[V]
  auto al16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
  const size_t off_vd = al16(sizeof(CamParams) * V);
  const size_t off_tb = al16(off_vd + sizeof(ViewDesc) * V);
  const size_t off_vt = al16(off_tb + sizeof(uint32_t) * V);
  const size_t vbytes = off_vt + sizeof(int2) * V;
  if (!ctx->vdesc_done) QGS_CU(cudaEventCreateWithFlags(&ctx->vdesc_done, cudaEventDisableTiming), "event");
  QGS_CU(cudaEventSynchronize(ctx->vdesc_done), "staging wait");
  if (ctx->h_vdesc_cap < vbytes) {
    if (ctx->h_vdesc) cudaFreeHost(ctx->h_vdesc);
    ctx->h_vdesc = nullptr;
    ctx->h_vdesc_cap = 0;
    QGS_CU(cudaHostAlloc((void**)&ctx->h_vdesc, vbytes, cudaHostAllocDefault), "alloc view staging");
    ctx->h_vdesc_cap = vbytes;
  }
  QGS_CU(ctx->vdesc.reserve(vbytes), "alloc view descriptors");
  bool extra = false;
  {
    uint8_t* h = ctx->h_vdesc;
    CamParams* hc = reinterpret_cast<CamParams*>(h);
    ViewDesc* hv = reinterpret_cast<ViewDesc*>(h + off_vd);
    uint32_t* hb = reinterpret_cast<uint32_t*>(h + off_tb);
    int2* ht = reinterpret_cast<int2*>(h + off_vt);
    for (int v = 0; v < V; ++v) {
      hc[v] = cps[v];
      hv[v].rp = rps[v];
      hv[v].rgb = outs[v].rgb;
      hv[v].alpha = outs[v].alpha;
      hv[v].depth = outs[v].depth;
      hv[v].normal = outs[v].normal;
      hv[v].T_final = nullptr;
      hv[v].n_contrib = nullptr;
      hv[v].ex = ExtraPlanes{outs[v].curvature, outs[v].distortion, outs[v].median_depth, nullptr};
      extra = extra || outs[v].curvature || outs[v].distortion || outs[v].median_depth;
      hb[v] = base[v];
      ht[v] = make_int2(cps[v].tiles_x, (int)base[v]);
    }
  }
  const CamParams* d_cp = reinterpret_cast<const CamParams*>(ctx->vdesc.p);
  const ViewDesc* d_vd = reinterpret_cast<const ViewDesc*>(ctx->vdesc.p + off_vd);
  const uint32_t* d_tb = reinterpret_cast<const uint32_t*>(ctx->vdesc.p + off_tb);
  const int2* d_vt = reinterpret_cast<const int2*>(ctx->vdesc.p + off_vt);

  const size_t n1 = (size_t)(VN > 0 ? VN : 1);
  QGS_CU(ctx->state.reserve(n1), "alloc state");
  QGS_CU(ctx->count.reserve(n1), "alloc count");
  QGS_CU(ctx->zkey.reserve(n1), "alloc zkey");
  QGS_CU(ctx->idx.reserve(n1), "alloc idx");
  QGS_CU(ctx->zkey2.reserve(n1), "alloc zkey2");
  QGS_CU(ctx->idx2.reserve(n1), "alloc idx2");
  QGS_CU(ctx->cnt_sorted.reserve(n1), "alloc cnt");
  QGS_CU(ctx->offs.reserve(n1 + 1), "alloc offs");
  QGS_CU(ctx->rect.reserve(n1), "alloc rect");
  QGS_CU(ctx->tslab.reserve(n1), "alloc tile slabs");
  QGS_CU(ctx->tbits_off.reserve(n1), "alloc tile mask offsets");
  if (ctx->tbits_want) QGS_CU(ctx->tbits.reserve(ctx->tbits_want), "alloc tile masks");
  const uint32_t cap_words =
      ctx->tbits_want ? (uint32_t)std::min<size_t>(std::min(ctx->tbits.cap, ctx->tbits_want), 0xFFFFFFF0u) : 0u;
  const bool tb_on = N > 0 && cap_words > 0;
  QGS_CU(ctx->ranges.reserve((size_t)T_all), "alloc ranges");
  QGS_CU(ctx->torder.reserve((size_t)T_all), "alloc tile order");
  QGS_CU(ctx->hist.reserve(radix_hist_elems((int64_t)n1)), "alloc hist");
  QGS_CU(ctx->scan_tmp.reserve(scan_tmp_elems((int64_t)radix_hist_elems((int64_t)n1) + (int64_t)n1)), "alloc scan");
  SortTemp tmp = sort_temp(ctx);

  const int64_t launches0 = launch_counter();
  QGS_CU(ctx->vpos.reserve(n1 + 1), "alloc visibility scan");
  QGS_CU(cudaMemcpyAsync(ctx->vdesc.p, ctx->h_vdesc, vbytes, cudaMemcpyHostToDevice, st), "upload views");
  QGS_CU(cudaEventRecord(ctx->vdesc_done, st), "event");
  QGS_CU(cudaMemsetAsync(ctx->dcount.p, 0, sizeof(uint32_t) * 3, st), "memset counters");
  SceneView sv{scene->mean, scene->quat, scene->scale, scene->curv, scene->opacity, scene->sh};
  if (N > 0) {
    k_preprocess_views<<<dim3(pre_blocks(N), (unsigned)V), 256, 0, st>>>(N, sv, d_cp, ctx->state.p, ctx->count.p,
                                                                   ctx->zkey.p, nullptr, ctx->rect.p, nullptr,
                                                                   ctx->tslab.p);
    ++launch_counter();
    QGS_CU(cudaGetLastError(), "k_preprocess_views");
    // keep each view's rectangle tiles that meet the parallelogram and the conic
    k_count_tiles<<<dim3((unsigned)((N + kCountBlock - 1) / kCountBlock), (unsigned)V), kCountBlock, 0, st>>>(
        N, ctx->tslab.p, 0, 0, ctx->count.p, ctx->rect.p, ctx->zkey.p, ctx->vpos.p, ctx->dcount.p,
        tb_on ? ctx->tbits.p : nullptr, ctx->tbits_off.p, cap_words, d_cp);
    ++launch_counter();
    QGS_CU(cudaGetLastError(), "k_count_tiles");
  }
  // the totals' read-back; the compaction of the visible (view, primitive) entries (index
  // order), which needs no total, runs during it
  QGS_CU(cudaMemcpyAsync(ctx->h_total, ctx->dcount.p, 4 * sizeof(uint32_t), cudaMemcpyDeviceToHost, st), "totals");
  if (!ctx->totals_ready) QGS_CU(cudaEventCreateWithFlags(&ctx->totals_ready, cudaEventDisableTiming), "event");
  QGS_CU(cudaEventRecord(ctx->totals_ready, st), "event");
  if (VN > 0) {
    QGS_CU(scan_exclusive_u32(ctx->vpos.p, ctx->vpos.p, VN, ctx->scan_tmp.p, ctx->scan_tmp.cap, st), "scan");
    k_compact<<<nblk(VN), 256, 0, st>>>(VN, ctx->count.p, ctx->zkey.p, ctx->vpos.p, ctx->zkey2.p, ctx->idx2.p);
    ++launch_counter();
    QGS_CU(cudaGetLastError(), "compact");
  }
  QGS_CU(cudaEventSynchronize(ctx->totals_ready), "sync");
  if (ctx->h_total[3]) {  // a radix sort of an earlier call gave up waiting for a chunk
    cudaMemsetAsync(ctx->dcount.p + 3, 0, sizeof(uint32_t), st);
    return fail(ctx, QGS_ECUDA, "a radix sort pass of an earlier call timed out in its look-back");
  }
  const int64_t Vv = (int64_t)ctx->h_total[0];
  const int64_t I = (int64_t)ctx->h_total[1];
  ctx->n_visible = Vv;
  if (tb_on && !ctx->tbits_fixed && (size_t)ctx->h_total[2] > cap_words)
    ctx->tbits_want = (size_t)ctx->h_total[2] + ctx->h_total[2] / 4;

  const size_t i1 = (size_t)(I > 0 ? I : 1);
  QGS_CU(ctx->inst.reserve(i1), "alloc inst");
  QGS_CU(ctx->inst2.reserve(i1), "alloc inst2");
  QGS_CU(ctx->dstate.reserve((size_t)(Vv > 0 ? Vv : 1)), "alloc ordered state");
  QGS_CU(ctx->hist.reserve(radix_hist_elems((int64_t)i1)), "alloc hist");
  QGS_CU(ctx->scan_tmp.reserve(scan_tmp_elems((int64_t)radix_hist_elems((int64_t)i1))), "alloc scan");
  tmp.hist = ctx->hist.p;
  tmp.hist_cap = ctx->hist.cap;
  tmp.scan_tmp = ctx->scan_tmp.p;
  tmp.scan_cap = ctx->scan_tmp.cap;

  // visible entries -> depth sort -> state, counts and offsets in depth order -> instances
  // (global tile << rb | depth rank) -> stable sort on the tile bits (render_forward's order
  // within each view: depth, then entry index)
  cudaError_t e = cudaSuccess;
  const bool fl0 = radix_sort_u32_pairs(ctx->zkey2.p, ctx->idx2.p, ctx->zkey.p, ctx->idx.p, Vv, 0, 32, tmp, st, &e);
  QGS_CU(e, "depth sort");
  const uint32_t* sidx = fl0 ? ctx->idx.p : ctx->idx2.p;
  if (Vv > 0) {
    k_gather_state<<<nblk(Vv * 8), 256, 0, st>>>(Vv, sidx, ctx->state.p, ctx->count.p, ctx->dstate.p,
                                                 ctx->cnt_sorted.p, tmp.err);
    ++launch_counter();
    QGS_CU(cudaGetLastError(), "gather state");
  }
  QGS_CU(scan_exclusive_u32(ctx->cnt_sorted.p, ctx->offs.p, Vv, ctx->scan_tmp.p, ctx->scan_tmp.cap, st), "scan");
  const int tb = bits_for(T_all);
  const int rb = bits_for(Vv > 1 ? Vv : 2);
  const bool packed = rb + tb <= 32;
  const void* sorted = ctx->inst.p;
  if (Vv > 0 && I > 0) {
    if (packed) {
      uint32_t* k0 = reinterpret_cast<uint32_t*>(ctx->inst.p);
      uint32_t* k1 = reinterpret_cast<uint32_t*>(ctx->inst2.p);
      k_emit_packed_views<uint32_t><<<emit_blocks(Vv), 256, 0, st>>>(
          Vv, sidx, ctx->cnt_sorted.p, ctx->rect.p, ctx->offs.p, (uint32_t)N, d_vt, d_cp, ctx->tslab.p,
          tb_on ? ctx->tbits.p : nullptr, ctx->tbits_off.p, rb, k0, tmp.err);
      ++launch_counter();
      QGS_CU(cudaGetLastError(), "emit");
      const bool f2 = radix_sort_u32_keys(k0, k1, I, rb, rb + tb, tmp, st, &e);
      QGS_CU(e, "tile sort");
      sorted = f2 ? (const void*)k1 : (const void*)k0;
    } else {
      k_emit_packed_views<uint64_t><<<emit_blocks(Vv), 256, 0, st>>>(
          Vv, sidx, ctx->cnt_sorted.p, ctx->rect.p, ctx->offs.p, (uint32_t)N, d_vt, d_cp, ctx->tslab.p,
          tb_on ? ctx->tbits.p : nullptr, ctx->tbits_off.p, 32, ctx->inst.p, tmp.err);
      ++launch_counter();
      QGS_CU(cudaGetLastError(), "emit");
      const bool f2 = radix_sort_u64_keys(ctx->inst.p, ctx->inst2.p, I, 32, 32 + tb, tmp, st, &e);
      QGS_CU(e, "tile sort");
      sorted = f2 ? (const void*)ctx->inst2.p : (const void*)ctx->inst.p;
    }
  }
  const uint32_t* ids = reinterpret_cast<const uint32_t*>(sorted);
  QGS_CU(cudaMemsetAsync(ctx->ranges.p, 0, sizeof(uint2) * (size_t)T_all, st), "memset ranges");
  if (I > 0) {
    if (packed)
      k_tile_ranges_x4<<<nblk((I + 3) / 4), 256, 0, st>>>(I, ids, rb, ctx->ranges.p, tmp.err, (uint32_t)T_all);
    else
      k_tile_ranges_t<uint64_t><<<nblk(I), 256, 0, st>>>(I, reinterpret_cast<const uint64_t*>(sorted), 32,
                                                         ctx->ranges.p, tmp.err);
    ++launch_counter();
    QGS_CU(cudaGetLastError(), "ranges");
  }
  k_tile_schedule<<<1, 1024, 0, st>>>((int)T_all, ctx->ranges.p, ctx->torder.p);
  ++launch_counter();
  QGS_CU(cudaGetLastError(), "tile schedule");
  s = enqueue_sort_check(ctx, st);
  if (s != QGS_OK) return s;
  const uint32_t* order = ctx->torder.p;
  QGS_CU(cudaMemsetAsync(ctx->stats.p, 0, sizeof(RasterStats), st), "memset stats");
  QGS_CU(launch_raster_fwd_views(ctx->cfg.density == 1, extra, (unsigned)T_all, st, ctx->ranges.p, ids,
                                 packed ? 1 : 2, packed ? (uint32_t)((1ull << rb) - 1ull) : 0xFFFFFFFFu,
                                 ctx->dstate.p, d_vd, V, d_tb, ctx->stats.p, order),
         "k_raster_fwd_views");
  ++launch_counter();
  ctx->launches_fwd = launch_counter() - launches0;
  ctx->launches_bwd = 0;
  ctx->have_stats = true;
  ctx->n = VN;
  ctx->n_inst = I;
  ctx->n_tiles_total = T_all;
  ctx->last_stream = st;
  return QGS_OK;
}

qgs_status render_backward(qgs_ctx* ctx, const qgs_scene* scene, const qgs_camera* cam, const qgs_image* grad_out,
                           const qgs_scene_grad* grad, qgs_stream stream) {
  if (!ctx) return QGS_EINVAL;
  ctx->err.clear();
  qgs_status s = check_scene(ctx, scene);
  if (s != QGS_OK) return s;
  if (!cam || !grad_out || !grad) return fail(ctx, QGS_EINVAL, "camera/grad_out/grad is NULL");
  if (!ctx->have_frame) return fail(ctx, QGS_ESTATE, "render_backward without a preceding render_forward");
  QGS_CU(cudaSetDevice(ctx->device), "cudaSetDevice");
  s = check_sorts(ctx);
  if (s != QGS_OK) return s;
  if (scene->n != ctx->n || scene->mean != ctx->scene_mean || cam->W != ctx->W || cam->H != ctx->H)
    return fail(ctx, QGS_ESTATE, "render_backward scene/camera differ from the last render_forward");
  if (grad_out->median_depth)
    return fail(ctx, QGS_EINVAL, "the median depth has no gradient: grad_out->median_depth must be NULL");
  if (grad_out->distortion && !ctx->have_resid)
    return fail(ctx, QGS_ESTATE, "a distortion gradient needs a forward that rendered an extra channel");
  if (scene->n > 0 && (!grad->mean || !grad->quat || !grad->scale || !grad->curv || !grad->opacity || !grad->sh))
    return fail(ctx, QGS_EINVAL, "gradient buffer is NULL");
  if (scene->n > 0 && ((((uintptr_t)grad->quat) & 15) || (((uintptr_t)grad->sh) & 15) ||
                       (((uintptr_t)grad->scale) & 7) || (((uintptr_t)grad->curv) & 7)))
    return fail(ctx, QGS_EINVAL, "grad quat/sh must be 16-byte aligned, scale/curv 8-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  QGS_CU(cudaSetDevice(ctx->device), "cudaSetDevice");
  const int64_t N = scene->n;
  if (N == 0) return QGS_OK;
  CamParams cp;
  RasterParams rp;
  make_params(ctx, cam, cp, rp);
  rp.id_mask = ctx->rp.id_mask;
  const int64_t NG = ctx->pgrad_by_pos ? ctx->n_visible : N;  // gradient records
  QGS_CU(ctx->pgrad.reserve((size_t)(NG > 0 ? NG : 1) * NGRAD_PAD), "alloc pgrad");
  if (NG > 0)
    QGS_CU(cudaMemsetAsync(ctx->pgrad.p, 0, sizeof(float) * (size_t)NG * NGRAD_PAD, st), "memset pgrad");
  const int64_t ntiles = (int64_t)cp.tiles_x * cp.tiles_y;
  const int64_t launches0 = launch_counter();
  const bool euclid = ctx->cfg.density == 1;
  const bool extra = grad_out->curvature || grad_out->distortion;
  const ExtraGrads eg{grad_out->curvature, grad_out->distortion, ctx->have_resid ? ctx->resid.p : nullptr};
  mark(ctx, 7, st);
  if (ctx->stp)
    QGS_CU(launch_raster_bwd_stp(euclid, extra, (unsigned)ntiles, st, ctx->ranges.p, ctx->ids, ctx->raster_state,
                                 rp, grad_out->rgb, grad_out->alpha, grad_out->depth, grad_out->normal,
                                 ctx->T_final.p, ctx->xres.p, eg, ctx->pgrad.p,
                                 ctx->pair_counters ? ctx->stats.p : nullptr, ctx->tile_order),
           "k_raster_bwd_stp");
  else
    QGS_CU(launch_raster_bwd(euclid, extra, (unsigned)ntiles, st, ctx->ranges.p, ctx->ids, ctx->id_stride,
                             ctx->raster_state, rp, grad_out->rgb, grad_out->alpha, grad_out->depth,
                             grad_out->normal, ctx->T_final.p, ctx->n_contrib.p, eg, ctx->pgrad.p,
                             ctx->pair_counters ? ctx->stats.p : nullptr, ctx->tile_order, ctx->inst_used.p),
           "k_raster_bwd");
  ctx->counted_bwd = ctx->pair_counters;
  ++launch_counter();
  mark(ctx, 8, st);
  SceneView sv{scene->mean, scene->quat, scene->scale, scene->curv, scene->opacity, scene->sh};
  GradView gv{grad->mean, grad->quat, grad->scale, grad->curv, grad->opacity, grad->sh};
  const int64_t nb = ctx->vis_list ? ctx->n_visible : N;
  if (nb > 0)
    k_preprocess_bwd<<<nblk(nb, 128), 128, 0, st>>>(nb, ctx->vis_list, sv, cp, ctx->count.p, ctx->pgrad.p,
                                               ctx->pgrad_by_pos, gv);
  ++launch_counter();
  QGS_CU(cudaGetLastError(), "k_preprocess_bwd");
  mark(ctx, 9, st);
  ctx->have_bwd_times = ctx->profiling;
  ctx->launches_bwd = launch_counter() - launches0;
  ctx->last_stream = st;
  return QGS_OK;
}

qgs_status qgs_get_frame_stats(qgs_ctx* ctx, qgs_frame_stats* out) {
  if (!ctx || !out) return QGS_EINVAL;
  if (!ctx->have_stats) return fail(ctx, QGS_ESTATE, "no frame rendered yet");
  QGS_CU(cudaSetDevice(ctx->device), "cudaSetDevice");
  const qgs_status s = check_sorts(ctx);
  if (s != QGS_OK) return s;
  QGS_CU(cudaStreamSynchronize(ctx->last_stream), "sync");
  RasterStats rs;
  QGS_CU(cudaMemcpy(&rs, ctx->stats.p, sizeof(rs), cudaMemcpyDeviceToHost), "stats");
  out->n_primitives = ctx->n;
  out->n_visible = ctx->n_visible;  // device counter read by the forward
  out->n_instances = ctx->n_inst;
  out->n_tiles = ctx->n_tiles_total;
  const int64_t nf = -1;  // counters not collected (qgs_set_pair_counters)
  out->pair_evals = ctx->counted_fwd ? (int64_t)rs.pair_evals : nf;
  out->pair_isect = ctx->counted_fwd ? (int64_t)rs.pair_isect : nf;
  out->pair_hits = ctx->counted_fwd ? (int64_t)rs.pair_hits : nf;
  out->pair_blended = ctx->counted_fwd ? (int64_t)rs.pair_blended : nf;
  out->grazing_resolves = ctx->counted_fwd ? (int64_t)rs.grazing : nf;
  out->bwd_pairs = ctx->counted_bwd ? (int64_t)rs.bwd_pairs : nf;
  out->bwd_contrib = ctx->counted_bwd ? (int64_t)rs.bwd_contrib : nf;
  out->launches_fwd = ctx->launches_fwd;
  out->launches_bwd = ctx->launches_bwd;
  auto el = [&](int a, int b) {
    float ms = -1.f;
    if (cudaEventElapsedTime(&ms, ctx->ev[a], ctx->ev[b]) != cudaSuccess) ms = -1.f;
    return ms;
  };
  out->ms_preprocess = ctx->have_fwd_times ? el(0, 1) : -1.f;
  out->ms_depth_sort = ctx->have_fwd_times ? el(1, 2) : -1.f;
  out->ms_emit = ctx->have_fwd_times ? el(3, 4) : -1.f;
  out->ms_tile_sort = ctx->have_fwd_times ? el(4, 5) : -1.f;
  out->ms_raster_fwd = ctx->have_fwd_times ? el(5, 6) : -1.f;
  out->ms_raster_bwd = ctx->have_bwd_times ? el(7, 8) : -1.f;
  out->ms_preprocess_bwd = ctx->have_bwd_times ? el(8, 9) : -1.f;
  return QGS_OK;
}

qgs_status qgs_set_profiling(qgs_ctx* ctx, int32_t enable) {
  if (!ctx) return QGS_EINVAL;
  QGS_CU(cudaSetDevice(ctx->device), "cudaSetDevice");
  if (enable && !ctx->ev[0]) {
    for (int i = 0; i < 10; ++i) QGS_CU(cudaEventCreate(&ctx->ev[i]), "cudaEventCreate");
  }
  ctx->profiling = enable != 0;
  return QGS_OK;
}

qgs_status qgs_set_pair_counters(qgs_ctx* ctx, int32_t enable) {
  if (!ctx) return QGS_EINVAL;
  ctx->pair_counters = enable != 0;
  return QGS_OK;
}

qgs_status qgs_set_tile_mask_capacity(qgs_ctx* ctx, int64_t words) {
  if (!ctx || words < 0) return QGS_EINVAL;
  ctx->tbits_want = (size_t)words;
  ctx->tbits_fixed = true;
  return QGS_OK;
}

qgs_status qgs_check_frame(qgs_ctx* ctx) {
  if (!ctx) return QGS_EINVAL;
  QGS_CU(cudaSetDevice(ctx->device), "cudaSetDevice");
  return check_sorts(ctx);
}

qgs_status qgs_debug_withhold_sort_chunk(qgs_ctx* ctx, int32_t spins) {
  if (!ctx) return QGS_EINVAL;
  if (spins <= 0) {
    ctx->test_withhold = 0;
    ctx->test_spins = kLookbackSpins;
    return QGS_OK;
  }
  ctx->test_withhold = 1;
  ctx->test_spins = spins;
  return QGS_OK;
}

qgs_status qgs_debug_check_word(int32_t device, int32_t* compiled_in, uint32_t* word) {
  if (!compiled_in || !word) return QGS_EINVAL;
  *compiled_in = kDebugChecks ? 1 : 0;
  *word = 0;
  if (!kDebugChecks) return QGS_OK;
#ifdef QGS_DEBUG_CHECKS
  if (cudaSetDevice(device) != cudaSuccess) return QGS_EINVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return QGS_ECUDA;
  uint32_t w = 0, ws = 0;
  const uint32_t zero = 0;
  if (cudaMemcpyFromSymbol(&w, g_check_api, sizeof(uint32_t)) != cudaSuccess ||
      cudaMemcpyToSymbol(g_check_api, &zero, sizeof(uint32_t)) != cudaSuccess || sort_check_word(&ws) != cudaSuccess)
    return QGS_ECUDA;
  *word = w | ws;
#endif
  return QGS_OK;
}

qgs_status qgs_copy_binning(qgs_ctx* ctx, uint64_t* keys, uint32_t* vals, int64_t cap, uint32_t* ranges,
                            int32_t* rects, int64_t* n_instances) {
  if (!ctx) return QGS_EINVAL;
  if (!ctx->have_frame) return fail(ctx, QGS_ESTATE, "no frame rendered yet");
  QGS_CU(cudaSetDevice(ctx->device), "cudaSetDevice");
  const qgs_status s = check_sorts(ctx);
  if (s != QGS_OK) return s;
  QGS_CU(cudaStreamSynchronize(ctx->last_stream), "sync");
  const int64_t I = ctx->n_inst;
  if (n_instances) *n_instances = I;
  if ((keys || vals) && cap < I) return fail(ctx, QGS_ECAPACITY, "key/value capacity smaller than the instance count");
  if ((keys || vals) && I > 0) {
    DevBuf<uint64_t> dk;
    DevBuf<uint32_t> dv;
    QGS_CU(dk.reserve((size_t)I), "alloc");
    if (dv.reserve((size_t)I) != cudaSuccess) {
      dk.release();
      return fail(ctx, QGS_ENOMEM, "alloc");
    }
    if (ctx->cfg.sort_mode == 0 && !ctx->stp) {
      if (ctx->packed32)
        k_debug_packed<uint32_t><<<nblk(I), 256>>>(I, reinterpret_cast<const uint32_t*>(ctx->sorted_keys),
                                                   ctx->rank_bits, ctx->vis_list, ctx->dstate.p, dk.p, dv.p);
      else
        k_debug_packed<uint64_t><<<nblk(I), 256>>>(I, reinterpret_cast<const uint64_t*>(ctx->sorted_keys),
                                                   ctx->rank_bits, ctx->vis_list, ctx->dstate.p, dk.p, dv.p);
    } else {
      cudaMemcpy(dk.p, ctx->sorted_keys, sizeof(uint64_t) * (size_t)I, cudaMemcpyDeviceToDevice);
      cudaMemcpy(dv.p, ctx->ids, sizeof(uint32_t) * (size_t)I, cudaMemcpyDeviceToDevice);
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess && keys) e = cudaMemcpy(keys, dk.p, sizeof(uint64_t) * (size_t)I, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && vals) e = cudaMemcpy(vals, dv.p, sizeof(uint32_t) * (size_t)I, cudaMemcpyDeviceToHost);
    dk.release();
    dv.release();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "copy keys");
  }
  if (ranges) {
    QGS_CU(cudaMemcpy(ranges, ctx->ranges.p, sizeof(uint2) * (size_t)ctx->tiles_x * ctx->tiles_y,
                      cudaMemcpyDeviceToHost),
           "copy ranges");
  }
  if (rects && ctx->n > 0) {
    std::vector<short4> r((size_t)ctx->n);
    QGS_CU(cudaMemcpy(r.data(), ctx->rect.p, sizeof(short4) * (size_t)ctx->n, cudaMemcpyDeviceToHost), "copy rects");
    for (int64_t i = 0; i < ctx->n; ++i) {
      rects[4 * i] = r[i].x;
      rects[4 * i + 1] = r[i].y;
      rects[4 * i + 2] = r[i].z;
      rects[4 * i + 3] = r[i].w;
    }
  }
  return QGS_OK;
}

qgs_status qgs_copy_residue(qgs_ctx* ctx, float* T_final, uint32_t* n_contrib) {
  if (!ctx) return QGS_EINVAL;
  if (!ctx->have_frame) return fail(ctx, QGS_ESTATE, "no frame rendered yet");
  QGS_CU(cudaSetDevice(ctx->device), "cudaSetDevice");
  const qgs_status s = check_sorts(ctx);
  if (s != QGS_OK) return s;
  QGS_CU(cudaStreamSynchronize(ctx->last_stream), "sync");
  const size_t P = (size_t)ctx->W * ctx->H;
  if (T_final) QGS_CU(cudaMemcpy(T_final, ctx->T_final.p, sizeof(float) * P, cudaMemcpyDeviceToHost), "copy T");
  if (n_contrib)
    QGS_CU(cudaMemcpy(n_contrib, ctx->n_contrib.p, sizeof(uint32_t) * P, cudaMemcpyDeviceToHost), "copy n");
  return QGS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// render_forward_noalloc: the forward render with every work buffer carved out of one
// statically sized device array (no cudaMalloc, cudaFree or allocating library call).
// It runs render_forward's kernels (preprocessing, the tile test against the
// parallelogram and the conic, the depth sort, the emission of the same tile lists, the
// tile sort, the compositing) with fixed capacities; only the intermediate layout differs
// (64-bit instances, primitive-indexed state, no tile-mask store), so the planes are the
// same bit for bit.
namespace {

constexpr int64_t NA_MAX_PRIMS = 32768;
constexpr int64_t NA_MAX_PIXELS = 262144;     // e.g. 512 x 512
constexpr int64_t NA_MAX_TILES = 4096;
constexpr int64_t NA_MAX_INSTANCES = 1 << 20;  // (tile, primitive) pairs per frame

constexpr size_t na_align(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t NA_HIST = (size_t)256 * ((NA_MAX_INSTANCES + kRadixChunk - 1) / kRadixChunk) + 1;  // u32
constexpr size_t NA_SCAN = 8192;                                                  // scan block sums (u32)
// byte offsets of each region inside the array
constexpr size_t NA_OFF_STATE = 0;
constexpr size_t NA_OFF_COUNT = NA_OFF_STATE + na_align(sizeof(PrimState) * NA_MAX_PRIMS);
constexpr size_t NA_OFF_ZKEY = NA_OFF_COUNT + na_align(4 * NA_MAX_PRIMS);
constexpr size_t NA_OFF_IDX = NA_OFF_ZKEY + na_align(4 * NA_MAX_PRIMS);
constexpr size_t NA_OFF_ZKEY2 = NA_OFF_IDX + na_align(4 * NA_MAX_PRIMS);
constexpr size_t NA_OFF_IDX2 = NA_OFF_ZKEY2 + na_align(4 * NA_MAX_PRIMS);
constexpr size_t NA_OFF_CNT = NA_OFF_IDX2 + na_align(4 * NA_MAX_PRIMS);
constexpr size_t NA_OFF_OFFS = NA_OFF_CNT + na_align(4 * NA_MAX_PRIMS);
constexpr size_t NA_OFF_RECT = NA_OFF_OFFS + na_align(4 * (NA_MAX_PRIMS + 1));
constexpr size_t NA_OFF_TSLAB = NA_OFF_RECT + na_align(sizeof(short4) * NA_MAX_PRIMS);
constexpr size_t NA_OFF_INST = NA_OFF_TSLAB + na_align(sizeof(TileSlab) * NA_MAX_PRIMS);
constexpr size_t NA_OFF_INST2 = NA_OFF_INST + na_align(8 * NA_MAX_INSTANCES);
constexpr size_t NA_OFF_RANGES = NA_OFF_INST2 + na_align(8 * NA_MAX_INSTANCES);
constexpr size_t NA_OFF_TFIN = NA_OFF_RANGES + na_align(sizeof(uint2) * NA_MAX_TILES);
constexpr size_t NA_OFF_NCON = NA_OFF_TFIN + na_align(4 * NA_MAX_PIXELS);
constexpr size_t NA_OFF_HIST = NA_OFF_NCON + na_align(4 * NA_MAX_PIXELS);
constexpr size_t NA_OFF_SCAN = NA_OFF_HIST + na_align(4 * NA_HIST);
constexpr size_t NA_OFF_STATS = NA_OFF_SCAN + na_align(4 * NA_SCAN);
constexpr size_t NA_OFF_VIS = NA_OFF_STATS + na_align(sizeof(RasterStats));
constexpr size_t NA_BYTES = NA_OFF_VIS + na_align(16);

// The scratch itself (about 27 MB). Every GPU that loads the library holds it until the
// process exits. Host code must not use this name as a device address.
__device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

std::mutex g_na_mutex;
unsigned char* g_na_ptr[64] = {};  // device address of the array, per device

}  // namespace

extern "C" qgs_status render_forward_noalloc(const qgs_scene* scene, const qgs_camera* cam, const qgs_image* out,
                                             qgs_stream stream) {
  qgs_ctx* ctx = nullptr;  // QGS_CU needs the name; there is no context here
  if (!scene || !cam || !out) return QGS_EINVAL;
  if (scene->n < 0) return QGS_EINVAL;
  if (scene->n > 0 && (!scene->mean || !scene->quat || !scene->scale || !scene->curv || !scene->opacity ||
                       !scene->sh))
    return QGS_EINVAL;
  if (scene->n > 0 && ((((uintptr_t)scene->quat) & 15) || (((uintptr_t)scene->sh) & 15) ||
                       (((uintptr_t)scene->scale) & 7) || (((uintptr_t)scene->curv) & 7)))
    return QGS_EINVAL;
  if (cam->W <= 0 || cam->H <= 0 || !finite_cam(cam)) return QGS_EINVAL;
  if (!out->rgb || !out->alpha || !out->depth || !out->normal) return QGS_EINVAL;
  if (out->curvature || out->distortion || out->median_depth) return QGS_EINVAL;  // base planes only
  const int64_t N = scene->n;
  const int64_t P = (int64_t)cam->W * cam->H;
  const int64_t TX = (cam->W + TILE - 1) / TILE, TY = (cam->H + TILE - 1) / TILE;
  if (N > NA_MAX_PRIMS || P > NA_MAX_PIXELS || TX * TY > NA_MAX_TILES) return QGS_ECAPACITY;

  int dev = 0;
  QGS_CU(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev < 0 || dev >= 64) return QGS_EINVAL;
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
      void* p = nullptr;
      QGS_CU(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress");
      g_na_ptr[dev] = static_cast<unsigned char*>(p);
    }
    base = g_na_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  PrimState* state = reinterpret_cast<PrimState*>(base + NA_OFF_STATE);
  uint32_t* count = reinterpret_cast<uint32_t*>(base + NA_OFF_COUNT);
  uint32_t* zkey = reinterpret_cast<uint32_t*>(base + NA_OFF_ZKEY);
  uint32_t* idx = reinterpret_cast<uint32_t*>(base + NA_OFF_IDX);
  uint32_t* zkey2 = reinterpret_cast<uint32_t*>(base + NA_OFF_ZKEY2);
  uint32_t* idx2 = reinterpret_cast<uint32_t*>(base + NA_OFF_IDX2);
  uint32_t* cnt_sorted = reinterpret_cast<uint32_t*>(base + NA_OFF_CNT);
  uint32_t* offs = reinterpret_cast<uint32_t*>(base + NA_OFF_OFFS);
  short4* rect = reinterpret_cast<short4*>(base + NA_OFF_RECT);
  TileSlab* tslab = reinterpret_cast<TileSlab*>(base + NA_OFF_TSLAB);
  uint64_t* inst = reinterpret_cast<uint64_t*>(base + NA_OFF_INST);
  uint64_t* inst2 = reinterpret_cast<uint64_t*>(base + NA_OFF_INST2);
  uint2* ranges = reinterpret_cast<uint2*>(base + NA_OFF_RANGES);
  float* T_final = reinterpret_cast<float*>(base + NA_OFF_TFIN);
  uint32_t* n_contrib = reinterpret_cast<uint32_t*>(base + NA_OFF_NCON);
  SortTemp tmp;
  tmp.hist = reinterpret_cast<uint32_t*>(base + NA_OFF_HIST);
  tmp.hist_cap = NA_HIST;
  tmp.scan_tmp = reinterpret_cast<uint32_t*>(base + NA_OFF_SCAN);
  tmp.scan_cap = NA_SCAN;
  RasterStats* stats = reinterpret_cast<RasterStats*>(base + NA_OFF_STATS);
  // [0] visible primitives, [1] tile instances, [2] unused, [3] sort failure word
  uint32_t* visible = reinterpret_cast<uint32_t*>(base + NA_OFF_VIS);
  tmp.err = visible + 3;

  qgs_config cfg;
  qgs_config_default(&cfg);
  qgs_ctx defaults;
  defaults.cfg = cfg;
  CamParams cp;
  RasterParams rp;
  make_params(&defaults, cam, cp, rp);
  const int64_t ntiles = TX * TY;

  // everything that must start at zero: the counters and the sort failure word, the tile
  // ranges, the pair counters
  QGS_CU(cudaMemsetAsync(visible, 0, 16, st), "memset");
  QGS_CU(cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)ntiles, st), "memset");
  QGS_CU(cudaMemsetAsync(stats, 0, sizeof(RasterStats), st), "memset");
  SceneView sv{scene->mean, scene->quat, scene->scale, scene->curv, scene->opacity, scene->sh};
  if (N > 0) {
    k_preprocess<<<pre_blocks(N), 256, 0, st>>>(N, sv, cp, state, count, zkey, idx, rect, nullptr, nullptr, tslab);
    QGS_CU(cudaGetLastError(), "k_preprocess");
    // keep the rectangle's tiles that meet the parallelogram and the conic (as render_forward)
    k_count_tiles<<<(unsigned)((N + kCountBlock - 1) / kCountBlock), kCountBlock, 0, st>>>(
        N, tslab, cam->W, cam->H, count, rect, zkey, nullptr, visible, nullptr, nullptr, 0u);
    QGS_CU(cudaGetLastError(), "k_count_tiles");
  }
  cudaError_t e = cudaSuccess;
  const bool fl = radix_sort_u32_pairs(zkey, idx, zkey2, idx2, N, 0, 32, tmp, st, &e);
  QGS_CU(e, "depth sort");
  const uint32_t* sidx = fl ? idx2 : idx;
  if (N > 0) {
    k_gather_u32<<<nblk(N), 256, 0, st>>>(N, sidx, count, cnt_sorted, tmp.err);
    QGS_CU(cudaGetLastError(), "gather");
  }
  QGS_CU(scan_exclusive_u32(cnt_sorted, offs, N, tmp.scan_tmp, tmp.scan_cap, st), "scan");
  uint32_t hv[4] = {0, 0, 0, 0};  // pageable host words: a copy, not an allocation
  QGS_CU(cudaMemcpyAsync(hv, visible, sizeof(hv), cudaMemcpyDeviceToHost, st), "totals");
  QGS_CU(cudaStreamSynchronize(st), "sync");
  if (hv[3]) return QGS_ECUDA;  // the depth sort gave up waiting in its look-back
  const int64_t I = (int64_t)hv[1];
  if (I > NA_MAX_INSTANCES) return QGS_ECAPACITY;
  const uint64_t* sorted = inst;
  if (N > 0 && I > 0) {
    k_emit<<<nblk(N), 256, 0, st>>>(N, sidx, count, rect, tslab, cam->W, cam->H, offs, nullptr, cp.tiles_x, inst,
                                    nullptr, nullptr, nullptr, tmp.err);
    QGS_CU(cudaGetLastError(), "emit");
    const bool f2 = radix_sort_u64_keys(inst, inst2, I, 32, 32 + bits_for(ntiles), tmp, st, &e);
    QGS_CU(e, "tile sort");
    sorted = f2 ? inst2 : inst;
    k_tile_ranges<<<nblk(I), 256, 0, st>>>(I, sorted, ranges, tmp.err);
    QGS_CU(cudaGetLastError(), "ranges");
  }
  QGS_CU(launch_raster_fwd(false, false, (unsigned)ntiles, st, ranges, reinterpret_cast<const uint32_t*>(sorted), 2,
                           state, rp, out->rgb, out->alpha, out->depth, out->normal, T_final, n_contrib,
                           ExtraPlanes{}, stats, nullptr, nullptr),
         "k_raster_fwd");
  // the tile sort's failure word (its look-back waits are bounded too)
  QGS_CU(cudaMemcpyAsync(hv + 3, visible + 3, sizeof(uint32_t), cudaMemcpyDeviceToHost, st), "sort status");
  QGS_CU(cudaStreamSynchronize(st), "sync");
  if (hv[3]) return QGS_ECUDA;
  return QGS_OK;
}
