// Device-wide exclusive scan and stable LSD radix sort (hand-written, no library).
//
// Scan: 4096 values per CTA, 16 per thread in registers (vector loads); a reduce pass
// writes the chunk sums, and the scan pass adds to each chunk the sum of the chunk sums
// before it (summed by the CTA itself while there are at most 2048 chunks).
//
// Radix sort: per pass of at most 8 bits (sorts of up to 2M keys run each pass as one
// kernel, see k_radix_downsweep's look-back),
//   1. upsweep  - each CTA histograms the digits of its 2048-key chunk into a
//                 digit-major count matrix hist[d * nblocks + b];
//   2. scan     - one exclusive scan of that matrix gives, for every (digit, chunk), the
//                 global position of the chunk's first key with that digit;
//   3. downsweep - each warp ranks its 256 keys in order (the lanes holding the same
//                 digit found with one ballot per digit bit), warp-level digit counters
//                 are scanned across the CTA's warps, and every key is written to
//                 base(d, chunk) + (keys with digit d in earlier warps) + rank in warp.
// Keys keep their relative order within a digit (stable), so successive passes from
// the least significant digit up sort by the whole bit range.
#include <algorithm>

#include "qgs_internal.cuh"

namespace qgs {

namespace {

constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_CHUNK = BLOCK * SCAN_ITEMS;  // 4096 values per CTA
constexpr int kScanDirectPrefix = 2048;          // chunks up to which each CTA sums its own prefix
constexpr int RS_WARPS = 8;
constexpr int RS_ITEMS = 8;                     // keys per lane
constexpr int RS_CHUNK = RS_WARPS * 32 * RS_ITEMS;  // 2048 keys per CTA
static_assert(RS_CHUNK == kRadixChunk, "histogram sizing assumes kRadixChunk keys per CTA");
constexpr unsigned FULL = 0xffffffffu;
#ifdef QGS_DEBUG_CHECKS
__device__ uint32_t g_check_sort;  // QGS_CHECK bits of this file's kernels
#endif

// Load / store 16 consecutive u32 of a chunk (vectorised when the addresses allow it).
__device__ __forceinline__ void load16(const uint32_t* in, int64_t i0, int64_t n, bool vec,
                                       uint32_t v[SCAN_ITEMS]) {
  if (vec && i0 + SCAN_ITEMS <= n) {
    const uint4* p = reinterpret_cast<const uint4*>(in + i0);
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS / 4; ++q) {
      const uint4 w = p[q];
      v[4 * q] = w.x; v[4 * q + 1] = w.y; v[4 * q + 2] = w.z; v[4 * q + 3] = w.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) v[k] = i0 + k < n ? in[i0 + k] : 0u;
  }
}

// Exclusive scan of the CTA's SCAN_CHUNK values held 16 per thread in registers (thread t
// holds items [16 t, 16 t + 16)): in-thread scan, warp shuffles over the thread totals,
// one pass over the warp totals. Returns the CTA total.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v[SCAN_ITEMS]) {
  __shared__ uint32_t warp_tot[BLOCK / 32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  uint32_t run = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    const uint32_t x = v[k];
    v[k] = run;
    run += x;
  }
  uint32_t inc = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(FULL, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  uint32_t wbase = 0, total = 0;
#pragma unroll
  for (int w = 0; w < BLOCK / 32; ++w) {
    const uint32_t x = warp_tot[w];
    if (w < warp) wbase += x;
    total += x;
  }
  const uint32_t base = wbase + inc - run;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) v[k] += base;
  return total;
}

__global__ void __launch_bounds__(BLOCK) k_scan_reduce(const uint32_t* __restrict__ in, int64_t n,
                                                       uint32_t* __restrict__ sums, bool vec) {
  __shared__ uint32_t red[BLOCK / 32];
  uint32_t v[SCAN_ITEMS];
  load16(in, (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_ITEMS, n, vec, v);
  uint32_t acc = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) acc += v[k];
  acc = __reduce_add_sync(FULL, acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < BLOCK / 32; ++w) t += red[w];
    sums[blockIdx.x] = t;
  }
}

// Scan of each chunk plus the sum of the chunk sums before it (each CTA adds up its own
// prefix from `sums`); the last CTA also writes the total to out[n]. in and out may be
// the same array (each thread reads its items before the CTA barrier, writes after).
__global__ void __launch_bounds__(BLOCK) k_scan_down(const uint32_t* in, int64_t n,
                                                     const uint32_t* __restrict__ sums, uint32_t* out,
                                                     bool vec) {
  __shared__ uint32_t red[BLOCK / 32];
  uint32_t off = 0;
  if (sums) {  // prefix of this chunk: sum of the earlier chunk sums
    uint32_t acc = 0;
    for (int b = threadIdx.x; b < (int)blockIdx.x; b += BLOCK) acc += sums[b];
    acc = __reduce_add_sync(FULL, acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
#pragma unroll
    for (int w = 0; w < BLOCK / 32; ++w) off += red[w];
  }
  const int64_t i0 = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_ITEMS;
  uint32_t v[SCAN_ITEMS];
  load16(in, i0, n, vec, v);
  const uint32_t total = block_exclusive_scan(v);
  if (vec && i0 + SCAN_ITEMS <= n) {
    uint4* p = reinterpret_cast<uint4*>(out + i0);
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS / 4; ++q)
      p[q] = make_uint4(v[4 * q] + off, v[4 * q + 1] + off, v[4 * q + 2] + off, v[4 * q + 3] + off);
  } else {
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k)
      if (i0 + k < n) out[i0 + k] = v[k] + off;
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = off + total;
}

// Scan of each chunk plus its precomputed offset offs[blockIdx.x] (many chunks).
__global__ void __launch_bounds__(BLOCK) k_scan_down_off(const uint32_t* in, int64_t n,
                                                         const uint32_t* __restrict__ offs, uint32_t* out,
                                                         bool vec) {
  const uint32_t off = offs[blockIdx.x];
  const int64_t i0 = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_ITEMS;
  uint32_t v[SCAN_ITEMS];
  load16(in, i0, n, vec, v);
  const uint32_t total = block_exclusive_scan(v);
  if (vec && i0 + SCAN_ITEMS <= n) {
    uint4* p = reinterpret_cast<uint4*>(out + i0);
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS / 4; ++q)
      p[q] = make_uint4(v[4 * q] + off, v[4 * q + 1] + off, v[4 * q + 2] + off, v[4 * q + 3] + off);
  } else {
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k)
      if (i0 + k < n) out[i0 + k] = v[k] + off;
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = off + total;
}

template <typename K>
__device__ __forceinline__ uint32_t digit_of(K key, int shift, uint32_t mask) {
  return (uint32_t)(key >> shift) & mask;
}

template <typename K>
__global__ void __launch_bounds__(BLOCK) k_radix_upsweep(const K* __restrict__ keys, int64_t n, int shift,
                                                         uint32_t mask, uint32_t* __restrict__ hist, int nblocks) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RS_CHUNK;
  K kk[RS_CHUNK / BLOCK];  // all loads in flight before the first count
#pragma unroll
  for (int it = 0; it < RS_CHUNK / BLOCK; ++it) {
    const int64_t i = base + it * BLOCK + threadIdx.x;
    kk[it] = i < n ? keys[i] : (K)0;
  }
#pragma unroll
  for (int it = 0; it < RS_CHUNK / BLOCK; ++it) {
    const int64_t i = base + it * BLOCK + threadIdx.x;
    if (i < n) atomicAdd(&h[digit_of(kk[it], shift, mask)], 1u);
  }
  __syncthreads();
  if (threadIdx.x <= mask) hist[(size_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

template <typename K, bool HAS_VAL>
constexpr size_t downsweep_smem() {
  return sizeof(K) * RS_CHUNK + (HAS_VAL ? sizeof(uint32_t) * RS_CHUNK : 0);
}

// Look-back status words of the single-pass scatter: bits 30..31 = 0 (not yet published),
// 1 (the chunk's own digit count) or 2 (the inclusive prefix over chunks 0..b), bits 0..29
// the count. A chunk waits at most `spins` polls for a predecessor, then sets the error
// word and continues (no hang; the result is then reported as a failure). Its keys still
// land inside the output: the digit offsets it found are never larger than the true ones.
// A pass that starts with the error word already set does nothing (its input would no
// longer match the digit counts taken before the first pass).
constexpr uint32_t kStAgg = 1u << 30, kStInc = 2u << 30, kStVal = (1u << 30) - 1u;
constexpr int kLookbackMaxChunks = 1024;  // sorts of up to 2M keys use the single-pass scatter
constexpr int kLookbackWindow = 8;        // predecessor status words read per round trip

// Stable scatter of one 2048-key chunk. Keys are ranked per warp (lanes of one digit found
// with one ballot per digit bit), the per-warp digit counts are scanned across warps and
// digits, the chunk is reordered by digit in shared memory, and then written out so that
// consecutive threads store consecutive keys of a digit run (coalesced). The chunk's
// global digit offsets come either from the scanned count matrix `offs` (LOOKBACK false)
// or, in a single pass (LOOKBACK true), from the whole array's digit counts `ghist` plus
// the counts of the earlier chunks, found by decoupled look-back: chunks take their index
// from a ticket, publish their own counts, then add up their predecessors' published
// counts until one that published its inclusive prefix (a chunk only ever waits for
// chunks with smaller tickets, which have already started and publish before waiting).
template <typename K, bool HAS_VAL, bool LOOKBACK>
__global__ void __launch_bounds__(BLOCK) k_radix_downsweep(const K* __restrict__ kin, K* __restrict__ kout,
                                                           const uint32_t* __restrict__ vin,
                                                           uint32_t* __restrict__ vout, int64_t n, int shift,
                                                           uint32_t mask, const uint32_t* __restrict__ offs,
                                                           int nblocks, const uint32_t* __restrict__ ghist,
                                                           uint32_t* status, uint32_t* ticket, uint32_t* err,
                                                           int spins_max) {
  extern __shared__ __align__(16) unsigned char dsm[];
  K* skeys = reinterpret_cast<K*>(dsm);
  uint32_t* svals = reinterpret_cast<uint32_t*>(skeys + RS_CHUNK);
  __shared__ uint32_t wh[RS_WARPS][256];
  __shared__ uint32_t boff[256];
  __shared__ uint32_t lstart[256];
  __shared__ uint32_t wsum[RS_WARPS];
  __shared__ uint32_t s_chunk, s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int chunk = blockIdx.x;
  if constexpr (LOOKBACK) {
    if (threadIdx.x == 0) {
      s_abort = *(volatile const uint32_t*)err;  // an earlier pass gave up: nothing to do
      s_chunk = atomicAdd(ticket, 1u);
    }
    __syncthreads();
    if (s_abort) return;
    chunk = (int)s_chunk;
  }
  const int64_t cbase = (int64_t)chunk * RS_CHUNK;
  const int64_t wbase = cbase + (int64_t)warp * 32 * RS_ITEMS;
  const uint32_t lt = (1u << lane) - 1u;
  const int nbits = 32 - __clz(mask);
  K kk[RS_ITEMS];
  uint32_t vv[RS_ITEMS];
  uint32_t rk[RS_ITEMS];
  // every global load first (the chunk's keys and its digit offsets, independent and in
  // flight together), then the ranking below, whose barriers would otherwise serialise
  // each load's latency
  uint32_t my_off = 0;
  if constexpr (LOOKBACK) {
    my_off = threadIdx.x <= mask ? ghist[threadIdx.x] : 0u;  // scanned into the global base below
  } else {
    my_off = threadIdx.x <= mask ? offs[(size_t)threadIdx.x * nblocks + blockIdx.x] : 0u;
  }
#pragma unroll
  for (int it = 0; it < RS_ITEMS; ++it) {
    const int64_t i = wbase + it * 32 + lane;
    kk[it] = i < n ? kin[i] : (K)0;
    if (HAS_VAL) vv[it] = i < n ? vin[i] : 0u;
  }
  for (int e = threadIdx.x; e < RS_WARPS * 256; e += BLOCK) (&wh[0][0])[e] = 0;
  if (!LOOKBACK && threadIdx.x <= mask) boff[threadIdx.x] = my_off;
  __syncthreads();
#pragma unroll
  for (int it = 0; it < RS_ITEMS; ++it) {
    const int64_t i = wbase + it * 32 + lane;
    const bool valid = i < n;
    const K key = kk[it];
    const uint32_t d = valid ? digit_of(key, shift, mask) : 0x100u + (uint32_t)lane;
    // lanes holding the same digit: one ballot per digit bit (invalid lanes carry a
    // lane-unique value above the digit range and match nobody; one match instruction
    // measured slower than these ballots)
    const uint32_t vmask = __ballot_sync(FULL, valid);  // every lane takes part in each ballot
    uint32_t peers = valid ? vmask : (1u << lane);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      if (b < nbits) {  // uniform across the grid
        const uint32_t bal = __ballot_sync(FULL, (d >> b) & 1u);
        peers &= ((d >> b) & 1u) ? bal : ~bal;
      }
    }
    if (!valid) peers = 1u << lane;
    const uint32_t before = valid ? wh[warp][d] : 0u;
    __syncwarp();
    if (valid && (peers & lt) == 0) wh[warp][d] = before + __popc(peers);
    __syncwarp();
    rk[it] = valid ? before + __popc(peers & lt) : 0xFFFFFFFFu;
  }
  __syncthreads();
  // per digit: exclusive scan across warps; digit totals -> exclusive scan across digits
  uint32_t tot = 0;
  {
    const int d = threadIdx.x;
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) {
      const uint32_t c = wh[w][d];
      wh[w][d] = tot;
      tot += c;
    }
    uint32_t inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(FULL, inc, o);
      if (lane >= o) inc += v;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    uint32_t base = 0;
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w)
      if (w < warp) base += wsum[w];
    lstart[d] = base + inc - tot;
  }
  if constexpr (LOOKBACK) {
    const int d = threadIdx.x;
    const bool live = (uint32_t)d <= mask;
    // publish this chunk's count of digit d (its inclusive prefix if it is the first)
    if (live) atomicExch(status + (size_t)chunk * 256 + d, (chunk == 0 ? kStInc : kStAgg) | tot);
    // the whole array's digit counts -> exclusive scan across digits (the digit's base)
    uint32_t inc = my_off;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(FULL, inc, o);
      if (lane >= o) inc += v;
    }
    __syncthreads();  // wsum is reused
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    uint32_t gbase = 0;
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w)
      if (w < warp) gbase += wsum[w];
    gbase += inc - my_off;
    // look back over the earlier chunks' counts of digit d, kLookbackWindow status words
    // per round trip (nearest first; a word not yet published is polled on its own)
    uint32_t excl = 0;
    if (live) {
      bool done = chunk == 0;
      for (int k0 = chunk - 1; !done && k0 >= 0; k0 -= kLookbackWindow) {
        uint32_t win[kLookbackWindow];
#pragma unroll
        for (int q = 0; q < kLookbackWindow; ++q)
          win[q] = k0 - q >= 0 ? *(volatile const uint32_t*)(status + (size_t)(k0 - q) * 256 + d) : kStInc;
#pragma unroll
        for (int q = 0; q < kLookbackWindow; ++q) {
          if (done) break;
          uint32_t sv = win[q];
          int spins = 0;
          while ((sv & ~kStVal) == 0u && spins < spins_max) {
            __nanosleep(32);
            sv = *(volatile const uint32_t*)(status + (size_t)(k0 - q) * 256 + d);
            ++spins;
          }
          if ((sv & ~kStVal) == 0u) {  // gave up: report, do not hang
            atomicOr(err, 1u);
            done = true;
            break;
          }
          excl += sv & kStVal;  // (past chunk 0 the window holds an empty inclusive word)
          if (sv & kStInc) done = true;
        }
      }
      if (chunk > 0) atomicExch(status + (size_t)chunk * 256 + d, kStInc | (excl + tot));
      boff[d] = gbase + excl;
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < RS_ITEMS; ++it) {
    if (rk[it] == 0xFFFFFFFFu) continue;
    const uint32_t d = digit_of(kk[it], shift, mask);
    const uint32_t lp = lstart[d] + wh[warp][d] + rk[it];
    if (!QGS_CHECK(g_check_sort, lp < (uint32_t)RS_CHUNK, kChkScatter)) continue;
    skeys[lp] = kk[it];
    if (HAS_VAL) svals[lp] = vv[it];
  }
  __syncthreads();
  const int cnt = (int)min((int64_t)RS_CHUNK, n - cbase);
  for (int i = threadIdx.x; i < cnt; i += BLOCK) {
    const K key = skeys[i];
    const uint32_t d = digit_of(key, shift, mask);
    const uint32_t pos = boff[d] + (uint32_t)i - lstart[d];
    if (!QGS_CHECK(g_check_sort, (int64_t)pos < n, kChkScatter)) continue;
    kout[pos] = key;
    if (HAS_VAL) vout[pos] = svals[i];
  }
}

__global__ void k_set_u32(uint32_t* p, uint32_t v) { *p = v; }

// Digit counts of every pass over the whole array, from one read of the keys.
struct PassSpec {
  int passes;
  int shift[8];
  uint32_t mask[8];
};
template <typename K>
__global__ void __launch_bounds__(BLOCK) k_radix_hist_all(const K* __restrict__ keys, int64_t n, PassSpec ps,
                                                          uint32_t* __restrict__ ghist) {
  __shared__ uint32_t h[8][256];
  for (int e = threadIdx.x; e < 8 * 256; e += BLOCK) (&h[0][0])[e] = 0u;
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * BLOCK + threadIdx.x; i < n; i += (int64_t)gridDim.x * BLOCK) {
    const K key = keys[i];
#pragma unroll
    for (int p = 0; p < 8; ++p)
      if (p < ps.passes) atomicAdd(&h[p][digit_of(key, ps.shift[p], ps.mask[p])], 1u);
  }
  __syncthreads();
#pragma unroll
  for (int p = 0; p < 8; ++p)
    if (p < ps.passes && (uint32_t)threadIdx.x <= ps.mask[p] && h[p][threadIdx.x])
      atomicAdd(&ghist[p * 256 + threadIdx.x], h[p][threadIdx.x]);
}

int scan_blocks(int64_t n) { return (int)((n + SCAN_CHUNK - 1) / SCAN_CHUNK); }

template <typename K, bool HAS_VAL>
bool radix_sort_impl(K* k0, uint32_t* v0, K* k1, uint32_t* v1, int64_t n, int begin_bit, int end_bit,
                     SortTemp& tmp, cudaStream_t st, cudaError_t* err) {
  *err = cudaSuccess;
  bool flipped = false;
  if (n <= 1 || end_bit <= begin_bit) return false;
  const int bits = end_bit - begin_bit;
  const int passes = (bits + 7) / 8;
  const int nblocks = (int)((n + RS_CHUNK - 1) / RS_CHUNK);
  constexpr size_t smem = downsweep_smem<K, HAS_VAL>();
  static bool attr_set[64] = {};  // per instantiation and device
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !attr_set[dev]) {
    *err = cudaFuncSetAttribute(k_radix_downsweep<K, HAS_VAL, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
    if (*err == cudaSuccess)
      *err = cudaFuncSetAttribute(k_radix_downsweep<K, HAS_VAL, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem);
    if (*err != cudaSuccess) return false;
    if (dev >= 0 && dev < 64) attr_set[dev] = true;
  }
  PassSpec ps{};
  ps.passes = passes;
  {
    int shift = begin_bit;
    for (int p = 0; p < passes; ++p) {
      const int pb = (bits - (shift - begin_bit) + (passes - p) - 1) / (passes - p);  // spread bits evenly
      ps.shift[p] = shift;
      ps.mask[p] = (1u << pb) - 1u;
      shift += pb;
    }
  }
  // single-pass scatter with look-back: status words [passes][nblocks][256], the passes'
  // digit counts [passes][256] and one ticket per pass, zeroed together
  const size_t lb_words = (size_t)passes * nblocks * 256 + (size_t)passes * 256 + passes + 1;
  // (for small sorts: its per-digit look-back walks grow with the chunks in flight, so large
  // sorts keep the count-matrix passes)
  if (nblocks <= kLookbackMaxChunks && passes <= 8 && lb_words <= tmp.hist_cap) {
    uint32_t* status = tmp.hist;
    uint32_t* ghist = status + (size_t)passes * nblocks * 256;
    uint32_t* tickets = ghist + (size_t)passes * 256;
    uint32_t* errw = tmp.err ? tmp.err : tickets + passes;  // a spare word when nobody reads the error
    *err = cudaMemsetAsync(status, 0, lb_words * sizeof(uint32_t), st);
    if (*err != cudaSuccess) return false;
    // test hook: the first pass's tickets start after the withheld chunks, which never run
    const int withheld = std::min(std::max(tmp.withhold_chunks, 0), nblocks - 1);
    tmp.withhold_chunks = 0;
    if (withheld > 0) {
      k_set_u32<<<1, 1, 0, st>>>(tickets, (uint32_t)withheld);
      ++launch_counter();
    }
    k_radix_hist_all<K><<<(unsigned)std::min(nblocks, 1024), BLOCK, 0, st>>>(k0, n, ps, ghist);
    ++launch_counter();
    for (int p = 0; p < passes; ++p) {
      K* kin = flipped ? k1 : k0;
      K* kout = flipped ? k0 : k1;
      uint32_t* vin = flipped ? v1 : v0;
      uint32_t* vout = flipped ? v0 : v1;
      const int ctas = nblocks - (p == 0 ? withheld : 0);
      k_radix_downsweep<K, HAS_VAL, true><<<ctas, BLOCK, smem, st>>>(
          kin, kout, vin, vout, n, ps.shift[p], ps.mask[p], nullptr, nblocks, ghist + (size_t)p * 256,
          status + (size_t)p * nblocks * 256, tickets + p, errw, tmp.spins);
      ++launch_counter();
      *err = cudaGetLastError();
      if (*err != cudaSuccess) return flipped;
      flipped = !flipped;
    }
    return flipped;
  }
  for (int p = 0; p < passes; ++p) {
    const int shift = ps.shift[p];
    const uint32_t mask = ps.mask[p];
    const int64_t m = (int64_t)(mask + 1) * nblocks;
    if ((size_t)m + 1 > tmp.hist_cap) {
      *err = cudaErrorInvalidValue;  // histogram buffer too small for this sort
      return flipped;
    }
    K* kin = flipped ? k1 : k0;
    K* kout = flipped ? k0 : k1;
    uint32_t* vin = flipped ? v1 : v0;
    uint32_t* vout = flipped ? v0 : v1;
    k_radix_upsweep<K><<<nblocks, BLOCK, 0, st>>>(kin, n, shift, mask, tmp.hist, nblocks);
    ++launch_counter();
    *err = scan_exclusive_u32(tmp.hist, tmp.hist, m, tmp.scan_tmp, tmp.scan_cap, st);
    if (*err != cudaSuccess) return flipped;
    k_radix_downsweep<K, HAS_VAL, false><<<nblocks, BLOCK, smem, st>>>(kin, kout, vin, vout, n, shift, mask, tmp.hist,
                                                                       nblocks, nullptr, nullptr, nullptr, nullptr, 0);
    ++launch_counter();
    *err = cudaGetLastError();
    if (*err != cudaSuccess) return flipped;
    flipped = !flipped;
  }
  return flipped;
}

}  // namespace

size_t scan_tmp_elems(int64_t n) {
  // block sums of each level plus their scans, with room for the totals
  size_t tot = 0;
  int64_t m = n;
  while (m > SCAN_CHUNK) {
    const int64_t b = scan_blocks(m);
    tot += 2 * (size_t)b + 2;
    m = b;
  }
  return tot + 16;
}

size_t radix_hist_elems(int64_t n) {
  // the single-pass scatter's status words, digit counts, tickets and a spare word for up
  // to 8 passes
  const int64_t nblocks = (n + RS_CHUNK - 1) / RS_CHUNK;
  return (size_t)8 * 256 * (size_t)(nblocks > 0 ? nblocks : 1) + 8 * 256 + 8 + 1;
}

cudaError_t scan_exclusive_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* tmp, size_t tmp_cap,
                               cudaStream_t st) {
  if (n <= 0) {
    return cudaMemsetAsync(out, 0, sizeof(uint32_t), st);
  }
  const bool vec = ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15) == 0;
  const int nb = scan_blocks(n);
  if (nb == 1) {
    k_scan_down<<<1, BLOCK, 0, st>>>(in, n, nullptr, out, vec);
    ++launch_counter();
    return cudaGetLastError();
  }
  if ((size_t)(2 * nb + 2) > tmp_cap) return cudaErrorInvalidValue;
  uint32_t* sums = tmp;
  k_scan_reduce<<<nb, BLOCK, 0, st>>>(in, n, sums, vec);
  ++launch_counter();
  if (nb <= kScanDirectPrefix) {
    // few chunks: each CTA of the second pass adds up its own prefix of the chunk sums
    k_scan_down<<<nb, BLOCK, 0, st>>>(in, n, sums, out, vec);
    ++launch_counter();
    return cudaGetLastError();
  }
  uint32_t* sums_scan = tmp + nb;  // nb + 1 slots
  cudaError_t e = scan_exclusive_u32(sums, sums_scan, nb, tmp + 2 * nb + 2, tmp_cap - (2 * nb + 2), st);
  if (e != cudaSuccess) return e;
  k_scan_down_off<<<nb, BLOCK, 0, st>>>(in, n, sums_scan, out, vec);
  ++launch_counter();
  return cudaGetLastError();
}

cudaError_t sort_check_word(uint32_t* word) {
  *word = 0;
#ifdef QGS_DEBUG_CHECKS
  cudaError_t e = cudaMemcpyFromSymbol(word, g_check_sort, sizeof(uint32_t));
  const uint32_t zero = 0;
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_check_sort, &zero, sizeof(uint32_t));
  return e;
#else
  return cudaSuccess;
#endif
}

bool radix_sort_u32_pairs(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, int64_t n, int begin_bit,
                          int end_bit, SortTemp& tmp, cudaStream_t st, cudaError_t* err) {
  return radix_sort_impl<uint32_t, true>(k0, v0, k1, v1, n, begin_bit, end_bit, tmp, st, err);
}

bool radix_sort_u32_keys(uint32_t* k0, uint32_t* k1, int64_t n, int begin_bit, int end_bit, SortTemp& tmp,
                         cudaStream_t st, cudaError_t* err) {
  return radix_sort_impl<uint32_t, false>(k0, nullptr, k1, nullptr, n, begin_bit, end_bit, tmp, st, err);
}

bool radix_sort_u64_keys(uint64_t* k0, uint64_t* k1, int64_t n, int begin_bit, int end_bit, SortTemp& tmp,
                         cudaStream_t st, cudaError_t* err) {
  return radix_sort_impl<uint64_t, false>(k0, nullptr, k1, nullptr, n, begin_bit, end_bit, tmp, st, err);
}

bool radix_sort_u64_pairs(uint64_t* k0, uint32_t* v0, uint64_t* k1, uint32_t* v1, int64_t n, int begin_bit,
                          int end_bit, SortTemp& tmp, cudaStream_t st, cudaError_t* err) {
  return radix_sort_impl<uint64_t, true>(k0, v0, k1, v1, n, begin_bit, end_bit, tmp, st, err);
}

}  // namespace qgs
