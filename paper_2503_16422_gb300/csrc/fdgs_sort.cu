// Onesweep LSD radix sort of packed 32/64-bit keys (one read and one write of the keys per
// digit pass, decoupled look-back for the per-digit partition prefixes).
//
// The rasterizer orders its (tile, depth) lists with two sorts of this kind: the visible
// Gaussians by depth (keys = depth bits << 32 | id, bits 32..63), then the emitted
// (tile << rank_bits | depth_rank) keys by their tile bits only. Emission happens in depth
// rank order and the sort is stable, so each tile's list comes out in (depth, id) order
// while the per-key sort moves only ceil(log2 tiles) bits.
#include <algorithm>

#include "fdgs_internal.h"

namespace fdgs {

namespace {

constexpr int kSortBlock = 256;
constexpr int kSortWarps = kSortBlock / 32;
constexpr int kRadix = 256;
constexpr int kItems = 16;
constexpr int kTileKeys = kSortBlock * kItems;   // keys per partition
constexpr int kMaxPasses = 8;                    // digit passes supported (64 bits)
constexpr int kAbortWord = 32;                   // index of the abort word after the counters

// Per-digit status word of the onesweep look-back: 2-bit flag | 30-bit count.
constexpr int kLookWin = 4;   // predecessors read per look-back step
constexpr uint32_t kStAgg = 1u << 30, kStPrefix = 2u << 30, kStValue = (1u << 30) - 1;

template <typename K>
__global__ void __launch_bounds__(kSortBlock)
k_histogram(const K *__restrict__ keys, const uint32_t *__restrict__ n_dev, int lo, int dbits,
            int npass, uint32_t *__restrict__ hist) {
  __shared__ uint32_t sh[kMaxPasses * kRadix];
  for (int i = threadIdx.x; i < npass * kRadix; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  const uint32_t n = *n_dev;
  const uint32_t mask = (1u << dbits) - 1u;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const K k = keys[i];
    for (int p = 0; p < npass; ++p)
      atomicAdd(&sh[p * kRadix + (uint32_t)((k >> (lo + p * dbits)) & mask)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < npass * kRadix; i += blockDim.x)
    if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// Exclusive scan of each pass's 256-bin histogram (one block per pass).
__global__ void __launch_bounds__(kRadix) k_hist_scan(uint32_t *hist) {
  __shared__ uint32_t warp_tot[kRadix / 32];
  uint32_t *h = hist + blockIdx.x * kRadix;
  const uint32_t v = h[threadIdx.x];
  uint32_t inc = warp_incl_scan(v);
  if (lane_id() == 31) warp_tot[threadIdx.x >> 5] = inc;
  __syncthreads();
  if (threadIdx.x < 32) {
    uint32_t w = threadIdx.x < kRadix / 32 ? warp_tot[threadIdx.x] : 0u;
    uint32_t wi = warp_incl_scan(w);
    if (threadIdx.x < kRadix / 32) warp_tot[threadIdx.x] = wi - w;
  }
  __syncthreads();
  h[threadIdx.x] = inc - v + warp_tot[threadIdx.x >> 5];
}

// Look-back waits give up after spin_limit polls; the first one to give up sets kErrTimeout in
// err and the call's abort word, every other waiter that sees the abort word gives up too,
// and later passes of the same sort skip their work. A waiter that gives up uses the partial
// prefix it has (never more than the true one), so every scatter address stays inside
// [0, n); the keys are then wrong but no access is out of bounds. withhold: a partition
// whose index equals it publishes nothing (failure injection on the host's request; ~0u
// otherwise).
// Three CTAs an SM (registers capped at 80): 0.55 -> 0.49 ms for the 64-frame batch's depth
// sort against two CTAs at the compiler's 128 registers (four CTAs, 64 registers and spills:
// 0.53 ms). The pass waits on shared memory (the warp ranking and the scatter into s_keys),
// so more resident warps hide more of it.
template <typename K>
__global__ void __launch_bounds__(kSortBlock, 3)
k_onesweep(const K *__restrict__ in, K *__restrict__ out, const uint32_t *__restrict__ n_dev,
           int shift, int dbits, const uint32_t *__restrict__ goff, uint32_t *status,
           uint32_t *part_ctr, uint32_t *err, uint32_t *abort_word, uint32_t spin_limit,
           uint32_t withhold) {
  __shared__ K s_keys[kTileKeys];
  __shared__ uint32_t s_wh[kSortWarps][kRadix + 1];
  __shared__ uint32_t s_bstart[kRadix];
  __shared__ uint32_t s_gbase[kRadix];
  __shared__ uint32_t s_wtot[kSortWarps];
  __shared__ uint32_t s_part;
  const uint32_t n = *n_dev;
  const uint32_t nparts = (n + kTileKeys - 1) / kTileKeys;
  const uint32_t mask = (1u << dbits) - 1u;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (ld_volatile_u32(abort_word)) return;   // an earlier pass of this sort timed out
  for (;;) {
    if (tid == 0) s_part = atomicAdd(part_ctr, 1u);
    for (int i = tid; i < kSortWarps * (kRadix + 1); i += kSortBlock) (&s_wh[0][0])[i] = 0;
    __syncthreads();
    const uint32_t part = s_part;
    if (part >= nparts) break;
    const uint32_t base = part * kTileKeys;
    K keys[kItems];
    uint32_t dig[kItems], rk[kItems];
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
      const uint32_t idx = base + warp * 32 * kItems + k * 32 + lane;
      if (idx < n) {
        keys[k] = in[idx];
        dig[k] = (uint32_t)((keys[k] >> shift) & mask);
      } else {
        keys[k] = 0;
        dig[k] = kRadix;   // dump bin: counted, never written
      }
    }
    // stable ranking within the warp, item by item
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
      const uint32_t d = dig[k];
      const uint32_t peers = __match_any_sync(0xffffffffu, d);
      const uint32_t prev = s_wh[warp][d];
      __syncwarp();
      if (lane == __ffs(peers) - 1) s_wh[warp][d] = prev + __popc(peers);
      __syncwarp();
      rk[k] = prev + __popc(peers & lanemask_lt());
    }
    __syncthreads();
    // digit `tid`: warp-exclusive offsets and block count
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
      const uint32_t c = s_wh[w][tid];
      s_wh[w][tid] = cnt;
      cnt += c;
    }
    // block-exclusive start of each digit
    {
      const uint32_t inc = warp_incl_scan(cnt);
      if (lane == 31) s_wtot[warp] = inc;
      __syncthreads();
      uint32_t wo = 0;
      for (int w = 0; w < warp; ++w) wo += s_wtot[w];
      s_bstart[tid] = inc - cnt + wo;
    }
    // decoupled look-back for digit `tid`
    {
      uint32_t *st = status + (size_t)part * kRadix + tid;
      const bool publish = part != withhold;
      uint32_t excl = 0;
      if (part == 0) {
        if (publish) st_volatile_u32(st, kStPrefix | cnt);
      } else {
        if (publish) st_volatile_u32(st, kStAgg | cnt);
        // the digit's status words of kLookWin predecessors are read at once, so the walk
        // back to the nearest inclusive prefix takes one L2 round trip per kLookWin of them
        int64_t j = (int64_t)part - 1;
        uint32_t spins = 0;
        while (j >= 0) {
          uint32_t sv[kLookWin];
#pragma unroll
          for (int w = 0; w < kLookWin; ++w)   // before partition 0 the prefix is 0
            sv[w] = j - w >= 0 ? ld_volatile_u32(status + (size_t)(j - w) * kRadix + tid)
                               : kStPrefix;
          int used = 0;         // entries summed; a word not yet published stops the window
          bool done = false;
#pragma unroll
          for (int w = 0; w < kLookWin; ++w) {
            if (done || used < w) continue;
            const uint32_t f = sv[w] & ~kStValue;
            if (f == 0) continue;
            excl += sv[w] & kStValue;
            used = w + 1;
            if (f == kStPrefix) done = true;
          }
          if (done) break;
          j -= used;
          if (used < kLookWin) {   // partition j has not published: wait for it
            if (++spins > spin_limit ||
                ((spins & 255) == 0 && ld_volatile_u32(abort_word))) {
              atomicOr(err, kErrTimeout);
              atomicOr(abort_word, 1u);
              break;
            }
            __nanosleep(20);
          }
        }
        if (publish) st_volatile_u32(st, kStPrefix | ((excl + cnt) & kStValue));
      }
      s_gbase[tid] = goff[tid] + excl;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kItems; ++k)
      if (dig[k] < kRadix) s_keys[s_bstart[dig[k]] + s_wh[warp][dig[k]] + rk[k]] = keys[k];
    __syncthreads();
    const uint32_t nvalid = min((uint32_t)kTileKeys, n - base);
    for (uint32_t i = tid; i < nvalid; i += kSortBlock) {
      const K k = s_keys[i];
      const uint32_t d = (uint32_t)((k >> shift) & mask);
      const uint32_t pos = s_gbase[d] + (i - s_bstart[d]);
      if (pos < n) out[pos] = k;   // always true unless a look-back gave up
    }
    __syncthreads();
  }
}

template <typename K>
int onesweep_grid() {
  static int g = 0;
  if (!g) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_onesweep<K>, kSortBlock, 0);
    g = std::max(1, per_sm) * num_sms();
  }
  return g;
}

size_t status_bytes(uint64_t n_cap) {
  const uint64_t parts = (n_cap + kTileKeys - 1) / kTileKeys;
  return std::max<uint64_t>(parts, 1) * kRadix * sizeof(uint32_t);
}

}  // namespace

int sort_passes(int bits) { return bits <= 0 ? 0 : (bits + 7) / 8; }
int sort_digit_bits(int bits) {
  const int np = sort_passes(bits);
  return np ? (bits + np - 1) / np : 0;
}

size_t sort_scratch_bytes(uint64_t n_cap, int bits) {
  const int np = std::max(1, sort_passes(bits));
  // hist [8][256] + 256 bytes of words (partition counters of the passes, the abort word)
  // + one status region per pass
  return kMaxPasses * kRadix * sizeof(uint32_t) + 256 + np * status_bytes(n_cap);
}

uint32_t g_debug_spin_limit = 0;
uint32_t g_debug_withhold = ~0u;

template <typename K>
K *radix_sort(K *a, K *b, const uint32_t *n_dev, uint64_t n_cap, int lo, int bits,
              void *scratch, cudaStream_t st, uint32_t *err_dev, bool hist_ready) {
  const int np = sort_passes(bits);
  if (np == 0 || n_cap == 0) return a;
  if (np > kMaxPasses) return a;   // wider than 64 bits: the histogram holds 8 passes
  const int dbits = (bits + np - 1) / np;
  uint32_t *hist = (uint32_t *)scratch;
  uint32_t *ctr = hist + kMaxPasses * kRadix;
  uint8_t *status0 = (uint8_t *)scratch + kMaxPasses * kRadix * sizeof(uint32_t) + 256;
  const size_t sb = status_bytes(n_cap);
  const size_t hist_bytes = kMaxPasses * kRadix * sizeof(uint32_t);
  if (hist_ready) {
    cudaMemsetAsync((uint8_t *)scratch + hist_bytes, 0,
                    sort_scratch_bytes(n_cap, bits) - hist_bytes, st);
  } else {
    cudaMemsetAsync(scratch, 0, sort_scratch_bytes(n_cap, bits), st);
    const int hgrid = (int)std::min<uint64_t>((n_cap + 4095) / 4096, (uint64_t)num_sms() * 4);
    k_histogram<K><<<std::max(1, hgrid), kSortBlock, 0, st>>>(a, n_dev, lo, dbits, np, hist);
    k_hist_scan<<<np, kRadix, 0, st>>>(hist);
  }
  const uint64_t parts = (n_cap + kTileKeys - 1) / kTileKeys;
  const int grid = (int)std::min<uint64_t>(parts, (uint64_t)onesweep_grid<K>());
  // per-call words after the partition counters: ctr[kAbortWord] is the call's abort flag
  // (zeroed with the rest of the scratch above)
  uint32_t *abort_word = ctr + kAbortWord;
  // injected failures apply to eager launches only: a captured graph would replay them
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cap);
  const bool eager = cap == cudaStreamCaptureStatusNone;
  const uint32_t spin = eager && g_debug_spin_limit ? g_debug_spin_limit : kSpinLimit;
  const uint32_t withhold = eager ? g_debug_withhold : ~0u;
  if (eager) g_debug_withhold = ~0u;   // one-shot: only the next sort pass withholds
  K *src = a, *dst = b;
  for (int p = 0; p < np; ++p) {
    k_onesweep<K><<<std::max(1, grid), kSortBlock, 0, st>>>(
        src, dst, n_dev, lo + p * dbits, dbits, hist + p * kRadix,
        (uint32_t *)(status0 + p * sb), ctr + p, err_dev, abort_word, spin,
        p == 0 ? withhold : ~0u);
    std::swap(src, dst);
  }
  return src;
}

template uint32_t *radix_sort<uint32_t>(uint32_t *, uint32_t *, const uint32_t *, uint64_t, int,
                                        int, void *, cudaStream_t, uint32_t *, bool);
template uint64_t *radix_sort<uint64_t>(uint64_t *, uint64_t *, const uint32_t *, uint64_t, int,
                                        int, void *, cudaStream_t, uint32_t *, bool);

}  // namespace fdgs
