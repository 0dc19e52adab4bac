// Batched rendering of many (camera, t, resolution) requests in one device-driven pipeline
// that is captured once in a CUDA graph and replayed:
//   k_pre_batch      per-Gaussian stage over all (request, partition) items; each item
//                    writes its visible keys to its own 256-key segment
//   k_part_scan      per-request scan of the segments' counts -> offsets, visible counts
//   k_batch_bases    per-request visible counts -> contiguous bases and 256-aligned slots
//   k_seg_compact    request segments -> one contiguous array of (request, depth, id) keys
//   radix_sort       one global depth sort (request bits on top keep requests apart)
//   k_gather_batch   blend-ready records and tile rectangles per slot, per-request key
//                    counts, coverage difference arrays and block-row/column bitmasks
//   k_tile_scan_batch  per-request tile counts and longest-first queue keys, block-list ranges
//                    (capacity-checked)
//   k_lists_blocks   block lists, a warp per 4x4 block of tiles: the block's entries from its
//                    bitmasks, each with the mask of the block's tiles it covers
//   radix_sort       queue keys by list length (descending)
//   k_blend_persist  persistent CTAs take tiles from the queue, longest first, and record
//                    each request's completion time (%globaltimer)
#include <math.h>

#include <algorithm>
#include <vector>

#include "fdgs_blend.cuh"
#include "fdgs_gauss.cuh"
#include "fdgs_internal.h"

namespace fdgs {

namespace {

constexpr int kB = 256;
constexpr int kW = kB / 32;
constexpr int kMaxReq = 128;
constexpr int kIdBits = kBatchIdBits;        // Gaussian id bits of the depth key
constexpr uint64_t kIdMask = (1ull << kIdBits) - 1;

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Index of the last base <= x in an ascending array of n bases (n >= 1).
__device__ __forceinline__ int find_segment(const uint32_t *bases, int n, uint32_t x) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int m = (lo + hi + 1) >> 1;
    if (bases[m] <= x) lo = m; else hi = m - 1;
  }
  return lo;
}

// ---------------------------------------------------------------------------------------
// The time- and camera-independent part of every Gaussian's forward, once per batch.
__global__ void __launch_bounds__(kB) k_cond_batch(BatchDev b) {
  for (uint32_t i = blockIdx.x * kB + threadIdx.x; i < b.n; i += gridDim.x * kB) {
    GaussState g;
    float inv_nt;
    gauss_cond(__ldg(&b.ls4[i]), __ldg(&b.ql[i]), __ldg(&b.qr[i]), __ldg(&b.opacity[i]), g,
               inv_nt);
    cond_store(g, inv_nt, b.cond + (size_t)i * kCond4);
  }
}

// Requests served by one item of the batched preprocess: the item's partition of 256
// Gaussians has its SH coefficients staged in shared memory and its conditional factors held
// in registers once for all of them (they do not depend on the request), instead of being
// read from L2 once per request.
constexpr int kPreGroup = 16;
// Dynamic shared memory of k_pre_batch: the staged SH planes of one partition.
inline size_t pre_smem_bytes(int deg, bool vq) {
  return (size_t)(vq ? 3 : (deg + 1) * (deg + 1) * 3) * kB * sizeof(float);
}

// Four CTAs an SM (registers capped at 64; the staged coefficients take 48 KB a CTA at degree
// 3): 0.63 ms per 64 requests for the one-request-per-item kernel, 0.50 with groups of 8 at 80
// registers, 0.44 with groups of 16 at 64.
template <bool kVQ>
__global__ void __launch_bounds__(kB, 4) k_pre_batch(BatchDev b) {
  __shared__ uint32_t s_item;
  __shared__ uint32_t s_wcnt[kW];
  extern __shared__ float s_sh[];   // [planes][kB]: plane k * 3 + c of the partition
  const uint32_t P = (b.n + kB - 1) / kB;
  const uint32_t G = (b.nreq + kPreGroup - 1) / kPreGroup;
  const uint32_t items = P * G;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int K = (b.deg + 1) * (b.deg + 1);
  const int planes = kVQ ? 3 : K * 3;
  for (;;) {
    if (tid == 0) s_item = atomicAdd(&b.ctr[BC_PRE_ITEM], 1u);
    __syncthreads();
    const uint32_t item = s_item;
    if (item >= items) break;
    // request-group-major, or partition-major (the groups of one partition back to back,
    // sharing its attributes in L2) for scenes too large for L2; segments and counts are
    // stored request-major (si)
    const uint32_t grp = b.part_major ? item % G : item / P;
    const uint32_t part = b.part_major ? item / G : item % P;
    const uint32_t i = part * kB + tid;
    const bool in = i < b.n;
    for (int pl = 0; pl < planes; ++pl)
      s_sh[pl * kB + tid] = in ? __ldg(&b.sh[(size_t)pl * b.n + i]) : 0.f;
    GaussState g0;
    float inv_nt = 0.f;
    float4 mean = make_float4(0.f, 0.f, 0.f, 0.f);
    if (in) {
      cond_load(b.cond + (size_t)i * kCond4, g0, inv_nt);
      mean = __ldg(&b.mean4[i]);
    }
    // the codebook row (vector-quantised SH): bands k >= 1
    const float *row = kVQ && in ? b.sh_cb + (size_t)__ldg(&b.sh_code[i]) * (size_t)(K - 1) * 3
                                 : nullptr;
    __syncthreads();   // the staged coefficients
    const uint32_t r_end = min((grp + 1) * (uint32_t)kPreGroup, (uint32_t)b.nreq);
    for (uint32_t r = grp * kPreGroup; r < r_end; ++r) {
      const uint32_t si = r * P + part;
      const ReqDesc &q = b.reqs[r];
      bool active = false, vis = false;
      uint64_t key = 0;
      if (in) {
        active = true;
        if (q.mask_l) {
          const uint32_t w = __ldg(&q.mask_l[i >> 5]) | __ldg(&q.mask_r[i >> 5]);
          active = (w >> (i & 31)) & 1u;
        }
        if (active) {
          GaussState g = g0;
          const uint8_t fl = gauss_forward_tail(q.cam, q.t, mean, inv_nt, g);
          if (fl & kFlagDet) {
            const float half = 0.5f * (g.c00 - g.c11);
            const float disc = half * half + g.c01 * g.c01;
            const float mid = 0.5f * (g.c00 + g.c11);
            const float lam = mid + sqrtf(fmaxf(kRadiusFloor, disc));
            const float rad = ceilf(3.f * sqrtf(lam));
            const float u = fmaf(q.cam.fx, g.xr, q.cam.cx);
            const float v = fmaf(q.cam.fy, g.yr, q.cam.cy);
            int x0, y0, x1, y1;
            tile_rect(u, v, rad, q.cam.gx, q.cam.gy, x0, y0, x1, y1);
            if (x1 > x0 && y1 > y0) {
              vis = true;
              float rgb[3];
              gauss_colour_from(q.cam, b.deg, g, rgb, [&](int k, int c) {
                return (kVQ && k > 0) ? __ldg(&row[(k - 1) * 3 + c])
                                      : s_sh[(k * 3 + c) * kB + tid];
              });
              // the blend-ready record by (request, id), and the alpha-tight tile rectangle:
              // the arithmetic of the per-frame record and gather, so records and lists equal
              // those of fdgs_render
              const float idet = 1.f / g.det;
              const float A = g.c11 * idet, B = -g.c01 * idet, C = g.c00 * idet;
              const float qa = -0.5f * kLog2e * A, qb = -kLog2e * B, qc = -0.5f * kLog2e * C;
              const size_t ri = (size_t)r * b.n + i;
              float4 *rp = reinterpret_cast<float4 *>(b.rec + ri * kRec);
              rp[0] = make_float4(u, v, qa, qb);
              rp[1] = make_float4(qc, log2f(g.a), rgb[0], rgb[1]);
              rp[2] = make_float4(rgb[2], -qb / (2.f * qa), -qb / (2.f * qc), rad);
              tighten_rect(u, v, A, B, C, g.a, x0, y0, x1, y1);
              if (!(x1 > x0 && y1 > y0)) x0 = y0 = x1 = y1 = 0;
              b.rect_id[ri] = make_uint2((uint32_t)x0 | ((uint32_t)x1 << 16),
                                         (uint32_t)y0 | ((uint32_t)y1 << 16));
              key = ((uint64_t)r << 57) | ((uint64_t)__float_as_uint(g.xc[2]) << kIdBits) |
                    (uint64_t)i;
            }
          }
        }
      }
      const uint32_t vb = __ballot_sync(0xffffffffu, vis);
      if (lane == 0) s_wcnt[warp] = __popc(vb);
      __syncthreads();
      if (tid == 0) {
        uint32_t tot = 0;
        for (int w = 0; w < kW; ++w) {
          const uint32_t c = s_wcnt[w];
          s_wcnt[w] = tot;
          tot += c;
        }
        b.part[si].x = tot;
      }
      __syncthreads();
      // the item's own 256-key segment, in id order; placed by k_seg_compact
      if (vis) b.vis_seg[(size_t)si * kB + s_wcnt[warp] + __popc(vb & lanemask_lt())] = key;
      __syncthreads();
    }
  }
}

// One CTA per request: exclusive scan of its partitions' visible counts -> segment offsets
// and the request's visible count.
constexpr int kPS = 1024;
__global__ void __launch_bounds__(kPS) k_part_scan(BatchDev b) {
  __shared__ uint32_t s_wsum[kPS / 32];
  __shared__ uint32_t s_carry;
  const uint32_t P = (b.n + kB - 1) / kB;
  uint2 *part = b.part + (size_t)blockIdx.x * P;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_carry = 0;
  __syncthreads();
  for (uint32_t p0 = 0; p0 < P; p0 += kPS) {
    const uint32_t i = p0 + tid;
    const uint32_t c = i < P ? part[i].x : 0u;
    const uint32_t inc = warp_incl_scan(c);
    if (lane == 31) s_wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      const uint32_t w = s_wsum[lane];
      s_wsum[lane] = warp_incl_scan(w) - w;
    }
    __syncthreads();
    const uint32_t excl = s_carry + s_wsum[warp] + inc - c;
    if (i < P) part[i].y = excl;
    __syncthreads();
    if (tid == kPS - 1) s_carry = excl + c;
    __syncthreads();
  }
  if (tid == 0) b.nv[blockIdx.x] = s_carry;
}

// Per-request bases (one warp; nreq <= 128): contiguous visible bases and 256-aligned slots.
__global__ void k_batch_bases(BatchDev b) {
  const int lane = threadIdx.x;
  uint32_t vcarry = 0, scarry = 0;
  for (int r0 = 0; r0 < b.nreq; r0 += 32) {
    const int r = r0 + lane;
    const uint32_t nv = r < b.nreq ? b.nv[r] : 0u;
    const uint32_t ns = (nv + kB - 1) / kB * kB;
    const uint32_t vi = warp_incl_scan(nv), si = warp_incl_scan(ns);
    if (r < b.nreq) {
      b.vis_base[r] = vcarry + vi - nv;
      b.slot_base[r] = scarry + si - ns;
    }
    vcarry += __shfl_sync(0xffffffffu, vi, 31);
    scarry += __shfl_sync(0xffffffffu, si, 31);
  }
  if (lane == 0) {
    b.ctr[BC_NVIS] = vcarry;
    b.ctr[BC_NSLOTS] = scarry;
    b.ctr[BC_NTILES] = b.ntiles;
  }
}

__global__ void k_seg_compact(BatchDev b) {
  const uint32_t P = (b.n + kB - 1) / kB;
  const uint64_t total = (uint64_t)b.nreq * P * kB;
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
       k += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t item = (uint32_t)(k / kB), i = (uint32_t)(k % kB);
    const uint2 pc = b.part[item];
    if (i < pc.x) b.vis[b.vis_base[item / P] + pc.y + i] = b.vis_seg[k];
  }
}

// The batched lists never leave the library, so they always use the alpha-tight tile sets
// (tighten_rect); images are those of the 3-sigma squares.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kB, 4) k_gather_batch(BatchDev b) {
  __shared__ uint32_t s_slot_base[kMaxReq];
  for (int r = threadIdx.x; r < b.nreq; r += kB) s_slot_base[r] = b.slot_base[r];
  __syncthreads();
  const uint32_t nparts = b.ctr[BC_NSLOTS] / kB;
  const int tid = threadIdx.x, lane = tid & 31;
  for (uint32_t part = blockIdx.x; part < nparts; part += gridDim.x) {
    const uint32_t s = part * kB + tid;
    const int r = find_segment(s_slot_base, b.nreq, part * kB);   // one request per partition
    const ReqDesc &q = b.reqs[r];
    const uint32_t l = s - s_slot_base[r];
    const bool valid = l < b.nv[r];
    uint32_t cnt = 0;
    int x0 = 0, y0 = 0, x1 = 0, y1 = 0;
    if (valid) {
      // the slot's Gaussian and its tile rectangle (computed with its record)
      const uint64_t key = b.vis_sorted[b.vis_base[r] + l];
      const uint32_t ri = r * b.n + (uint32_t)(key & kIdMask);
      const uint2 rc = b.rect_id[ri];
      b.rect[s] = rc;
      b.ridx[s] = ri;
      x0 = (int)(rc.x & 0xFFFFu);
      x1 = (int)(rc.x >> 16);
      y0 = (int)(rc.y & 0xFFFFu);
      y1 = (int)(rc.y >> 16);
      if (x1 > x0 && y1 > y0) cnt = (uint32_t)((x1 - x0) * (y1 - y0));
    }
    // block-row and block-column coverage bitmasks of the request (a block row holds
    // kListBlock tile rows); the warp owns local word l / 32
    {
      const int bgx = (q.cam.gx + kListBlock - 1) / kListBlock;
      const int bgy = (q.cam.gy + kListBlock - 1) / kListBlock;
      const size_t mw = b.mask_words;
      uint32_t *rows = b.masks + q.mask_base + (l >> 5);
      uint32_t *cols = rows + (size_t)bgy * mw;
      const int e = kListBlock - 1;
      warp_coverage_words(y0 / kListBlock, (y1 + e) / kListBlock, bgy, rows, mw);
      warp_coverage_words(x0 / kListBlock, (x1 + e) / kListBlock, bgx, cols, mw);
    }
    // the request's key count (its lists' total length); the partition's part of it
    const uint32_t ws = warp_sum(cnt);
    if (lane == 0 && ws) atomicAdd(&b.key_cnt[r], (unsigned long long)ws);
  }
}

// One CTA per request: the request's list totals, the capacity check (empty block ranges if
// the lists would overflow it), and the block lists' ranges from the block coverage counts.
constexpr int kTS = 1024;

// Exclusive scan, in cell order, of the counts of a w x h grid (row stride w); emit(cell,
// start, count) for every cell.
template <class Cnt, class F>
__device__ void scan_cells(const Cnt *d, int w, int h, uint32_t *s_wsum, uint32_t &s_carry,
                           F &&emit) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t cells = (uint32_t)w * h;
  if (tid == 0) s_carry = 0;
  __syncthreads();
  for (uint32_t c0 = 0; c0 < cells; c0 += kTS) {
    const uint32_t t = c0 + tid;
    const uint32_t c = t < cells ? (uint32_t)d[t] : 0u;
    const uint32_t inc = warp_incl_scan(c);
    if (lane == 31) s_wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      const uint32_t v = s_wsum[lane];
      s_wsum[lane] = warp_incl_scan(v) - v;
    }
    __syncthreads();
    const uint32_t start = s_carry + s_wsum[warp] + inc - c;
    if (t < cells) emit(t, start, c);
    __syncthreads();
    if (tid == kTS - 1) s_carry = start + c;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kTS) k_tile_scan_batch(BatchDev b) {
  __shared__ uint32_t s_wsum[kTS / 32];
  __shared__ uint32_t s_carry;
  const int r = blockIdx.x;
  const ReqDesc &q = b.reqs[r];
  const int bgx = (q.cam.gx + kListBlock - 1) / kListBlock;
  const int bgy = (q.cam.gy + kListBlock - 1) / kListBlock;
  // the request's first block-list entry: the counts of the requests before it
  uint64_t nkeys = 0, bbase = 0, nbkeys = 0;
  for (int i = 0; i < b.nreq; ++i) {
    const uint64_t c = b.key_cnt[i], cb = b.bkey_cnt[i];
    if (i < r) bbase += cb;
    nkeys += c;
    nbkeys += cb;
  }
  if (r == 0 && threadIdx.x == 0) {
    b.ctr[BC_NKEYS_LO] = (uint32_t)nkeys;
    b.ctr[BC_NKEYS_HI] = (uint32_t)(nkeys >> 32);
    b.ctr[BC_NBKEYS_LO] = (uint32_t)nbkeys;
    b.ctr[BC_NBKEYS_HI] = (uint32_t)(nbkeys >> 32);
  }
  const bool overflow = nbkeys > b.key_cap;
  if (overflow && threadIdx.x == 0) atomicOr(b.err, kErrCapacity);
  scan_cells(b.bcount + q.block_base, bgx, bgy, s_wsum, s_carry,
             [&](uint32_t k, uint32_t start, uint32_t c) {
               const uint32_t st = (uint32_t)(bbase + start);
               b.branges[q.block_base + k] = overflow ? make_uint2(0, 0) : make_uint2(st, st + c);
             });
}

// Block lists: one warp per block of kListBlock x kListBlock tiles writes, in rank order, the
// record indices (request x n + id) of the Gaussians whose tile rectangles meet the block,
// each with the 16-bit mask of the block's tiles the rectangle covers. The warp ANDs the block's row and column bitmasks
// 64 words at a time (two per lane, the next words in flight) and queues the entries found;
// all lanes together then form the new entries' tile masks from their rectangles
// (independent loads) and write the queue out with coalesced stores. A tile's list is the
// entries of its block list whose mask holds its bit, in order: the blend reads it that way.
// The queue holds kLQ entries; a round of 64 words with more entries than fit is queued in
// parts (each lane keeps its remaining bits), so the queue stays small and many warps fit.
constexpr int kLW = 4;                          // warps per CTA
constexpr uint32_t kLQ = 288;                   // queue entries per warp
static_assert(kListBlock == 4, "the tile masks below hold 4 x 4 tiles in 16 bits");

// Per-tile entry counts of a block list, kept by each lane for the entries it handles: the
// 16-bit tile mask of an entry is spread four bits to a word of byte fields (bit j of a nibble
// to bit 8 j) and added to four lane-local words; tile_counts_flush sums those words over the
// warp into lane t < 16's count of tile t and clears them. A field grows by at most one per
// entry, so a lane flushes at least every 255 entries.
__device__ __forceinline__ void tile_counts_add(uint32_t tm, uint32_t acc[4]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) acc[k] += (((tm >> (4 * k)) & 0xFu) * 0x204081u) & 0x01010101u;
}
__device__ __forceinline__ void tile_counts_flush(uint32_t acc[4], uint32_t lane,
                                                  uint32_t &tcnt) {
  uint32_t red[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    // per byte field: sum over the warp without carries between fields (each field of a
    // lane is at most 255, so the four fields are summed as separate 16-bit halves)
    const uint32_t lo = __reduce_add_sync(0xffffffffu, acc[k] & 0x00FF00FFu);
    const uint32_t hi = __reduce_add_sync(0xffffffffu, (acc[k] >> 8) & 0x00FF00FFu);
    red[k] = lane < 16 ? ((lane & 1) ? hi : lo) : 0u;
    acc[k] = 0u;
  }
  const uint32_t k = lane >> 2;
  const uint32_t w = k == 0 ? red[0] : k == 1 ? red[1] : k == 2 ? red[2] : red[3];
  // field f = lane & 3 of the word: bytes 0 and 2 went to lo (halves), 1 and 3 to hi
  if (lane < 16) tcnt += (w >> (16 * ((lane & 3) >> 1))) & 0xFFFFu;
}

// Entries of every block list: per block (a warp), the popcount of the AND of its row and
// column bitmasks, and the request's total.
__global__ void __launch_bounds__(kLW * 32) k_block_counts(BatchDev b) {
  __shared__ uint32_t s_block_base[kMaxReq];
  for (int r = threadIdx.x; r < b.nreq; r += kLW * 32) s_block_base[r] = b.reqs[r].block_base;
  __syncthreads();
  const int warp = threadIdx.x >> 5;
  const uint32_t lane = lane_id();
  const size_t mw = b.mask_words;
  for (uint32_t gb = blockIdx.x * kLW + warp; gb < b.nblocks; gb += gridDim.x * kLW) {
    const int r = find_segment(s_block_base, b.nreq, gb);
    const ReqDesc &q = b.reqs[r];
    const int bgx = (q.cam.gx + kListBlock - 1) / kListBlock;
    const int bgy = (q.cam.gy + kListBlock - 1) / kListBlock;
    const uint32_t lb = gb - q.block_base;
    const uint32_t words = (b.nv[r] + 31) / 32;
    const uint4 *rows = reinterpret_cast<const uint4 *>(b.masks + q.mask_base +
                                                        (size_t)(lb / bgx) * mw);
    const uint4 *cols = reinterpret_cast<const uint4 *>(b.masks + q.mask_base +
                                                        (size_t)(bgy + lb % bgx) * mw);
    // four words per lane per step (masks zero up to the 256-slot boundary)
    const uint32_t quads = (words + 3) / 4;
    uint32_t c = 0;
    for (uint32_t i = lane; i < quads; i += 32) {
      const uint4 x = __ldg(&rows[i]), y = __ldg(&cols[i]);
      c += __popc(x.x & y.x) + __popc(x.y & y.y) + __popc(x.z & y.z) + __popc(x.w & y.w);
    }
    c = warp_sum(c);
    if (lane == 0) {
      b.bcount[gb] = c;
      if (c) atomicAdd(&b.bkey_cnt[r], (unsigned long long)c);
    }
  }
}

__global__ void __launch_bounds__(kLW * 32) k_lists_blocks(BatchDev b) {
  __shared__ uint32_t s_slot[kLW][kLQ];
  __shared__ uint32_t s_block_base[kMaxReq];
  for (int r = threadIdx.x; r < b.nreq; r += kLW * 32) s_block_base[r] = b.reqs[r].block_base;
  __syncthreads();
  const int warp = threadIdx.x >> 5;
  const uint32_t lane = lane_id();
  uint32_t *qs = s_slot[warp];
  const uint2 *__restrict__ rect = b.rect;
  const uint32_t *__restrict__ ridx = b.ridx;
  uint32_t *__restrict__ lists = b.lists;
  uint16_t *__restrict__ ltm = b.ltm;
  const uint32_t *__restrict__ masks = b.masks;
  const size_t mw = b.mask_words;
  const int nreq = b.nreq;
  for (uint32_t gb = blockIdx.x * kLW + warp; gb < b.nblocks; gb += gridDim.x * kLW) {
    const uint2 brg = b.branges[gb];
    const int r = find_segment(s_block_base, nreq, gb);
    const ReqDesc &q = b.reqs[r];
    const int gx = q.cam.gx, gy = q.cam.gy;
    const int bgx = (gx + kListBlock - 1) / kListBlock;
    const int bgy = (gy + kListBlock - 1) / kListBlock;
    const uint32_t lb = gb - q.block_base;
    const int bx0 = (int)(lb % bgx) * kListBlock, by0 = (int)(lb / bgx) * kListBlock;
    const uint32_t words = (b.nv[r] + 31) / 32, base = b.slot_base[r];
    const uint32_t *rows = masks + q.mask_base + (size_t)(by0 / kListBlock) * mw;
    const uint32_t *cols = masks + q.mask_base + (size_t)bgy * mw + (size_t)(bx0 / kListBlock) * mw;
    uint32_t out = brg.x;                        // next list position (warp-uniform)
    uint32_t tcnt = 0;                           // lane t < 16: entries of the block's tile t
    uint32_t tacc[4] = {0u, 0u, 0u, 0u}, tn = 0;  // lane-local counts, entries since a flush
    // two words per lane per round (64-bit loads; the masks are zero up to the request's
    // 256-slot boundary, so the pair of the last word is readable and empty); the words of
    // the next round are loaded while this round is processed
    const uint2 *rows2 = reinterpret_cast<const uint2 *>(rows);
    const uint2 *cols2 = reinterpret_cast<const uint2 *>(cols);
    const uint32_t pairs = brg.y > brg.x ? (words + 1) / 2 : 0u;   // an empty list: no pass
    uint2 nr = lane < pairs ? __ldg(&rows2[lane]) : make_uint2(0u, 0u);
    uint2 nc = lane < pairs ? __ldg(&cols2[lane]) : make_uint2(0u, 0u);
    for (uint32_t p0 = 0; p0 < pairs; p0 += 32) {
      const uint32_t sb = base + (p0 + lane) * 64;
      uint64_t m = ((uint64_t)(nr.y & nc.y) << 32) | (nr.x & nc.x);
      const uint32_t pn = p0 + 32 + lane;
      nr = pn < pairs ? __ldg(&rows2[pn]) : make_uint2(0u, 0u);
      nc = pn < pairs ? __ldg(&cols2[pn]) : make_uint2(0u, 0u);
      uint32_t pc = __popcll(m);
      uint32_t inc = warp_incl_scan(pc);
      uint32_t tot = __shfl_sync(0xffffffffu, inc, 31);
      while (tot) {
        uint32_t pos = inc - pc;
        while (m && pos < kLQ) {
          qs[pos++] = sb + (uint32_t)(__ffsll(m) - 1);
          m &= m - 1;
        }
        const uint32_t qn = min(tot, kLQ);
        __syncwarp();
        // tile masks from the rectangles (independent loads), coalesced stores
        for (uint32_t e0 = 0; e0 < qn; e0 += 32) {
          const uint32_t e = e0 + lane;
          uint32_t tm = 0;
          if (e < qn) {
            const uint32_t slot = qs[e];
            const uint2 rc = __ldg(&rect[slot]);
            const uint32_t ri = __ldg(&ridx[slot]);
            const int rx0 = max((int)(rc.x & 0xFFFFu) - bx0, 0);
            const int rx1 = min((int)(rc.x >> 16) - bx0, kListBlock);
            const int ry0 = max((int)(rc.y & 0xFFFFu) - by0, 0);
            const int ry1 = min((int)(rc.y >> 16) - by0, kListBlock);
            if (rx1 > rx0 && ry1 > ry0) {
              const uint32_t xm = (1u << rx1) - (1u << rx0);
              const uint32_t ym = (1u << (kListBlock * ry1)) - (1u << (kListBlock * ry0));
              tm = (xm * 0x1111u) & ym;
            }
            if (out + e < brg.y) {               // the block's range bounds every store
              lists[out + e] = ri;
              ltm[out + e] = (uint16_t)tm;
            } else {
              tm = 0;
            }
          }
          tile_counts_add(tm, tacc);
          if (++tn == 255u) {                     // uniform: every lane counts each step
            tile_counts_flush(tacc, lane, tcnt);
            tn = 0;
          }
        }
        out += qn;
        __syncwarp();
        if (tot <= kLQ) break;
        pc = __popcll(m);                          // bits the full queue could not take
        inc = warp_incl_scan(pc);
        tot = __shfl_sync(0xffffffffu, inc, 31);
      }
    }
    tile_counts_flush(tacc, lane, tcnt);
    // the block's tiles: list lengths (as [0, length) ranges: the blend skips empty tiles)
    // and the keys of the longest-first queue
    if (lane < kListBlock * kListBlock) {
      const int tx = bx0 + (int)(lane % kListBlock), ty = by0 + (int)(lane / kListBlock);
      if (tx < gx && ty < gy) {
        const uint32_t gt = q.tile_base + (uint32_t)(ty * gx + tx);
        b.ranges[gt] = make_uint2(0u, tcnt);
        const uint32_t len = min(tcnt, 0xFFFFFFu);
        b.qkeys[gt] = ((uint64_t)(0xFFFFFFu - len) << 32) | gt;
      }
    }
  }
}

// Persistent blend over the longest-first queue of all requests' tiles.
// Only the images are written: nothing reads a batched frame's transmittance or n_contrib.
// kWeights (score pass): also the per-slot blend weights and stop flags.
// The minimum resident CTAs cap the registers at 69 (four pixels a lane) so that 14 CTAs fit
// an SM (measured: 9.42 ms per 64 frames at 14 CTAs against 9.88 ms at the compiler's own 80
// registers, 12 CTAs).
// kTma: records staged by TMA gather4 through b.rec_map (the map lives in the kernel's
// parameter space, hence __grid_constant__); a stage wait that gives up ends the CTA's work
// with kErrTimeout set.
// kBlack: every request of the batch has a black background, so only the T = 0 colour blend
// is compiled in (fewer registers: 64 against 71 for four pixels a lane).
template <int FW, int PX, bool kCount, bool kWeights = false, bool kTma = false,
          bool kBlack = false>
__global__ void __launch_bounds__(256 / PX, PX == 8 ? 24 : (PX == 4 ? 14 : (PX == 2 ? 7 : 4)))
    k_blend_persist(const __grid_constant__ BatchDev b) {
  constexpr int NT = 256 / PX;
  __shared__ BlendSmem<NT, kTma> sm;
  __shared__ uint32_t s_q;
  __shared__ uint32_t s_tile_base[kMaxReq];
  for (int r = threadIdx.x; r < b.nreq; r += NT) s_tile_base[r] = b.reqs[r].tile_base;
  uint32_t tma_ph = 0;
  if constexpr (kTma) {
    if (threadIdx.x == 0) {
      mbar_init((uint32_t)__cvta_generic_to_shared(&sm.stage.bar[0]), NT / 4);
      mbar_init((uint32_t)__cvta_generic_to_shared(&sm.stage.bar[1]), NT / 4);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
  }
  for (;;) {
    if (threadIdx.x == 0) s_q = atomicAdd(&b.ctr[BC_QUEUE], 1u);
    __syncthreads();
    const uint32_t qi = s_q;
    if (qi >= b.ntiles) break;
    const uint32_t gt = (uint32_t)b.queue[qi];
    const int r = find_segment(s_tile_base, b.nreq, gt);
    const ReqDesc &q = b.reqs[r];
    const uint32_t t = gt - q.tile_base;
    BlendTile bt;
    bt.tx = t % q.cam.gx;
    bt.ty = t / q.cam.gx;
    bt.W = q.cam.W;
    bt.H = q.cam.H;
    // the tile reads its block's list and stages the entries that hold its bit; a tile with
    // no entries of its own composites nothing (background only)
    const uint2 own = b.ranges[gt];
    const int bgx = (q.cam.gx + kListBlock - 1) / kListBlock;
    bt.range = own.y > own.x
                   ? b.branges[q.block_base + (uint32_t)((bt.ty / kListBlock) * bgx +
                                                         bt.tx / kListBlock)]
                   : make_uint2(0, 0);
    bt.tmask = b.ltm;
    bt.tbit = (bt.ty % kListBlock) * kListBlock + bt.tx % kListBlock;
    bt.rec_sorted = b.rec;                       // blend-ready records by record index
    bt.rgb = q.rgb;
    bt.T_final = nullptr;
    bt.n_contrib = nullptr;
    bt.bg0 = q.bg[0];
    bt.bg1 = q.bg[1];
    bt.bg2 = q.bg[2];
    bt.w_sum = kWeights ? b.w_sum : nullptr;
    bt.stop_mark = kWeights ? b.stop_mark : nullptr;
    bt.evals = b.evals;
    bt.tmap = &b.rec_map;
    bt.err = b.err;
    bt.tma_skip = b.tma_skip;
    bt.tma_spin = b.tma_spin;
    static_assert(!kBlack || (!kWeights && !kCount), "kBlack: plain colour blend only");
    bool ok;
    if constexpr (kBlack)
      ok = blend_tile<uint32_t, FW, PX, false, false, false, true, true, kTma>(
          bt, b.lists, 0xFFFFFFFFu, sm, tma_ph);
    else if (!kWeights && !kCount && q.bg[0] == 0.f && q.bg[1] == 0.f && q.bg[2] == 0.f)
      ok = blend_tile<uint32_t, FW, PX, false, false, false, true, true, kTma>(
          bt, b.lists, 0xFFFFFFFFu, sm, tma_ph);
    else
      ok = blend_tile<uint32_t, FW, PX, kWeights, kCount, false, true, false, kTma>(
          bt, b.lists, 0xFFFFFFFFu, sm, tma_ph);
    if (!ok) break;                              // uniform over the CTA
    __syncthreads();
    if (threadIdx.x == 0) atomicMax(&b.done_ns[r], (unsigned long long)global_timer_ns());
  }
}

__global__ void k_batch_start(BatchDev b) {
  if (threadIdx.x == 0) *b.t0_ns = global_timer_ns();
}

__global__ void k_stamp(unsigned long long *stamps, int i) { stamps[i] = global_timer_ns(); }

int grid_of(const void *kernel, int threads, int per_sm_cap, size_t smem = 0) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
  per_sm = std::max(1, std::min(per_sm, per_sm_cap));
  return per_sm * num_sms();
}

}  // namespace

// Enqueues the whole batch on `st` (capturable: no host synchronisation, grid sizes depend
// only on the plan). The caller zeroes nothing: the memsets are part of the sequence.
void launch_batch(const BatchDev &b, BatchLaunch &L, cudaStream_t st) {
  cudaMemsetAsync(b.ctr, 0, BC_COUNT * sizeof(uint32_t), st);
  cudaMemsetAsync(b.key_cnt, 0, b.nreq * sizeof(unsigned long long), st);
  cudaMemsetAsync(b.bkey_cnt, 0, b.nreq * sizeof(unsigned long long), st);
  cudaMemsetAsync(b.done_ns, 0, b.nreq * sizeof(unsigned long long), st);
  if (b.evals) cudaMemsetAsync(b.evals, 0, 3 * sizeof(unsigned long long), st);
  if (b.w_sum) {
    cudaMemsetAsync(b.w_sum, 0, L.wsum_len * sizeof(float), st);
    cudaMemsetAsync(b.stop_mark, 0, L.wsum_len * sizeof(uint32_t), st);
  }
  // stage boundaries: a one-thread kernel stamps %globaltimer (events recorded inside a
  // captured graph cannot be timed); stream order makes each difference a stage duration
  auto mark = [&](int i) { k_stamp<<<1, 1, 0, st>>>(b.stamps, i); };
  k_batch_start<<<1, 32, 0, st>>>(b);
  mark(0);
  static int g_pre = 0, g_gather = 0;
  k_cond_batch<<<(int)std::min<uint64_t>((b.n + kB - 1) / kB, (uint64_t)num_sms() * 8), kB, 0,
                 st>>>(b);
  const size_t pre_smem = pre_smem_bytes(b.deg, b.sh_cb != nullptr);
  static size_t pre_smem_set = 0;
  if (pre_smem > pre_smem_set) {   // above 48 KB the kernels must opt in
    cudaFuncSetAttribute(k_pre_batch<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)pre_smem);
    cudaFuncSetAttribute(k_pre_batch<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)pre_smem);
    pre_smem_set = pre_smem;
    g_pre = 0;
  }
  if (!g_pre) g_pre = grid_of((const void *)k_pre_batch<false>, kB, 64, pre_smem);
  if (!g_gather) g_gather = grid_of((const void *)k_gather_batch, kB, 64);
  const uint64_t pre_items = (uint64_t)((b.n + kB - 1) / kB) *
                             (uint64_t)((b.nreq + kPreGroup - 1) / kPreGroup);
  if (b.sh_cb)
    k_pre_batch<true><<<(int)std::min<uint64_t>(pre_items, g_pre), kB, pre_smem, st>>>(b);
  else
    k_pre_batch<false><<<(int)std::min<uint64_t>(pre_items, g_pre), kB, pre_smem, st>>>(b);
  mark(1);
  k_part_scan<<<b.nreq, kPS, 0, st>>>(b);
  k_batch_bases<<<1, 32, 0, st>>>(b);
  const uint64_t rn = (uint64_t)b.nreq * b.n;
  const uint64_t segs = (uint64_t)((b.n + kB - 1) / kB) * b.nreq;   // (request, partition)
  k_seg_compact<<<(int)std::min<uint64_t>(segs, (uint64_t)num_sms() * 16), kB, 0, st>>>(b);
  uint64_t *srt = radix_sort<uint64_t>(b.vis, b.vis_alt, b.ctr + BC_NVIS, rn, kIdBits,
                                       64 - kIdBits, L.sort_scratch, st, b.err);
  mark(2);
  BatchDev b2 = b;
  b2.vis_sorted = srt;
  L.vis_sorted = srt;
  const uint64_t slot_parts = (rn + (uint64_t)b.nreq * kB) / kB;
  k_gather_batch<<<(int)std::min<uint64_t>(slot_parts, g_gather), kB, 0, st>>>(b2);
  mark(3);
  k_block_counts<<<(int)std::min<uint64_t>((b.nblocks + kLW - 1) / kLW,
                                            (uint64_t)num_sms() * 32),
                   kLW * 32, 0, st>>>(b2);
  k_tile_scan_batch<<<b.nreq, kTS, 0, st>>>(b2);
  mark(4);
  k_lists_blocks<<<(int)std::min<uint64_t>((b.nblocks + kLW - 1) / kLW,
                                            (uint64_t)num_sms() * 32),
                   kLW * 32, 0, st>>>(b2);
  mark(5);
  uint64_t *qs = radix_sort<uint64_t>(b.qkeys, b.qkeys_alt, b.ctr + BC_NTILES, b.ntiles, 32, 24,
                                      L.sort_scratch, st, b.err);
  b2.queue = qs;
  mark(6);
  const int grid = L.blend_ctas_per_sm * num_sms();
  if (b.w_sum) {
    // weighted passes: one weighted variant (8x16 footprint, four pixels per lane), then
    // the per-Gaussian score accumulation or contributor marks
    static int per_sm = 0;
    if (!per_sm) {
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_blend_persist<8, 4, false, true>,
                                                    64, 0);
      per_sm = std::max(1, per_sm);
    }
    if (L.staging == 1 && b.rec_map_ok)
      k_blend_persist<8, 4, false, true, true><<<per_sm * num_sms(), 64, 0, st>>>(b2);
    else
      k_blend_persist<8, 4, false, true><<<per_sm * num_sms(), 64, 0, st>>>(b2);
    if (b.score) launch_score_batch(b2, st);
    if (b.mark) launch_mark_batch(b2, st);
  } else {
    const bool tma = L.staging == 1 && b.rec_map_ok;
    const bool black = L.black != 0;
    with_blend_shape(L.footprint, [&](auto fw, auto px) {
      constexpr int FW = decltype(fw)::value, PX = decltype(px)::value;
      if constexpr (PX == 4) {
        // the gather4 staging is built for the four-pixels-a-lane shapes
        if (tma) {
          if (b.evals)
            k_blend_persist<FW, PX, true, false, true><<<grid, 256 / PX, 0, st>>>(b2);
          else if (black)
            k_blend_persist<FW, PX, false, false, true, true><<<grid, 256 / PX, 0, st>>>(b2);
          else
            k_blend_persist<FW, PX, false, false, true><<<grid, 256 / PX, 0, st>>>(b2);
          return;
        }
      }
      if (b.evals)
        k_blend_persist<FW, PX, true><<<grid, 256 / PX, 0, st>>>(b2);
      else if (black)
        k_blend_persist<FW, PX, false, false, false, true><<<grid, 256 / PX, 0, st>>>(b2);
      else
        k_blend_persist<FW, PX, false><<<grid, 256 / PX, 0, st>>>(b2);
    });
  }
  mark(7);
}

__global__ void k_copy_words(WordJobs j) {
  for (int k = 0; k < j.count; ++k)
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < j.n[k];
         i += gridDim.x * blockDim.x)
      j.dst[k][i] = j.src[k][i];
}

void launch_copy_words(const WordJobs &j, cudaStream_t st) {
  k_copy_words<<<4, 256, 0, st>>>(j);
}

bool encode_record_map(BatchDev &b, uint64_t rows) {
  using Encode = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                              const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                              const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  // the driver's encoder, fetched once (no link against the driver library)
  static const Encode enc = []() -> Encode {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                         cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return reinterpret_cast<Encode>(fn);
  }();
  b.rec_map_ok = 0;
  // gather4 row coordinates are 32-bit signed; the base must be 16-byte aligned
  if (!enc || !b.rec || rows == 0 || rows >= (1ull << 31) || ((uintptr_t)b.rec & 15)) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)kRec, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)kRec * sizeof(float)};   // 48 B rows
  const cuuint32_t box[2] = {(cuuint32_t)kRec, 1};                      // one row high
  const cuuint32_t estr[2] = {1, 1};
  if (enc(&b.rec_map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)b.rec, dims, strides, box,
          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  b.rec_map_ok = 1;
  return true;
}

int batch_blend_max_ctas_per_sm(int shape, bool black) {
  int per_sm = 0;
  with_blend_shape(shape, [&](auto fw, auto px) {
    constexpr int FW = decltype(fw)::value, PX = decltype(px)::value;
    if (black)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &per_sm, k_blend_persist<FW, PX, false, false, false, true>, 256 / PX, 0);
    else
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_blend_persist<FW, PX, false>,
                                                    256 / PX, 0);
  });
  return std::max(1, per_sm);
}

}  // namespace fdgs
