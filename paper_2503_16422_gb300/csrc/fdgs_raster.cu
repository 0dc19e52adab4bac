// Rasterizer kernels of the GB300 masked 4D Gaussian splatting path.
//
// Frame pipeline (all on one stream, counts stay on the device):
//   k_preprocess   per Gaussian: key-frame mask gate (Sec. 4.2.2), slice (Eq. 1, Eq. 3),
//                  temporal cull, EWA projection, tile rectangle, SH colour; writes the
//                  48-byte record by id and compacts the visible ones as
//                  (depth bits << 32 | id) keys with a chained scan (decoupled look-back).
//   radix sort     visible keys by depth (fdgs_sort.cu) -> depth rank order.
//   k_gather_scan  records into rank order + exclusive scan of tile counts (key offsets).
//   k_emit         one key (tile << rank_bits | rank) per covered tile, warp-cooperative.
//   radix sort     keys by tile bits only (stable) -> per-tile lists in (depth, id) order.
//   k_ranges       [start, end) of each tile's list.
//   k_blend        per 16x16 tile: front-to-back compositing (Eq. 2) with early stop.
// Reverse: k_blend_bwd (reverse replay per tile) and k_preprocess_bwd (chain to 4D params).
#include <algorithm>

#include "fdgs_gauss.cuh"
#include "fdgs_internal.h"

namespace fdgs {

int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

namespace {

constexpr int kBlock = 256;
constexpr int kWarps = kBlock / 32;

template <typename F>
int persistent_grid(F kernel, uint64_t parts) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, 0);
  uint64_t g = (uint64_t)std::max(1, per_sm) * num_sms();
  return (int)std::max<uint64_t>(1, std::min<uint64_t>(g, parts));
}

// ---------------------------------------------------------------------------------------
// Per-Gaussian stage with fused compaction of the visible Gaussians.
// ---------------------------------------------------------------------------------------
template <bool kVQ>
__global__ void __launch_bounds__(kBlock) k_preprocess(PreArgs a) {
  __shared__ uint32_t s_part;
  __shared__ uint32_t s_wcnt[kWarps];
  __shared__ uint64_t s_base;
  const uint32_t nparts = (a.n + kBlock - 1) / kBlock;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (;;) {
    if (tid == 0) s_part = atomicAdd(&a.ctr[C_PART0], 1u);
    __syncthreads();
    const uint32_t part = s_part;
    if (part >= nparts) break;
    const uint32_t i = part * kBlock + tid;
    bool active = false, vis = false;
    uint64_t key = 0;
    if (i < a.n) {
      active = true;
      if (a.mask_l) {
        const uint32_t w = __ldg(&a.mask_l[i >> 5]) | __ldg(&a.mask_r[i >> 5]);
        active = (w >> (i & 31)) & 1u;
      }
      uint8_t fl = 0;
      if (active) {
        GaussState g;
        fl = gauss_forward(a.cam, a.t, __ldg(&a.mean4[i]), __ldg(&a.ls4[i]), __ldg(&a.ql[i]),
                           __ldg(&a.qr[i]), __ldg(&a.opacity[i]), g, !a.no_cull);
        if (fl & kFlagDet) {
          const float half = 0.5f * (g.c00 - g.c11);
          const float disc = half * half + g.c01 * g.c01;
          const float mid = 0.5f * (g.c00 + g.c11);
          const float lam = mid + sqrtf(fmaxf(kRadiusFloor, disc));
          const float r = ceilf(3.f * sqrtf(lam));
          const float u = fmaf(a.cam.fx, g.xr, a.cam.cx);
          const float v = fmaf(a.cam.fy, g.yr, a.cam.cy);
          int x0, y0, x1, y1;
          tile_rect(u, v, r, a.cam.gx, a.cam.gy, x0, y0, x1, y1);
          if (x1 > x0 && y1 > y0) {
            vis = true;
            fl |= kFlagVisible;
            float rgb[3];
            gauss_colour<kVQ>(a.cam, a.sh, a.sh_cb, a.sh_code, a.deg, a.n, i, g, rgb);
            const float idet = 1.f / g.det;
            float4 *rp = reinterpret_cast<float4 *>(a.rec + (size_t)i * kRec);
            rp[0] = make_float4(u, v, g.c11 * idet, -g.c01 * idet);
            rp[1] = make_float4(g.c00 * idet, g.a, rgb[0], rgb[1]);
            rp[2] = make_float4(rgb[2], g.xc[2], r, (float)((x1 - x0) * (y1 - y0)));
            key = ((uint64_t)__float_as_uint(g.xc[2]) << 32) | (uint64_t)i;
          }
        }
      }
      if (a.flags) a.flags[i] = fl;
    }
    const uint32_t vb = __ballot_sync(0xffffffffu, vis);
    const uint32_t ab = __ballot_sync(0xffffffffu, active);
    if (lane == 0) {
      s_wcnt[warp] = __popc(vb);
      if (ab) atomicAdd(&a.ctr[C_NACTIVE], (uint32_t)__popc(ab));
    }
    __syncthreads();
    if (warp == 0) {
      uint32_t tot = 0;
      if (lane == 0)
        for (int w = 0; w < kWarps; ++w) {
          const uint32_t c = s_wcnt[w];
          s_wcnt[w] = tot;
          tot += c;
        }
      tot = __shfl_sync(0xffffffffu, tot, 0);
      const uint64_t base = lookback_warp(a.status, part, tot, a.err);
      if (lane == 0) {
        s_base = base;
        if (part == nparts - 1) a.ctr[C_NVIS] = (uint32_t)(base + tot);
      }
    }
    __syncthreads();
    if (vis) a.vis_keys[s_base + s_wcnt[warp] + __popc(vb & lanemask_lt())] = key;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// Records into depth-rank order (blend-ready form) + exclusive scan of the per-Gaussian
// tile counts (key offsets) + per-tile coverage counts as a 2D difference array (four
// atomics per Gaussian; k_tile_scan integrates it).
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock, 4)
k_gather_scan(const uint64_t *__restrict__ sorted, const uint32_t *__restrict__ nv_dev,
              const float *__restrict__ rec, float *__restrict__ rec_sorted,
              uint32_t *__restrict__ offsets, uint64_t *status, uint32_t *ctr, uint32_t *err,
              int gx, int gy, int *__restrict__ diff, uint32_t *__restrict__ rowmask,
              uint32_t *__restrict__ colmask, uint32_t mask_words, int tight) {
  __shared__ uint32_t s_part;
  __shared__ uint32_t s_wtot[kWarps];
  __shared__ uint64_t s_base;
  const uint32_t nv = *nv_dev;
  const uint32_t nparts = (nv + kBlock - 1) / kBlock;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (;;) {
    if (tid == 0) s_part = atomicAdd(&ctr[C_PART0 + 1], 1u);
    __syncthreads();
    const uint32_t part = s_part;
    if (part >= nparts) break;
    const uint32_t r = part * kBlock + tid;
    uint32_t cnt = 0;
    int x0 = 0, y0 = 0, x1 = 0, y1 = 0;
    if (r < nv) {
      const uint32_t id = (uint32_t)sorted[r];
      const float4 *src = reinterpret_cast<const float4 *>(rec + (size_t)id * kRec);
      float4 *dst = reinterpret_cast<float4 *>(rec_sorted + (size_t)r * kRecS);
      const float4 a0 = src[0], a1 = src[1], a2 = src[2];
      // a0 = (u, v, A, B), a1 = (C, a, r, g), a2 = (b, depth, radius, count)
      const float qa = -0.5f * kLog2e * a0.z, qb = -kLog2e * a0.w, qc = -0.5f * kLog2e * a1.x;
      dst[0] = make_float4(a0.x, a0.y, qa, qb);
      dst[1] = make_float4(qc, log2f(a1.y), a1.z, a1.w);
      dst[2] = make_float4(a2.x, -qb / (2.f * qa), -qb / (2.f * qc), a2.z);
      dst[3] = make_float4(a0.z, a0.w, a1.x, a1.y);
      tile_rect(a0.x, a0.y, a2.z, gx, gy, x0, y0, x1, y1);
      if (tight) tighten_rect(a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, x0, y0, x1, y1);
      if (x1 > x0 && y1 > y0) {
        cnt = (uint32_t)((x1 - x0) * (y1 - y0));
        const int W1 = gx + 1;
        atomicAdd(&diff[y0 * W1 + x0], 1);
        atomicAdd(&diff[y0 * W1 + x1], -1);
        atomicAdd(&diff[y1 * W1 + x0], -1);
        atomicAdd(&diff[y1 * W1 + x1], 1);
      } else {
        x0 = y0 = x1 = y1 = 0;
      }
    }
    if (rowmask) {
      // coverage bitmasks by depth rank: bit (r & 31) of word r / 32 of tile row y / column x
      // is set iff the Gaussian of rank r covers that row / column. Each warp owns one word.
      const uint32_t word = r >> 5;
      warp_coverage_words(y0, y1, gy, rowmask + word, mask_words);
      warp_coverage_words(x0, x1, gx, colmask + word, mask_words);
    }
    const uint32_t inc = warp_incl_scan(cnt);
    if (lane == 31) s_wtot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      uint32_t tot = 0;
      if (lane == 0)
        for (int w = 0; w < kWarps; ++w) {
          const uint32_t c = s_wtot[w];
          s_wtot[w] = tot;
          tot += c;
        }
      tot = __shfl_sync(0xffffffffu, tot, 0);
      const uint64_t base = lookback_warp(status, part, tot, err);
      if (lane == 0) {
        s_base = base;
        if (part == nparts - 1) {
          const uint64_t total = base + tot;
          ctr[C_NKEYS_LO] = (uint32_t)total;
          ctr[C_NKEYS_HI] = (uint32_t)(total >> 32);
        }
      }
    }
    __syncthreads();
    if (r < nv) offsets[r] = (uint32_t)(s_base + s_wtot[warp] + inc - cnt);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// Per-tile coverage counts from the difference array -> tile ranges [start, end) and the
// exclusive digit offsets of each pass of the tile sort (so the sort skips its histogram).
// One CTA; diff is [gy + 1][gx + 1] and is integrated in place.
// ---------------------------------------------------------------------------------------
constexpr int kScanBlock = 1024;
// Length buckets of the blend's longest-first tile order: 16 list entries each, two per
// scan thread; lists of 32752 entries or more share the first bucket.
constexpr int kOrderBuckets = 2 * kScanBlock;
__device__ __forceinline__ uint32_t order_bucket(uint32_t len) {
  return (uint32_t)(kOrderBuckets - 1) - min(len >> 4, (uint32_t)(kOrderBuckets - 1));
}
__global__ void __launch_bounds__(kScanBlock)
k_tile_scan(int *__restrict__ diff, int gx, int gy, int npass, int dbits, uint2 *ranges,
            uint32_t *__restrict__ hist, uint32_t *__restrict__ order, uint64_t cap,
            unsigned long long *need, uint32_t *err) {
  __shared__ uint32_t s_hist[4 * 256];
  __shared__ uint32_t s_ord[kOrderBuckets];
  __shared__ uint32_t s_wsum[kScanBlock / 32];
  __shared__ uint32_t s_carry;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int W1 = gx + 1;
  for (int i = tid; i < 4 * 256; i += kScanBlock) s_hist[i] = 0;
  for (int i = tid; i < kOrderBuckets; i += kScanBlock) s_ord[i] = 0;
  // rows: prefix along x (one warp per row)
  for (int y = warp; y < gy; y += kScanBlock / 32) {
    int carry = 0;
    for (int x0 = 0; x0 < gx; x0 += 32) {
      const int x = x0 + lane;
      int v = x < gx ? diff[y * W1 + x] : 0;
      v = warp_incl_scan(v) + carry;
      if (x < gx) diff[y * W1 + x] = v;
      carry = __shfl_sync(0xffffffffu, v, 31);
    }
  }
  __syncthreads();
  // columns: prefix along y (one thread per column)
  for (int x = tid; x < gx; x += kScanBlock) {
    int acc = 0;
    for (int y = 0; y < gy; ++y) {
      acc += diff[y * W1 + x];
      diff[y * W1 + x] = acc;
    }
  }
  __syncthreads();
  // exclusive scan over tiles in id order (ty * gx + tx), chunked by the block
  const uint32_t tiles = (uint32_t)gx * gy;
  const uint32_t mask = (1u << dbits) - 1u;
  if (tid == 0) s_carry = 0;
  __syncthreads();
  for (uint32_t t0 = 0; t0 < tiles; t0 += kScanBlock) {
    const uint32_t t = t0 + tid;
    uint32_t c = 0;
    if (t < tiles) c = (uint32_t)diff[(t / gx) * W1 + (t % gx)];
    const uint32_t inc = warp_incl_scan(c);
    if (lane == 31) s_wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      const uint32_t w = s_wsum[lane];
      const uint32_t wi = warp_incl_scan(w);
      s_wsum[lane] = wi - w;
    }
    __syncthreads();
    const uint32_t start = s_carry + s_wsum[warp] + inc - c;
    if (t < tiles) {
      ranges[t] = make_uint2(start, start + c);
      if (order) atomicAdd(&s_ord[order_bucket(c)], 1u);
      for (int p = 0; p < npass; ++p)
        if (c) atomicAdd(&s_hist[p * 256 + ((t >> (p * dbits)) & mask)], c);
    }
    __syncthreads();
    if (tid == kScanBlock - 1) s_carry = start + c;
    __syncthreads();
  }
  // a list capacity fixed before the launch (renders sized without a host synchronisation):
  // when the lists do not fit, every range is emptied (nothing is written or read beyond the
  // capacity, the frame composites no Gaussian) and the length needed is recorded
  if (cap && (uint64_t)s_carry > cap) {
    if (tid == 0) {
      atomicOr(err, kErrCapacity);
      atomicMax(need, (unsigned long long)s_carry);
    }
    for (uint32_t t = tid; t < tiles; t += kScanBlock) ranges[t] = make_uint2(0u, 0u);
    // the length buckets of the tile order were counted with the lengths before: now every
    // tile is in the bucket of empty lists (else the order's slots would run past its end)
    for (int i = tid; i < kOrderBuckets; i += kScanBlock)
      s_ord[i] = i == kOrderBuckets - 1 ? tiles : 0u;
    __syncthreads();
  }
  // exclusive digit offsets per pass (threads 0..255 = warps 0..7 hold the 256 digits)
  for (int p = 0; p < npass; ++p) {
    uint32_t v = 0, inc = 0;
    if (tid < 256) {
      v = s_hist[p * 256 + tid];
      inc = warp_incl_scan(v);
      if (lane == 31) s_wsum[warp] = inc;
    }
    __syncthreads();
    if (tid < 256) {
      uint32_t wo = 0;
      for (int w = 0; w < warp; ++w) wo += s_wsum[w];
      hist[p * 256 + tid] = wo + inc - v;
    }
    __syncthreads();
  }
  if (order) {
    // longest lists first: exclusive scan of the length buckets (two a thread), then every
    // tile takes a slot of its bucket (the ranges written above are visible to the block)
    const uint32_t h0 = s_ord[2 * tid], h1 = s_ord[2 * tid + 1];
    const uint32_t inc = warp_incl_scan(h0 + h1);
    if (lane == 31) s_wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      const uint32_t w = s_wsum[lane];
      s_wsum[lane] = warp_incl_scan(w) - w;
    }
    __syncthreads();
    const uint32_t ex = s_wsum[warp] + inc - (h0 + h1);
    s_ord[2 * tid] = ex;
    s_ord[2 * tid + 1] = ex + h0;
    __syncthreads();
    for (uint32_t t = tid; t < tiles; t += kScanBlock) {
      const uint2 rg = ranges[t];
      order[atomicAdd(&s_ord[order_bucket(rg.y - rg.x)], 1u)] = t;
    }
  }
}

// ---------------------------------------------------------------------------------------
// Key emission: a warp takes 32 consecutive ranks and writes their keys one Gaussian at a
// time, the 32 lanes walking the tile rectangle in row-major order (consecutive addresses,
// one integer division per Gaussian and lane).
// ---------------------------------------------------------------------------------------
// Tile lists without a sort (dense coverage): the list of tile (tx, ty) is the set bits of
// rowmask[ty] AND colmask[tx], i.e. the ranks of the Gaussians whose rectangle covers the
// tile, already in depth order. One warp per tile writes them from ranges[tile].x on.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock)
k_tile_lists(const uint32_t *__restrict__ rowmask, const uint32_t *__restrict__ colmask,
             uint32_t mask_words, uint32_t words, const uint32_t *__restrict__ nv_dev,
             int gx, int gy, const uint2 *__restrict__ ranges, uint32_t *__restrict__ lists) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t tiles = (uint32_t)gx * gy;
  // the visible count from the device when the host did not read it
  if (nv_dev) words = (*nv_dev + 31) / 32;
  for (uint32_t t = blockIdx.x * kWarps + warp; t < tiles; t += gridDim.x * kWarps) {
    const uint32_t *rows = rowmask + (size_t)(t / gx) * mask_words;
    const uint32_t *cols = colmask + (size_t)(t % gx) * mask_words;
    // one word per lane per step: a frame has one wave of tile warps, so the shorter steps
    // (and lower register count) win here; the batched builder reads four words per lane
    const uint2 rg = ranges[t];
    if (rg.y == rg.x) continue;   // no entries (or ranges emptied by a capacity overflow)
    uint32_t off = rg.x;
    // the words of group g+2 are loading while group g is written out
    uint32_t nr0 = lane < words ? __ldg(&rows[lane]) : 0u;
    uint32_t nc0 = lane < words ? __ldg(&cols[lane]) : 0u;
    uint32_t nr1 = lane + 32 < words ? __ldg(&rows[lane + 32]) : 0u;
    uint32_t nc1 = lane + 32 < words ? __ldg(&cols[lane + 32]) : 0u;
    for (uint32_t c0 = 0; c0 < words; c0 += 32) {
      const uint32_t c = c0 + lane;
      uint32_t m = nr0 & nc0;
      nr0 = nr1;
      nc0 = nc1;
      nr1 = c + 64 < words ? __ldg(&rows[c + 64]) : 0u;
      nc1 = c + 64 < words ? __ldg(&cols[c + 64]) : 0u;
      const uint32_t pc = __popc(m);
      const uint32_t inc = warp_incl_scan(pc);
      uint32_t o = off + inc - pc;
      while (m) {
        const int b = __ffs(m) - 1;
        m &= m - 1;
        lists[o++] = c * 32 + b;
      }
      off += __shfl_sync(0xffffffffu, inc, 31);
    }
  }
}

// ---------------------------------------------------------------------------------------
template <typename K>
__global__ void __launch_bounds__(kBlock)
k_emit(const float *__restrict__ rec_sorted, const uint32_t *__restrict__ offsets, uint32_t nv,
       int gx, int gy, int rb, int tight, K *__restrict__ keys) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t total_warps = gridDim.x * kWarps;
  for (uint32_t chunk = blockIdx.x * kWarps + warp; (uint64_t)chunk * 32 < nv;
       chunk += total_warps) {
    const uint32_t r = chunk * 32 + lane;
    int x0 = 0, y0 = 0, w = 1;
    uint32_t cnt = 0, off = 0;
    if (r < nv) {
      const float4 g0 = *reinterpret_cast<const float4 *>(rec_sorted + (size_t)r * kRecS);
      const float rad = rec_sorted[(size_t)r * kRecS + kRecSRadius];
      int x1, y1;
      tile_rect(g0.x, g0.y, rad, gx, gy, x0, y0, x1, y1);
      if (tight) {
        const float4 g3 = *reinterpret_cast<const float4 *>(rec_sorted + (size_t)r * kRecS + 12);
        tighten_rect(g0.x, g0.y, g3.x, g3.y, g3.z, g3.w, x0, y0, x1, y1);
      }
      if (x1 > x0 && y1 > y0) {
        w = x1 - x0;
        cnt = (uint32_t)(w * (y1 - y0));
      } else {
        x0 = y0 = 0;
        w = 1;
        cnt = 0;
      }
      off = offsets[r];
    }
    const uint32_t nlanes = min(32u, nv - chunk * 32);
    for (uint32_t g = 0; g < nlanes; ++g) {
      const uint32_t gc = __shfl_sync(0xffffffffu, cnt, g);
      const int gw = __shfl_sync(0xffffffffu, w, g);
      const int gx0 = __shfl_sync(0xffffffffu, x0, g);
      const int gy0 = __shfl_sync(0xffffffffu, y0, g);
      const uint32_t goff = __shfl_sync(0xffffffffu, off, g);
      const K rank = (K)(chunk * 32 + g);
      int row = lane / gw, col = lane - row * gw;
      const int srow = 32 / gw, scol = 32 - srow * gw;
      for (uint32_t j = lane; j < gc; j += 32) {
        keys[goff + j] = ((K)((uint32_t)(gy0 + row) * (uint32_t)gx + (uint32_t)(gx0 + col)) << rb) | rank;
        col += scol;
        row += srow;
        if (col >= gw) {
          col -= gw;
          ++row;
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// Per-Gaussian reverse: recompute the forward of each visible Gaussian and chain the
// gradients of its 2D record back to the 4D parameters (gradients are added in place).
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_preprocess_bwd(PreBwdArgs a) {
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < a.nv;
       r += gridDim.x * blockDim.x) {
    const uint32_t i = (uint32_t)a.sorted[r];
    const float *g2 = a.g2d + (size_t)r * 9;
    float gg[9];
    bool any = false;
#pragma unroll
    for (int f = 0; f < 9; ++f) {
      gg[f] = g2[f];
      any |= gg[f] != 0.f;
    }
    if (!any) continue;
    GaussState g;
    const uint8_t fl = gauss_forward(a.cam, a.t, __ldg(&a.mean4[i]), __ldg(&a.ls4[i]),
                                     __ldg(&a.ql[i]), __ldg(&a.qr[i]), __ldg(&a.opacity[i]), g);
    if (!(fl & kFlagDet)) continue;
    float rgb[3];
    gauss_colour<false>(a.cam, a.sh, nullptr, nullptr, a.deg, a.n, i, g, rgb);
    GaussGrad out;
    const float grgb[3] = {gg[6], gg[7], gg[8]};
    gauss_backward(a.cam, a.sh, a.deg, a.n, i, g, gg[0], gg[1], gg[2], gg[3], gg[4], gg[5],
                   grgb, out, a.g_sh);
    if (a.g_mean4)
      for (int k = 0; k < 4; ++k) a.g_mean4[(size_t)i * 4 + k] += out.mean[k];
    if (a.g_ls4)
      for (int k = 0; k < 4; ++k) a.g_ls4[(size_t)i * 4 + k] += out.ls[k];
    if (a.g_ql)
      for (int k = 0; k < 4; ++k) a.g_ql[(size_t)i * 4 + k] += out.ql[k];
    if (a.g_qr)
      for (int k = 0; k < 4; ++k) a.g_qr[(size_t)i * 4 + k] += out.qr[k];
    if (a.g_op) a.g_op[i] += out.o;
  }
}

}  // namespace

// ---- launchers ------------------------------------------------------------------------

void launch_preprocess(const PreArgs &a, cudaStream_t st) {
  if (a.n == 0) return;
  const uint64_t parts = (a.n + kBlock - 1) / kBlock;
  static int grid_cap = 0;
  if (!grid_cap) grid_cap = persistent_grid(k_preprocess<false>, ~0ull);
  if (a.sh_cb)
    k_preprocess<true><<<(int)std::min<uint64_t>(parts, grid_cap), kBlock, 0, st>>>(a);
  else
    k_preprocess<false><<<(int)std::min<uint64_t>(parts, grid_cap), kBlock, 0, st>>>(a);
}

void launch_gather_scan(const uint64_t *sorted, const uint32_t *ctr_nvis, uint32_t n_cap,
                        const float *rec, float *rec_sorted, uint32_t *offsets,
                        uint64_t *status, uint32_t *ctr, uint32_t *err, int gx, int gy,
                        int *diff, uint32_t *rowmask, uint32_t *colmask, uint32_t mask_words,
                        int tight, cudaStream_t st) {
  if (n_cap == 0) return;
  const uint64_t parts = (n_cap + kBlock - 1) / kBlock;
  static int grid_cap = 0;
  if (!grid_cap) grid_cap = persistent_grid(k_gather_scan, ~0ull);
  k_gather_scan<<<(int)std::min<uint64_t>(parts, grid_cap), kBlock, 0, st>>>(
      sorted, ctr_nvis, rec, rec_sorted, offsets, status, ctr, err, gx, gy, diff, rowmask,
      colmask, mask_words, tight);
}

void launch_tile_scan(int *diff, int gx, int gy, int npass, int dbits, uint2 *ranges,
                      uint32_t *hist, uint32_t *order, cudaStream_t st, uint64_t cap,
                      unsigned long long *need, uint32_t *err) {
  k_tile_scan<<<1, kScanBlock, 0, st>>>(diff, gx, gy, npass, dbits, ranges, hist, order, cap,
                                        need, err);
}

void launch_tile_lists(const uint32_t *rowmask, const uint32_t *colmask, uint32_t mask_words,
                       uint32_t nv, int gx, int gy, const uint2 *ranges, uint32_t *lists,
                       cudaStream_t st, const uint32_t *nv_dev) {
  const uint64_t tiles = (uint64_t)gx * gy;
  if (tiles == 0 || (nv == 0 && !nv_dev)) return;
  const int grid = (int)std::min<uint64_t>((tiles + kWarps - 1) / kWarps,
                                           (uint64_t)num_sms() * 8);
  k_tile_lists<<<grid, kBlock, 0, st>>>(rowmask, colmask, mask_words, (nv + 31) / 32, nv_dev,
                                        gx, gy, ranges, lists);
}

template <typename K>
void launch_emit(const float *rec_sorted, const uint32_t *offsets, uint32_t nv, int gx, int gy,
                 int rb, int tight, K *keys, cudaStream_t st) {
  if (nv == 0) return;
  const uint64_t chunks = (nv + 31) / 32;
  const int grid = (int)std::min<uint64_t>((chunks + kWarps - 1) / kWarps,
                                           (uint64_t)num_sms() * 8);
  k_emit<K><<<grid, kBlock, 0, st>>>(rec_sorted, offsets, nv, gx, gy, rb, tight, keys);
}

void launch_preprocess_bwd(const PreBwdArgs &a, cudaStream_t st) {
  if (a.nv == 0) return;
  const int grid = (int)std::min<uint64_t>((a.nv + 127) / 128, (uint64_t)num_sms() * 8);
  k_preprocess_bwd<<<grid, 128, 0, st>>>(a);
}

template void launch_emit<uint32_t>(const float *, const uint32_t *, uint32_t, int, int, int,
                                    int, uint32_t *, cudaStream_t);
template void launch_emit<uint64_t>(const float *, const uint32_t *, uint32_t, int, int, int,
                                    int, uint64_t *, cudaStream_t);

}  // namespace fdgs
