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
                           __ldg(&a.qr[i]), __ldg(&a.opacity[i]), g);
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
            gauss_colour(a.cam, a.sh, a.deg, a.n, i, g, rgb);
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
    if (tid == 0) {
      uint32_t tot = 0;
      for (int w = 0; w < kWarps; ++w) {
        const uint32_t c = s_wcnt[w];
        s_wcnt[w] = tot;
        tot += c;
      }
      const uint64_t base = lookback_single(a.status, part, tot, a.err);
      s_base = base;
      if (part == nparts - 1) a.ctr[C_NVIS] = (uint32_t)(base + tot);
    }
    __syncthreads();
    if (vis) a.vis_keys[s_base + s_wcnt[warp] + __popc(vb & lanemask_lt())] = key;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// Records into depth-rank order + exclusive scan of the per-Gaussian tile counts.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock)
k_gather_scan(const uint64_t *__restrict__ sorted, const uint32_t *__restrict__ nv_dev,
              const float *__restrict__ rec, float *__restrict__ rec_sorted,
              uint32_t *__restrict__ offsets, uint64_t *status, uint32_t *ctr, uint32_t *err) {
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
    if (r < nv) {
      const uint32_t id = (uint32_t)sorted[r];
      const float4 *src = reinterpret_cast<const float4 *>(rec + (size_t)id * kRec);
      float4 *dst = reinterpret_cast<float4 *>(rec_sorted + (size_t)r * kRec);
      const float4 a0 = src[0], a1 = src[1], a2 = src[2];
      dst[0] = a0;
      dst[1] = a1;
      dst[2] = a2;
      cnt = (uint32_t)a2.w;
    }
    const uint32_t inc = warp_incl_scan(cnt);
    if (lane == 31) s_wtot[warp] = inc;
    __syncthreads();
    if (tid == 0) {
      uint32_t tot = 0;
      for (int w = 0; w < kWarps; ++w) {
        const uint32_t c = s_wtot[w];
        s_wtot[w] = tot;
        tot += c;
      }
      const uint64_t base = lookback_single(status, part, tot, err);
      s_base = base;
      if (part == nparts - 1) {
        const uint64_t total = base + tot;
        ctr[C_NKEYS_LO] = (uint32_t)total;
        ctr[C_NKEYS_HI] = (uint32_t)(total >> 32);
      }
    }
    __syncthreads();
    if (r < nv) offsets[r] = (uint32_t)(s_base + s_wtot[warp] + inc - cnt);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// Key emission: each warp expands the tile rectangles of 32 consecutive ranks into
// contiguous, coalesced key writes.
// ---------------------------------------------------------------------------------------
template <typename K>
__global__ void __launch_bounds__(kBlock)
k_emit(const float *__restrict__ rec_sorted, const uint32_t *__restrict__ offsets, uint32_t nv,
       int gx, int gy, int rb, K *__restrict__ keys) {
  __shared__ uint32_t s_excl[kWarps][32];
  __shared__ int s_x0[kWarps][32], s_y0[kWarps][32], s_w[kWarps][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t total_warps = gridDim.x * kWarps;
  for (uint32_t chunk = blockIdx.x * kWarps + warp; (uint64_t)chunk * 32 < nv;
       chunk += total_warps) {
    const uint32_t r = chunk * 32 + lane;
    uint32_t cnt = 0;
    int x0 = 0, y0 = 0, w = 1;
    if (r < nv) {
      const float *rp = rec_sorted + (size_t)r * kRec;
      int x1, y1;
      tile_rect(rp[R_U], rp[R_V], rp[R_RADIUS], gx, gy, x0, y0, x1, y1);
      w = x1 - x0;
      cnt = (uint32_t)(w * (y1 - y0));
    }
    const uint32_t inc = warp_incl_scan(cnt);
    const uint32_t total = __shfl_sync(0xffffffffu, inc, 31);
    s_excl[warp][lane] = inc - cnt;
    s_x0[warp][lane] = x0;
    s_y0[warp][lane] = y0;
    s_w[warp][lane] = w;
    const uint32_t base = __shfl_sync(0xffffffffu, r < nv ? offsets[r] - (inc - cnt) : 0u, 0);
    __syncwarp();
    for (uint32_t j = lane; j < total; j += 32) {
      int lo = 0, hi = 31;
      while (lo < hi) {
        const int m = (lo + hi + 1) >> 1;
        if (s_excl[warp][m] <= j) lo = m; else hi = m - 1;
      }
      const uint32_t q = j - s_excl[warp][lo];
      const uint32_t ww = (uint32_t)s_w[warp][lo];
      const uint32_t tx = s_x0[warp][lo] + q % ww;
      const uint32_t ty = s_y0[warp][lo] + q / ww;
      keys[base + j] = ((K)(ty * (uint32_t)gx + tx) << rb) | (K)(chunk * 32 + lo);
    }
    __syncwarp();
  }
}

template <typename K>
__global__ void k_ranges(const K *__restrict__ keys, uint32_t nkeys, int rb,
                         uint2 *__restrict__ ranges) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nkeys;
       i += gridDim.x * blockDim.x) {
    const uint32_t t = (uint32_t)(keys[i] >> rb);
    if (i == 0 || (uint32_t)(keys[i - 1] >> rb) != t) ranges[t].x = i;
    if (i == nkeys - 1 || (uint32_t)(keys[i + 1] >> rb) != t) ranges[t].y = i + 1;
  }
}

// ---------------------------------------------------------------------------------------
// Forward blend: one CTA per 16x16 tile, one thread per pixel. Records are staged in
// shared memory 256 at a time; the CTA leaves as soon as every pixel has stopped.
// ---------------------------------------------------------------------------------------
template <typename K, bool kWeights, bool kCount>
__global__ void __launch_bounds__(kBlock) k_blend(BlendArgs a, const K *__restrict__ keys,
                                                  uint32_t rmask) {
  __shared__ float2 s_xy[kBlock];
  __shared__ float4 s_co[kBlock];
  __shared__ float4 s_rgb[kBlock];
  const int tile = blockIdx.x;
  const int tx = tile % a.gx, ty = tile / a.gx;
  const int tid = threadIdx.x;
  const int px = tx * kTile + (tid & (kTile - 1)), py = ty * kTile + (tid >> 4);
  const bool inside = px < a.W && py < a.H;
  const uint2 range = a.ranges[tile];
  const float fpx = (float)px, fpy = (float)py;
  float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
  uint32_t last = 0, nevals = 0;
  bool done = !inside;
  for (uint32_t start = range.x; start < range.y; start += kBlock) {
    if (__syncthreads_count(done) == kBlock) break;
    const uint32_t idx = start + tid;
    if (idx < range.y) {
      const uint32_t r = (uint32_t)(keys[idx] & (K)rmask);
      const float4 *rp = reinterpret_cast<const float4 *>(a.rec_sorted + (size_t)r * kRec);
      const float4 r0 = rp[0], r1 = rp[1];
      const float r2 = a.rec_sorted[(size_t)r * kRec + 8];
      s_xy[tid] = make_float2(r0.x, r0.y);
      s_co[tid] = make_float4(r0.z, r0.w, r1.x, r1.y);
      s_rgb[tid] = make_float4(r1.z, r1.w, r2, __uint_as_float(r));
    }
    __syncthreads();
    const int nb = (int)min((uint32_t)kBlock, range.y - start);
    for (int j = 0; j < nb; ++j) {
      float wgt = 0.f;
      if (!done) {
        const float2 xy = s_xy[j];
        const float4 co = s_co[j];
        float alpha, G, dx, dy;
        if (kCount) ++nevals;
        if (eval_alpha(xy.x, xy.y, co.x, co.y, co.z, co.w, fpx, fpy, alpha, G, dx, dy)) {
          const float nT = T * (1.f - alpha);
          if (nT < kTStop) {
            done = true;
          } else {
            const float4 c = s_rgb[j];
            wgt = alpha * T;
            C0 = fmaf(c.x, wgt, C0);
            C1 = fmaf(c.y, wgt, C1);
            C2 = fmaf(c.z, wgt, C2);
            T = nT;
            last = start - range.x + j + 1;
          }
        }
      }
      if (kWeights) {
        if (__any_sync(0xffffffffu, wgt != 0.f)) {
          const float s = warp_sum(wgt);
          if ((tid & 31) == 0) atomicAdd(&a.w_sum[__float_as_uint(s_rgb[j].w)], s);
        }
      } else if (done) {
        break;
      }
    }
  }
  if (kCount) {
    const uint32_t ws = warp_sum(nevals);
    if ((tid & 31) == 0 && ws) atomicAdd(a.evals, (unsigned long long)ws);
  }
  if (inside) {
    const size_t pix = (size_t)py * a.W + px, hw = (size_t)a.W * a.H;
    a.rgb[pix] = C0 + T * a.bg[0];
    a.rgb[hw + pix] = C1 + T * a.bg[1];
    a.rgb[2 * hw + pix] = C2 + T * a.bg[2];
    a.T_final[pix] = T;
    a.n_contrib[pix] = last;
  }
}

// ---------------------------------------------------------------------------------------
// Backward blend: reverse replay of each tile list from the largest n_contrib down to 0.
// Transmittance is recovered as T_i = T_{i+1} / (1 - alpha_i) from T_final.
// ---------------------------------------------------------------------------------------
template <typename K>
__global__ void __launch_bounds__(kBlock) k_blend_bwd(BlendBwdArgs a, const K *__restrict__ keys,
                                                      uint32_t rmask) {
  __shared__ float2 s_xy[kBlock];
  __shared__ float4 s_co[kBlock];
  __shared__ float4 s_rgb[kBlock];
  __shared__ uint32_t s_max;
  const int tile = blockIdx.x;
  const int tx = tile % a.gx, ty = tile / a.gx;
  const int tid = threadIdx.x, lane = tid & 31;
  const int px = tx * kTile + (tid & (kTile - 1)), py = ty * kTile + (tid >> 4);
  const bool inside = px < a.W && py < a.H;
  const uint2 range = a.ranges[tile];
  const size_t pix = (size_t)py * a.W + px, hw = (size_t)a.W * a.H;
  if (tid == 0) s_max = 0;
  __syncthreads();
  uint32_t nc = 0;
  float T = 1.f, dL0 = 0.f, dL1 = 0.f, dL2 = 0.f;
  if (inside) {
    nc = a.n_contrib[pix];
    T = a.T_final[pix];
    dL0 = a.dL_drgb[pix];
    dL1 = a.dL_drgb[hw + pix];
    dL2 = a.dL_drgb[2 * hw + pix];
    atomicMax(&s_max, nc);
  }
  const float Tf = T;
  const float bg_dot = a.bg[0] * dL0 + a.bg[1] * dL1 + a.bg[2] * dL2;
  float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, last_a = 0.f, lc0 = 0.f, lc1 = 0.f, lc2 = 0.f;
  const float fpx = (float)px, fpy = (float)py;
  __syncthreads();
  const int maxnc = (int)s_max;
  for (int bend = maxnc; bend > 0; bend -= kBlock) {
    const int bstart = max(0, bend - kBlock);
    __syncthreads();
    if (bstart + tid < bend) {
      const uint32_t r = (uint32_t)(keys[range.x + bstart + tid] & (K)rmask);
      const float4 *rp = reinterpret_cast<const float4 *>(a.rec_sorted + (size_t)r * kRec);
      const float4 r0 = rp[0], r1 = rp[1];
      const float r2 = a.rec_sorted[(size_t)r * kRec + 8];
      s_xy[tid] = make_float2(r0.x, r0.y);
      s_co[tid] = make_float4(r0.z, r0.w, r1.x, r1.y);
      s_rgb[tid] = make_float4(r1.z, r1.w, r2, __uint_as_float(r));
    }
    __syncthreads();
    for (int jj = bend - bstart - 1; jj >= 0; --jj) {
      const int pos = bstart + jj;
      float g[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      bool contrib = false;
      if ((uint32_t)pos < nc) {
        const float2 xy = s_xy[jj];
        const float4 co = s_co[jj];
        float alpha, G, dx, dy;
        if (eval_alpha(xy.x, xy.y, co.x, co.y, co.z, co.w, fpx, fpy, alpha, G, dx, dy)) {
          contrib = true;
          const float4 c = s_rgb[jj];
          const float om = 1.f - alpha;
          T = T / om;
          const float wgt = alpha * T;
          acc0 = last_a * lc0 + (1.f - last_a) * acc0;
          acc1 = last_a * lc1 + (1.f - last_a) * acc1;
          acc2 = last_a * lc2 + (1.f - last_a) * acc2;
          float dLda = (c.x - acc0) * dL0 + (c.y - acc1) * dL1 + (c.z - acc2) * dL2;
          dLda = dLda * T - Tf / om * bg_dot;
          g[6] = wgt * dL0;
          g[7] = wgt * dL1;
          g[8] = wgt * dL2;
          last_a = alpha;
          lc0 = c.x; lc1 = c.y; lc2 = c.z;
          if (__fmul_rn(co.w, G) < kAlphaMax) {
            g[5] = G * dLda;
            const float gp = alpha * dLda;
            g[0] = gp * (-co.x * dx - co.y * dy);
            g[1] = gp * (-co.z * dy - co.y * dx);
            g[2] = gp * (-0.5f * dx * dx);
            g[3] = gp * (-dx * dy);
            g[4] = gp * (-0.5f * dy * dy);
          }
        }
      }
      if (__any_sync(0xffffffffu, contrib)) {
#pragma unroll
        for (int f = 0; f < 9; ++f) g[f] = warp_sum(g[f]);
        if (lane == 0) {
          float *dst = a.g2d + (size_t)__float_as_uint(s_rgb[jj].w) * 9;
#pragma unroll
          for (int f = 0; f < 9; ++f)
            if (g[f] != 0.f) atomicAdd(&dst[f], g[f]);
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
    gauss_colour(a.cam, a.sh, a.deg, a.n, i, g, rgb);
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
  if (!grid_cap) grid_cap = persistent_grid(k_preprocess, ~0ull);
  k_preprocess<<<(int)std::min<uint64_t>(parts, grid_cap), kBlock, 0, st>>>(a);
}

void launch_gather_scan(const uint64_t *sorted, const uint32_t *ctr_nvis, uint32_t n_cap,
                        const float *rec, float *rec_sorted, uint32_t *offsets,
                        uint64_t *status, uint32_t *ctr, uint32_t *err, cudaStream_t st) {
  if (n_cap == 0) return;
  const uint64_t parts = (n_cap + kBlock - 1) / kBlock;
  static int grid_cap = 0;
  if (!grid_cap) grid_cap = persistent_grid(k_gather_scan, ~0ull);
  k_gather_scan<<<(int)std::min<uint64_t>(parts, grid_cap), kBlock, 0, st>>>(
      sorted, ctr_nvis, rec, rec_sorted, offsets, status, ctr, err);
}

template <typename K>
void launch_emit(const float *rec_sorted, const uint32_t *offsets, uint32_t nv, int gx, int gy,
                 int rb, K *keys, cudaStream_t st) {
  if (nv == 0) return;
  const uint64_t chunks = (nv + 31) / 32;
  const int grid = (int)std::min<uint64_t>((chunks + kWarps - 1) / kWarps,
                                           (uint64_t)num_sms() * 8);
  k_emit<K><<<grid, kBlock, 0, st>>>(rec_sorted, offsets, nv, gx, gy, rb, keys);
}

template <typename K>
void launch_ranges(const K *keys, uint32_t nkeys, int rb, uint2 *ranges, cudaStream_t st) {
  if (nkeys == 0) return;
  const int grid = (int)std::min<uint64_t>((nkeys + kBlock - 1) / kBlock,
                                           (uint64_t)num_sms() * 16);
  k_ranges<K><<<grid, kBlock, 0, st>>>(keys, nkeys, rb, ranges);
}

template <typename K>
void launch_blend(const BlendArgs &a, const K *keys, uint32_t rmask, cudaStream_t st) {
  const int tiles = a.gx * a.gy;
  if (tiles == 0) return;
  if (a.w_sum)
    k_blend<K, true, false><<<tiles, kBlock, 0, st>>>(a, keys, rmask);
  else if (a.evals)
    k_blend<K, false, true><<<tiles, kBlock, 0, st>>>(a, keys, rmask);
  else
    k_blend<K, false, false><<<tiles, kBlock, 0, st>>>(a, keys, rmask);
}

template <typename K>
void launch_blend_bwd(const BlendBwdArgs &a, const K *keys, uint32_t rmask, cudaStream_t st) {
  const int tiles = a.gx * a.gy;
  if (tiles == 0) return;
  k_blend_bwd<K><<<tiles, kBlock, 0, st>>>(a, keys, rmask);
}

void launch_preprocess_bwd(const PreBwdArgs &a, cudaStream_t st) {
  if (a.nv == 0) return;
  const int grid = (int)std::min<uint64_t>((a.nv + 127) / 128, (uint64_t)num_sms() * 8);
  k_preprocess_bwd<<<grid, 128, 0, st>>>(a);
}

#define FDGS_INST(K)                                                                      \
  template void launch_emit<K>(const float *, const uint32_t *, uint32_t, int, int, int, K *, \
                               cudaStream_t);                                             \
  template void launch_ranges<K>(const K *, uint32_t, int, uint2 *, cudaStream_t);        \
  template void launch_blend<K>(const BlendArgs &, const K *, uint32_t, cudaStream_t);    \
  template void launch_blend_bwd<K>(const BlendBwdArgs &, const K *, uint32_t, cudaStream_t);
FDGS_INST(uint32_t)
FDGS_INST(uint64_t)
#undef FDGS_INST

}  // namespace fdgs
