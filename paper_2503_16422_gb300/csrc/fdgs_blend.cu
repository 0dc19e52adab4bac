// Per-tile front-to-back compositing (Eq. 2 with Eq. 3's alpha) and its reverse replay.
//
// One CTA of 256 threads per 16x16 tile; each warp owns an FW x (32/FW) pixel footprint of
// the tile, one pixel per lane. The tile's records are staged 256 at a time with cp.async
// into a double buffer (the copy of batch b+1 is in flight while batch b is composited; the
// keys of batch b+2 are already loading into registers).
//
// Warp-ballot culling: the 32 lanes of a warp each test one of 32 staged Gaussians against
// the warp's footprint rectangle (the largest exponent over the rectangle, exact for the
// concave quadratic, minus a margin) and __ballot_sync the hits; the warp then evaluates only
// those Gaussians, one at a time, for its 32 pixels. A culled Gaussian has alpha < 1/255 at
// every pixel of the footprint, so it would have been skipped pixel by pixel anyway: the
// result is identical to evaluating every list entry at every pixel. A warp stops when all
// its pixels have stopped; the CTA stops when all warps have.
#include <algorithm>

#include "fdgs_internal.h"

namespace fdgs {

namespace {

constexpr int kBatch = 256;

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Pixel of lane `lane` in warp `warp` of tile (tx, ty) for an FW-wide warp footprint.
template <int FW>
struct Footprint {
  static constexpr int FH = 32 / FW;
  static constexpr int WX = kTile / FW;
  int x0, y0;       // footprint origin (pixels)
  int px, py;       // this lane's pixel
  __device__ __forceinline__ Footprint(int tx, int ty, int warp, int lane) {
    x0 = tx * kTile + (warp % WX) * FW;
    y0 = ty * kTile + (warp / WX) * FH;
    px = x0 + lane % FW;
    py = y0 + lane / FW;
  }
  // Whether the Gaussian can reach alpha >= 1/255 at some pixel of the footprint.
  __device__ __forceinline__ bool may_hit(float4 g0, float c2, float lga, float kx,
                                          float ky) const {
    const float qmax = quad_max_rect(g0.z, g0.w, c2, kx, ky, g0.x - (float)(x0 + FW - 1),
                                     g0.x - (float)x0, g0.y - (float)(y0 + FH - 1),
                                     g0.y - (float)y0);
    return qmax + lga >= kLog2AlphaMin - kCullMargin;
  }
};

template <typename K, int FW, bool kWeights, bool kCount>
__global__ void __launch_bounds__(256)
k_blend(BlendArgs a, const K *__restrict__ keys, uint32_t rmask) {
  constexpr int NT = 256;
  constexpr int E = kBatch / NT;
  __shared__ __align__(16) float4 s_g0[2][kBatch];   // u, v, a2, b2
  __shared__ __align__(16) float4 s_g1[2][kBatch];   // c2, lga, r, g
  __shared__ __align__(16) float4 s_g2[2][kBatch];   // b, kx, ky, radius
  __shared__ uint32_t s_rk[kWeights ? 2 : 1][kBatch];
  const int tile = blockIdx.x;
  const int tx = tile % a.gx, ty = tile / a.gx;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const Footprint<FW> fp(tx, ty, warp, lane);
  const uint2 range = a.ranges[tile];
  const uint32_t n = range.y - range.x;
  const int nb = (int)((n + kBatch - 1) / kBatch);
  const bool inside = fp.px < a.W && fp.py < a.H;
  const float fpx = (float)fp.px, fpy = (float)fp.py;
  float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
  uint32_t last = 0, nevals = 0;
  bool done = !inside;
  bool warp_done = __all_sync(0xffffffffu, done);

  K kr[E];
  auto load_keys = [&](int b) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const uint32_t i = (uint32_t)b * kBatch + e * NT + tid;
      kr[e] = i < n ? keys[range.x + i] : (K)0;
    }
  };
  auto issue = [&](int b) {
    const int st = b & 1;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const uint32_t i = (uint32_t)b * kBatch + e * NT + tid;
      if (i < n) {
        const uint32_t r = (uint32_t)(kr[e] & (K)rmask);
        const float *rp = a.rec_sorted + (size_t)r * kRecS;
        const int j = e * NT + tid;
        cp_async16(&s_g0[st][j], rp);
        cp_async16(&s_g1[st][j], rp + 4);
        cp_async16(&s_g2[st][j], rp + 8);
        if (kWeights) s_rk[st][j] = r;
      }
    }
    cp_async_commit();
  };

  if (nb > 0) {
    load_keys(0);
    issue(0);
    if (nb > 1) load_keys(1);
  }
  for (int b = 0; b < nb; ++b) {
    if (b + 1 < nb) {
      issue(b + 1);
      if (b + 2 < nb) load_keys(b + 2);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const int st = b & 1;
    const int cnt = (int)min((uint32_t)kBatch, n - (uint32_t)b * kBatch);
    const uint32_t pos0 = (uint32_t)b * kBatch;
    for (int j0 = 0; j0 < cnt && !warp_done; j0 += 32) {
      bool hit = false;
      if (j0 + lane < cnt) {
        const float4 g0 = s_g0[st][j0 + lane];
        const float2 g1 = *reinterpret_cast<const float2 *>(&s_g1[st][j0 + lane]);
        const float4 g2 = s_g2[st][j0 + lane];
        hit = fp.may_hit(g0, g1.x, g1.y, g2.y, g2.z);
      }
      uint32_t m = __ballot_sync(0xffffffffu, hit);
      while (m) {
        const int j = j0 + __ffs(m) - 1;
        m &= m - 1;
        float w = 0.f;
        if (!done) {
          if (kCount) ++nevals;
          const float4 g0 = s_g0[st][j];
          const float4 g1 = s_g1[st][j];
          float alpha, raw, dx, dy;
          if (splat_alpha(g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, fpx, fpy, alpha, raw, dx, dy)) {
            const float nT = T * (1.f - alpha);
            if (nT < kTStop) {
              done = true;
            } else {
              w = alpha * T;
              C0 = fmaf(g1.z, w, C0);
              C1 = fmaf(g1.w, w, C1);
              C2 = fmaf(s_g2[st][j].x, w, C2);
              T = nT;
              last = pos0 + j + 1;
            }
          }
        }
        if (kWeights) {
          if (__any_sync(0xffffffffu, w != 0.f)) {
            const float s = warp_sum(w);
            if (lane == 0) atomicAdd(&a.w_sum[s_rk[st][j]], s);
          }
        }
      }
      warp_done = __all_sync(0xffffffffu, done);
    }
    if (__syncthreads_and(warp_done)) {
      cp_async_wait<0>();
      break;
    }
  }
  if (kCount) {
    const uint32_t ws = warp_sum(nevals);
    if (lane == 0 && ws) atomicAdd(a.evals, (unsigned long long)ws);
  }
  if (inside) {
    const size_t hw = (size_t)a.W * a.H;
    const size_t pix = (size_t)fp.py * a.W + fp.px;
    a.rgb[pix] = C0 + T * a.bg[0];
    a.rgb[hw + pix] = C1 + T * a.bg[1];
    a.rgb[2 * hw + pix] = C2 + T * a.bg[2];
    a.T_final[pix] = T;
    a.n_contrib[pix] = last;
  }
}

// Reverse replay of each tile list from the largest n_contrib down to 0, with the same
// warp-footprint culling (a culled Gaussian was skipped by every pixel of the footprint).
template <typename K, int FW>
__global__ void __launch_bounds__(256)
k_blend_bwd(BlendBwdArgs a, const K *__restrict__ keys, uint32_t rmask) {
  __shared__ __align__(16) float4 s_g0[kBatch];   // u, v, a2, b2
  __shared__ __align__(16) float4 s_g1[kBatch];   // c2, lga, r, g
  __shared__ __align__(16) float4 s_g2[kBatch];   // b, kx, ky, radius
  __shared__ __align__(16) float4 s_g3[kBatch];   // A, B, C, a
  __shared__ uint32_t s_rk[kBatch];
  __shared__ uint32_t s_max;
  const int tile = blockIdx.x;
  const int tx = tile % a.gx, ty = tile / a.gx;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const Footprint<FW> fp(tx, ty, warp, lane);
  const bool inside = fp.px < a.W && fp.py < a.H;
  const uint2 range = a.ranges[tile];
  const size_t pix = (size_t)fp.py * a.W + fp.px, hw = (size_t)a.W * a.H;
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
  const uint32_t warp_nc = __reduce_max_sync(0xffffffffu, nc);
  const float Tf = T;
  const float bg_dot = a.bg[0] * dL0 + a.bg[1] * dL1 + a.bg[2] * dL2;
  float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, last_a = 0.f, lc0 = 0.f, lc1 = 0.f, lc2 = 0.f;
  const float fpx = (float)fp.px, fpy = (float)fp.py;
  __syncthreads();
  const int maxnc = (int)s_max;
  for (int bend = maxnc; bend > 0; bend -= kBatch) {
    const int bstart = max(0, bend - kBatch);
    __syncthreads();
    if (bstart + tid < bend) {
      const uint32_t r = (uint32_t)(keys[range.x + bstart + tid] & (K)rmask);
      const float4 *rp = reinterpret_cast<const float4 *>(a.rec_sorted + (size_t)r * kRecS);
      s_g0[tid] = rp[0];
      s_g1[tid] = rp[1];
      s_g2[tid] = rp[2];
      s_g3[tid] = rp[3];
      s_rk[tid] = r;
    }
    __syncthreads();
    // groups of 32 entries, last group first; entries at or beyond the warp's largest
    // n_contrib are never blended by its pixels
    const int wend = min(bend, (int)warp_nc) - bstart;
    for (int g0i = ((wend - 1) >> 5) << 5; wend > 0 && g0i >= 0; g0i -= 32) {
      bool hit = false;
      const int jl = g0i + lane;
      if (jl < wend) {
        const float4 g0 = s_g0[jl];
        const float2 g1 = *reinterpret_cast<const float2 *>(&s_g1[jl]);
        const float4 g2 = s_g2[jl];
        hit = fp.may_hit(g0, g1.x, g1.y, g2.y, g2.z);
      }
      uint32_t m = __ballot_sync(0xffffffffu, hit);
      while (m) {
        const int bit = 31 - __clz(m);
        m &= ~(1u << bit);
        const int jj = g0i + bit;
        const int pos = bstart + jj;
        float g[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        bool contrib = false;
        if ((uint32_t)pos < nc) {
          const float4 g0 = s_g0[jj];
          const float4 g1 = s_g1[jj];
          float alpha, raw, dx, dy;
          if (splat_alpha(g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, fpx, fpy, alpha, raw, dx, dy)) {
            contrib = true;
            const float cb = s_g2[jj].x;
            const float om = 1.f - alpha;
            T = T / om;
            const float wgt = alpha * T;
            acc0 = last_a * lc0 + (1.f - last_a) * acc0;
            acc1 = last_a * lc1 + (1.f - last_a) * acc1;
            acc2 = last_a * lc2 + (1.f - last_a) * acc2;
            float dLda = (g1.z - acc0) * dL0 + (g1.w - acc1) * dL1 + (cb - acc2) * dL2;
            dLda = dLda * T - Tf / om * bg_dot;
            g[6] = wgt * dL0;
            g[7] = wgt * dL1;
            g[8] = wgt * dL2;
            last_a = alpha;
            lc0 = g1.z; lc1 = g1.w; lc2 = cb;
            if (raw < kAlphaMax) {
              const float4 g3 = s_g3[jj];          // A, B, C, a
              g[5] = raw / g3.w * dLda;            // d alpha / d a = exp(power)
              const float gp = alpha * dLda;       // d alpha / d power = alpha
              g[0] = gp * (-g3.x * dx - g3.y * dy);
              g[1] = gp * (-g3.z * dy - g3.y * dx);
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
            float *dst = a.g2d + (size_t)s_rk[jj] * 9;
#pragma unroll
            for (int f = 0; f < 9; ++f)
              if (g[f] != 0.f) atomicAdd(&dst[f], g[f]);
          }
        }
      }
    }
  }
}

template <typename K, int FW>
void blend_fw(const BlendArgs &a, const K *keys, uint32_t rmask, cudaStream_t st) {
  const int tiles = a.gx * a.gy;
  if (a.w_sum)
    k_blend<K, FW, true, false><<<tiles, 256, 0, st>>>(a, keys, rmask);
  else if (a.evals)
    k_blend<K, FW, false, true><<<tiles, 256, 0, st>>>(a, keys, rmask);
  else
    k_blend<K, FW, false, false><<<tiles, 256, 0, st>>>(a, keys, rmask);
}

}  // namespace

int g_blend_shape = 1;   // warp footprint: 0 -> 16x2, 1 -> 8x4, 2 -> 4x8 pixels

template <typename K>
void launch_blend(const BlendArgs &a, const K *keys, uint32_t rmask, cudaStream_t st) {
  if (a.gx * a.gy == 0) return;
  switch (g_blend_shape) {
    case 0: blend_fw<K, 16>(a, keys, rmask, st); break;
    case 2: blend_fw<K, 4>(a, keys, rmask, st); break;
    default: blend_fw<K, 8>(a, keys, rmask, st); break;
  }
}

template <typename K>
void launch_blend_bwd(const BlendBwdArgs &a, const K *keys, uint32_t rmask, cudaStream_t st) {
  const int tiles = a.gx * a.gy;
  if (tiles == 0) return;
  k_blend_bwd<K, 8><<<tiles, 256, 0, st>>>(a, keys, rmask);
}

template void launch_blend<uint32_t>(const BlendArgs &, const uint32_t *, uint32_t, cudaStream_t);
template void launch_blend<uint64_t>(const BlendArgs &, const uint64_t *, uint32_t, cudaStream_t);
template void launch_blend_bwd<uint32_t>(const BlendBwdArgs &, const uint32_t *, uint32_t,
                                         cudaStream_t);
template void launch_blend_bwd<uint64_t>(const BlendBwdArgs &, const uint64_t *, uint32_t,
                                         cudaStream_t);

}  // namespace fdgs
