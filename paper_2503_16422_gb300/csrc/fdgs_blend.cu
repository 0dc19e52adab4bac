// Blend kernels: the per-tile forward (one CTA per 16x16 tile, body in fdgs_blend.cuh) and the
// reverse replay used by the backward.
#include <algorithm>

#include "fdgs_blend.cuh"

namespace fdgs {

namespace {

template <typename K, int FW, int PX, bool kWeights, bool kCount>
__global__ void __launch_bounds__(256 / PX)
k_blend(BlendArgs a, const K *__restrict__ keys, uint32_t rmask) {
  __shared__ BlendSmem<256 / PX> sm;
  BlendTile bt;
  bt.tx = blockIdx.x % a.gx;
  bt.ty = blockIdx.x / a.gx;
  bt.W = a.W;
  bt.H = a.H;
  bt.range = a.ranges[blockIdx.x];
  bt.rec_sorted = a.rec_sorted;
  bt.rgb = a.rgb;
  bt.T_final = a.T_final;
  bt.n_contrib = a.n_contrib;
  bt.bg0 = a.bg[0];
  bt.bg1 = a.bg[1];
  bt.bg2 = a.bg[2];
  bt.w_sum = a.w_sum;
  bt.stop_mark = a.stop_mark;
  bt.evals = a.evals;
  blend_tile<K, FW, PX, kWeights, kCount, true>(bt, keys, rmask, sm);
}

// Sums of eight per-lane values over the warp by a transposed butterfly: at offsets 16, 8
// and 4 each lane keeps half of its partial sums and adds its partner's copy of them (7
// shuffles for 8 values instead of 40), then offsets 2 and 1 finish one sum per lane. Lane L
// ends with the full sum of value fi = 4 ((L >> 4) & 1) + 2 ((L >> 3) & 1) + ((L >> 2) & 1),
// so lanes 0, 4, ..., 28 hold the eight sums.
__device__ __forceinline__ float warp_sum8_transposed(const float v[8], int &fi) {
  const int lane = (int)lane_id();
  const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
  float w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float send = h16 ? v[i] : v[i + 4];
    const float keep = h16 ? v[i + 4] : v[i];
    w[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  float x[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float send = h8 ? w[i] : w[i + 2];
    const float keep = h8 ? w[i + 2] : w[i];
    x[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  float y = (h4 ? x[1] : x[0]) + __shfl_xor_sync(0xffffffffu, h4 ? x[0] : x[1], 4);
  y += __shfl_xor_sync(0xffffffffu, y, 2);
  y += __shfl_xor_sync(0xffffffffu, y, 1);
  fi = (h16 ? 4 : 0) + (h8 ? 2 : 0) + (h4 ? 1 : 0);
  return y;
}

// Reverse replay of each tile list from the largest n_contrib down to 0, one pixel per
// lane, with the warp-footprint culling of the forward (a culled Gaussian was skipped by
// every pixel of the footprint). Transmittance is recovered as T_i = T_{i+1} / (1 - alpha_i).
template <typename K, int FW>
__global__ void __launch_bounds__(256)
k_blend_bwd(BlendBwdArgs a, const K *__restrict__ keys, uint32_t rmask) {
  constexpr int FH = 32 / FW;
  constexpr int WX = kTile / FW;
  constexpr int kB = 256;
  __shared__ __align__(16) float4 s_g0[kB];   // u, v, a2, b2
  __shared__ __align__(16) float4 s_g1[kB];   // c2, lga, r, g
  __shared__ __align__(16) float4 s_g2[kB];   // b, kx, ky, radius
  __shared__ __align__(16) float4 s_g3[kB];   // A, B, C, 1/a (from the record's a)
  __shared__ uint32_t s_rk[kB];
  __shared__ uint32_t s_max;
  const int tile = blockIdx.x;
  const int tx = tile % a.gx, ty = tile / a.gx;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int fx0 = tx * kTile + (warp % WX) * FW, fy0 = ty * kTile + (warp / WX) * FH;
  const int px = fx0 + lane % FW, py = fy0 + lane / FW;
  const float fxl = (float)fx0, fxh = (float)(fx0 + FW - 1);
  const float fyl = (float)fy0, fyh = (float)(fy0 + FH - 1);
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
  const uint32_t warp_nc = __reduce_max_sync(0xffffffffu, nc);
  const float Tf = T;
  const float bg_dot = a.bg[0] * dL0 + a.bg[1] * dL1 + a.bg[2] * dL2;
  float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, last_a = 0.f, lc0 = 0.f, lc1 = 0.f, lc2 = 0.f;
  const float fpx = (float)px, fpy = (float)py;
  __syncthreads();
  const int maxnc = (int)s_max;
  for (int bend = maxnc; bend > 0; bend -= kB) {
    const int bstart = max(0, bend - kB);
    __syncthreads();
    if (bstart + tid < bend) {
      const uint32_t r = (uint32_t)(keys[range.x + bstart + tid] & (K)rmask);
      const float4 *rp = reinterpret_cast<const float4 *>(a.rec_sorted + (size_t)r * kRecS);
      s_g0[tid] = rp[0];
      s_g1[tid] = rp[1];
      s_g2[tid] = rp[2];
      float4 g3 = rp[3];
      g3.w = 1.f / g3.w;                      // once per staged entry, not per hit
      s_g3[tid] = g3;
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
        hit = may_hit_rect(g0, g1.x, g1.y, g2.y, g2.z, fxl, fxh, fyl, fyh);
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
            // 1 - alpha >= 0.01: the fast reciprocal is within 2 ulp, far inside the
            // gradient tolerance, and replaces three IEEE divisions per hit
            const float iom = __fdividef(1.f, om);
            T = T * iom;
            const float wgt = alpha * T;
            acc0 = last_a * lc0 + (1.f - last_a) * acc0;
            acc1 = last_a * lc1 + (1.f - last_a) * acc1;
            acc2 = last_a * lc2 + (1.f - last_a) * acc2;
            float dLda = (g1.z - acc0) * dL0 + (g1.w - acc1) * dL1 + (cb - acc2) * dL2;
            dLda = dLda * T - Tf * iom * bg_dot;
            g[6] = wgt * dL0;
            g[7] = wgt * dL1;
            g[8] = wgt * dL2;
            last_a = alpha;
            lc0 = g1.z; lc1 = g1.w; lc2 = cb;
            if (raw < kAlphaMax) {
              const float4 g3 = s_g3[jj];          // A, B, C, 1/a
              g[5] = raw * g3.w * dLda;            // d alpha / d a = exp(power)
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
          float *dst = a.g2d + (size_t)s_rk[jj] * 9;
          int fi;
          const float s8 = warp_sum8_transposed(g, fi);   // g[0..7]: lane owns sum fi
          const float s9 = warp_sum(g[8]);
          if ((lane & 3) == 0 && s8 != 0.f) atomicAdd(&dst[fi], s8);
          if (lane == 4 && s9 != 0.f) atomicAdd(&dst[8], s9);
        }
      }
    }
  }
}

}  // namespace

int g_blend_shape = 3;   // launch shape of the forward blend (see with_blend_shape)

template <typename K>
void launch_blend(const BlendArgs &a, const K *keys, uint32_t rmask, cudaStream_t st) {
  const int tiles = a.gx * a.gy;
  if (tiles == 0) return;
  with_blend_shape(g_blend_shape, [&](auto fw, auto px) {
    constexpr int FW = decltype(fw)::value, PX = decltype(px)::value;
    if (a.w_sum)
      k_blend<K, FW, PX, true, false><<<tiles, 256 / PX, 0, st>>>(a, keys, rmask);
    else if (a.evals)
      k_blend<K, FW, PX, false, true><<<tiles, 256 / PX, 0, st>>>(a, keys, rmask);
    else
      k_blend<K, FW, PX, false, false><<<tiles, 256 / PX, 0, st>>>(a, keys, rmask);
  });
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
