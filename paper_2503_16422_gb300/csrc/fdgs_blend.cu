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
  const int tile = a.order ? (int)a.order[blockIdx.x] : (int)blockIdx.x;
  BlendTile bt;
  bt.tx = tile % a.gx;
  bt.ty = tile / a.gx;
  bt.W = a.W;
  bt.H = a.H;
  bt.range = a.ranges[tile];
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
  uint32_t no_tma = 0;
  blend_tile<K, FW, PX, kWeights, kCount, true>(bt, keys, rmask, sm, no_tma);
}

// The forward-only blend of a single render on a black background (no frame kept, so no
// transmittance or n_contrib is written): the T = 0 stop encoding and, with an even number of
// pixels a lane, the paired FP32 evaluation of the batched blend; images are bit-identical to
// the flag form's.
template <typename K, int FW, int PX>
__global__ void __launch_bounds__(256 / PX)
k_blend_fwd(BlendArgs a, const K *__restrict__ keys, uint32_t rmask) {
  __shared__ BlendSmem<256 / PX> sm;
  const int tile = a.order ? (int)a.order[blockIdx.x] : (int)blockIdx.x;
  BlendTile bt;
  bt.tx = tile % a.gx;
  bt.ty = tile / a.gx;
  bt.W = a.W;
  bt.H = a.H;
  bt.range = a.ranges[tile];
  bt.rec_sorted = a.rec_sorted;
  bt.rgb = a.rgb;
  bt.T_final = nullptr;
  bt.n_contrib = nullptr;
  bt.bg0 = bt.bg1 = bt.bg2 = 0.f;
  bt.w_sum = nullptr;
  bt.stop_mark = nullptr;
  bt.evals = nullptr;
  uint32_t no_tma = 0;
  blend_tile<K, FW, PX, false, false, false, false, true>(bt, keys, rmask, sm, no_tma);
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

// Reverse replay of each tile list from the largest n_contrib down to 0, with the
// warp-footprint culling of the forward (a culled Gaussian was skipped by every pixel of the
// footprint). Transmittance is recovered as T_i = T_{i+1} / (1 - alpha_i). A CTA of 256 / PX
// threads replays one tile (tiles in the forward's longest-first order when it is given); each
// lane owns PX pixels of one footprint row, FW / PX apart, and sums their gradient terms
// before the warp reduction. As in the forward, the evaluation has no branches: an entry a
// pixel did not blend takes alpha = 0 and leaves its state unchanged.
// kCount: also count (into a.evals) the entry evaluations at pixels whose replay has reached
// them (list position below n_contrib), the ones that were blended, and the atomics issued.
template <typename K, int FW, int PX, bool kCount = false>
__global__ void __launch_bounds__(256 / PX)
k_blend_bwd(BlendBwdArgs a, const K *__restrict__ keys, uint32_t rmask) {
  constexpr int NT = 256 / PX;
  constexpr int NW = NT / 32;
  constexpr int FH = 32 * PX / FW;
  constexpr int HW = FW / PX;
  constexpr int WX = kTile / FW;
  constexpr int kB = NT;
  __shared__ __align__(16) float4 s_g0[kB];   // u, v, a2, b2
  __shared__ __align__(16) float4 s_g1[kB];   // c2, lga, r, g
  __shared__ __align__(16) float4 s_g2[kB];   // b, kx, ky, radius
  __shared__ __align__(16) float4 s_g3[kB];   // A, B, C, 1/a (from the record's a)
  __shared__ uint32_t s_rk[kB];
  // per warp, the footprint hits of the current group of 32 entries in entry order
  __shared__ __align__(16) float4 h0[NW][32], h1[NW][32], h3[NW][32];
  __shared__ float2 h2[NW][32];               // b, entry index within the batch
  __shared__ uint32_t s_max;
  const int tile = a.order ? (int)a.order[blockIdx.x] : (int)blockIdx.x;
  const int tx = tile % a.gx, ty = tile / a.gx;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int fx0 = tx * kTile + (warp % WX) * FW, fy0 = ty * kTile + (warp / WX) * FH;
  const int px0 = fx0 + lane % HW, py = fy0 + lane / HW;
  const float fxl = (float)fx0, fxh = (float)(fx0 + FW - 1);
  const float fyl = (float)fy0, fyh = (float)(fy0 + FH - 1);
  const uint2 range = a.ranges[tile];
  const size_t hw = (size_t)a.W * a.H;
  if (tid == 0) s_max = 0;
  __syncthreads();
  uint32_t nc[PX];
  float T[PX], Tf[PX], dL0[PX], dL1[PX], dL2[PX], bg_dot[PX];
  float acc0[PX], acc1[PX], acc2[PX], last_a[PX], lc0[PX], lc1[PX], lc2[PX];
  uint32_t lane_nc = 0;
#pragma unroll
  for (int p = 0; p < PX; ++p) {
    const int px = px0 + p * HW;
    nc[p] = 0;
    T[p] = 1.f;
    dL0[p] = dL1[p] = dL2[p] = 0.f;
    if (px < a.W && py < a.H) {
      const size_t pix = (size_t)py * a.W + px;
      nc[p] = a.n_contrib[pix];
      T[p] = a.T_final[pix];
      dL0[p] = a.dL_drgb[pix];
      dL1[p] = a.dL_drgb[hw + pix];
      dL2[p] = a.dL_drgb[2 * hw + pix];
    }
    lane_nc = max(lane_nc, nc[p]);
    Tf[p] = T[p];
    bg_dot[p] = a.bg[0] * dL0[p] + a.bg[1] * dL1[p] + a.bg[2] * dL2[p];
    acc0[p] = acc1[p] = acc2[p] = last_a[p] = lc0[p] = lc1[p] = lc2[p] = 0.f;
  }
  uint32_t n_eval = 0, n_valid = 0, n_atomic = 0;
  const uint32_t warp_nc = __reduce_max_sync(0xffffffffu, lane_nc);
  if (lane == 0) atomicMax(&s_max, warp_nc);
  const float fpy = (float)py;
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
      float4 g0, g1;
      if (jl < wend) {
        g0 = s_g0[jl];
        g1 = s_g1[jl];
        const float4 g2 = s_g2[jl];
        hit = may_hit_rect(g0, g1.x, g1.y, g2.y, g2.z, fxl, fxh, fyl, fyh);
      }
      const uint32_t m = __ballot_sync(0xffffffffu, hit);
      if (hit) {
        const int hp = __popc(m & lanemask_lt());
        h0[warp][hp] = g0;
        h1[warp][hp] = g1;
        h3[warp][hp] = s_g3[jl];
        h2[warp][hp] = make_float2(s_g2[jl].x, __int_as_float(jl));
      }
      __syncwarp();
      for (int k = __popc(m) - 1; k >= 0; --k) {
        const float4 e0 = h0[warp][k];
        const float4 e1 = h1[warp][k];
        const float2 e2 = h2[warp][k];
        const float4 e3 = h3[warp][k];        // A, B, C, 1/a
        const int jj = __float_as_int(e2.y);
        const uint32_t pos = (uint32_t)(bstart + jj);
        // the exponent as in the forward, with the row terms shared by the lane's pixels
        const float dy = __fsub_rn(e0.y, fpy);
        const float b2dy = __fmul_rn(e0.w, dy);
        const float c2l = __fmaf_rn(__fmul_rn(e1.x, dy), dy, e1.y);
        float G[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        bool any = false;
#pragma unroll
        for (int p = 0; p < PX; ++p) {
          const float dx = __fsub_rn(e0.x, (float)(px0 + p * HW));
          const float e = __fmaf_rn(dx, __fmaf_rn(e0.z, dx, b2dy), c2l);
          const bool valid = pos < nc[p] && e >= kLog2AlphaMin;
          if (kCount) {
            n_eval += pos < nc[p] ? 1u : 0u;
            n_valid += valid ? 1u : 0u;
          }
          any = any || valid;
          const float raw = ex2_approx(e);
          const float alpha = valid ? fminf(kAlphaMax, raw) : 0.f;
          // 1 - alpha >= 0.01: the fast reciprocal is within 2 ulp, far inside the gradient
          // tolerance, and replaces three IEEE divisions per hit
          const float iom = __fdividef(1.f, 1.f - alpha);
          T[p] = valid ? T[p] * iom : T[p];
          const float wgt = alpha * T[p];
          const float la = last_a[p];
          acc0[p] = valid ? la * lc0[p] + (1.f - la) * acc0[p] : acc0[p];
          acc1[p] = valid ? la * lc1[p] + (1.f - la) * acc1[p] : acc1[p];
          acc2[p] = valid ? la * lc2[p] + (1.f - la) * acc2[p] : acc2[p];
          float dLda = (e1.z - acc0[p]) * dL0[p] + (e1.w - acc1[p]) * dL1[p] +
                       (e2.x - acc2[p]) * dL2[p];
          dLda = dLda * T[p] - Tf[p] * iom * bg_dot[p];
          G[6] += wgt * dL0[p];
          G[7] += wgt * dL1[p];
          G[8] += wgt * dL2[p];
          last_a[p] = valid ? alpha : la;
          lc0[p] = valid ? e1.z : lc0[p];
          lc1[p] = valid ? e1.w : lc1[p];
          lc2[p] = valid ? e2.x : lc2[p];
          const bool unclamped = valid && raw < kAlphaMax;
          G[5] += unclamped ? raw * e3.w * dLda : 0.f;   // d alpha / d a = exp(power)
          const float gp = unclamped ? alpha * dLda : 0.f; // d alpha / d power = alpha
          G[0] += gp * (-e3.x * dx - e3.y * dy);
          G[1] += gp * (-e3.z * dy - e3.y * dx);
          G[2] += gp * (-0.5f * dx * dx);
          G[3] += gp * (-dx * dy);
          G[4] += gp * (-0.5f * dy * dy);
        }
        if (__any_sync(0xffffffffu, any)) {
          float *dst = a.g2d + (size_t)s_rk[jj] * 9;
          int fi;
          const float s8 = warp_sum8_transposed(G, fi);   // G[0..7]: lane owns sum fi
          const float s9 = warp_sum(G[8]);
          if ((lane & 3) == 0 && s8 != 0.f) atomicAdd(&dst[fi], s8);
          if (lane == 4 && s9 != 0.f) atomicAdd(&dst[8], s9);
          if (kCount) n_atomic += ((lane & 3) == 0 && s8 != 0.f) + (lane == 4 && s9 != 0.f);
        }
      }
      __syncwarp();                    // the list is rewritten by the next group
    }
  }
  if (kCount) {
    const uint32_t e = warp_sum(n_eval), v = warp_sum(n_valid), t = warp_sum(n_atomic);
    if (lane == 0 && e) atomicAdd(&a.evals[0], (unsigned long long)e);
    if (lane == 0 && v) atomicAdd(&a.evals[1], (unsigned long long)v);
    if (lane == 0 && t) atomicAdd(&a.evals[2], (unsigned long long)t);
  }
}

}  // namespace

int g_blend_shape = kBlendShapeDefault;
int g_blend_shape_fwd = kBlendShapeFwdDefault;

template <typename K>
void launch_blend(const BlendArgs &a, const K *keys, uint32_t rmask, cudaStream_t st) {
  const int tiles = a.gx * a.gy;
  if (tiles == 0) return;
  // no transmittance to write: the forward-only blend (the caller passes a null T_final only
  // for an uncounted, unweighted render on a black background)
  if (!a.T_final) {
    with_blend_shape(g_blend_shape_fwd, [&](auto fw, auto px) {
      constexpr int FW = decltype(fw)::value, PX = decltype(px)::value;
      k_blend_fwd<K, FW, PX><<<tiles, 256 / PX, 0, st>>>(a, keys, rmask);
    });
    return;
  }
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
  // 8x16 warp footprints, four pixels per lane (0.66 vs 0.95 ms for one pixel per lane with
  // branches, alpha-tight frames of the 200k scene at 1352x1014, including the per-Gaussian
  // backward)
  if (a.evals)
    k_blend_bwd<K, 8, 4, true><<<tiles, 64, 0, st>>>(a, keys, rmask);
  else
    k_blend_bwd<K, 8, 4><<<tiles, 64, 0, st>>>(a, keys, rmask);
}

template void launch_blend<uint32_t>(const BlendArgs &, const uint32_t *, uint32_t, cudaStream_t);
template void launch_blend<uint64_t>(const BlendArgs &, const uint64_t *, uint32_t, cudaStream_t);
template void launch_blend_bwd<uint32_t>(const BlendBwdArgs &, const uint32_t *, uint32_t,
                                         cudaStream_t);
template void launch_blend_bwd<uint64_t>(const BlendBwdArgs &, const uint64_t *, uint32_t,
                                         cudaStream_t);

}  // namespace fdgs
