// Per-tile front-to-back compositing (Eq. 2 with Eq. 3's alpha): the device-side body shared
// by the one-CTA-per-tile kernel and the persistent batched kernel.
//
// A CTA of 256 threads composites one 16x16 tile; each warp owns an FW x (32/FW) pixel
// footprint, one pixel per lane. The tile's records are staged 256 at a time with cp.async
// into a double buffer (the copy of batch b+1 is in flight while batch b is composited; the
// keys of batch b+2 are already loading into registers). Two culling levels, both exact for
// the concave exponent and conservative by a margin, so no per-pixel decision changes:
//   1. staging: each thread tests its staged Gaussian against the whole tile; survivors are
//      compacted (block ballot + prefix) into an index list that keeps list order;
//   2. warps: lanes test 32 survivors at a time against the warp's footprint and
//      __ballot_sync the hits; each hitting lane writes its record to the warp's hit list, and
//      the warp evaluates the list in order, one Gaussian at a time, for 32 pixels.
// A culled Gaussian has alpha < 1/255 at every pixel it is culled for, so it would have been
// skipped pixel by pixel anyway: results equal evaluating every entry at every pixel.
#pragma once
#include "fdgs_internal.h"

namespace fdgs {

constexpr int kBlendBatch = 256;
constexpr int kBlendThreads = 256;

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

// Whether a Gaussian (blend-ready record fields) can reach alpha >= 1/255 somewhere in the
// pixel rectangle [x0, x1] x [y0, y1] (pixel coordinates, inclusive).
__device__ __forceinline__ bool may_hit_rect(float4 g0, float c2, float lga, float kx, float ky,
                                             float x0, float x1, float y0, float y1) {
  const float qmax = quad_max_rect(g0.z, g0.w, c2, kx, ky, g0.x - x1, g0.x - x0, g0.y - y1,
                                   g0.y - y0);
  return qmax + lga >= kLog2AlphaMin - kCullMargin;
}

struct BlendSmem {
  float4 g0[2][kBlendBatch];   // u, v, a2, b2
  float4 g1[2][kBlendBatch];   // c2, lga, r, g
  float4 g2[2][kBlendBatch];   // b, kx, ky, radius
  uint32_t rk[2][kBlendBatch]; // rank (score weights)
  uint16_t idx[kBlendBatch];   // compacted survivors of the tile test
  uint32_t wcnt[kBlendThreads / 32];
  uint32_t ncomp;
  // per warp, the records of the footprint-test hits in hit order, written by the lanes that
  // tested them: u, v, a2, b2 | c2, lga, r, g | b, stage index
  float4 h0[kBlendThreads / 32][32];
  float4 h1[kBlendThreads / 32][32];
  float2 h2[kBlendThreads / 32][32];
};

// Where one tile's inputs and outputs live.
struct BlendTile {
  int tx, ty, W, H;
  uint2 range;                 // [start, end) into keys
  const float *rec_sorted;     // blend-ready records [rank][16]
  float *rgb;                  // [3][H][W]
  float *T_final;              // [H][W]
  uint32_t *n_contrib;         // [H][W]
  float bg0, bg1, bg2;
  float *w_sum;                // per-rank weights (score pass) or null
  uint32_t *stop_mark;         // per-rank flag: the entry stopped a pixel (with w_sum)
  unsigned long long *evals;   // [2] evaluations, culling tests (profiling) or null
};

template <typename K, int FW, bool kWeights, bool kCount>
__device__ __forceinline__ void blend_tile(const BlendTile &bt, const K *__restrict__ keys,
                                           uint32_t rmask, BlendSmem &sm) {
  constexpr int NT = kBlendThreads;
  constexpr int FH = 32 / FW;
  constexpr int WX = kTile / FW;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int fx0 = bt.tx * kTile + (warp % WX) * FW, fy0 = bt.ty * kTile + (warp / WX) * FH;
  const int px = fx0 + lane % FW, py = fy0 + lane / FW;
  const float tx0 = (float)(bt.tx * kTile), ty0 = (float)(bt.ty * kTile);
  const float fxl = (float)fx0, fxh = (float)(fx0 + FW - 1);
  const float fyl = (float)fy0, fyh = (float)(fy0 + FH - 1);
  const uint32_t n = bt.range.y - bt.range.x;
  const int nb = (int)((n + kBlendBatch - 1) / kBlendBatch);
  const bool inside = px < bt.W && py < bt.H;
  const float fpx = (float)px, fpy = (float)py;
  float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
  uint32_t last = 0, nevals = 0, ntests = 0;
  bool done = !inside;
  bool warp_done = __all_sync(0xffffffffu, done);

  K kr = (K)0;
  auto load_key = [&](int b) {
    const uint32_t i = (uint32_t)b * kBlendBatch + tid;
    kr = i < n ? keys[bt.range.x + i] : (K)0;
  };
  auto issue = [&](int b) {
    const int st = b & 1;
    const uint32_t i = (uint32_t)b * kBlendBatch + tid;
    if (i < n) {
      const uint32_t r = (uint32_t)(kr & (K)rmask);
      const float *rp = bt.rec_sorted + (size_t)r * kRecS;
      cp_async16(&sm.g0[st][tid], rp);
      cp_async16(&sm.g1[st][tid], rp + 4);
      cp_async16(&sm.g2[st][tid], rp + 8);
      if (kWeights) sm.rk[st][tid] = r;
    }
    cp_async_commit();
  };

  if (nb > 0) {
    load_key(0);
    issue(0);
    if (nb > 1) load_key(1);
  }
  for (int b = 0; b < nb; ++b) {
    if (b + 1 < nb) {
      issue(b + 1);
      if (b + 2 < nb) load_key(b + 2);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const int st = b & 1;
    const int cnt = (int)min((uint32_t)kBlendBatch, n - (uint32_t)b * kBlendBatch);
    const uint32_t pos0 = (uint32_t)b * kBlendBatch;
    // 1. tile-level test of the thread's own staged Gaussian, block compaction
    bool keep = false;
    if (kCount && tid < cnt) ++ntests;
    if (tid < cnt) {
      const float4 g0 = sm.g0[st][tid];
      const float2 g1 = *reinterpret_cast<const float2 *>(&sm.g1[st][tid]);
      const float4 g2 = sm.g2[st][tid];
      keep = may_hit_rect(g0, g1.x, g1.y, g2.y, g2.z, tx0, tx0 + (kTile - 1), ty0,
                          ty0 + (kTile - 1));
    }
    const uint32_t kb = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) sm.wcnt[warp] = __popc(kb);
    __syncthreads();
    if (keep) {
      uint32_t off = __popc(kb & lanemask_lt());
      for (int w = 0; w < warp; ++w) off += sm.wcnt[w];
      sm.idx[off] = (uint16_t)tid;
    }
    if (tid == 0) {
      uint32_t tot = 0;
      for (int w = 0; w < NT / 32; ++w) tot += sm.wcnt[w];
      sm.ncomp = tot;
    }
    __syncthreads();
    const int ncomp = (int)sm.ncomp;
    // 2. warp footprint tests on the survivors, evaluation of the hits
    for (int c0 = 0; c0 < ncomp && !warp_done; c0 += 32) {
      bool hit = false;
      int j = 0;
      float4 g0, g1, g2;
      if (kCount && c0 + lane < ncomp) ++ntests;
      if (c0 + lane < ncomp) {
        j = sm.idx[c0 + lane];
        g0 = sm.g0[st][j];
        g1 = sm.g1[st][j];
        g2 = sm.g2[st][j];
        hit = may_hit_rect(g0, g1.x, g1.y, g2.y, g2.z, fxl, fxh, fyl, fyh);
      }
      const uint32_t m = __ballot_sync(0xffffffffu, hit);
      if (hit) {                       // hand the record to the warp's hit list
        const int p = __popc(m & lanemask_lt());
        sm.h0[warp][p] = g0;
        sm.h1[warp][p] = g1;
        sm.h2[warp][p] = make_float2(g2.x, __int_as_float(j));
      }
      __syncwarp();
      const int nh = __popc(m);
      for (int k = 0; k < nh; ++k) {
        float w = 0.f;
        if (!done) {
          if (kCount) ++nevals;
          const float4 h0 = sm.h0[warp][k];
          const float4 h1 = sm.h1[warp][k];
          float alpha, raw, dx, dy;
          if (splat_alpha(h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, fpx, fpy, alpha, raw, dx, dy)) {
            const float nT = T * (1.f - alpha);
            if (nT < kTStop) {
              done = true;
              // the entry ends this pixel's list: the key-frame masks keep it
              if (kWeights) bt.stop_mark[sm.rk[st][__float_as_int(sm.h2[warp][k].y)]] = 1u;
            } else {
              const float2 h2 = sm.h2[warp][k];
              w = alpha * T;
              C0 = fmaf(h1.z, w, C0);
              C1 = fmaf(h1.w, w, C1);
              C2 = fmaf(h2.x, w, C2);
              T = nT;
              last = pos0 + (uint32_t)__float_as_int(h2.y) + 1;
            }
          }
        }
        if (kWeights) {
          if (__any_sync(0xffffffffu, w != 0.f)) {
            const float s = warp_sum(w);
            if (lane == 0) atomicAdd(&bt.w_sum[sm.rk[st][__float_as_int(sm.h2[warp][k].y)]], s);
          }
        }
      }
      __syncwarp();                    // the list is rewritten by the next round
      warp_done = __all_sync(0xffffffffu, done);
    }
    if (__syncthreads_and(warp_done)) {
      cp_async_wait<0>();
      break;
    }
  }
  if (kCount) {
    const uint32_t ws = warp_sum(nevals), wt = warp_sum(ntests);
    if (lane == 0 && ws) atomicAdd(&bt.evals[0], (unsigned long long)ws);
    if (lane == 0 && wt) atomicAdd(&bt.evals[1], (unsigned long long)wt);
  }
  if (inside) {
    const size_t hw = (size_t)bt.W * bt.H;
    const size_t pix = (size_t)py * bt.W + px;
    bt.rgb[pix] = C0 + T * bt.bg0;
    bt.rgb[hw + pix] = C1 + T * bt.bg1;
    bt.rgb[2 * hw + pix] = C2 + T * bt.bg2;
    bt.T_final[pix] = T;
    bt.n_contrib[pix] = last;
  }
}

}  // namespace fdgs
