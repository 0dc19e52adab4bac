// Per-tile front-to-back compositing (Eq. 2 with Eq. 3's alpha): the device-side body shared
// by the one-CTA-per-tile kernel and the persistent batched kernel.
//
// A CTA of 256 / PX threads composites one 16x16 tile; each warp owns an FW x (32 PX / FW)
// pixel footprint and each lane PX pixels of one footprint row, FW / PX apart (so the row
// terms of the exponent are shared). The tile's records are staged one per thread at a time
// with cp.async into a double buffer (the copy of batch b+1 is in flight while batch b is
// composited; the keys of batch b+2 are already loading into registers). Two culling levels,
// both exact for the concave exponent and conservative by a margin, so no per-pixel decision
// changes:
//   1. staging: each thread tests its staged Gaussian against the whole tile; survivors are
//      compacted per warp (ballot) into index segments that, read in turn, keep list order;
//   2. warps: lanes test 32 survivors at a time against the warp's footprint and
//      __ballot_sync the hits; each hitting lane writes its record to the warp's hit list, and
//      the warp evaluates the list in order, one Gaussian at a time, for 32 PX pixels. With
//      eight pixels a lane one warp covers the tile: the CTA is that warp, its barriers are
//      warp-level, and the footprint test is the tile test already made.
// A culled Gaussian has alpha < 1/255 at every pixel it is culled for, so it would have been
// skipped pixel by pixel anyway: results equal evaluating every entry at every pixel.
//
// The per-pixel evaluation has no branches: a pixel whose exponent fails a test, or which has
// already stopped, takes alpha = 0, and T - 0 T, fma(c, 0, C) leave its transmittance and
// colour sums bit-for-bit unchanged. So the arithmetic of every pixel, and every result, is
// the same for every footprint, every PX and the one-pixel-per-branch formulation.
//
// The plain colour blend of the batched path (kTz) with an even PX evaluates the lane's pixels
// in pairs with the paired FP32 instructions of sm_100-class GPUs (one fma.rn.f32x2 does the
// two IEEE fmas of a pixel pair): the exponent, the weight, the transmittance step and the
// colour sums of two pixels take one instruction each; every value is the one of the scalar
// form bit for bit. The colour sums are kept negated (fma(c, -w, -C) = -fma(c, w, C) exactly
// under round-to-nearest), so the weight's sign needs no extra instruction per hit.
#pragma once
#include <type_traits>

#include "fdgs_internal.h"

namespace fdgs {

// Launch shapes of the forward blend (kBlendShapes of them): warp footprint FW x (32 PX / FW)
// pixels, PX pixels per lane.
//   0: 16x2, 1: 8x4, 2: 4x8 (one pixel per lane), 3: 8x8 (two), 4: 16x8, 5: 8x16 (four),
//   6: 16x16 (eight; one warp per tile, so the tile test is the footprint test)
template <class F>
inline void with_blend_shape(int shape, F &&f) {
  switch (shape) {
    case 0: f(std::integral_constant<int, 16>{}, std::integral_constant<int, 1>{}); break;
    case 2: f(std::integral_constant<int, 4>{}, std::integral_constant<int, 1>{}); break;
    case 3: f(std::integral_constant<int, 8>{}, std::integral_constant<int, 2>{}); break;
    case 4: f(std::integral_constant<int, 16>{}, std::integral_constant<int, 4>{}); break;
    case 5: f(std::integral_constant<int, 8>{}, std::integral_constant<int, 4>{}); break;
    case 6: f(std::integral_constant<int, 16>{}, std::integral_constant<int, 8>{}); break;
    default: f(std::integral_constant<int, 8>{}, std::integral_constant<int, 1>{}); break;
  }
}

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

// The staged records of a batch of NT list entries, double-buffered. cp.async (per thread,
// 16 bytes at a time) fills three structure-of-arrays planes; TMA (tile::gather4, four
// 48-byte rows of the record tensor per instruction) fills rows, four to a 256-byte chunk
// whose start is 128-byte aligned as tensor copies require, with one transaction-counting
// mbarrier per buffer.
template <int NT>
struct StageSoa {
  float4 g0[2][NT];            // u, v, a2, b2
  float4 g1[2][NT];            // c2, lga, r, g
  float4 g2[2][NT];            // b, kx, ky, radius
};
template <int NT>
struct StageRows {
  alignas(128) unsigned char c[2][NT / 4][256];
  unsigned long long bar[2];
};

template <int NT, bool kTma = false>
struct BlendSmem {
  typename std::conditional<kTma, StageRows<NT>, StageSoa<NT>>::type stage;
  uint32_t rk[2][NT];          // rank (score weights)
  uint16_t idx[NT];            // compacted survivors of the tile test
  uint32_t wcnt[NT / 32];
  // per warp, the records of the footprint-test hits in hit order, written by the lanes that
  // tested them: u, v, a2, b2 | c2, lga, r, g | b, stage index
  float4 h0[NT / 32][32];
  float4 h1[NT / 32][32];
  float2 h2[NT / 32][32];
  // one-warp CTAs on block lists: the tile's entries (record indices) in list order, between
  // the scan of the list and their staging (kRing of them, a power of two)
  uint32_t ring[NT == 32 ? 256 : 1];
  uint32_t cand[NT == 32 ? 128 : 1];   // ... and the entries of one scan with the tile's bit
};

// mbarrier and TMA helpers of the gather4 staging (shared-window addresses).
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_arrive(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Four rows (r0..r3) of a 2D float tensor, columns [0, box width), into dst.
__device__ __forceinline__ void tma_gather4(uint32_t dst, const void *tmap, uint32_t bar,
                                            uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cta.global.tile::gather4.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
      "l"(tmap), "r"(0), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(bar)
      : "memory");
}
// Spin limit of a stage wait (each try_wait may itself suspend for a while): far above any
// legitimate copy time, so it only ends a broken protocol.
constexpr uint32_t kTmaSpin = 1u << 20;

// Where one tile's inputs and outputs live.
struct BlendTile {
  int tx, ty, W, H;
  uint2 range;                 // [start, end) into keys
  const uint16_t *tmask;       // block lists: per entry, the block's tiles it covers
  int tbit;                    // block lists: this tile's bit in those masks
  const float *rec_sorted;     // blend-ready records: [rank][16] for tile lists, [record][12]
                               // for block lists (kBlk)
  float *rgb;                  // [3][H][W]
  float *T_final;              // [H][W] (written when kAux)
  uint32_t *n_contrib;         // [H][W] (written when kAux)
  float bg0, bg1, bg2;
  float *w_sum;                // per-rank weights (score pass) or null
  uint32_t *stop_mark;         // per-rank flag: the entry stopped a pixel (with w_sum)
  unsigned long long *evals;   // [3] evaluations, culling tests, alpha >= 1/255 evaluations
                               // (profiling) or null
  const void *tmap = nullptr;  // kTma: tensor map of the 12-float records (kBlk)
  uint32_t *err = nullptr;     // kTma: error word (kErrTimeout when a stage wait gives up)
  uint32_t tma_skip = 0;       // kTma: failure injection, thread 0 withholds its arrivals
  uint32_t tma_spin = 0;       // kTma: stage-wait poll limit (0: kTmaSpin)
};

// kAux: also write the final transmittance and 1 + the list position of the last blended
// entry per pixel (what the reverse replay of the backward starts from).
// kBlk: keys[range] is the list of the tile's block of tiles, entries (indices of 12-float
// records) in rank order with a mask of the block's tiles each covers; only entries with bit
// tbit are staged and tested (the others are flagged per thread and skip the tile test), and
// the tile composites exactly its own list. One-warp CTAs (kCompact) stage only the tile's
// hits, in full stages: the list is scanned 128 positions at a time; the entries with bit tbit
// take the tile test on their records (read from global memory), and those that pass go to a
// ring of record indices, from which every stage takes 32. The hits are then read straight
// from the stage, with no test or hit list.
// kTz (black background, no weights, counts or side outputs): the loop keeps no per-pixel
// stop flags. T is updated at every entry, and an entry blends only when its T - alpha T is
// at least 1e-4. T never grows, so the first entry that fails the test (the one that stops
// the pixel) is followed only by entries that fail it too: the colour sums are those of the
// flag form bit for bit, and the final T, which differs after a stop, is multiplied by the
// black background. Pixels outside the image start at T = 0.
// kTma (block lists only): records are staged by TMA gather4 (four per instruction, issued by
// every fourth thread for its own entry and the next three) instead of per-thread cp.async;
// tma_ph carries the two buffers' mbarrier phases across the tiles of a persistent CTA.
// Returns false when a stage wait gave up (kErrTimeout set; nothing is in flight).
template <typename K, int FW, int PX, bool kWeights, bool kCount, bool kAux, bool kBlk = false,
          bool kTz = false, bool kTma = false>
__device__ __forceinline__ bool blend_tile(const BlendTile &bt, const K *__restrict__ keys,
                                           uint32_t rmask, BlendSmem<256 / PX, kTma> &sm,
                                           uint32_t &tma_ph) {
  constexpr int NT = 256 / PX;   // threads = records staged per batch
  constexpr int FH = 32 * PX / FW;
  constexpr int HW = FW / PX;    // lanes per footprint row
  constexpr int WX = kTile / FW;
  static_assert(FW % PX == 0 && FW <= kTile && FH * (NT / 32) == kTile * WX, "shape");
  static_assert(!kTz || (!kWeights && !kCount && !kAux), "kTz: plain colour blend only");
  static_assert(!kTma || (kBlk && NT % 4 == 0), "kTma: block lists, whole chunks");
  // one warp covers the whole tile: a survivor of the tile test is a hit of the warp
  constexpr bool kWholeTile = FW == kTile && FH == kTile;
  // one-warp CTAs on block lists with cp.async staging: compacted stages (see above)
  constexpr bool kCompact = kBlk && !kTma && NT == 32;
  static_assert(!kCompact || !kAux, "kCompact: no list positions");
  // CTA barriers; a one-warp CTA needs only warp-level ones
  auto cta_sync = [] {
    if constexpr (NT == 32) __syncwarp(); else __syncthreads();
  };
  auto cta_and = [](bool v) -> bool {
    if constexpr (NT == 32) return __all_sync(0xffffffffu, v); else return __syncthreads_and(v);
  };
  auto cta_or = [](bool v) -> bool {
    if constexpr (NT == 32) return __any_sync(0xffffffffu, v); else return __syncthreads_or(v);
  };
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int fx0 = bt.tx * kTile + (warp % WX) * FW, fy0 = bt.ty * kTile + (warp / WX) * FH;
  const int px0 = fx0 + lane % HW, py = fy0 + lane / HW;
  const float tx0 = (float)(bt.tx * kTile), ty0 = (float)(bt.ty * kTile);
  const float fxl = (float)fx0, fxh = (float)(fx0 + FW - 1);
  const float fyl = (float)fy0, fyh = (float)(fy0 + FH - 1);
  const uint32_t n = bt.range.y - bt.range.x;
  const int nb = (int)((n + NT - 1) / NT);
  const float fpy = (float)py;
  float T[PX], C0[PX], C1[PX], C2[PX];
  uint32_t last[PX];
  bool done[PX];
  bool lane_done = true;
#pragma unroll
  for (int p = 0; p < PX; ++p) {
    T[p] = 1.f;
    C0[p] = C1[p] = C2[p] = 0.f;
    last[p] = 0;
    done[p] = !(px0 + p * HW < bt.W && py < bt.H);
    if (kTz) T[p] = done[p] ? 0.f : 1.f;
    lane_done = lane_done && done[p];
  }
  uint32_t nevals = 0, ntests = 0, npass = 0;
  // the paired form (kTz, even PX): pixel pairs (2q, 2q + 1) of the lane, the negated pixel
  // x coordinates (dx = u + (-px) is u - px exactly)
  constexpr bool kPair = kTz && PX % 2 == 0;
  constexpr int PH = PX / 2 > 0 ? PX / 2 : 1;
  float2 T2[PH], C02[PH], C12[PH], C22[PH], npx2[PH];
  if constexpr (kPair) {
#pragma unroll
    for (int q = 0; q < PH; ++q) {
      T2[q] = make_float2(T[2 * q], T[2 * q + 1]);
      C02[q] = C12[q] = C22[q] = make_float2(0.f, 0.f);
      npx2[q] = make_float2(-(float)(px0 + 2 * q * HW), -(float)(px0 + (2 * q + 1) * HW));
    }
  }
  bool warp_done = __all_sync(0xffffffffu, lane_done);

  constexpr K kNone = ~(K)0;     // block lists: the entry does not cover this tile
  K kr = (K)0;
  auto load_key = [&](int b) {
    const uint32_t i = (uint32_t)b * NT + tid;
    kr = i < n ? keys[bt.range.x + i] : (K)0;
    if (kBlk && i < n && !((bt.tmask[bt.range.x + i] >> bt.tbit) & 1u)) kr = kNone;
  };
  uint32_t none_bits = 0;        // kBlk: bit st set when this thread's entry of buffer st
                                 // does not cover the tile (nothing is staged for it with
                                 // cp.async; TMA stages its record anyway); it skips the tests
  auto issue = [&](int b) {
    const int st = b & 1;
    const uint32_t i = (uint32_t)b * NT + tid;
    if constexpr (kTma) {
      const bool mine = i < n && kr != kNone;
      const uint32_t r = mine ? (uint32_t)(kr & (K)rmask) : 0u;   // row 0 fills the tail
      none_bits = (none_bits & ~(1u << st)) | (mine ? 0u : (1u << st));
      if (kWeights) sm.rk[st][tid] = r;
      const uint32_t r1 = __shfl_down_sync(0xffffffffu, r, 1);
      const uint32_t r2 = __shfl_down_sync(0xffffffffu, r, 2);
      const uint32_t r3 = __shfl_down_sync(0xffffffffu, r, 3);
      if ((tid & 3) == 0 && !(bt.tma_skip && tid == 0)) {
        const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&sm.stage.bar[st]);
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&sm.stage.c[st][tid >> 2][0]);
        // the buffer was last read through the generic proxy (ordered by the CTA barrier)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_arrive(bar, 4u * kRec * 4u);
        tma_gather4(dst, bt.tmap, bar, r, r1, r2, r3);
      }
    } else {
      if (kBlk) none_bits = (none_bits & ~(1u << st)) | ((i < n && kr == kNone) ? (1u << st) : 0u);
      if (i < n && (!kBlk || kr != kNone)) {
        const uint32_t r = (uint32_t)(kr & (K)rmask);
        // block lists index the batch's 12-float records by (request, id); tile lists the
        // per-frame 16-float records by depth rank
        const float *rp = bt.rec_sorted + (size_t)r * (kBlk ? kRec : kRecS);
        cp_async16(&sm.stage.g0[st][tid], rp);
        cp_async16(&sm.stage.g1[st][tid], rp + 4);
        cp_async16(&sm.stage.g2[st][tid], rp + 8);
        if (kWeights) sm.rk[st][tid] = r;
      }
      cp_async_commit();
    }
  };
  // kTma: waits for buffer st's copies (bounded); false when the wait gave up
  auto wait_parity = [&](int st, uint32_t ph) -> bool {
    if constexpr (kTma) {
      const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&sm.stage.bar[st]);
      const uint32_t limit = bt.tma_spin ? bt.tma_spin : kTmaSpin;
      bool ok = false;
      for (uint32_t it = 0; it < limit && !ok; ++it) ok = mbar_try_wait(bar, ph);
      return ok;
    } else {
      return true;
    }
  };
  auto wait_buf = [&](int st) -> bool {
    const bool ok = wait_parity(st, (tma_ph >> st) & 1u);
    tma_ph ^= 1u << st;
    return ok;
  };
  // kTma: a stage wait gave up. Records kErrTimeout and settles the buffers whose copies may
  // be in flight (the one that timed out and, with in_flight, the other one): every thread
  // waits again (bounded) before the CTA leaves. Under the injected failure, whose phases lack
  // exactly thread 0's arrival, thread 0 supplies it first, so they complete once the copies
  // issued have landed and none is left in flight.
  auto give_up = [&](int st, bool in_flight) {
    if constexpr (kTma) {
      if (tid == 0) atomicOr(bt.err, kErrTimeout);
      for (int k = 0; k < (in_flight ? 2 : 1); ++k) {
        const int sb = k == 0 ? st : (st ^ 1);
        const uint32_t ph = ((tma_ph >> sb) & 1u) ^ 1u;   // the phase waited on (bit flipped)
        if (tid == 0 && bt.tma_skip)
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(
                           (uint32_t)__cvta_generic_to_shared(&sm.stage.bar[sb]))
                       : "memory");
        wait_parity(sb, ph);
      }
      cta_sync();
    }
  };
  // the three float4 of staged record j of buffer st
  auto staged = [&](int st, int j, float4 &a, float4 &b4, float4 &c) {
    if constexpr (kTma) {
      const float4 *q = reinterpret_cast<const float4 *>(&sm.stage.c[st][j >> 2][(j & 3) * 48]);
      a = q[0];
      b4 = q[1];
      c = q[2];
    } else {
      a = sm.stage.g0[st][j];
      b4 = sm.stage.g1[st][j];
      c = sm.stage.g2[st][j];
    }
  };

  // Evaluation of nh hits of stage buffer st in list order: get(k, h0, h1, h2) reads hit k's
  // record (h2.x the blue coefficient, h2.y the stage slot as an int); pos1 - 1 is the list
  // position of the buffer's slot 0. The paired loop reads each next record one hit ahead.
  auto run_hits = [&](int nh, int st, uint32_t pos1, auto get) {
    if constexpr (kPair) {
      float4 h0, h1;
      float2 h2;
      get(0, h0, h1, h2);
      for (int k = 0; k < nh; ++k) {
        float4 n0, n1;
        float2 n2;
        get(min(k + 1, 31), n0, n1, n2);
        // row terms (shared by the lane's pixels), log2 opacity folded into the constant term
        const float dy = __fsub_rn(h0.y, fpy);
        const float b2dy = __fmul_rn(h0.w, dy);
        const float c2l = __fmaf_rn(__fmul_rn(h1.x, dy), dy, h1.y);
        const float2 uu = make_float2(h0.x, h0.x), aa = make_float2(h0.z, h0.z);
        const float2 bd = make_float2(b2dy, b2dy), cl = make_float2(c2l, c2l);
        const float2 cr = make_float2(h1.z, h1.z), cg = make_float2(h1.w, h1.w);
        const float2 cb = make_float2(h2.x, h2.x);
#pragma unroll
        for (int q = 0; q < PH; ++q) {
          const float2 dx = __fadd2_rn(uu, npx2[q]);
          const float2 e = __ffma2_rn(dx, __ffma2_rn(aa, dx, bd), cl);
          // -alpha = -min(0.99, 2^e) where e >= log2(1/255), else -0 (the 0 that a 0/1 multiplier
          // would give; a select keeps it off the FMA pipe, the busiest here)
          const float2 na = make_float2(
              e.x >= kLog2AlphaMin ? fmaxf(-kAlphaMax, -ex2_approx(e.x)) : -0.f,
              e.y >= kLog2AlphaMin ? fmaxf(-kAlphaMax, -ex2_approx(e.y)) : -0.f);
          const float2 nw = __fmul2_rn(na, T2[q]);          // -alpha T
          const float2 nT = __fadd2_rn(T2[q], nw);          // T - alpha T
          // the entry that takes T below 1e-4 stops the pixel and blends nothing. T never
          // grows (T - alpha T <= T), so it keeps being updated: every later entry finds
          // T - alpha T below 1e-4 as well and blends nothing, as a stopped pixel must. A
          // select on the test keeps the colour weight's product off the FMA pipe.
          const bool k0 = nT.x >= kTStop, k1 = nT.y >= kTStop;
          const float2 nwi = make_float2(k0 ? nw.x : 0.f, k1 ? nw.y : 0.f);   // -(weight)
          C02[q] = __ffma2_rn(cr, nwi, C02[q]);     // the negated colour sums
          C12[q] = __ffma2_rn(cg, nwi, C12[q]);
          C22[q] = __ffma2_rn(cb, nwi, C22[q]);
          T2[q] = nT;
        }
        h0 = n0;
        h1 = n1;
        h2 = n2;
      }
    } else {
      for (int k = 0; k < nh; ++k) {
        float4 h0, h1;
        float2 h2;
        get(k, h0, h1, h2);
        // the row terms of the exponent are shared by the lane's pixels
        const float dy = __fsub_rn(h0.y, fpy);
        const float b2dy = __fmul_rn(h0.w, dy);
        const float c2l = __fmaf_rn(__fmul_rn(h1.x, dy), dy, h1.y);
        float w = 0.f;
#pragma unroll
        for (int p = 0; p < PX; ++p) {
          const float dx = __fsub_rn(h0.x, (float)(px0 + p * HW));
          const float e = __fmaf_rn(dx, __fmaf_rn(h0.z, dx, b2dy), c2l);
          if constexpr (kTz) {
            const bool valid = e >= kLog2AlphaMin;
            const float alpha = valid ? fminf(kAlphaMax, ex2_approx(e)) : 0.f;
            const float wa = alpha * T[p];
            const float nT = T[p] - wa;
            // T keeps being updated after the stop: it never grows, so every later entry
            // fails the test too and blends nothing
            const bool stop = nT < kTStop;
            const float wi = stop ? 0.f : wa;
            C0[p] = fmaf(h1.z, wi, C0[p]);
            C1[p] = fmaf(h1.w, wi, C1[p]);
            C2[p] = fmaf(h2.x, wi, C2[p]);
            T[p] = nT;
            continue;
          }
          const bool valid = !done[p] && e >= kLog2AlphaMin;
          if (kCount && !done[p]) ++nevals;
          if (kCount && valid) ++npass;
          const float alpha = valid ? fminf(kAlphaMax, ex2_approx(e)) : 0.f;
          // Eq. 2's transmittance step T (1 - alpha), taken as T - alpha T: the weight alpha T
          // is needed anyway, so this saves the subtraction 1 - alpha
          const float wa = alpha * T[p];
          const float nT = T[p] - wa;
          // only a valid entry can stop a pixel: an unfinished pixel has T >= kTStop
          const bool stop = nT < kTStop;
          // the entry that ends this pixel's list: the key-frame masks keep it
          if (kWeights && stop) bt.stop_mark[sm.rk[st][__float_as_int(h2.y)]] = 1u;
          done[p] = done[p] || stop;
          const bool use = valid && !stop;
          const float wi = stop ? 0.f : wa;
          C0[p] = fmaf(h1.z, wi, C0[p]);
          C1[p] = fmaf(h1.w, wi, C1[p]);
          C2[p] = fmaf(h2.x, wi, C2[p]);
          T[p] = use ? nT : T[p];
          if (kAux) last[p] = use ? pos1 + (uint32_t)__float_as_int(h2.y) : last[p];
          if (kWeights) w += wi;
        }
        if (kWeights) {
          if (__any_sync(0xffffffffu, w != 0.f)) {
            const float s = warp_sum(w);
            if (lane == 0) atomicAdd(&bt.w_sum[sm.rk[st][__float_as_int(h2.y)]], s);
          }
        }
      }
    }
  };
  auto check_done = [&] {
    lane_done = true;
#pragma unroll
    for (int p = 0; p < PX; ++p) {
      if constexpr (kPair)
        lane_done = lane_done && ((p & 1) ? T2[p >> 1].y : T2[p >> 1].x) < kTStop;
      else
        lane_done = lane_done && (kTz ? T[p] < kTStop : done[p]);
    }
    warp_done = __all_sync(0xffffffffu, lane_done);
  };

  if constexpr (kCompact) {
    // ring of the tile's hits, filled 128 list positions at a time while fewer than 32 wait:
    // at most 159 are held, so a slot is rewritten only after its stage has read it
    constexpr uint32_t kRing = 256;
    uint32_t sp = 0, rh = 0, rt = 0;   // list positions scanned; ring entries read, written
    auto refill = [&] {
      while (rt - rh < 32u && sp < n) {
        uint32_t kk[4], tw[4];
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          const uint32_t i = sp + (uint32_t)(32 * g) + (uint32_t)lane;
          kk[g] = i < n ? keys[bt.range.x + i] : (K)0;
          tw[g] = i < n ? bt.tmask[bt.range.x + i] : 0u;
        }
        // the entries with the tile's bit, in list order
        uint32_t nc = 0;
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          const bool cv = (tw[g] >> bt.tbit) & 1u;
          const uint32_t bm = __ballot_sync(0xffffffffu, cv);
          if (cv) sm.cand[nc + __popc(bm & lanemask_lt())] = (uint32_t)(kk[g] & (K)rmask);
          nc += __popc(bm);
        }
        sp += 128;
        __syncwarp();
        // their tile tests, 32 at a time; the hits go to the ring in order
        for (uint32_t c0 = 0; c0 < nc; c0 += 32) {
          bool hit = false;
          uint32_t r = 0;
          if (c0 + (uint32_t)lane < nc) {
            if (kCount) ++ntests;
            r = sm.cand[c0 + lane];
            const float4 *rp = reinterpret_cast<const float4 *>(bt.rec_sorted + (size_t)r * kRec);
            const float4 g0 = __ldg(rp), g1 = __ldg(rp + 1), g2 = __ldg(rp + 2);
            hit = may_hit_rect(g0, g1.x, g1.y, g2.y, g2.z, tx0, tx0 + (kTile - 1), ty0,
                               ty0 + (kTile - 1));
          }
          const uint32_t bm = __ballot_sync(0xffffffffu, hit);
          if (hit) sm.ring[(rt + __popc(bm & lanemask_lt())) & (kRing - 1)] = r;
          rt += __popc(bm);
        }
        __syncwarp();                    // the candidates are rewritten by the next scan
      }
    };
    // stages the next (up to) 32 ring entries into buffer st; one commit group each call
    auto issue_c = [&](int st) -> int {
      const uint32_t c = min(32u, rt - rh);
      if ((uint32_t)lane < c) {
        const uint32_t r = sm.ring[(rh + lane) & (kRing - 1)];
        const float *rp = bt.rec_sorted + (size_t)r * kRec;
        cp_async16(&sm.stage.g0[st][lane], rp);
        cp_async16(&sm.stage.g1[st][lane], rp + 4);
        cp_async16(&sm.stage.g2[st][lane], rp + 8);
        if (kWeights) sm.rk[st][lane] = r;
      }
      cp_async_commit();
      rh += c;
      return (int)c;
    };
    refill();
    int cnt = issue_c(0);
    refill();
    for (int b = 0; cnt > 0 && !warp_done; ++b) {
      const int st = b & 1;
      const int cnt_next = issue_c(st ^ 1);
      cp_async_wait<1>();
      __syncwarp();
      run_hits(cnt, st, 0u, [&](int k, float4 &a, float4 &b4, float2 &c) {
        a = sm.stage.g0[st][k];
        b4 = sm.stage.g1[st][k];
        c = make_float2(sm.stage.g2[st][k].x, __int_as_float(k));
      });
      check_done();
      if (!warp_done) refill();          // the entries of the stage after the next
      __syncwarp();                      // buffer st is staged into again by the next call
      cnt = cnt_next;
    }
    cp_async_wait<0>();
  } else {
  if (nb > 0) {
    load_key(0);
    issue(0);
    if (nb > 1) load_key(1);
  }
  for (int b = 0; b < nb; ++b) {
    if (b + 1 < nb) {
      issue(b + 1);
      if (b + 2 < nb) load_key(b + 2);
      if constexpr (!kTma) cp_async_wait<1>();
    } else {
      if constexpr (!kTma) cp_async_wait<0>();
    }
    if constexpr (kTma) {
      // every thread waits for the buffer's copies; a wait that gives up ends the tile (and
      // the CTA's work) after the other buffer's copies, if any are in flight, are waited for
      const bool ok = wait_buf(b & 1);
      if (cta_or(!ok)) {
        if (b + 1 < nb) tma_ph ^= 1u << ((b + 1) & 1);   // its phase is settled below
        give_up(b & 1, b + 1 < nb);
        return false;
      }
    } else {
      cta_sync();
    }
    const int st = b & 1;
    const int cnt = (int)min((uint32_t)NT, n - (uint32_t)b * NT);
    const uint32_t pos1 = (uint32_t)b * NT + 1;
    // 1. tile-level test of the thread's own staged Gaussian, block compaction
    bool keep = false;
    if (kCount && tid < cnt) ++ntests;
    if (tid < cnt && !(kBlk && ((none_bits >> st) & 1u))) {
      float4 g0, g1, g2;
      staged(st, tid, g0, g1, g2);
      keep = may_hit_rect(g0, g1.x, g1.y, g2.y, g2.z, tx0, tx0 + (kTile - 1), ty0,
                          ty0 + (kTile - 1));
    }
    // survivors are compacted per warp: warp w's in idx[32 w, 32 w + wcnt[w]), so one barrier
    // publishes them; the list of all survivors in rank order is the warps' segments in turn
    const uint32_t kb = __ballot_sync(0xffffffffu, keep);
    if (keep) sm.idx[warp * 32 + __popc(kb & lanemask_lt())] = (uint16_t)tid;
    if (lane == 0) sm.wcnt[warp] = __popc(kb);
    cta_sync();
    int seg0[NT / 32];               // first survivor position of each warp's segment
    int ncomp = 0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) {
      seg0[w] = ncomp;
      ncomp += (int)sm.wcnt[w];
    }
    // 2. warp footprint tests on the survivors, evaluation of the hits
    for (int c0 = 0; c0 < ncomp && !warp_done; c0 += 32) {
      bool hit = false;
      int j = 0;
      float4 g0, g1, g2;
      if (kCount && !kWholeTile && c0 + lane < ncomp) ++ntests;
      if (c0 + lane < ncomp) {
        const int pos = c0 + lane;
        int slot = pos;                // in warp 0's segment, else in the last one it reaches
#pragma unroll
        for (int v = 1; v < NT / 32; ++v) slot = pos >= seg0[v] ? v * 32 + pos - seg0[v] : slot;
        j = sm.idx[slot];
        staged(st, j, g0, g1, g2);
        hit = kWholeTile || may_hit_rect(g0, g1.x, g1.y, g2.y, g2.z, fxl, fxh, fyl, fyh);
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
      run_hits(nh, st, pos1, [&](int k, float4 &a, float4 &b4, float2 &c) {
        a = sm.h0[warp][k];
        b4 = sm.h1[warp][k];
        c = sm.h2[warp][k];
      });
      __syncwarp();                    // the list is rewritten by the next round
      check_done();
    }
    if (cta_and(warp_done)) {
      if constexpr (kTma) {
        // the next buffer's copies are in flight: consume its phase before leaving
        if (b + 1 < nb && cta_or(!wait_buf((b + 1) & 1))) {
          give_up((b + 1) & 1, false);
          return false;
        }
      } else {
        cp_async_wait<0>();
      }
      break;
    }
  }
  }
  if (kCount) {
    const uint32_t ws = warp_sum(nevals), wt = warp_sum(ntests), wp = warp_sum(npass);
    if (lane == 0 && ws) atomicAdd(&bt.evals[0], (unsigned long long)ws);
    if (lane == 0 && wt) atomicAdd(&bt.evals[1], (unsigned long long)wt);
    if (lane == 0 && wp) atomicAdd(&bt.evals[2], (unsigned long long)wp);
  }
  if constexpr (kPair) {
#pragma unroll
    for (int q = 0; q < PH; ++q) {
      T[2 * q] = T2[q].x;
      T[2 * q + 1] = T2[q].y;
      C0[2 * q] = -C02[q].x;
      C0[2 * q + 1] = -C02[q].y;
      C1[2 * q] = -C12[q].x;
      C1[2 * q + 1] = -C12[q].y;
      C2[2 * q] = -C22[q].x;
      C2[2 * q + 1] = -C22[q].y;
    }
  }
  const size_t hw = (size_t)bt.W * bt.H;
#pragma unroll
  for (int p = 0; p < PX; ++p) {
    const int px = px0 + p * HW;
    if (px < bt.W && py < bt.H) {
      const size_t pix = (size_t)py * bt.W + px;
      bt.rgb[pix] = C0[p] + T[p] * bt.bg0;
      bt.rgb[hw + pix] = C1[p] + T[p] * bt.bg1;
      bt.rgb[2 * hw + pix] = C2[p] + T[p] * bt.bg2;
      if (kAux) {
        bt.T_final[pix] = T[p];
        bt.n_contrib[pix] = last[p];
      }
    }
  }
  return true;
}

}  // namespace fdgs
