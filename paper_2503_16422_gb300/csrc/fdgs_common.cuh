// Shared device definitions of the GB300 4D Gaussian rasterizer.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fdgs {

// Blending thresholds of the 3DGS-family renderer the paper builds on (Sec. 3, Eq. 2 and
// Eq. 3 give only the compositing sum; these constants are the renderer's).
constexpr float kAlphaMin = 1.0f / 255.0f;   // alpha below this is skipped
constexpr float kAlphaMax = 0.99f;           // alpha is clamped to this
constexpr float kTStop = 1e-4f;              // stop before transmittance drops below this
constexpr float kDilation = 0.3f;            // px^2 added to the 2D covariance diagonal
constexpr float kFovClamp = 1.3f;            // Jacobian clamp, times tan(fov/2)
constexpr float kRadiusFloor = 0.1f;         // floor of the eigenvalue discriminant
constexpr int kTile = 16;                    // gating tile side (pixels)
constexpr int kTilePixels = kTile * kTile;

// Device error bits (scene status word).
constexpr uint32_t kErrTimeout = 1u;
constexpr uint32_t kErrCapacity = 2u;

// Spin-wait limit of every decoupled look-back (iterations of roughly 0.1-1 us each). Once
// any waiter gives up it sets kErrTimeout in the error word, and every other waiter that
// sees the bit gives up too, so a broken protocol costs one limit in total, not one per wait.
constexpr uint32_t kSpinLimit = 1u << 20;

// Per-Gaussian decision flags (exported for tests).
constexpr uint8_t kFlagMask = 1, kFlagTemporal = 2, kFlagNear = 4, kFlagDet = 8,
                  kFlagVisible = 16;

// Record of a projected Gaussian, 12 floats (48 B): the per-frame state the blend reads.
constexpr int kRec = 12;
enum RecField { R_U = 0, R_V, R_A, R_B, R_C, R_OPA, R_R, R_G, R_BL, R_DEPTH, R_RADIUS, R_COUNT };

struct DevCam {
  float R[9];       // world->camera rotation, row-major
  float tv[3];      // world->camera translation
  float eye[3];     // camera centre in world coordinates (-R^T tv)
  float fx, fy, cx, cy;
  float limx, limy; // Jacobian clamp limits (1.3 tan(fov/2))
  float znear;
  int W, H, gx, gy;
};

// Counters kept on the device for one frame.
enum Counter {
  C_NVIS = 0,      // visible Gaussians (u32)
  C_NACTIVE = 1,   // Gaussians through the mask gate (u32)
  C_NKEYS_LO = 2,  // number of keys (u64 split in two words)
  C_NKEYS_HI = 3,
  C_ERR = 4,       // device error bits of this frame
  C_PART0 = 8,     // partition counters of persistent kernels (8..31)
  C_COUNT = 32
};

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ void nanosleep_ns(uint32_t ns) { __nanosleep(ns); }

// Volatile (L2-coherent) 64-bit load/store for look-back status words.
__device__ __forceinline__ uint64_t ld_volatile_u64(const uint64_t *p) {
  uint64_t v;
  asm volatile("ld.volatile.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_volatile_u64(uint64_t *p, uint64_t v) {
  asm volatile("st.volatile.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_volatile_u32(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.volatile.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_volatile_u32(uint32_t *p, uint32_t v) {
  asm volatile("st.volatile.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Status word of a single-value decoupled look-back: 2-bit flag in the top bits.
constexpr uint64_t kLbAgg = 1ull << 62, kLbPrefix = 2ull << 62, kLbValue = (1ull << 62) - 1;

template <typename T>
__device__ __forceinline__ T warp_sum(T v);

// Look-back of partition `part` with aggregate `agg`, walked by a whole warp (all 32 lanes
// call it; every decision is uniform over the warp). Lane 0 publishes the aggregate; the
// lanes read the status words of 32 predecessors at once (partitions j, j - 1, ..., j - 31),
// so the walk back to the nearest inclusive prefix takes one L2 round trip per 32 of them;
// a predecessor that has not published yet is waited for (bounded spin). Lane 0 publishes
// the inclusive prefix; every lane returns the exclusive one. On timeout sets kErrTimeout and
// returns the partial sum, so that every waiting successor still terminates.
__device__ __forceinline__ uint64_t lookback_warp(uint64_t *status, uint32_t part,
                                                  uint64_t agg, uint32_t *err) {
  const uint32_t lane = lane_id();
  if (part == 0) {
    if (lane == 0) st_volatile_u64(&status[0], kLbPrefix | agg);
    return 0;
  }
  if (lane == 0) st_volatile_u64(&status[part], kLbAgg | agg);
  uint64_t excl = 0;
  int64_t j = (int64_t)part - 1;   // the nearest predecessor not summed yet
  uint32_t spins = 0;
  for (;;) {
    const int64_t jj = j - (int64_t)lane;
    // before partition 0 the prefix is 0
    const uint64_t s = jj >= 0 ? ld_volatile_u64(&status[jj]) : kLbPrefix;
    const uint64_t f = s & ~kLbValue;
    const uint32_t nr = __ballot_sync(0xffffffffu, f == 0);
    const uint32_t pf = __ballot_sync(0xffffffffu, f == kLbPrefix);
    const int first_nr = nr ? __ffs(nr) - 1 : 32;
    const int first_pf = pf ? __ffs(pf) - 1 : 32;
    if (first_pf < first_nr) {
      // aggregates up to the nearest inclusive prefix, which ends the walk
      excl += warp_sum<uint64_t>((int)lane <= first_pf ? (s & kLbValue) : 0ull);
      break;
    }
    // the aggregates before the nearest partition that has not published yet
    excl += warp_sum<uint64_t>((int)lane < first_nr ? (s & kLbValue) : 0ull);
    j -= first_nr;
    if (first_nr < 32) {
      const bool give_up =
          ++spins > kSpinLimit || ((spins & 255) == 0 && (ld_volatile_u32(err) & kErrTimeout));
      if (__any_sync(0xffffffffu, give_up)) {
        if (lane == 0) atomicOr(err, kErrTimeout);
        break;
      }
      nanosleep_ns(32);
    }
  }
  if (lane == 0) st_volatile_u64(&status[part], kLbPrefix | (excl + agg));
  return excl;
}

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T n = __shfl_up_sync(0xffffffffu, v, o);
    if ((int)lane_id() >= o) v += n;
  }
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Tile rectangle [xmin, xmax) x [ymin, ymax) of a Gaussian with image centre (u, v) and
// integer radius r: floor((u - r) / 16) .. floor((u + r + 15) / 16), clamped to the grid.
// Used by the per-Gaussian stage and again by key emission; identical float operations.
__device__ __forceinline__ void tile_rect(float u, float v, float r, int gx, int gy,
                                          int &xmin, int &ymin, int &xmax, int &ymax) {
  const float inv = 1.0f / kTile;
  float x0 = floorf(__fmul_rn(__fsub_rn(u, r), inv));
  float y0 = floorf(__fmul_rn(__fsub_rn(v, r), inv));
  float x1 = floorf(__fmul_rn(__fadd_rn(__fadd_rn(u, r), (float)(kTile - 1)), inv));
  float y1 = floorf(__fmul_rn(__fadd_rn(__fadd_rn(v, r), (float)(kTile - 1)), inv));
  xmin = (int)fminf(fmaxf(x0, 0.f), (float)gx);
  ymin = (int)fminf(fmaxf(y0, 0.f), (float)gy);
  xmax = (int)fminf(fmaxf(x1, 0.f), (float)gx);
  ymax = (int)fminf(fmaxf(y1, 0.f), (float)gy);
}

// ---- blend-ready record (depth-rank order), 16 floats = 64 B -----------------------------
// [0..3]  u, v, a2 = -A/2 log2(e), b2 = -B log2(e)       (image centre, scaled conic)
// [4..7]  c2 = -C/2 log2(e), lga = log2(a), r, g        (a = sigmoid(o) p(t))
// [8..11] b, kx = -b2 / (2 a2), ky = -b2 / (2 c2), radius
// [12..15] A, B, C, a                                   (raw conic and opacity: backward, and
//                                                        the alpha-tight tile sets)
constexpr int kRecS = 16;
constexpr int kRecSRadius = 11;
// Footprint culling margin (log2 units): a Gaussian is culled for a pixel footprint only if
// its largest exponent over the footprint rectangle is below log2(1/255) by more than this,
// far beyond float32 rounding of the per-pixel exponent, so per-pixel decisions never change.
constexpr float kCullMargin = 0.01f;

// Largest value of q(d) = a2 dx^2 + b2 dx dy + c2 dy^2 (a concave quadratic) over the
// rectangle of offsets d in [dxl, dxh] x [dyl, dyh]: 0 if the rectangle holds d = 0, else
// the best of its four edges (on each edge the 1D maximiser, kx*Y or ky*X, clamped).
__device__ __forceinline__ float quad_max_rect(float a2, float b2, float c2, float kx, float ky,
                                               float dxl, float dxh, float dyl, float dyh) {
  if (dxl <= 0.f && dxh >= 0.f && dyl <= 0.f && dyh >= 0.f) return 0.f;
  float best = -INFINITY;
  {
    const float dy = fminf(fmaxf(ky * dxl, dyl), dyh);
    best = fmaxf(best, dxl * (a2 * dxl + b2 * dy) + c2 * dy * dy);
  }
  {
    const float dy = fminf(fmaxf(ky * dxh, dyl), dyh);
    best = fmaxf(best, dxh * (a2 * dxh + b2 * dy) + c2 * dy * dy);
  }
  {
    const float dx = fminf(fmaxf(kx * dyl, dxl), dxh);
    best = fmaxf(best, dx * (a2 * dx + b2 * dyl) + c2 * dyl * dyl);
  }
  {
    const float dx = fminf(fmaxf(kx * dyh, dxl), dxh);
    best = fmaxf(best, dx * (a2 * dx + b2 * dyh) + c2 * dyh * dyh);
  }
  return best;
}
// Coverage words of one warp's 32 ranks: for each row r < n, bit `lane` of word r is set when
// the lane's interval [lo, hi) holds r; word r goes to dst[r * stride]. One ballot per row;
// lane k keeps the word of row 32 c + k and stores it once per 32 rows.
__device__ __forceinline__ void warp_coverage_words(int lo, int hi, int n, uint32_t *dst,
                                                    size_t stride) {
  const uint32_t lane = lane_id();
  const uint32_t span = (uint32_t)max(hi - lo, 0);
  for (int c = 0; c < n; c += 32) {
    uint32_t mine = 0;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      const uint32_t bb = __ballot_sync(0xffffffffu, (uint32_t)(c + k - lo) < span);
      if (lane == (uint32_t)k) mine = bb;
    }
    if (c + (int)lane < n) dst[(size_t)(c + lane) * stride] = mine;
  }
}

// Alpha-tight tile set (the batched path always; the per-frame API on request): a pixel p of
// the 3-sigma square can only take alpha >= 1/255 from the Gaussian where its exponent
// reaches log2(1/255), i.e. inside
// the ellipse d^T Sigma^-1 d <= 2 ln(255 a), d = p - (u, v), whose bounding box has
// half-widths sqrt(Q Sigma_xx), sqrt(Q Sigma_yy). The box (Q widened by 0.1% + 0.1, far more
// than the float error of the blend's exponent) is intersected with the square's tiles
// [x0, x1) x [y0, y1); every (pixel, Gaussian) pair the blend would composite keeps its
// tile, so images are unchanged. Conic A, B, C = Sigma^-1; a = opacity x temporal weight.
__device__ __forceinline__ void tighten_rect(float u, float v, float A, float B, float C, float a,
                                             int &x0, int &y0, int &x1, int &y1) {
  const float det = A * C - B * B;
  if (!(det > 0.f)) return;                 // degenerate conic: keep the square
  const float Q = 2.f * logf(255.f * a) * 1.001f + 0.1f;
  if (!(Q > 0.f)) {
    x1 = x0;
    y1 = y0;
    return;
  }
  const float hx = sqrtf(Q * C / det), hy = sqrtf(Q * A / det);
  const float inv = 1.f / (float)kTile;
  x0 = max(x0, (int)floorf((u - hx) * inv));
  x1 = min(x1, (int)floorf((u + hx) * inv) + 1);
  y0 = max(y0, (int)floorf((v - hy) * inv));
  y1 = min(y1, (int)floorf((v + hy) * inv) + 1);
}

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLog2AlphaMin = -7.9943534368588578f;   // log2(1/255)

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// The exponent of one (Gaussian, pixel) pair from the blend-ready record. The forward blend
// (blend_tile) and the backward replay (k_blend_bwd) evaluate it with the same explicit
// rounding, so both take the same decisions bit for bit:
//   dy = v - py, b2dy = b2 dy, c2l = fma(c2 dy, dy, log2(a))   (row terms, once per pixel row)
//   dx = u - px, e = fma(dx, fma(a2, dx, b2dy), c2l)
// with d = mean2D - pixel and e = log2(a exp(power)), power = -1/2 (A dx^2 + 2 B dx dy +
// C dy^2). The pair is skipped when e puts a exp(power) below 1/255; otherwise alpha =
// min(0.99, 2^e). The renderer's "power > 0 is skipped" rule needs no test: the conic is the
// inverse of J Sigma J^T + 0.3 I, positive definite by construction, so power <= 0 exactly,
// and a float32 power that rounds above 0 belongs to an exact power within rounding of 0,
// which the reference rule would blend (alpha = a to within that rounding). (Written out in
// both kernels: factored into helper functions the same arithmetic compiled 12% slower in the
// persistent blend.)

}  // namespace fdgs
