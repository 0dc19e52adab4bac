// Spatial-Temporal Variation Score helpers (Sec. 4.2.1, Eqs. 4-7), pruning keep-set, and
// frame export kernels.
#include <algorithm>

#include "fdgs_gauss.cuh"
#include "fdgs_internal.h"

namespace fdgs {

namespace {

constexpr int kB = 256;

int grid_for(uint64_t n, int per_sm = 16) {
  return (int)std::max<uint64_t>(1, std::min<uint64_t>((n + kB - 1) / kB,
                                                        (uint64_t)num_sms() * per_sm));
}

template <typename K>
__global__ void k_keys_to_ids(const K *__restrict__ keys, uint32_t nkeys, uint32_t rmask,
                              const uint64_t *__restrict__ sorted, uint32_t *__restrict__ ids) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nkeys; i += gridDim.x * blockDim.x)
    ids[i] = (uint32_t)sorted[(uint32_t)(keys[i] & (K)rmask)];
}

__global__ void k_export_records(const uint64_t *__restrict__ sorted, uint32_t nv,
                                 const float *__restrict__ rec, float *__restrict__ out) {
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < nv; r += gridDim.x * blockDim.x) {
    const uint32_t id = (uint32_t)sorted[r];
    for (int k = 0; k < kRec; ++k) out[(size_t)id * kRec + k] = rec[(size_t)id * kRec + k];
  }
}

__global__ void k_volume_bits(const float4 *__restrict__ ls4, uint32_t n, uint32_t *vbits) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float4 l = ls4[i];
    vbits[i] = __float_as_uint(expf(l.x + l.y + l.z + l.w));
  }
}

// Per-Gaussian constants of the score pass, once per pass: gamma_i = clamp(V_i / V_p90, 0,
// 1)^0.1 (V_p90 = vsorted[k]) and the temporal variance Sigma_t,i = |row t of R diag(s)|^2 in
// FP64. f_i(t) (Eqs. 5-6) takes the difference (t - mu_t)^2 / Sigma_t - 1, which cancels at
// the inflection points of p(t): there a float32 Sigma_t (a sum of four products after two
// quaternion normalisations and four exponentials, a few ulps off) would move f by up to 1e-3
// relative for short-lived Gaussians (Sigma_t ~ 3e-4), so Sigma_t is formed in FP64 from the
// float32 attributes, once per Gaussian.
__global__ void k_score_consts(const float4 *__restrict__ ls4, const float4 *__restrict__ ql,
                               const float4 *__restrict__ qr, uint32_t n,
                               const uint32_t *__restrict__ vsorted, uint32_t k, float *gamma,
                               double *sig_t) {
  const float vref = __uint_as_float(vsorted[k]);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float4 l = ls4[i];
    const float v = expf(l.x + l.y + l.z + l.w);
    const float x = fminf(fmaxf(v / vref, 0.f), 1.f);
    gamma[i] = powf(x, 0.1f);
    const float4 a4 = ql[i], b4 = qr[i];
    const double na = rsqrt((double)a4.x * a4.x + (double)a4.y * a4.y + (double)a4.z * a4.z +
                            (double)a4.w * a4.w);
    const double nb = rsqrt((double)b4.x * b4.x + (double)b4.y * b4.y + (double)b4.z * b4.z +
                            (double)b4.w * b4.w);
    // row t of the left-multiplication matrix of q_l = (a, b, c, d): (d, -c, b, a)
    const double L3[4] = {a4.w * na, -a4.z * na, a4.y * na, a4.x * na};
    // the right-multiplication matrix of q_r = (p, x, r, s), row-major
    const double p_ = b4.x * nb, x_ = b4.y * nb, r_ = b4.z * nb, s_ = b4.w * nb;
    const double R[16] = {p_, -x_, -r_, -s_, x_, p_, s_, -r_, r_, -s_, p_, x_, s_, r_, -x_, p_};
    const double sc[4] = {exp((double)l.x), exp((double)l.y), exp((double)l.z),
                          exp((double)l.w)};
    double acc = 0.0;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      double e = 0.0;
#pragma unroll
      for (int j = 0; j < 4; ++j) e = fma(L3[j], R[j * 4 + m], e);
      e *= sc[m];
      acc = fma(e, e, acc);
    }
    sig_t[i] = acc;
  }
}

// f_i(t) of Eqs. 5-6: the second time derivative of the temporal opacity p_i(t) =
// exp(-(t - mu_t)^2 / (2 Sigma_t)), p'' = ((t - mu_t)^2 / Sigma_t - 1) / Sigma_t p, mapped
// through tanh into [1, 2] (its reciprocal half-plus-half form). The difference is taken in
// FP64 (t - mu_t is exact there); p and tanh are float32.
__device__ __forceinline__ float variation_factor(float t, float mu_t, double st) {
  const double dt = (double)t - (double)mu_t;
  const double inv = 1.0 / st;
  const double x = dt * dt * inv;
  const float p = expf(-0.5f * (float)x);
  const float p2 = (float)((x - 1.0) * inv) * p;
  return 1.f / (0.5f * tanhf(fabsf(p2)) + 0.5f);
}

// The factor of score variant (d) of the ablation (Table 4): p^(1)(t) = -(t - mu_t) / Sigma_t
// p(t) in place of p^(2) in Eq. 6.
__device__ __forceinline__ float variation_factor_d1(float t, float mu_t, double st) {
  const double dt = (double)t - (double)mu_t;
  const float p = expf(-0.5f * (float)(dt * dt / st));
  const float p1 = -(float)(dt / st) * p;
  return 1.f / (0.5f * tanhf(fabsf(p1)) + 0.5f);
}

// The per-(Gaussian, t) factor that multiplies the blend weight w_i(t, view) in each rendered
// score variant (fdgs_score_variant): f gamma (Eq. 7, ours), 1 (spatial only), f1 gamma
// (p^(1) in place of p^(2)), Sigma_t gamma (Sigma_t in place of S^TV).
__device__ __forceinline__ float score_factor(int variant, float t, float mu_t, double st,
                                              float gamma) {
  switch (variant) {
    case 1: return 1.f;
    case 3: return variation_factor_d1(t, mu_t, st) * gamma;
    case 4: return (float)st * gamma;
    default: return variation_factor(t, mu_t, st) * gamma;
  }
}

__global__ void k_score_accumulate(const uint64_t *__restrict__ sorted,
                                   const uint32_t *__restrict__ nv_dev,
                                   const float *__restrict__ w_sum,
                                   const float4 *__restrict__ mean4,
                                   const double *__restrict__ sig_t,
                                   const float *__restrict__ gamma, float t, float *score,
                                   int variant) {
  const uint32_t nv = *nv_dev;
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < nv; r += gridDim.x * blockDim.x) {
    const float w = w_sum[r];
    if (w == 0.f) continue;
    const uint32_t id = (uint32_t)sorted[r];
    score[id] += w * score_factor(variant, t, mean4[id].w, sig_t[id], gamma[id]);
  }
}

// Temporal-only score (variant (c) of Table 4): S_i += f_i(t) gamma_i for one t, no render.
__global__ void k_score_temporal(const float4 *__restrict__ mean4,
                                 const double *__restrict__ sig_t,
                                 const float *__restrict__ gamma, uint32_t n, float t,
                                 float *score) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    score[i] += variation_factor(t, mean4[i].w, sig_t[i]) * gamma[i];
}

// The batched score pass: the weight of Gaussian i over the pixels of request r sits at
// record index r n + i; it is added to the score with the request's f_i(t) (the requests of
// one batch share Gaussians, hence the atomics).
__global__ void k_score_batch(BatchDev b) {
  const uint64_t total = (uint64_t)b.nreq * b.n;
  for (uint64_t ri = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; ri < total;
       ri += (uint64_t)gridDim.x * blockDim.x) {
    const float w = b.w_sum[ri];
    if (w == 0.f) continue;
    const uint32_t r = (uint32_t)(ri / b.n), id = (uint32_t)(ri % b.n);
    atomicAdd(&b.score[id], w * score_factor(b.score_variant, b.reqs[r].t, b.mean4[id].w,
                                             b.sig_t[id], b.gamma[id]));
  }
}

// The batched mask pass: the contributors of each request (blended at one pixel at least, or
// stopped a pixel) set their bits in the request's key-frame row.
__global__ void k_mark_batch(BatchDev b) {
  const uint64_t total = (uint64_t)b.nreq * b.n;
  for (uint64_t ri = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; ri < total;
       ri += (uint64_t)gridDim.x * blockDim.x) {
    if (!(b.w_sum[ri] > 0.f) && !b.stop_mark[ri]) continue;
    const uint32_t r = (uint32_t)(ri / b.n), id = (uint32_t)(ri % b.n);
    uint32_t *row = b.reqs[r].mark_row;
    if (row) atomicOr(&row[id >> 5], 1u << (id & 31));
  }
}

// Visibility mask of one view (Sec. 4.2.2): every visible rank blended at one pixel at least
// (positive blend weight) or that stopped a pixel sets its Gaussian's bit in the word row.
__global__ void k_mark_contributors(const uint64_t *__restrict__ sorted,
                                    const uint32_t *__restrict__ nv_dev,
                                    const float *__restrict__ w_sum,
                                    const uint32_t *__restrict__ stop_mark, uint32_t *row) {
  const uint32_t nv = *nv_dev;
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < nv; r += gridDim.x * blockDim.x) {
    if (!(w_sum[r] > 0.f) && !stop_mark[r]) continue;
    const uint32_t id = (uint32_t)sorted[r];
    atomicOr(&row[id >> 5], 1u << (id & 31));
  }
}

// Word row -> packed bytes, LSB first: byte b holds bits 8b .. 8b + 7.
__global__ void k_pack_mask_row(const uint32_t *__restrict__ row, uint32_t nbytes,
                                uint8_t *__restrict__ out) {
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < nbytes;
       b += gridDim.x * blockDim.x)
    out[b] = (uint8_t)(row[b >> 2] >> ((b & 3) * 8));
}

__global__ void k_score_keys(const float *__restrict__ score, uint32_t n, uint64_t *keys) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    keys[i] = ((uint64_t)__float_as_uint(score[i]) << 32) | i;
}

// The id bounds check only matters after a sort whose look-back gave up (its output can hold
// stale keys); a complete sort is a permutation of 0..n-1.
__global__ void k_keep_from_sorted(const uint64_t *__restrict__ sorted, uint32_t n,
                                   uint32_t n_drop, uint8_t *keep) {
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const uint32_t id = (uint32_t)sorted[j];
    if (id < n) keep[id] = j >= n_drop ? 1 : 0;
  }
}

}  // namespace

template <typename K>
void launch_keys_to_ids(const K *keys, uint32_t nkeys, uint32_t rmask, const uint64_t *sorted,
                        uint32_t *ids, cudaStream_t st) {
  if (nkeys == 0) return;
  k_keys_to_ids<K><<<grid_for(nkeys), kB, 0, st>>>(keys, nkeys, rmask, sorted, ids);
}
template void launch_keys_to_ids<uint32_t>(const uint32_t *, uint32_t, uint32_t,
                                           const uint64_t *, uint32_t *, cudaStream_t);
template void launch_keys_to_ids<uint64_t>(const uint64_t *, uint32_t, uint32_t,
                                           const uint64_t *, uint32_t *, cudaStream_t);

void launch_export_records(const uint64_t *sorted, uint32_t nv, const float *rec,
                           float *out, cudaStream_t st) {
  if (nv == 0) return;
  k_export_records<<<grid_for(nv), kB, 0, st>>>(sorted, nv, rec, out);
}

void launch_volume_bits(const float4 *ls4, uint32_t n, uint32_t *vbits, cudaStream_t st) {
  if (n == 0) return;
  k_volume_bits<<<grid_for(n), kB, 0, st>>>(ls4, n, vbits);
}

void launch_score_consts(const float4 *ls4, const float4 *ql, const float4 *qr, uint32_t n,
                         const uint32_t *vsorted, uint32_t k, float *gamma, double *sig_t,
                         cudaStream_t st) {
  if (n == 0) return;
  k_score_consts<<<grid_for(n), kB, 0, st>>>(ls4, ql, qr, n, vsorted, k, gamma, sig_t);
}

void launch_score_batch(const BatchDev &b, cudaStream_t st) {
  k_score_batch<<<grid_for((uint64_t)b.nreq * b.n), kB, 0, st>>>(b);
}

void launch_mark_batch(const BatchDev &b, cudaStream_t st) {
  k_mark_batch<<<grid_for((uint64_t)b.nreq * b.n), kB, 0, st>>>(b);
}

void launch_score_accumulate(const uint64_t *sorted, const uint32_t *nv_dev, uint32_t nv_cap,
                             const float *w_sum, const float4 *mean4, const double *sig_t,
                             const float *gamma, float t, float *score, int variant,
                             cudaStream_t st) {
  if (nv_cap == 0) return;
  k_score_accumulate<<<grid_for(nv_cap), kB, 0, st>>>(sorted, nv_dev, w_sum, mean4, sig_t, gamma,
                                                      t, score, variant);
}

void launch_score_temporal(const float4 *mean4, const double *sig_t, const float *gamma,
                           uint32_t n, float t, float *score, cudaStream_t st) {
  if (n == 0) return;
  k_score_temporal<<<grid_for(n), kB, 0, st>>>(mean4, sig_t, gamma, n, t, score);
}

void launch_mark_contributors(const uint64_t *sorted, const uint32_t *nv_dev, uint32_t nv_cap,
                              const float *w_sum, const uint32_t *stop_mark, uint32_t *row,
                              cudaStream_t st) {
  if (nv_cap == 0) return;
  k_mark_contributors<<<grid_for(nv_cap), kB, 0, st>>>(sorted, nv_dev, w_sum, stop_mark, row);
}

void launch_pack_mask_row(const uint32_t *row, uint32_t nbytes, uint8_t *out, cudaStream_t st) {
  if (nbytes == 0) return;
  k_pack_mask_row<<<grid_for(nbytes), kB, 0, st>>>(row, nbytes, out);
}

void launch_score_keys(const float *score, uint32_t n, uint64_t *keys, cudaStream_t st) {
  if (n == 0) return;
  k_score_keys<<<grid_for(n), kB, 0, st>>>(score, n, keys);
}

void launch_keep_from_sorted(const uint64_t *sorted, uint32_t n, uint32_t n_drop,
                             uint8_t *keep, cudaStream_t st) {
  if (n == 0) return;
  k_keep_from_sorted<<<grid_for(n), kB, 0, st>>>(sorted, n, n_drop, keep);
}

}  // namespace fdgs
