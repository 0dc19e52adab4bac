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

__global__ void k_gamma(const float4 *__restrict__ ls4, uint32_t n,
                        const uint32_t *__restrict__ vsorted, uint32_t k, float *gamma) {
  const float vref = __uint_as_float(vsorted[k]);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float4 l = ls4[i];
    const float v = expf(l.x + l.y + l.z + l.w);
    const float x = fminf(fmaxf(v / vref, 0.f), 1.f);
    gamma[i] = powf(x, 0.1f);
  }
}

// Temporal variance Sigma_t = |row t of R diag(s)|^2 of one Gaussian.
__device__ __forceinline__ float temporal_variance(float4 ls, float4 ql, float4 qr) {
  float qn_l[4], qn_r[4], il, ir, L[16], Rr[16];
  quat_unit(ql, qn_l, il);
  quat_unit(qr, qn_r, ir);
  left_mat(qn_l, L);
  right_mat(qn_r, Rr);
  const float s[4] = {expf(ls.x), expf(ls.y), expf(ls.z), expf(ls.w)};
  float v = 0.f;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    float r = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) r = fmaf(L[12 + k], Rr[k * 4 + m], r);
    const float e = r * s[m];
    v = fmaf(e, e, v);
  }
  return v;
}

// f_i(t) of Eqs. 5-6: the second time derivative of the temporal opacity p_i(t) mapped
// through tanh into [1, 2] (its reciprocal half-plus-half form).
__device__ __forceinline__ float variation_factor(float t, float4 m4, float4 ls, float4 ql,
                                                  float4 qr) {
  const float st = temporal_variance(ls, ql, qr);
  const float dt = t - m4.w;
  const float p = expf(-0.5f * dt * dt / st);
  const float p2 = (dt * dt / (st * st) - 1.f / st) * p;
  return 1.f / (0.5f * tanhf(fabsf(p2)) + 0.5f);
}

__global__ void k_score_accumulate(const uint64_t *__restrict__ sorted,
                                   const uint32_t *__restrict__ nv_dev,
                                   const float *__restrict__ w_sum,
                                   const float4 *__restrict__ mean4, const float4 *__restrict__ ls4,
                                   const float4 *__restrict__ ql, const float4 *__restrict__ qr,
                                   const float *__restrict__ gamma, float t, float *score) {
  const uint32_t nv = *nv_dev;
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < nv; r += gridDim.x * blockDim.x) {
    const float w = w_sum[r];
    if (w == 0.f) continue;
    const uint32_t id = (uint32_t)sorted[r];
    const float f = variation_factor(t, mean4[id], ls4[id], ql[id], qr[id]);
    score[id] += w * f * gamma[id];
  }
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
    const float f = variation_factor(b.reqs[r].t, b.mean4[id], b.ls4[id], b.ql[id], b.qr[id]);
    atomicAdd(&b.score[id], w * f * b.gamma[id]);
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

void launch_gamma(const float4 *ls4, uint32_t n, const uint32_t *vsorted, uint32_t k,
                  float *gamma, cudaStream_t st) {
  if (n == 0) return;
  k_gamma<<<grid_for(n), kB, 0, st>>>(ls4, n, vsorted, k, gamma);
}

void launch_score_batch(const BatchDev &b, cudaStream_t st) {
  k_score_batch<<<grid_for((uint64_t)b.nreq * b.n), kB, 0, st>>>(b);
}

void launch_mark_batch(const BatchDev &b, cudaStream_t st) {
  k_mark_batch<<<grid_for((uint64_t)b.nreq * b.n), kB, 0, st>>>(b);
}

void launch_score_accumulate(const uint64_t *sorted, const uint32_t *nv_dev, uint32_t nv_cap,
                             const float *w_sum, const float4 *mean4, const float4 *ls4,
                             const float4 *ql, const float4 *qr, const float *gamma, float t,
                             float *score, cudaStream_t st) {
  if (nv_cap == 0) return;
  k_score_accumulate<<<grid_for(nv_cap), kB, 0, st>>>(sorted, nv_dev, w_sum, mean4, ls4, ql, qr,
                                                      gamma, t, score);
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
