// Kernels of one post-pruning fine-tuning iteration (Sec. 4.2.1 "Pruning": the pruned scene
// is optimised further, through the filter of Sec. 4.2.2): the L1 loss of a render against
// its target with the loss's image gradient, and one Adam update of every attribute array.
#include <algorithm>

#include "fdgs_internal.h"

namespace fdgs {

namespace {

constexpr int kB = 256;

// dL[i] = sign(img[i] - target[i]) / n (0 where equal) and loss += sum |img - target| / n.
__global__ void __launch_bounds__(kB)
    k_l1_grad(const float *__restrict__ img, const float *__restrict__ target, uint32_t n,
              float inv_n, float *__restrict__ dL, float *loss) {
  __shared__ float s_part[kB / 32];
  float acc = 0.f;
  for (uint32_t i = blockIdx.x * kB + threadIdx.x; i < n; i += gridDim.x * kB) {
    const float d = img[i] - target[i];
    dL[i] = d > 0.f ? inv_n : (d < 0.f ? -inv_n : 0.f);
    acc += fabsf(d);
  }
  acc = warp_sum(acc);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) s_part[warp] = acc;
  __syncthreads();
  if (warp == 0) {
    float v = lane < kB / 32 ? s_part[lane] : 0.f;
    v = warp_sum(v);
    if (lane == 0 && v != 0.f) atomicAdd(loss, v * inv_n);
  }
}

// Adam (Kingma and Ba) over the segments of one concatenated parameter space, in PyTorch's
// formulation: m += (1 - b1) (g - m), v = b2 v + (1 - b2) g^2,
// p -= step_size m / (sqrt(v) / sqrt(bc2) + eps), step_size = lr / bc1, bcK = 1 - bK^step.
__global__ void __launch_bounds__(kB) k_adam(AdamArgs a) {
  const uint64_t total = a.off[a.nseg];
  for (uint64_t i = blockIdx.x * (uint64_t)kB + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * kB) {
    int s = 0;
    while (s + 1 < a.nseg && i >= a.off[s + 1]) ++s;
    const uint64_t j = i - a.off[s];
    const float g = a.grad[i];
    const float m = fmaf(1.f - a.b1, g - a.m[i], a.m[i]);
    const float v = fmaf(a.b2, a.v[i], (1.f - a.b2) * g * g);
    a.m[i] = m;
    a.v[i] = v;
    const float denom = sqrtf(v) / a.sqrt_bc2 + a.eps;
    a.param[s][j] -= a.step_size[s] * (m / denom);
  }
}

int grid_for(uint64_t n) {
  return (int)std::max<uint64_t>(1, std::min<uint64_t>((n + kB - 1) / kB,
                                                        (uint64_t)num_sms() * 8));
}

}  // namespace

void launch_l1_grad(const float *img, const float *target, uint32_t n, float *dL, float *loss,
                    cudaStream_t st) {
  if (n == 0) return;
  k_l1_grad<<<grid_for(n), kB, 0, st>>>(img, target, n, 1.f / (float)n, dL, loss);
}

void launch_adam(const AdamArgs &a, cudaStream_t st) {
  const uint64_t total = a.off[a.nseg];
  if (total == 0) return;
  k_adam<<<grid_for(total), kB, 0, st>>>(a);
}

}  // namespace fdgs
