// Pruning keep-set selection that allocates no device memory.
//
// fdgs_select_keep keeps its sort buffers in the scene's grow-only workspace, which means a
// cudaMalloc the first time (and whenever n grows) and a cudaFree when it grows again. Some
// callers cannot allow that: a pruning step inside a real-time render or training loop must
// not pay the implicit device-wide synchronisation of cudaMalloc/cudaFree, and a process whose
// HBM is already fully reserved by another allocator (a framework's caching pool, a fixed
// serving budget) cannot obtain fresh device memory at all. fdgs_select_keep_noalloc does the
// same selection with every scratch byte in one file-scope static device array, held by every
// device that loads this module until the process exits. The runtime reserves that array when
// it loads the module on a device: at the module's first use there (its first call here, under
// the default lazy module loading) or when the library is loaded (CUDA_MODULE_LOADING=EAGER).
// A caller that can allow no allocation at all after start-up makes one warm-up call first.
#include <mutex>

#include "fdgs.h"
#include "fdgs_internal.h"

namespace {

// Largest n accepted: the score-pass workload size (1M Gaussians) rounded up to 2^20.
constexpr uint32_t kNoAllocMaxN = 1u << 20;
// Layout: [0, 16 MiB) two ping-pong arrays of kNoAllocMaxN 64-bit sort keys,
// [16 MiB, +256) count and error words, [16 MiB + 256, ...) radix-sort scratch.
constexpr size_t kKeysBytes = 2ull * kNoAllocMaxN * sizeof(uint64_t);
constexpr size_t kWordsBytes = 256;
constexpr size_t kScratchBytes = 18ull << 20;   // 18 MiB in total

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Host code must not take the address of g_noalloc_scratch directly (that is a host-side
// stand-in, not a device address): it asks the runtime, once per device, and caches the
// answer. After cudaDeviceReset the module may be reloaded elsewhere and the cached address
// is stale, so calls after a reset of that device are not supported.
std::mutex g_mu;
constexpr int kMaxDevices = 64;
void *g_dev_ptr[kMaxDevices] = {};

int scratch_on_current_device(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    fdgs::set_error_message("fdgs_select_keep_noalloc: no usable current CUDA device");
    return FDGS_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_dev_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      fdgs::set_error_message("fdgs_select_keep_noalloc: cudaGetSymbolAddress failed");
      return FDGS_ERR_CUDA;
    }
    g_dev_ptr[dev] = p;
  }
  *out = g_dev_ptr[dev];
  return FDGS_OK;
}

// Writes the key count read by the sort and clears the error word.
__global__ void k_put_count(uint32_t *words, uint32_t n) {
  words[0] = n;
  words[1] = 0;
}

}  // namespace

extern "C" int fdgs_select_keep_noalloc(const float *score_dev, int64_t n, float prune_ratio,
                                        uint8_t *keep_out_dev, fdgs_stream stream) {
  if (!score_dev || !keep_out_dev || n < 0) {
    fdgs::set_error_message("fdgs_select_keep_noalloc: null pointer or negative n");
    return FDGS_ERR_INVALID;
  }
  if (n > (int64_t)kNoAllocMaxN) {
    fdgs::set_error_message("fdgs_select_keep_noalloc: n exceeds the static scratch limit of "
                            "1048576 scores");
    return FDGS_ERR_CAPACITY;
  }
  if (!(prune_ratio >= 0.f && prune_ratio <= 1.f)) {
    fdgs::set_error_message("fdgs_select_keep_noalloc: prune_ratio must be in [0, 1]");
    return FDGS_ERR_INVALID;
  }
  if (n == 0) return FDGS_OK;
  void *base = nullptr;
  int rc = scratch_on_current_device(&base);
  if (rc != FDGS_OK) return rc;
  const uint32_t N = (uint32_t)n;
  if (kKeysBytes + kWordsBytes + fdgs::sort_scratch_bytes(kNoAllocMaxN, 32) > kScratchBytes) {
    fdgs::set_error_message("fdgs_select_keep_noalloc: static scratch layout too small");
    return FDGS_ERR_CAPACITY;
  }
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char *b = static_cast<unsigned char *>(base);
  uint64_t *keys_a = reinterpret_cast<uint64_t *>(b);
  uint64_t *keys_b = keys_a + kNoAllocMaxN;
  uint32_t *words = reinterpret_cast<uint32_t *>(b + kKeysBytes);
  void *sort_scratch = b + kKeysBytes + kWordsBytes;
  k_put_count<<<1, 1, 0, st>>>(words, N);
  fdgs::launch_score_keys(score_dev, N, keys_a, st);
  uint64_t *srt = fdgs::radix_sort<uint64_t>(keys_a, keys_b, words, N, 32, 32, sort_scratch, st,
                                             words + 1);
  const uint32_t n_drop = (uint32_t)((double)prune_ratio * (double)N);
  fdgs::launch_keep_from_sorted(srt, N, n_drop, keep_out_dev, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    fdgs::set_error_message(cudaGetErrorString(e));
    return FDGS_ERR_CUDA;
  }
  // The call has no scene whose status word a later call could read, so it waits for its own
  // work and reports a look-back that gave up (the keep-set is then unspecified).
  uint32_t dev_err = 0;
  e = cudaMemcpyAsync(&dev_err, words + 1, sizeof dev_err, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    fdgs::set_error_message(cudaGetErrorString(e));
    return FDGS_ERR_CUDA;
  }
  if (dev_err & fdgs::kErrTimeout) {
    fdgs::set_error_message("fdgs_select_keep_noalloc: a sort look-back reached its spin-wait "
                            "limit; the keep-set is unspecified");
    return FDGS_ERR_TIMEOUT;
  }
  return FDGS_OK;
}
