// Internal host-side interfaces between the C ABI and the kernel files.
#pragma once
#include <cuda.h>            // CUtensorMap (types only; the encoder is fetched at run time)
#include <cuda_runtime.h>
#include <stdint.h>

#include "fdgs_common.cuh"

namespace fdgs {

// ---- radix sort (fdgs_sort.cu) ---------------------------------------------------------
// Stable LSD onesweep sort of packed keys on bits [lo, lo + bits). The key count is read
// from device memory (n_dev) so launches need no host synchronisation; n_cap bounds it.
// Returns the buffer that holds the result (a or b). scratch must hold
// sort_scratch_bytes(n_cap, bits) bytes.
size_t sort_scratch_bytes(uint64_t n_cap, int bits);
// With hist_ready the caller has already written each pass's exclusive digit offsets into
// sort_hist(scratch) (256 words per pass) and the histogram kernels are skipped.
template <typename K>
K *radix_sort(K *a, K *b, const uint32_t *n_dev, uint64_t n_cap, int lo, int bits,
              void *scratch, cudaStream_t st, uint32_t *err_dev, bool hist_ready = false);
int sort_passes(int bits);
// Failure injection for tests (fdgs_debug_inject): a spin-wait limit for the sort's look-backs
// (0 = kSpinLimit) and a partition whose look-back publish the next sort pass withholds
// (~0u = none; reset by that pass).
extern uint32_t g_debug_spin_limit;
extern uint32_t g_debug_withhold;
int sort_digit_bits(int bits);
inline uint32_t *sort_hist(void *scratch) { return static_cast<uint32_t *>(scratch); }
constexpr uint64_t kSortMaxKeys = (1ull << 30) - 1;

// ---- rasterizer kernels (fdgs_raster.cu) -----------------------------------------------
struct PreArgs {
  const float4 *mean4, *ls4, *ql, *qr;
  const float *opacity, *sh;
  const float *sh_cb;                // SH codebook [n_code][K-1][3] or null
  const uint16_t *sh_code;           // [n] codes (with sh_cb)
  int deg;
  uint32_t n;
  const uint32_t *mask_l, *mask_r;   // null = no mask
  float t;
  DevCam cam;
  float *rec;          // [n][12] by Gaussian id
  uint64_t *vis_keys;  // compacted (depth bits << 32 | id), id order
  uint8_t *flags;      // optional [n]
  uint64_t *status;    // chained-scan status [ceil(n/256)]
  uint32_t *ctr;       // frame counters
  uint32_t *err;       // scene status word (device error bits)
  int no_cull = 0;     // keep Gaussians with a = sigmoid(o) p(t) < 1/255 (same image)
};
void launch_preprocess(const PreArgs &a, cudaStream_t st);

// rec_sorted is the blend-ready record [nv][16] (see fdgs_common.cuh); diff is the
// [gy + 1][gx + 1] tile-coverage difference array (zeroed by the caller). tight: tile sets
// cut to the alpha >= 1/255 ellipse (tighten_rect), else the 3-sigma squares.
void launch_gather_scan(const uint64_t *sorted, const uint32_t *ctr_nvis, uint32_t n_cap,
                        const float *rec, float *rec_sorted, uint32_t *offsets,
                        uint64_t *status, uint32_t *ctr, uint32_t *err, int gx, int gy,
                        int *diff, uint32_t *rowmask, uint32_t *colmask, uint32_t mask_words,
                        int tight, cudaStream_t st);
// Tile lists by coverage bitmasks (rowmask/colmask written by the gather when non-null,
// [gy or gx][mask_words] words): lists[ranges[t].x ..] = ranks covering tile t, ascending.
// nv_dev (optional): the visible count on the device, read by the kernel instead of nv.
// Tiles whose range is empty are skipped.
void launch_tile_lists(const uint32_t *rowmask, const uint32_t *colmask, uint32_t mask_words,
                       uint32_t nv, int gx, int gy, const uint2 *ranges, uint32_t *lists,
                       cudaStream_t st, const uint32_t *nv_dev = nullptr);
// Tile-list builder: 0 auto (cost model), 1 emit + radix sort, 2 coverage bitmasks.
extern int g_list_mode;
// Integrates diff into per-tile counts; writes tile ranges and the tile sort's digit offsets.
// order (optional): tile ids by descending list length, in buckets of 16 entries (order
// within a bucket unspecified), so that the one-CTA-per-tile blend starts its longest tiles
// first. cap (0: none): the list capacity; longer lists set kErrCapacity in err, raise
// *need to their total length and empty every range.
void launch_tile_scan(int *diff, int gx, int gy, int npass, int dbits, uint2 *ranges,
                      uint32_t *hist, uint32_t *order, cudaStream_t st, uint64_t cap = 0,
                      unsigned long long *need = nullptr, uint32_t *err = nullptr);

template <typename K>
void launch_emit(const float *rec_sorted, const uint32_t *offsets, uint32_t nv, int gx, int gy,
                 int rb, int tight, K *keys, cudaStream_t st);

struct BlendArgs {
  const uint2 *ranges;
  const float *rec_sorted;
  int W, H, gx, gy;
  float bg[3];
  float *rgb;          // [3][H][W]
  float *T_final;      // [H][W], or null for a forward-only render (then n_contrib too)
  uint32_t *n_contrib; // [H][W]
  float *w_sum;        // optional [nv] per-rank blend-weight sums (score pass)
  uint32_t *stop_mark; // with w_sum: [nv] per-rank flag, set where the entry stopped a pixel
  unsigned long long *evals;  // optional evaluation counters [3] (profiling)
  const uint32_t *order = nullptr;  // optional [tiles] launch order (longest list first)
};
template <typename K>
void launch_blend(const BlendArgs &a, const K *keys, uint32_t rmask, cudaStream_t st);

struct BlendBwdArgs {
  const uint2 *ranges;
  const float *rec_sorted;
  int W, H, gx, gy;
  float bg[3];
  const float *dL_drgb;
  const float *T_final;
  const uint32_t *n_contrib;
  float *g2d;          // [nv][9] per rank: u, v, A, B, C, a, r, g, b
  const uint32_t *order = nullptr;  // optional [tiles] launch order (the forward's)
  unsigned long long *evals = nullptr;  // optional counters [3] (profiling; see k_blend_bwd)
};
template <typename K>
void launch_blend_bwd(const BlendBwdArgs &a, const K *keys, uint32_t rmask, cudaStream_t st);

struct PreBwdArgs {
  const float4 *mean4, *ls4, *ql, *qr;
  const float *opacity, *sh;
  int deg;
  uint32_t n, nv;
  float t;
  DevCam cam;
  const uint64_t *sorted;  // rank -> (depth, id)
  const float *g2d;
  float *g_mean4, *g_ls4, *g_ql, *g_qr, *g_op, *g_sh;
};
void launch_preprocess_bwd(const PreBwdArgs &a, cudaStream_t st);

// ---- frame export, score pass and keep-set helpers (fdgs_score.cu) ----------------------
template <typename K>
void launch_keys_to_ids(const K *keys, uint32_t nkeys, uint32_t rmask, const uint64_t *sorted,
                        uint32_t *ids, cudaStream_t st);
void launch_export_records(const uint64_t *sorted, uint32_t nv, const float *rec,
                           float *out, cudaStream_t st);
// V_i = prod of the four scales, as float bits (positive floats sort as unsigned ints)
void launch_volume_bits(const float4 *ls4, uint32_t n, uint32_t *vbits, cudaStream_t st);
// per Gaussian: gamma_i = clamp(V_i / V_sorted[k], 0, 1)^0.1 with V_sorted the ascending
// volumes, and the temporal variance Sigma_t,i in FP64
void launch_score_consts(const float4 *ls4, const float4 *ql, const float4 *qr, uint32_t n,
                         const uint32_t *vsorted, uint32_t k, float *gamma, double *sig_t,
                         cudaStream_t st);
// score[id] += w_sum[rank] * factor_id(t) for every visible rank, the factor of the score
// variant (fdgs_score_variant; 0: f_id(t) gamma[id], the score of Eq. 7)
void launch_score_accumulate(const uint64_t *sorted, const uint32_t *nv_dev, uint32_t nv_cap,
                             const float *w_sum, const float4 *mean4, const double *sig_t,
                             const float *gamma, float t, float *score, int variant,
                             cudaStream_t st);
// the temporal-only score variant: score[i] += f_i(t) gamma[i] for every Gaussian
void launch_score_temporal(const float4 *mean4, const double *sig_t, const float *gamma,
                           uint32_t n, float t, float *score, cudaStream_t st);
void launch_score_keys(const float *score, uint32_t n, uint64_t *keys, cudaStream_t st);
// key-frame masks: row[id / 32] |= bit id % 32 for visible ranks blended somewhere
// (w_sum > 0) or that stopped a pixel (stop_mark); rows packed into LSB-first bytes
void launch_mark_contributors(const uint64_t *sorted, const uint32_t *nv_dev, uint32_t nv_cap,
                              const float *w_sum, const uint32_t *stop_mark, uint32_t *row,
                              cudaStream_t st);
void launch_pack_mask_row(const uint32_t *row, uint32_t nbytes, uint8_t *out, cudaStream_t st);
void launch_keep_from_sorted(const uint64_t *sorted, uint32_t n, uint32_t n_drop,
                             uint8_t *keep, cudaStream_t st);

// ---- batched rendering (fdgs_batch.cu) -------------------------------------------------
// One request of a batch, as the kernels read it (uploaded once per batch).
struct ReqDesc {
  DevCam cam;
  float t;
  const uint32_t *mask_l, *mask_r;   // null = unmasked
  float bg[3];
  float *rgb;                        // [3][H][W]
  uint32_t tile_base;                // first global tile id of the request
  uint32_t block_base;               // first global tile-block id (kListBlock^2 tiles each)
  uint64_t mask_base;                // offset of its block-row and block-column bitmasks
  uint32_t *mark_row;                // mask pass: the key-frame word row it marks, or null
};
// Side, in tiles, of the square tile blocks the batched list builder works on: bitmasks are
// kept per block row and block column, and one warp builds the lists of a block's tiles.
constexpr int kListBlock = 4;
enum BatchCounter {
  BC_PRE_ITEM = 0, BC_NVIS = 1, BC_NSLOTS = 2, BC_NTILES = 3, BC_NKEYS_LO = 5,
  BC_NKEYS_HI = 6, BC_QUEUE = 7, BC_NBKEYS_LO = 8, BC_NBKEYS_HI = 9, BC_COUNT = 16
};
struct BatchDev {
  const ReqDesc *reqs;
  int nreq;
  uint32_t n, ntiles, nblocks, mask_words;
  int part_major;                    // preprocess order: partition-major (large scenes)
  uint64_t key_cap;
  const float4 *mean4, *ls4, *ql, *qr;
  const float *opacity, *sh;
  float4 *cond;                      // [n][5] conditional factors of every Gaussian
  const float *sh_cb;                // SH codebook or null
  const uint16_t *sh_code;
  int deg;
  uint32_t *ctr, *err;
  uint2 *part;                       // [nreq][partitions]: visible count, segment offset
  float *rec;                        // [nreq][n][12] blend-ready records by (request, id)
  uint2 *rect_id;                    // [nreq][n] alpha-tight tile rectangles by (request, id)
  uint32_t *ridx;                    // [slots] record index (request x n + id) of each slot
  uint64_t *vis_seg, *vis, *vis_alt; // visible keys: per-partition segments, contiguous, alt
  const uint64_t *vis_sorted;
  uint32_t *nv, *vis_base, *slot_base;
  unsigned long long *key_cnt;       // [nreq] list entries per request
  uint2 *rect;                       // [slots] tile rectangle: x0 | x1 << 16, y0 | y1 << 16
  uint32_t *masks;
  uint2 *ranges;                     // [ntiles] [0, list length) of each tile's list
                                     // (written with the block lists; the entries live
                                     // in the block lists)
  uint2 *branges;                    // [nblocks] [start, end) into lists / ltm
  uint32_t *bcount;                  // [nblocks] block-list entries
  unsigned long long *bkey_cnt;      // [nreq] block-list entries per request
  uint64_t *qkeys, *qkeys_alt;
  const uint64_t *queue;
  uint32_t *lists;                   // [key_cap] block lists: record indices, rank order
  uint16_t *ltm;                     // [key_cap] block lists: the block's tiles each covers
  unsigned long long *done_ns, *t0_ns;
  unsigned long long *evals;         // [3] blend counters (see BlendTile), or null
  // weighted passes (null for renders): blend weights and stop flags per record index
  // [nreq][n]; the score pass adds them, with the Gaussians' volume factors gamma, into
  // score (Eqs. 4-7); the mask pass marks the contributing Gaussians in each request's
  // mark_row
  float *w_sum;
  uint32_t *stop_mark;
  const float *gamma;
  const double *sig_t;               // [n] temporal variances (score pass)
  float *score;
  int score_variant;                 // fdgs_score_variant of the score pass
  int mark;
  unsigned long long *stamps;        // [kBatchStages + 1] %globaltimer at stage boundaries
  // TMA descriptor of rec as a 2D tensor (12 floats x nreq n rows, 48-byte rows, box 12 x 1)
  // for the blend's gather4 staging; valid when rec_map_ok
  alignas(64) CUtensorMap rec_map;
  int rec_map_ok;
  uint32_t tma_skip;                 // failure injection: thread 0 skips its stage arrivals
  uint32_t tma_spin;                 // stage-wait poll limit (0: kTmaSpin)
};
struct BatchLaunch {
  void *sort_scratch;
  int footprint;                     // launch shape of the blend (with_blend_shape)
  int blend_ctas_per_sm;             // persistent blend grid = this x SMs
  const uint64_t *vis_sorted;        // out: the buffer that holds the sorted depth keys
  uint64_t wsum_len;                 // entries of the weighted passes' buffers (nreq x n)
  int staging;                       // blend record staging: 0 cp.async, 1 TMA gather4
  int black;                         // every request's background is black
};
// ---- post-pruning fine-tuning (fdgs_finetune.cu) ----------------------------------------
// dL = sign(img - target) / n, loss += mean |img - target| (n floats)
void launch_l1_grad(const float *img, const float *target, uint32_t n, float *dL, float *loss,
                    cudaStream_t st);
// One Adam step over nseg segments of a concatenated parameter space: segment s is
// [off[s], off[s + 1]) of grad, m and v, and updates param[s] in place with its step size
// lr_s / (1 - b1^step); sqrt_bc2 = sqrt(1 - b2^step).
struct AdamArgs {
  int nseg;
  uint64_t off[9];
  float *param[8];
  float step_size[8];
  const float *grad;
  float *m, *v;
  float b1, b2, eps, sqrt_bc2;
};
void launch_adam(const AdamArgs &a, cudaStream_t st);

// Encodes b.rec_map over b.rec with the given row count (nreq x n); false (and
// b.rec_map_ok = 0) when the driver offers no tensor-map encoder or rejects the layout.
bool encode_record_map(BatchDev &b, uint64_t rows);
// Record staging of the batched blend for plans captured from now on (fdgs_set_batch_staging).
extern int g_batch_staging;
// Failure injection (fdgs_debug_inject): the next eager TMA-staged batch withholds one arrival
// (and its copy) on every stage barrier.
extern uint32_t g_debug_tma_skip;
// Gaussian id bits at the bottom of the batched depth keys (request | depth | id).
constexpr int kBatchIdBits = 25;
// Stages timed by the device stamps: preprocess, depth_sort (bases, compaction, sort),
// gather, tile_scan, lists, queue_sort, blend.
constexpr int kBatchStages = 7;
void launch_batch(const BatchDev &b, BatchLaunch &L, cudaStream_t st);
// Word copies run by one small kernel (up to kWordJobs of them): the batch uploads its request
// descriptors from, and reads its counters back into, pinned host memory that the GPU
// addresses directly, so that no copy engine is involved and they never wait behind the
// caller's own host copies on other streams.
constexpr int kWordJobs = 6;
struct WordJobs {
  const uint32_t *src[kWordJobs];
  uint32_t *dst[kWordJobs];
  uint32_t n[kWordJobs];
  int count;
};
void launch_copy_words(const WordJobs &j, cudaStream_t st);
// Score pass of a batch: adds w_sum[r][i] * f_i(t_r) * gamma_i to score[i] for every request
// r and Gaussian i (after the weighted blend of the batch).
void launch_score_batch(const BatchDev &b, cudaStream_t st);
// Mask pass of a batch: sets bit id of request r's mark_row for every Gaussian that was
// blended somewhere in r (weight > 0) or stopped one of its pixels.
void launch_mark_batch(const BatchDev &b, cudaStream_t st);
// Resident CTAs per SM of the persistent blend of a launch shape (black: the variant for
// batches whose requests all have a black background).
int batch_blend_max_ctas_per_sm(int shape, bool black = false);

int num_sms();
extern int g_blend_shape;   // launch shape of the forward blend (with_blend_shape)
extern int g_blend_shape_fwd;   // ... of the forward-only blend on black backgrounds
constexpr int kBlendShapes = 7;
// 8x8 footprint, two pixels a lane, for the blend that writes transmittance; 8x16, four
// pixels a lane, for the forward-only blend (0.430 against 0.436 ms for 16x16 and 0.447 for
// 8x8, masked 200k-Gaussian frames at 1352x1014)
constexpr int kBlendShapeDefault = 3, kBlendShapeFwdDefault = 5;

// Sets the message returned by fdgs_last_error() on this thread.
void set_error_message(const char *msg);

}  // namespace fdgs
