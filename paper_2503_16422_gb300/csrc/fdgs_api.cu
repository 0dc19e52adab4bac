// C ABI of the GB300 masked 4D Gaussian rasterizer: scene and frame lifecycle, workspace
// management and the stream-ordered launch sequence of each call (declared in fdgs.h).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <set>
#include <string>
#include <vector>

#include "fdgs.h"
#include "fdgs_internal.h"
#include <nvtx3/nvToolsExt.h>

using namespace fdgs;

// An NVTX range around each entry point's host work, for profilers that show them (ncu
// --nvtx filters, Nsight Systems timelines); without a profiler attached it costs a call.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CK(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(FDGS_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));        \
  } while (0)

#define TRY(expr)            \
  do {                       \
    int rc_ = (expr);        \
    if (rc_ != FDGS_OK) return rc_; \
  } while (0)

// Grow-only device buffer.
struct Buf {
  void *p = nullptr;
  size_t n = 0;
  template <typename T>
  T *as() const { return static_cast<T *>(p); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
};

// Host-side failure injection (fdgs_debug_inject): the next g_fail_allocs growths fail as a
// refused cudaMalloc would.
int g_fail_allocs = 0;

int grow(Buf &b, size_t bytes) {
  if (bytes <= b.n && b.p) return FDGS_OK;
  if (g_fail_allocs > 0) {
    --g_fail_allocs;
    return fail(FDGS_ERR_OOM, "device allocation of %zu bytes refused (injected failure)",
                bytes + bytes / 4);
  }
  b.release();
  const size_t nb = std::max<size_t>(bytes + bytes / 4, 256);
  if (cudaMalloc(&b.p, nb) != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return fail(FDGS_ERR_OOM, "cudaMalloc of %zu bytes failed", nb);
  }
  b.n = nb;
  return FDGS_OK;
}

int ceil_log2(uint64_t x) {  // bits needed to represent 0..x-1 (>= 1)
  int b = 1;
  while (b < 63 && (1ull << b) < x) ++b;
  return b;
}

// Per-render buffers. One per frame in flight plus the scene's own.
struct Workspace {
  Buf ctr;                       // u32[C_COUNT]
  uint32_t *hctr = nullptr;      // pinned host mirror of ctr
  Buf pre_status, scan_status;   // u64 per partition of 256 Gaussians
  Buf rec, rec_sorted;           // f32[n][12]
  Buf vis[2];                    // u64[n] visible (depth, id) keys, ping-pong
  Buf offsets;                   // u32[n]
  Buf flags;                     // u8[n]
  Buf keys[2];                   // packed (tile, rank) keys, ping-pong
  Buf ranges;                    // uint2[tiles]
  Buf order;                     // u32[tiles] blend launch order (longest list first)
  Buf Tf, nc;                    // f32 / u32 [pixels]
  Buf scratch;                   // sort scratch
  Buf g2d;                       // f32[n][9] backward accumulators
  Buf wsum;                      // f32[n] per-rank blend weights (score pass)
  Buf stopmark;                  // u32[n] per-rank "stopped a pixel" flags (with wsum)
  Buf diff;                      // i32[gy + 1][gx + 1] tile-coverage difference array
  Buf rowmask, colmask;          // u32 coverage bitmasks by depth rank per tile row / column
  // renders without a host synchronisation (fdgs_render_async): the tile-list capacity in
  // entries (0 until the first, sizing call) and the u64 list length an overflowing render
  // needed (atomicMax on the device, read and cleared by fdgs_status_sync)
  uint64_t key_cap = 0;
  Buf need;
  ~Workspace() {
    Buf *all[] = {&ctr, &pre_status, &scan_status, &rec, &rec_sorted, &vis[0], &vis[1],
                  &offsets, &flags, &keys[0], &keys[1], &ranges, &order, &Tf, &nc, &scratch, &g2d,
                  &wsum, &stopmark, &diff, &rowmask, &colmask, &need};
    for (Buf *b : all) b->release();
    if (hctr) cudaFreeHost(hctr);
  }
};

struct FrameMeta {
  DevCam cam{};
  float t = 0.f;
  int W = 0, H = 0, gx = 0, gy = 0, l = -1, r = -1;
  uint32_t n_active = 0, nv = 0;
  uint64_t nkeys = 0;
  int key64 = 0, rb = 1, builder = 1;
  uint64_t *sorted = nullptr;
  void *keys = nullptr;
  float bg[3] = {0.f, 0.f, 0.f};
  cudaStream_t stream = nullptr;
};

}  // namespace

namespace {

// Buffers, captured graph and tuning of one batch geometry (request count, resolutions,
// mask use, scene attribute pointers). Built on the first batch call of that geometry.
struct BatchPlan {
  int nreq = 0;
  std::vector<int> W, H;
  bool masked = false;
  fdgs_scene_desc d{};
  const uint64_t *vis_sorted = nullptr;    // sorted depth keys of the last batch (device)
  bool weighted = false;                   // next runs: a weighted pass (eager, no graph)
  float *score_out = nullptr;              // score pass: accumulate into this (else null)
  int score_variant = 0;                   // score pass: fdgs_score_variant
  const float *gamma = nullptr;
  const double *sig_t = nullptr;           // score pass: temporal variances (FP64)
  bool mark = false;                       // mask pass: requests carry mark_row
  Buf wsum, stop;                          // weighted passes: per-slot weights, stop flags
  const float *sh_cb = nullptr;            // codebook pointers captured in the graph
  const uint16_t *sh_code = nullptr;
  uint32_t ntiles = 0, nblocks = 0, mask_words = 0;
  uint64_t key_cap = 0, rn = 0, slot_cap = 0, mask_total = 0;
  std::vector<ReqDesc> tmpl;
  Buf reqs, ctr, part, rec, vis_seg, vis, vis_alt, nv, vis_base, slot_base, key_cnt,
      rect_id, ridx, rect, masks, ranges, branges, bcount, bkey_cnt, qkeys, qkeys_alt,
      lists, ltm, done, t0, scratch, cond;
  // pinned host memory that the GPU also addresses (mapped; d_* are the device pointers)
  ReqDesc *h_reqs = nullptr;
  uint32_t *h_ctr = nullptr;
  unsigned long long *h_done = nullptr;   // [nreq] completion, then t0
  uint32_t *h_status = nullptr;           // the status word, read back with the counters
  ReqDesc *d_h_reqs = nullptr;
  uint32_t *d_h_ctr = nullptr, *d_h_status = nullptr;
  unsigned long long *d_h_done = nullptr, *d_h_stamps = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr;
  int footprint = 6, ctas = 0;
  int staging = -1;                            // record staging the graph was captured with
  int black = 1;                               // this call's requests have black backgrounds
  int cap_black = -1;                          // ... and those the graph was captured for
  bool tuned = false;
  std::vector<float> lat_ms;
  Buf stamps;                                  // u64[kBatchStages + 1] %globaltimer
  unsigned long long *h_stamps = nullptr;      // pinned mirror
  float stage_ms[kBatchStages] = {};
  ~BatchPlan() {
    stamps.release();
    wsum.release();
    stop.release();
    if (h_stamps) cudaFreeHost(h_stamps);
    Buf *all[] = {&reqs, &ctr, &part, &rec, &vis_seg, &vis, &vis_alt, &nv, &vis_base,
                  &slot_base, &key_cnt, &rect_id, &ridx, &rect, &masks, &ranges, &branges,
                  &bcount, &bkey_cnt, &qkeys, &qkeys_alt, &lists, &ltm, &done, &t0, &scratch,
                  &cond};
    for (Buf *b : all) b->release();
    if (h_reqs) cudaFreeHost(h_reqs);
    if (h_ctr) cudaFreeHost(h_ctr);
    if (h_done) cudaFreeHost(h_done);
    if (h_status) cudaFreeHost(h_status);
    if (exec) cudaGraphExecDestroy(exec);
    if (cap) cudaStreamDestroy(cap);
  }
};

}  // namespace

struct fdgs_scene {
  fdgs_scene_desc d{};
  int device = 0;
  BatchPlan *plan = nullptr;
  uint64_t list_cap_hint = 0;   // initial block-list capacity of new plans (0: heuristic)
  Buf masks;
  size_t row_words = 0;
  int n_key = 0;
  std::vector<float> key_times;
  Workspace main;
  Workspace nosync;   // fdgs_render_async's own buffers (no other call reallocates them)
  std::vector<Workspace *> pool;
  std::set<fdgs_frame *> live;
  Buf status;     // u32 device error bits
  Buf aux[6];     // score pass / keep-set buffers: 0 keys, 1 gamma, 2 sort scratch,
                  // 3 device scalar, 4 score-pass image, 5 key-frame mask word row
  int prof = 0;   // profiling flags (fdgs_profile_enable)
  // stage events: [0..8] bound the forward's eight stages, [9..11] the backward's two
  cudaEvent_t ev[FDGS_PROFILE_STAGES + 2] = {};
  Buf evals;      // u64[3] blend evaluations, culling tests, alpha >= 1/255 evaluations
  const float *sh_cb = nullptr;        // borrowed SH codebook (fdgs_set_sh_codebook) or null
  const uint16_t *sh_code = nullptr;
  int n_code = 0;
  // fine-tuning (fdgs_finetune_step): image, its gradient, the concatenated gradients and
  // Adam moments of every attribute array, the loss scratch, Adam's step count
  Buf ft_img, ft_dL, ft_grad, ft_m, ft_v, ft_loss;
  uint64_t ft_total = 0;
  int ft_step = 0;
  // launch shape of new batch plans (fdgs_set_batch_shape): blend shape, CTAs per SM (0: the
  // occupancy limit)
  int batch_footprint = 6, batch_ctas = 0;
};

struct fdgs_frame {
  fdgs_scene *scene;
  Workspace *ws;
  FrameMeta m;
};

namespace {

int check_desc(const fdgs_scene_desc *d) {
  if (!d) return fail(FDGS_ERR_INVALID, "null scene description");
  if (d->n < 0 || d->n >= (1ll << 30)) return fail(FDGS_ERR_INVALID, "n out of range");
  if (d->sh_degree < 0 || d->sh_degree > 3)
    return fail(FDGS_ERR_INVALID, "sh_degree must be 0..3");
  if (d->n > 0 && (!d->mean4 || !d->logscale4 || !d->q_left || !d->q_right ||
                   !d->opacity_logit || !d->sh))
    return fail(FDGS_ERR_INVALID, "null attribute pointer");
  const void *v[] = {d->mean4, d->logscale4, d->q_left, d->q_right};
  for (const void *p : v)
    if (((uintptr_t)p) & 15) return fail(FDGS_ERR_INVALID, "[n][4] arrays must be 16-byte aligned");
  return FDGS_OK;
}

int make_cam(const fdgs_camera *c, DevCam &dc) {
  if (!c) return fail(FDGS_ERR_INVALID, "null camera");
  if (c->width < 1 || c->height < 1 || c->width > 16384 || c->height > 16384)
    return fail(FDGS_ERR_INVALID, "image size out of range");
  if (!(c->fx > 0.f) || !(c->fy > 0.f)) return fail(FDGS_ERR_INVALID, "focal length <= 0");
  for (int r = 0; r < 3; ++r) {
    for (int k = 0; k < 3; ++k) dc.R[r * 3 + k] = c->viewmat[r * 4 + k];
    dc.tv[r] = c->viewmat[r * 4 + 3];
  }
  for (int k = 0; k < 3; ++k)
    dc.eye[k] = -(dc.R[0 * 3 + k] * dc.tv[0] + dc.R[1 * 3 + k] * dc.tv[1] +
                  dc.R[2 * 3 + k] * dc.tv[2]);
  dc.fx = c->fx; dc.fy = c->fy; dc.cx = c->cx; dc.cy = c->cy;
  dc.limx = kFovClamp * ((float)c->width / (2.f * c->fx));
  dc.limy = kFovClamp * ((float)c->height / (2.f * c->fy));
  dc.znear = c->znear;
  dc.W = c->width; dc.H = c->height;
  dc.gx = (c->width + kTile - 1) / kTile;
  dc.gy = (c->height + kTile - 1) / kTile;
  return FDGS_OK;
}

void keyframe_pair(const std::vector<float> &kt, float t, int &l, int &r) {
  const int n = (int)kt.size();
  l = 0;
  for (int i = 0; i < n; ++i)
    if (kt[i] <= t) l = i;
  r = std::min(l + 1, n - 1);
}

int check_device_errors(fdgs_scene *s, cudaStream_t st) {
  uint32_t e = 0;
  CK(cudaMemcpyAsync(&e, s->status.p, 4, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (e) {
    // a render without host synchronisation that overflowed its list capacity recorded the
    // length it needed: the capacity grows to fit it (the buffer is allocated here, outside
    // any stream capture), so that the render can be repeated
    Workspace &ws = s->nosync;
    if ((e & kErrCapacity) && ws.need.p) {
      unsigned long long need = 0;
      CK(cudaMemcpyAsync(&need, ws.need.p, 8, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      if (need > ws.key_cap) {
        ws.key_cap = need + need / 4;
        TRY(grow(ws.keys[0], ws.key_cap * 4));
      }
      CK(cudaMemsetAsync(ws.need.p, 0, 8, st));
    }
    CK(cudaMemsetAsync(s->status.p, 0, 4, st));
    if (e & kErrTimeout) return fail(FDGS_ERR_TIMEOUT, "device spin-wait limit reached");
    return fail(FDGS_ERR_CAPACITY, "device capacity exceeded");
  }
  return FDGS_OK;
}

// Key emission in depth-rank order, then the stable sort on the tile bits (the digit
// offsets were written by the tile scan). Returns the buffer holding the sorted keys.
template <typename K>
K *emit_and_sort(Workspace &ws, uint32_t nv, uint64_t nkeys, int gx, int gy, int rb, int tb,
                 int tight, uint32_t *ctr, uint32_t *err, cudaEvent_t *ev, cudaStream_t st) {
  K *k0 = ws.keys[0].as<K>(), *k1 = ws.keys[1].as<K>();
  K *out = k0;
  if (nkeys)
    launch_emit<K>(ws.rec_sorted.as<float>(), ws.offsets.as<uint32_t>(), nv, gx, gy, rb, tight,
                   k0, st);
  if (ev) cudaEventRecord(ev[6], st);
  if (nkeys)
    out = radix_sort<K>(k0, k1, ctr + C_NKEYS_LO, nkeys, rb, tb, ws.scratch.p, st, err, true);
  if (ev) cudaEventRecord(ev[7], st);
  return out;
}

// One render into workspace ws. want_flags: also write per-Gaussian decision flags.
// wsum: per-rank blend weights are accumulated (score pass); the buffer is zeroed here.
// no_sync: nothing waits for the device (fdgs_render_async): the coverage-bitmask lists are
// built into the workspace's fixed capacity ws.key_cap from device-side counts; lists that do
// not fit empty the frame's ranges and are reported through the status word.
int render_impl(fdgs_scene *s, Workspace &ws, const fdgs_camera *cam, float t,
                const fdgs_render_opts *opts, float *rgb, bool want_flags, bool want_wsum,
                bool use_mask_override, FrameMeta &m, cudaStream_t st, bool no_sync = false) {
  DevCam dc;
  TRY(make_cam(cam, dc));
  if (!rgb) return fail(FDGS_ERR_INVALID, "null output image");
  const uint32_t N = (uint32_t)s->d.n;
  const int W = dc.W, H = dc.H, gx = dc.gx, gy = dc.gy;
  const uint64_t tiles = (uint64_t)gx * gy, pixels = (uint64_t)W * H;
  const uint64_t parts = std::max<uint64_t>(1, (N + 255) / 256);
  const uint64_t n1 = std::max<uint64_t>(N, 1);
  const int tight = opts && opts->tile_sets == 1;
  TRY(grow(ws.ctr, C_COUNT * 4));
  if (!ws.hctr) CK(cudaMallocHost(&ws.hctr, C_COUNT * 4));
  TRY(grow(ws.pre_status, parts * 8));
  TRY(grow(ws.scan_status, parts * 8));
  TRY(grow(ws.rec, n1 * kRec * 4));
  TRY(grow(ws.rec_sorted, n1 * kRecS * 4));
  TRY(grow(ws.diff, (uint64_t)(gx + 1) * (gy + 1) * 4));
  // coverage bitmasks (one bit per depth rank, per tile row and per tile column) are written
  // by the gather whenever the bitmask list builder may be chosen after the key count is known
  const uint32_t mask_words = (uint32_t)((N + 255) / 256 * 8);
  const uint64_t mask_bytes = (uint64_t)(gx + gy) * mask_words * 4;
  const bool want_masks = g_list_mode != 1 && N > 0 && mask_bytes <= (512ull << 20);
  if (no_sync && ((N > 0 && !want_masks) || want_flags || want_wsum))
    return fail(FDGS_ERR_INVALID,
                "a render without host synchronisation needs the coverage-bitmask list builder "
                "(list mode 0 or 2, (tiles_x + tiles_y) * ceil(n / 256) * 32 B <= 512 MiB) and "
                "keeps no frame");
  if (want_masks) {
    TRY(grow(ws.rowmask, (uint64_t)gy * mask_words * 4));
    TRY(grow(ws.colmask, (uint64_t)gx * mask_words * 4));
  }
  TRY(grow(ws.vis[0], n1 * 8));
  TRY(grow(ws.vis[1], n1 * 8));
  TRY(grow(ws.offsets, n1 * 4));
  if (want_flags) TRY(grow(ws.flags, n1));
  TRY(grow(ws.ranges, tiles * 8));
  TRY(grow(ws.order, tiles * 4));
  TRY(grow(ws.Tf, pixels * 4));
  TRY(grow(ws.nc, pixels * 4));
  TRY(grow(ws.scratch, sort_scratch_bytes(n1, 32)));
  if (want_wsum) {
    TRY(grow(ws.wsum, n1 * 4));
    TRY(grow(ws.stopmark, n1 * 4));
  }

  const bool use_mask = use_mask_override && opts && opts->use_mask && s->n_key > 0;
  const uint32_t *ml = nullptr, *mr = nullptr;
  m.l = m.r = -1;
  if (use_mask) {
    keyframe_pair(s->key_times, t, m.l, m.r);
    ml = s->masks.as<uint32_t>() + (size_t)m.l * s->row_words;
    mr = s->masks.as<uint32_t>() + (size_t)m.r * s->row_words;
  }
  const bool prof = (s->prof & 1) && s->ev[0];
  const bool count = (s->prof & 2) && s->evals.p;
  if (count) CK(cudaMemsetAsync(s->evals.p, 0, 24, st));
  if (prof) CK(cudaEventRecord(s->ev[0], st));
  CK(cudaMemsetAsync(ws.ctr.p, 0, C_COUNT * 4, st));
  CK(cudaMemsetAsync(ws.pre_status.p, 0, parts * 8, st));
  CK(cudaMemsetAsync(ws.scan_status.p, 0, parts * 8, st));
  CK(cudaMemsetAsync(ws.diff.p, 0, (size_t)(gx + 1) * (gy + 1) * 4, st));
  uint32_t *ctr = ws.ctr.as<uint32_t>();
  uint32_t *err = s->status.as<uint32_t>();

  PreArgs pa;
  pa.mean4 = (const float4 *)s->d.mean4;
  pa.ls4 = (const float4 *)s->d.logscale4;
  pa.ql = (const float4 *)s->d.q_left;
  pa.qr = (const float4 *)s->d.q_right;
  pa.opacity = s->d.opacity_logit;
  pa.sh = s->d.sh;
  pa.sh_cb = s->sh_cb;
  pa.sh_code = s->sh_code;
  pa.deg = s->d.sh_degree;
  pa.n = N;
  pa.mask_l = ml;
  pa.mask_r = mr;
  pa.t = t;
  pa.cam = dc;
  pa.rec = ws.rec.as<float>();
  pa.vis_keys = ws.vis[0].as<uint64_t>();
  pa.flags = want_flags ? ws.flags.as<uint8_t>() : nullptr;
  pa.status = ws.pre_status.as<uint64_t>();
  pa.ctr = ctr;
  pa.err = err;
  pa.no_cull = opts && opts->no_temporal_cull ? 1 : 0;
  launch_preprocess(pa, st);
  if (prof) CK(cudaEventRecord(s->ev[1], st));
  uint64_t *sorted = radix_sort<uint64_t>(ws.vis[0].as<uint64_t>(), ws.vis[1].as<uint64_t>(),
                                          ctr + C_NVIS, N, 32, 32, ws.scratch.p, st, err);
  if (prof) CK(cudaEventRecord(s->ev[2], st));
  launch_gather_scan(sorted, ctr + C_NVIS, N, ws.rec.as<float>(), ws.rec_sorted.as<float>(),
                     ws.offsets.as<uint32_t>(), ws.scan_status.as<uint64_t>(), ctr, err, gx, gy,
                     ws.diff.as<int>(), want_masks ? ws.rowmask.as<uint32_t>() : nullptr,
                     want_masks ? ws.colmask.as<uint32_t>() : nullptr, mask_words, tight, st);
  if (prof) CK(cudaEventRecord(s->ev[3], st));
  CK(cudaGetLastError());
  uint32_t nv = 0;
  uint64_t nkeys = 0;
  const int tb = ceil_log2(std::max<uint64_t>(tiles, 2));
  bool use_masks = true;
  int rb = 32, key64 = 0;
  if (no_sync) {
    // lists into the fixed capacity, counts left on the device
    TRY(grow(ws.keys[0], std::max<uint64_t>(ws.key_cap, 1) * 4));
    if (!ws.need.p) {
      TRY(grow(ws.need, 8));
      CK(cudaMemsetAsync(ws.need.p, 0, 8, st));
    }
  } else {
    CK(cudaMemcpyAsync(ws.hctr, ctr, C_COUNT * 4, cudaMemcpyDeviceToHost, st));
    TRY(check_device_errors(s, st));   // synchronises the stream

    nv = ws.hctr[C_NVIS];
    nkeys = (uint64_t)ws.hctr[C_NKEYS_LO] | ((uint64_t)ws.hctr[C_NKEYS_HI] << 32);
    if (nkeys > kSortMaxKeys)
      return fail(FDGS_ERR_CAPACITY, "%llu tile keys exceed the sort limit",
                  (unsigned long long)nkeys);
    // List builder: coverage bitmasks read tiles x ceil(nv/32) word pairs from L2; emit + sort
    // move the keys through DRAM (1 write + 2 per pass). Bitmasks win when coverage is dense.
    const uint64_t words = (nv + 31) / 32;
    const int rb_sort = ceil_log2(std::max<uint32_t>(nv, 2));
    const uint64_t kb_sort = (rb_sort + tb) > 32 ? 8 : 4;
    use_masks = want_masks && nkeys > 0 &&
                (g_list_mode == 2 ||
                 tiles * words * 8 < 2 * nkeys * kb_sort * (1 + 2 * (uint64_t)sort_passes(tb)));
    rb = use_masks ? 32 : rb_sort;
    key64 = use_masks ? 0 : (rb + tb) > 32;
    const size_t kb = key64 ? 8 : 4;
    const uint64_t k1 = std::max<uint64_t>(nkeys, 1);
    TRY(grow(ws.keys[0], k1 * kb));
    if (!use_masks) TRY(grow(ws.keys[1], k1 * kb));
    TRY(grow(ws.scratch, std::max(sort_scratch_bytes(n1, 32), sort_scratch_bytes(k1, tb))));
  }
  if (want_wsum) {
    CK(cudaMemsetAsync(ws.wsum.p, 0, n1 * 4, st));
    CK(cudaMemsetAsync(ws.stopmark.p, 0, n1 * 4, st));
  }
  const uint32_t rmask = (uint32_t)((1ull << rb) - 1);
  BlendArgs ba;
  ba.ranges = ws.ranges.as<uint2>();
  ba.rec_sorted = ws.rec_sorted.as<float>();
  ba.W = W; ba.H = H; ba.gx = gx; ba.gy = gy;
  for (int c = 0; c < 3; ++c) ba.bg[c] = opts ? opts->bg[c] : 0.f;
  ba.rgb = rgb;
  // a render that keeps no frame, uncounted, on a black background needs no transmittance or
  // n_contrib: the forward-only blend (launch_blend takes it exactly when T_final is null)
  const bool fwd_only = !want_flags && !want_wsum && !count && ba.bg[0] == 0.f &&
                        ba.bg[1] == 0.f && ba.bg[2] == 0.f;
  ba.T_final = fwd_only ? nullptr : ws.Tf.as<float>();
  ba.n_contrib = fwd_only ? nullptr : ws.nc.as<uint32_t>();
  ba.w_sum = want_wsum ? ws.wsum.as<float>() : nullptr;
  ba.stop_mark = want_wsum ? ws.stopmark.as<uint32_t>() : nullptr;
  ba.evals = count ? s->evals.as<unsigned long long>() : nullptr;
  if (prof) CK(cudaEventRecord(s->ev[4], st));   // ev[3] -> ev[4]: the host synchronisation
  // tile ranges and the tile sort's digit offsets, straight from the coverage counts
  launch_tile_scan(ws.diff.as<int>(), gx, gy, use_masks ? 0 : sort_passes(tb),
                   sort_digit_bits(tb), ws.ranges.as<uint2>(), sort_hist(ws.scratch.p),
                   ws.order.as<uint32_t>(), st, no_sync ? std::max<uint64_t>(ws.key_cap, 1) : 0,
                   no_sync ? ws.need.as<unsigned long long>() : nullptr, err);
  ba.order = ws.order.as<uint32_t>();
  if (prof) CK(cudaEventRecord(s->ev[5], st));
  void *skeys;
  if (use_masks) {
    // lists of plain ranks straight in tile-major, depth order (the "emit" stage; no sort)
    launch_tile_lists(ws.rowmask.as<uint32_t>(), ws.colmask.as<uint32_t>(), mask_words, nv, gx,
                      gy, ws.ranges.as<uint2>(), ws.keys[0].as<uint32_t>(), st,
                      no_sync ? ctr + C_NVIS : nullptr);
    if (prof) CK(cudaEventRecord(s->ev[6], st));
    if (prof) CK(cudaEventRecord(s->ev[7], st));
    skeys = ws.keys[0].p;
  } else {
    skeys = key64 ? (void *)emit_and_sort<uint64_t>(ws, nv, nkeys, gx, gy, rb, tb, tight, ctr,
                                                     err, prof ? s->ev : nullptr, st)
                  : (void *)emit_and_sort<uint32_t>(ws, nv, nkeys, gx, gy, rb, tb, tight, ctr,
                                                     err, prof ? s->ev : nullptr, st);
  }
  if (key64)
    launch_blend<uint64_t>(ba, (const uint64_t *)skeys, rmask, st);
  else
    launch_blend<uint32_t>(ba, (const uint32_t *)skeys, rmask, st);
  if (prof) CK(cudaEventRecord(s->ev[8], st));
  CK(cudaGetLastError());
  m.cam = dc;
  m.t = t;
  m.W = W; m.H = H; m.gx = gx; m.gy = gy;
  m.n_active = ws.hctr[C_NACTIVE];
  m.nv = nv;
  m.nkeys = nkeys;
  m.key64 = key64;
  m.rb = rb;
  m.builder = use_masks ? 2 : 1;
  m.sorted = sorted;
  m.keys = skeys;
  for (int c = 0; c < 3; ++c) m.bg[c] = ba.bg[c];
  m.stream = st;
  return FDGS_OK;
}

Workspace *take_workspace(fdgs_scene *s) {
  if (!s->pool.empty()) {
    Workspace *w = s->pool.back();
    s->pool.pop_back();
    return w;
  }
  return new Workspace();
}

// ---- batched rendering -------------------------------------------------------------------

bool plan_matches(const BatchPlan *p, const fdgs_scene *s, const fdgs_camera *cams, int n,
                  bool masked) {
  if (!p || p->nreq != n || p->masked != masked || memcmp(&p->d, &s->d, sizeof(s->d)) != 0 ||
      p->sh_cb != s->sh_cb || p->sh_code != s->sh_code)
    return false;
  for (int i = 0; i < n; ++i)
    if (p->W[i] != cams[i].width || p->H[i] != cams[i].height) return false;
  return true;
}

// Grows the block lists to the plan's capacity. On failure the plan is marked unusable (its
// captured graph, which holds the old list pointers, is destroyed, and it matches no batch
// geometry), so that the next batch call builds a new plan.
int plan_alloc_lists(BatchPlan &p) {
  int rc = grow(p.lists, std::max<uint64_t>(p.key_cap, 1) * 4);
  if (rc == FDGS_OK) rc = grow(p.ltm, std::max<uint64_t>(p.key_cap, 1) * 2);
  if (rc != FDGS_OK) {
    if (p.exec) cudaGraphExecDestroy(p.exec);
    p.exec = nullptr;
    p.W.clear();
    p.H.clear();
    p.nreq = -1;
  }
  return rc;
}

int plan_build(fdgs_scene *s, BatchPlan &p, const fdgs_camera *cams, int n, bool masked);

// The plan of this batch geometry: the current one if it matches, else a new one. A plan
// whose construction failed (a refused allocation, a bad camera) is discarded, so that the
// next call starts again instead of matching a half-built plan.
int plan_prepare(fdgs_scene *s, const fdgs_camera *cams, int n, bool masked) {
  if (plan_matches(s->plan, s, cams, n, masked)) return FDGS_OK;
  delete s->plan;
  s->plan = new BatchPlan();
  const int rc = plan_build(s, *s->plan, cams, n, masked);
  if (rc != FDGS_OK) {
    delete s->plan;
    s->plan = nullptr;
  }
  return rc;
}

int plan_build(fdgs_scene *s, BatchPlan &p, const fdgs_camera *cams, int n, bool masked) {
  p.nreq = n;
  p.masked = masked;
  p.d = s->d;
  p.sh_cb = s->sh_cb;
  p.sh_code = s->sh_code;
  const uint32_t N = (uint32_t)s->d.n;
  p.mask_words = (N + 255) / 256 * 8;
  p.tmpl.resize(n);
  uint64_t tiles = 0, blocks = 0, mask = 0;
  for (int i = 0; i < n; ++i) {
    DevCam dc;
    TRY(make_cam(&cams[i], dc));
    p.W.push_back(dc.W);
    p.H.push_back(dc.H);
    ReqDesc &q = p.tmpl[i];
    memset(&q, 0, sizeof q);
    q.tile_base = (uint32_t)tiles;
    q.mask_base = mask;
    q.block_base = (uint32_t)blocks;
    const uint64_t bgx = (dc.gx + kListBlock - 1) / kListBlock;
    const uint64_t bgy = (dc.gy + kListBlock - 1) / kListBlock;
    blocks += bgx * bgy;
    tiles += (uint64_t)dc.gx * dc.gy;
    mask += (bgx + bgy) * p.mask_words;
  }
  if (tiles >= (1ull << 32))
    return fail(FDGS_ERR_INVALID, "batch too large");
  p.ntiles = (uint32_t)tiles;
  p.nblocks = (uint32_t)blocks;
  p.mask_total = mask;
  p.rn = (uint64_t)n * N;
  p.slot_cap = p.rn + (uint64_t)n * 256;
  // block-list entries; a batch that needs more regrows the lists and reruns
  p.key_cap = s->list_cap_hint ? s->list_cap_hint : std::max<uint64_t>(p.rn * 8, 1 << 20);
  const uint64_t P = (N + 255) / 256;
  TRY(grow(p.reqs, n * sizeof(ReqDesc)));
  TRY(grow(p.ctr, BC_COUNT * 4));
  TRY(grow(p.part, std::max<uint64_t>(P * n, 1) * 8));
  if ((uint64_t)n * N >= (1ull << 32))
    return fail(FDGS_ERR_INVALID, "batch too large: requests x Gaussians must stay below 2^32");
  TRY(grow(p.rec, std::max<uint64_t>(p.rn, 1) * kRec * 4));
  TRY(grow(p.rect_id, std::max<uint64_t>(p.rn, 1) * 8));
  TRY(grow(p.vis_seg, std::max<uint64_t>(P * n * 256, 1) * 8));
  TRY(grow(p.vis, std::max<uint64_t>(p.rn, 1) * 8));
  TRY(grow(p.vis_alt, std::max<uint64_t>(p.rn, 1) * 8));
  TRY(grow(p.nv, n * 4));
  TRY(grow(p.vis_base, n * 4));
  TRY(grow(p.slot_base, n * 4));
  TRY(grow(p.key_cnt, n * 8));
  TRY(grow(p.ridx, p.slot_cap * 4));
  TRY(grow(p.rect, p.slot_cap * 8));
  TRY(grow(p.cond, std::max<uint64_t>(N, 1) * 80));
  TRY(grow(p.masks, std::max<uint64_t>(mask, 1) * 4));
  TRY(grow(p.ranges, tiles * 8));
  TRY(grow(p.branges, std::max<uint64_t>(blocks, 1) * 8));
  TRY(grow(p.bcount, std::max<uint64_t>(blocks, 1) * 4));
  TRY(grow(p.bkey_cnt, n * 8));
  TRY(grow(p.qkeys, tiles * 8));
  TRY(grow(p.qkeys_alt, tiles * 8));
  TRY(grow(p.done, n * 8));
  TRY(grow(p.t0, 8));
  TRY(grow(p.scratch, std::max(sort_scratch_bytes(std::max<uint64_t>(p.rn, 1), 39),
                               sort_scratch_bytes(tiles, 24))));
  TRY(plan_alloc_lists(p));
  CK(cudaHostAlloc(&p.h_reqs, n * sizeof(ReqDesc), cudaHostAllocMapped));
  CK(cudaHostAlloc(&p.h_ctr, BC_COUNT * 4, cudaHostAllocMapped));
  CK(cudaHostAlloc(&p.h_done, (n + 1) * 8, cudaHostAllocMapped));
  CK(cudaHostAlloc(&p.h_status, 4, cudaHostAllocMapped));
  CK(cudaStreamCreateWithFlags(&p.cap, cudaStreamNonBlocking));
  TRY(grow(p.stamps, (kBatchStages + 1) * 8));
  CK(cudaHostAlloc(&p.h_stamps, (kBatchStages + 1) * 8, cudaHostAllocMapped));
  CK(cudaHostGetDevicePointer((void **)&p.d_h_reqs, p.h_reqs, 0));
  CK(cudaHostGetDevicePointer((void **)&p.d_h_ctr, p.h_ctr, 0));
  CK(cudaHostGetDevicePointer((void **)&p.d_h_done, p.h_done, 0));
  CK(cudaHostGetDevicePointer((void **)&p.d_h_status, p.h_status, 0));
  CK(cudaHostGetDevicePointer((void **)&p.d_h_stamps, p.h_stamps, 0));
  p.footprint = s->batch_footprint;
  p.ctas = s->batch_ctas ? s->batch_ctas : batch_blend_max_ctas_per_sm(p.footprint);
  return FDGS_OK;
}

// Per-call request contents: camera, time, mask rows of the two nearest key-frames, output.
int plan_fill(fdgs_scene *s, BatchPlan &p, const fdgs_camera *cams, const float *ts,
              const fdgs_render_opts *opts, float *const *rgb) {
  for (int i = 0; i < p.nreq; ++i) {
    ReqDesc q = p.tmpl[i];
    TRY(make_cam(&cams[i], q.cam));
    if (!rgb[i]) return fail(FDGS_ERR_INVALID, "null output image for request %d", i);
    q.t = ts[i];
    q.rgb = rgb[i];
    for (int c = 0; c < 3; ++c) q.bg[c] = opts ? opts->bg[c] : 0.f;
    if (i == 0) p.black = q.bg[0] == 0.f && q.bg[1] == 0.f && q.bg[2] == 0.f;
    q.mask_l = q.mask_r = nullptr;
    if (p.masked) {
      int l, r;
      keyframe_pair(s->key_times, ts[i], l, r);
      q.mask_l = s->masks.as<uint32_t>() + (size_t)l * s->row_words;
      q.mask_r = s->masks.as<uint32_t>() + (size_t)r * s->row_words;
    }
    p.h_reqs[i] = q;
  }
  return FDGS_OK;
}

void plan_dev(const fdgs_scene *s, BatchPlan &p, BatchDev &b, BatchLaunch &L) {
  b.reqs = p.reqs.as<ReqDesc>();
  b.nreq = p.nreq;
  b.n = (uint32_t)s->d.n;
  b.ntiles = p.ntiles;
  b.nblocks = p.nblocks;
  {
    // partition-major preprocess when the attributes (and SH) outgrow half of L2: each
    // partition's attributes are then read once from DRAM for all requests (measured on 3M
    // Gaussians: 9.0 vs 11.3 ms per 64 requests; on 200k, which fits, 0.63 vs 0.60 ms)
    static int l2 = -1;
    if (l2 < 0) {
      int dev = 0;
      cudaGetDevice(&dev);
      if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess) l2 = 0;
    }
    const uint64_t k = (uint64_t)(s->d.sh_degree + 1) * (s->d.sh_degree + 1);
    const uint64_t bytes = (uint64_t)s->d.n * (68 + 12 * k);
    b.part_major = l2 > 0 && bytes > (uint64_t)l2 / 2 ? 1 : 0;
  }
  b.mask_words = p.mask_words;
  b.key_cap = p.key_cap;
  b.mean4 = (const float4 *)s->d.mean4;
  b.ls4 = (const float4 *)s->d.logscale4;
  b.ql = (const float4 *)s->d.q_left;
  b.qr = (const float4 *)s->d.q_right;
  b.opacity = s->d.opacity_logit;
  b.sh = s->d.sh;
  b.sh_cb = s->sh_cb;
  b.sh_code = s->sh_code;
  b.deg = s->d.sh_degree;
  b.ctr = p.ctr.as<uint32_t>();
  b.err = s->status.as<uint32_t>();
  b.part = p.part.as<uint2>();
  b.rec = p.rec.as<float>();
  b.vis_seg = p.vis_seg.as<uint64_t>();
  b.vis = p.vis.as<uint64_t>();
  b.vis_alt = p.vis_alt.as<uint64_t>();
  b.vis_sorted = nullptr;
  b.nv = p.nv.as<uint32_t>();
  b.vis_base = p.vis_base.as<uint32_t>();
  b.slot_base = p.slot_base.as<uint32_t>();
  b.key_cnt = p.key_cnt.as<unsigned long long>();
  b.rect_id = p.rect_id.as<uint2>();
  b.ridx = p.ridx.as<uint32_t>();
  b.cond = p.cond.as<float4>();
  b.rect = p.rect.as<uint2>();
  b.masks = p.masks.as<uint32_t>();
  b.ranges = p.ranges.as<uint2>();
  b.branges = p.branges.as<uint2>();
  b.bcount = p.bcount.as<uint32_t>();
  b.bkey_cnt = p.bkey_cnt.as<unsigned long long>();
  b.ltm = p.ltm.as<uint16_t>();
  b.qkeys = p.qkeys.as<uint64_t>();
  b.qkeys_alt = p.qkeys_alt.as<uint64_t>();
  b.queue = nullptr;
  b.lists = p.lists.as<uint32_t>();
  b.done_ns = p.done.as<unsigned long long>();
  b.t0_ns = p.t0.as<unsigned long long>();
  b.evals = nullptr;
  b.stamps = p.stamps.as<unsigned long long>();
  b.w_sum = p.weighted ? p.wsum.as<float>() : nullptr;
  b.stop_mark = p.weighted ? p.stop.as<uint32_t>() : nullptr;
  b.gamma = p.gamma;
  b.sig_t = p.sig_t;
  b.score = p.score_out;
  b.score_variant = p.score_variant;
  b.mark = p.mark ? 1 : 0;
  L.wsum_len = p.rn;
  L.sort_scratch = p.scratch.p;
  L.footprint = p.footprint;
  L.blend_ctas_per_sm = p.ctas;
  L.staging = g_batch_staging;
  L.black = p.black;
  b.tma_skip = g_debug_tma_skip;
  b.tma_spin = g_debug_tma_skip ? 4096u : 0u;
  b.rec_map_ok = 0;
  if (g_batch_staging == 1) encode_record_map(b, p.rn);   // cp.async staging if it fails
}

// The request descriptors from the mapped host array to the device, by a kernel.
static_assert(sizeof(ReqDesc) % 4 == 0, "descriptors are copied as 32-bit words");
void upload_reqs(BatchPlan &p, cudaStream_t st) {
  WordJobs j{};
  j.src[0] = reinterpret_cast<const uint32_t *>(p.d_h_reqs);
  j.dst[0] = static_cast<uint32_t *>(p.reqs.p);
  j.n[0] = (uint32_t)(p.nreq * sizeof(ReqDesc) / 4);
  j.count = 1;
  launch_copy_words(j, st);
}

int plan_capture(fdgs_scene *s, BatchPlan &p) {
  if (p.exec) {
    cudaGraphExecDestroy(p.exec);
    p.exec = nullptr;
  }
  BatchDev b;
  BatchLaunch L;
  plan_dev(s, p, b, L);
  b.w_sum = nullptr;   // a graph never holds a weighted pass (they run eagerly)
  b.stop_mark = nullptr;
  b.gamma = nullptr;
  b.sig_t = nullptr;
  b.score = nullptr;
  b.score_variant = 0;
  b.mark = 0;
  b.tma_skip = 0;      // injections never enter a captured graph
  b.tma_spin = 0;
  p.staging = g_batch_staging;
  p.cap_black = p.black;
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(p.cap, cudaStreamCaptureModeRelaxed));
  upload_reqs(p, p.cap);
  launch_batch(b, L, p.cap);
  p.vis_sorted = L.vis_sorted;
  const cudaError_t e = cudaStreamEndCapture(p.cap, &g);
  if (e != cudaSuccess) return fail(FDGS_ERR_CUDA, "batch graph capture: %s", cudaGetErrorString(e));
  const cudaError_t e2 = cudaGraphInstantiate(&p.exec, g, 0);
  cudaGraphDestroy(g);
  if (e2 != cudaSuccess) {
    p.exec = nullptr;
    return fail(FDGS_ERR_CUDA, "batch graph instantiate: %s", cudaGetErrorString(e2));
  }
  return FDGS_OK;
}

// Runs the batch (graph replay when captured, else eagerly), synchronises the stream, grows
// the list capacity and reruns if it overflowed, records per-request latencies.
int plan_run(fdgs_scene *s, BatchPlan &p, cudaStream_t st) {
  // a counting profile (fdgs_profile_enable bit1) runs the batch eagerly with the counting
  // blend variant, so that fdgs_profile_read returns its evaluation and test counts
  const bool count = (s->prof & 2) && s->evals.p;
  if (p.exec && (p.staging != g_batch_staging || p.cap_black != p.black))
    TRY(plan_capture(s, p));
  // an injected stage-barrier failure runs the batch eagerly, once
  const bool inject = g_debug_tma_skip != 0 && g_batch_staging == 1;
  for (int attempt = 0; attempt < 4; ++attempt) {
    if (p.exec && !count && !p.weighted && !inject) {
      CK(cudaGraphLaunch(p.exec, st));
    } else {
      BatchDev b;
      BatchLaunch L;
      plan_dev(s, p, b, L);
      if (count) b.evals = s->evals.as<unsigned long long>();
      upload_reqs(p, st);
      launch_batch(b, L, st);
      p.vis_sorted = L.vis_sorted;
      if (inject) g_debug_tma_skip = 0;
    }
    // counters, completion times, stage stamps and the status word, written by the GPU
    // straight into pinned host memory
    WordJobs j{};
    auto job = [&](const void *src, void *dst, size_t bytes) {
      j.src[j.count] = static_cast<const uint32_t *>(src);
      j.dst[j.count] = static_cast<uint32_t *>(dst);
      j.n[j.count] = (uint32_t)(bytes / 4);
      ++j.count;
    };
    job(p.ctr.p, p.d_h_ctr, BC_COUNT * 4);
    job(p.done.p, p.d_h_done, p.nreq * 8);
    job(p.t0.p, p.d_h_done + p.nreq, 8);
    job(p.stamps.p, p.d_h_stamps, (kBatchStages + 1) * 8);
    job(s->status.p, p.d_h_status, 4);
    launch_copy_words(j, st);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    const uint32_t e = *(volatile uint32_t *)p.h_status;
    if (e & kErrTimeout) {
      CK(cudaMemset(s->status.p, 0, 4));
      return fail(FDGS_ERR_TIMEOUT, "device spin-wait limit reached");
    }
    if (e & kErrCapacity) {
      CK(cudaMemset(s->status.p, 0, 4));
      const uint64_t nkeys =
          (uint64_t)p.h_ctr[BC_NBKEYS_LO] | ((uint64_t)p.h_ctr[BC_NBKEYS_HI] << 32);
      if (nkeys >= (1ull << 32)) return fail(FDGS_ERR_CAPACITY, "batch has >= 2^32 list entries");
      p.key_cap = nkeys + nkeys / 8 + 1024;
      TRY(plan_alloc_lists(p));
      if (p.exec) TRY(plan_capture(s, p));
      continue;
    }
    for (int i = 0; i < kBatchStages; ++i)
      p.stage_ms[i] = p.h_stamps[i + 1] > p.h_stamps[i]
                          ? (float)((p.h_stamps[i + 1] - p.h_stamps[i]) * 1e-6)
                          : 0.f;
    p.lat_ms.resize(p.nreq);
    const unsigned long long t0 = p.h_done[p.nreq];
    for (int i = 0; i < p.nreq; ++i)
      p.lat_ms[i] = p.h_done[i] > t0 ? (float)((p.h_done[i] - t0) * 1e-6) : 0.f;
    return FDGS_OK;
  }
  return fail(FDGS_ERR_CAPACITY, "batch list capacity kept overflowing");
}

int batch_args_ok(fdgs_scene *s, const fdgs_camera *cams, const float *ts, int n_req,
                  float *const *rgb) {
  if (!s) return fail(FDGS_ERR_INVALID, "null scene");
  if (n_req < 0 || n_req > 128 || (n_req > 0 && (!cams || !ts || !rgb)))
    return fail(FDGS_ERR_INVALID, "bad batch arguments (1..128 requests)");
  if (s->d.n >= (1ll << 25)) return fail(FDGS_ERR_INVALID, "batched path needs n < 2^25");
  return FDGS_OK;
}

}  // namespace

void fdgs::set_error_message(const char *msg) { g_err = msg ? msg : ""; }
int fdgs::g_list_mode = 0;
int fdgs::g_batch_staging = 0;
uint32_t fdgs::g_debug_tma_skip = 0;

extern "C" {

const char *fdgs_last_error(void) { return g_err.c_str(); }
const char *fdgs_version(void) { return "fdgs 0.1 (sm_103a)"; }

int fdgs_create_scene(const fdgs_scene_desc *desc, fdgs_scene **out) {
  if (!out) return fail(FDGS_ERR_INVALID, "null output pointer");
  *out = nullptr;
  TRY(check_desc(desc));
  fdgs_scene *s = new fdgs_scene();
  s->d = *desc;
  cudaGetDevice(&s->device);
  if (grow(s->status, 4) != FDGS_OK) {
    delete s;
    return FDGS_ERR_OOM;
  }
  if (cudaMemset(s->status.p, 0, 4) != cudaSuccess) {
    delete s;
    return fail(FDGS_ERR_CUDA, "cudaMemset failed");
  }
  *out = s;
  return FDGS_OK;
}

int fdgs_update_scene(fdgs_scene *s, const fdgs_scene_desc *desc) {
  if (!s) return fail(FDGS_ERR_INVALID, "null scene");
  TRY(check_desc(desc));
  if (desc->n != s->d.n && s->n_key > 0) {
    s->n_key = 0;
    s->key_times.clear();
  }
  s->d = *desc;
  return FDGS_OK;
}

int fdgs_destroy_scene(fdgs_scene *s) {
  if (!s) return FDGS_OK;
  cudaDeviceSynchronize();
  for (fdgs_frame *f : s->live) {
    delete f->ws;
    delete f;
  }
  for (Workspace *w : s->pool) delete w;
  delete s->plan;
  s->masks.release();
  s->status.release();
  s->evals.release();
  for (auto &e : s->ev)
    if (e) cudaEventDestroy(e);
  for (Buf &b : s->aux) b.release();
  delete s;
  return FDGS_OK;
}

int fdgs_set_active_mask(fdgs_scene *s, const uint8_t *bits_dev, const float *key_times,
                         int n_key, fdgs_stream stream) {
  NvtxRange nvtx_range_("fdgs_set_active_mask");
  if (!s) return fail(FDGS_ERR_INVALID, "null scene");
  cudaStream_t st = (cudaStream_t)stream;
  if (n_key < 0) return fail(FDGS_ERR_INVALID, "n_key < 0");
  if (n_key == 0) {
    s->n_key = 0;
    s->key_times.clear();
    return FDGS_OK;
  }
  if (!bits_dev || !key_times) return fail(FDGS_ERR_INVALID, "null mask pointer");
  for (int i = 1; i < n_key; ++i)
    if (!(key_times[i] >= key_times[i - 1]))
      return fail(FDGS_ERR_INVALID, "key-frame times must be ascending");
  const size_t n = (size_t)s->d.n;
  const size_t row_bytes = (n + 7) / 8;
  const size_t words = ((n + 31) / 32 + 3) / 4 * 4;   // padded to 16 bytes
  TRY(grow(s->masks, std::max<size_t>(words * 4 * n_key, 16)));
  CK(cudaMemsetAsync(s->masks.p, 0, words * 4 * n_key, st));
  if (row_bytes)
    CK(cudaMemcpy2DAsync(s->masks.p, words * 4, bits_dev, row_bytes, row_bytes, n_key,
                         cudaMemcpyDeviceToDevice, st));
  s->row_words = words;
  s->n_key = n_key;
  s->key_times.assign(key_times, key_times + n_key);
  return FDGS_OK;
}

int fdgs_render(fdgs_scene *s, const fdgs_camera *cam, float t, const fdgs_render_opts *opts,
                float *rgb_out_dev, fdgs_frame **frame_out, fdgs_stream stream) {
  NvtxRange nvtx_range_("fdgs_render");
  if (!s) return fail(FDGS_ERR_INVALID, "null scene");
  cudaStream_t st = (cudaStream_t)stream;
  if (frame_out) *frame_out = nullptr;
  if (!frame_out) {
    FrameMeta m;
    return render_impl(s, s->main, cam, t, opts, rgb_out_dev, false, false, true, m, st);
  }
  Workspace *ws = take_workspace(s);
  fdgs_frame *f = new fdgs_frame{s, ws, FrameMeta()};
  int rc = render_impl(s, *ws, cam, t, opts, rgb_out_dev, true, false, true, f->m, st);
  if (rc != FDGS_OK) {
    s->pool.push_back(ws);
    delete f;
    return rc;
  }
  s->live.insert(f);
  *frame_out = f;
  return FDGS_OK;
}

int fdgs_render_async(fdgs_scene *s, const fdgs_camera *cam, float t,
                      const fdgs_render_opts *opts, float *rgb_out_dev, fdgs_stream stream) {
  NvtxRange nvtx_range_("fdgs_render_async");
  if (!s) return fail(FDGS_ERR_INVALID, "null scene");
  cudaStream_t st = (cudaStream_t)stream;
  DevCam dc;
  TRY(make_cam(cam, dc));
  const uint64_t mask_bytes = (uint64_t)(dc.gx + dc.gy) * (((uint64_t)s->d.n + 255) / 256 * 8) * 4;
  if (g_list_mode == 1 || mask_bytes > (512ull << 20))
    return fail(FDGS_ERR_INVALID,
                "fdgs_render_async needs the coverage-bitmask list builder (list mode 0 or 2, "
                "(tiles_x + tiles_y) * ceil(n / 256) * 32 B <= 512 MiB)");
  Workspace &ws = s->nosync;
  FrameMeta m;
  if (ws.key_cap == 0) {
    // the first call sizes the list capacity with one synchronised render: twice its lists
    // (4 bytes an entry), room for the other frames of a sequence
    TRY(render_impl(s, ws, cam, t, opts, rgb_out_dev, false, false, true, m, st));
    ws.key_cap = 2 * m.nkeys + 65536;
    TRY(grow(ws.keys[0], ws.key_cap * 4));
    if (!ws.need.p) {
      TRY(grow(ws.need, 8));
      CK(cudaMemsetAsync(ws.need.p, 0, 8, st));
    }
    return FDGS_OK;
  }
  return render_impl(s, ws, cam, t, opts, rgb_out_dev, false, false, true, m, st, true);
}

int fdgs_reserve_render_lists(fdgs_scene *s, uint64_t entries) {
  if (!s) return fail(FDGS_ERR_INVALID, "null scene");
  if (entries > kSortMaxKeys) return fail(FDGS_ERR_INVALID, "entries above the list limit");
  Workspace &ws = s->nosync;
  ws.key_cap = entries;
  if (entries) {
    TRY(grow(ws.keys[0], entries * 4));
    if (!ws.need.p) {
      TRY(grow(ws.need, 8));
      CK(cudaMemset(ws.need.p, 0, 8));
    }
  }
  return FDGS_OK;
}

int fdgs_frame_release(fdgs_frame *f) {
  if (!f) return FDGS_OK;
  fdgs_scene *s = f->scene;
  if (s->live.erase(f) == 0) return fail(FDGS_ERR_STATE, "frame not live");
  s->pool.push_back(f->ws);
  delete f;
  return FDGS_OK;
}

int fdgs_frame_get_stats(fdgs_frame *f, fdgs_frame_stats *o) {
  if (!f || !o) return fail(FDGS_ERR_INVALID, "null argument");
  CK(cudaStreamSynchronize(f->m.stream));
  o->n_active = f->m.n_active;
  o->n_visible = f->m.nv;
  o->n_keys = (int64_t)f->m.nkeys;
  o->width = f->m.W;
  o->height = f->m.H;
  o->tiles_x = f->m.gx;
  o->tiles_y = f->m.gy;
  o->key_l = f->m.l;
  o->key_r = f->m.r;
  o->key_bytes = f->m.key64 ? 8 : 4;
  o->list_builder = f->m.builder;
  return FDGS_OK;
}

int fdgs_frame_export(fdgs_frame *f, uint32_t *tile_ranges_dev, uint32_t *tile_ids_dev,
                      float *T_final_dev, uint32_t *n_contrib_dev, uint8_t *gauss_flags_dev,
                      float *records_dev, fdgs_stream stream) {
  if (!f) return fail(FDGS_ERR_INVALID, "null frame");
  cudaStream_t st = (cudaStream_t)stream;
  const FrameMeta &m = f->m;
  Workspace &ws = *f->ws;
  const size_t tiles = (size_t)m.gx * m.gy, pixels = (size_t)m.W * m.H;
  if (tile_ranges_dev)
    CK(cudaMemcpyAsync(tile_ranges_dev, ws.ranges.p, tiles * 8, cudaMemcpyDeviceToDevice, st));
  if (tile_ids_dev && m.nkeys) {
    const uint32_t rmask = (uint32_t)((1ull << m.rb) - 1);
    if (m.key64)
      launch_keys_to_ids<uint64_t>((const uint64_t *)m.keys, (uint32_t)m.nkeys, rmask, m.sorted,
                                   tile_ids_dev, st);
    else
      launch_keys_to_ids<uint32_t>((const uint32_t *)m.keys, (uint32_t)m.nkeys, rmask, m.sorted,
                                   tile_ids_dev, st);
  }
  if (T_final_dev)
    CK(cudaMemcpyAsync(T_final_dev, ws.Tf.p, pixels * 4, cudaMemcpyDeviceToDevice, st));
  if (n_contrib_dev)
    CK(cudaMemcpyAsync(n_contrib_dev, ws.nc.p, pixels * 4, cudaMemcpyDeviceToDevice, st));
  if (gauss_flags_dev && f->scene->d.n)
    CK(cudaMemcpyAsync(gauss_flags_dev, ws.flags.p, (size_t)f->scene->d.n,
                       cudaMemcpyDeviceToDevice, st));
  if (records_dev)
    launch_export_records(m.sorted, m.nv, ws.rec.as<float>(), records_dev, st);
  CK(cudaGetLastError());
  return FDGS_OK;
}

int fdgs_render_backward(fdgs_scene *s, fdgs_frame *f, const float *dL_drgb_dev,
                         float *g_mean4, float *g_logscale4, float *g_q_left, float *g_q_right,
                         float *g_opacity_logit, float *g_sh, fdgs_stream stream) {
  NvtxRange nvtx_range_("fdgs_render_backward");
  if (!s || !f) return fail(FDGS_ERR_INVALID, "null argument");
  if (f->scene != s || !s->live.count(f)) return fail(FDGS_ERR_STATE, "frame not of this scene");
  if (!dL_drgb_dev) return fail(FDGS_ERR_INVALID, "null dL/drgb");
  if (s->sh_cb)
    return fail(FDGS_ERR_STATE, "backward needs full SH coefficients (a codebook is set)");
  cudaStream_t st = (cudaStream_t)stream;
  const FrameMeta &m = f->m;
  Workspace &ws = *f->ws;
  if (m.nv == 0) return FDGS_OK;
  TRY(grow(ws.g2d, (size_t)m.nv * 9 * 4));
  CK(cudaMemsetAsync(ws.g2d.p, 0, (size_t)m.nv * 9 * 4, st));
  BlendBwdArgs ba;
  ba.ranges = ws.ranges.as<uint2>();
  ba.rec_sorted = ws.rec_sorted.as<float>();
  ba.W = m.W; ba.H = m.H; ba.gx = m.gx; ba.gy = m.gy;
  for (int c = 0; c < 3; ++c) ba.bg[c] = m.bg[c];
  ba.dL_drgb = dL_drgb_dev;
  ba.T_final = ws.Tf.as<float>();
  ba.n_contrib = ws.nc.as<uint32_t>();
  ba.g2d = ws.g2d.as<float>();
  ba.order = ws.order.as<uint32_t>();   // the forward's longest-first tile order
  if ((s->prof & 2) && s->evals.p) {
    CK(cudaMemsetAsync(s->evals.p, 0, 24, st));
    ba.evals = s->evals.as<unsigned long long>();
  }
  const uint32_t rmask = (uint32_t)((1ull << m.rb) - 1);
  const bool prof = (s->prof & 1) && s->ev[0];
  if (prof) CK(cudaEventRecord(s->ev[9], st));
  if (m.key64)
    launch_blend_bwd<uint64_t>(ba, (const uint64_t *)m.keys, rmask, st);
  else
    launch_blend_bwd<uint32_t>(ba, (const uint32_t *)m.keys, rmask, st);
  if (prof) CK(cudaEventRecord(s->ev[10], st));
  PreBwdArgs pa;
  pa.mean4 = (const float4 *)s->d.mean4;
  pa.ls4 = (const float4 *)s->d.logscale4;
  pa.ql = (const float4 *)s->d.q_left;
  pa.qr = (const float4 *)s->d.q_right;
  pa.opacity = s->d.opacity_logit;
  pa.sh = s->d.sh;
  pa.deg = s->d.sh_degree;
  pa.n = (uint32_t)s->d.n;
  pa.nv = m.nv;
  pa.t = m.t;
  pa.cam = m.cam;
  pa.sorted = m.sorted;
  pa.g2d = ws.g2d.as<float>();
  pa.g_mean4 = g_mean4;
  pa.g_ls4 = g_logscale4;
  pa.g_ql = g_q_left;
  pa.g_qr = g_q_right;
  pa.g_op = g_opacity_logit;
  pa.g_sh = g_sh;
  launch_preprocess_bwd(pa, st);
  if (prof) CK(cudaEventRecord(s->ev[11], st));
  CK(cudaGetLastError());
  return FDGS_OK;
}

int fdgs_render_batch(fdgs_scene *s, const fdgs_camera *cams, const float *ts, int n_req,
                      const fdgs_render_opts *opts, float *const *rgb_out_dev,
                      fdgs_stream stream) {
  NvtxRange nvtx_range_("fdgs_render_batch");
  TRY(batch_args_ok(s, cams, ts, n_req, rgb_out_dev));
  if (n_req == 0 || s->d.n == 0) {
    for (int i = 0; i < n_req; ++i) {   // empty scene: background only
      FrameMeta m;
      TRY(render_impl(s, s->main, &cams[i], ts[i], opts, rgb_out_dev[i], false, false, true, m,
                      (cudaStream_t)stream));
    }
    return FDGS_OK;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const bool masked = opts && opts->use_mask && s->n_key > 0;
  TRY(plan_prepare(s, cams, n_req, masked));
  BatchPlan &p = *s->plan;
  TRY(plan_fill(s, p, cams, ts, opts, rgb_out_dev));
  const bool first = !p.exec;
  TRY(plan_run(s, p, st));
  if (first) TRY(plan_capture(s, p));   // later calls of this geometry replay the graph
  return FDGS_OK;
}

int fdgs_batch_autotune(fdgs_scene *s, const fdgs_camera *cams, const float *ts, int n_req,
                        const fdgs_render_opts *opts, float *const *rgb_out_dev,
                        fdgs_stream stream) {
  NvtxRange nvtx_range_("fdgs_batch_autotune");
  TRY(batch_args_ok(s, cams, ts, n_req, rgb_out_dev));
  if (n_req == 0 || s->d.n == 0) return FDGS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const bool masked = opts && opts->use_mask && s->n_key > 0;
  TRY(plan_prepare(s, cams, n_req, masked));
  BatchPlan &p = *s->plan;
  TRY(plan_fill(s, p, cams, ts, opts, rgb_out_dev));
  TRY(plan_run(s, p, st));   // sizes the list capacity
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_f = p.footprint, best_c = p.ctas;
  for (int f = 0; f < kBlendShapes; ++f) {
    // resident CTAs per SM: the occupancy limit and half of it
    const int maxc = batch_blend_max_ctas_per_sm(f, p.black != 0);
    std::vector<int> ctas = {std::max(1, maxc / 2), maxc};
    ctas.erase(std::unique(ctas.begin(), ctas.end()), ctas.end());
    for (int c : ctas) {
      p.footprint = f;
      p.ctas = c;
      TRY(plan_capture(s, p));
      TRY(plan_run(s, p, st));   // warm
      float tot = 0.f;
      for (int rep = 0; rep < 3; ++rep) {
        CK(cudaEventRecord(e0, st));
        CK(cudaGraphLaunch(p.exec, st));
        CK(cudaEventRecord(e1, st));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        tot += ms;
      }
      if (tot < best) {
        best = tot;
        best_f = f;
        best_c = c;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  p.footprint = best_f;
  p.ctas = best_c;
  p.tuned = true;
  TRY(plan_capture(s, p));
  return plan_run(s, p, st);
}

int fdgs_batch_info(fdgs_scene *s, float *latency_ms, int n, int *footprint,
                    int *ctas_per_sm, float *stage_ms) {
  if (!s) return fail(FDGS_ERR_INVALID, "null scene");
  if (!s->plan) return fail(FDGS_ERR_STATE, "no batch has been rendered");
  BatchPlan &p = *s->plan;
  if (stage_ms)
    for (int i = 0; i < kBatchStages; ++i) stage_ms[i] = p.stage_ms[i];
  if (latency_ms)
    for (int i = 0; i < std::min(n, (int)p.lat_ms.size()); ++i) latency_ms[i] = p.lat_ms[i];
  if (footprint) *footprint = p.footprint;
  if (ctas_per_sm) *ctas_per_sm = p.ctas;
  return FDGS_OK;
}

int fdgs_build_keyframe_masks(fdgs_scene *s, const fdgs_camera *cams, int n_cam,
                              const float *key_times, int n_key, uint8_t *bits_out_dev,
                              fdgs_stream stream) {
  NvtxRange nvtx_range_("fdgs_build_keyframe_masks");
  if (!s) return fail(FDGS_ERR_INVALID, "null scene");
  if (n_cam < 0 || n_key < 0 || (n_key > 0 && (!key_times || !bits_out_dev)) ||
      (n_cam > 0 && !cams))
    return fail(FDGS_ERR_INVALID, "bad key-frame mask arguments");
  cudaStream_t st = (cudaStream_t)stream;
  const uint32_t N = (uint32_t)s->d.n;
  const uint32_t nbytes = (N + 7) / 8, words = (N + 31) / 32;
  if (n_key == 0) return FDGS_OK;
  CK(cudaMemsetAsync(bits_out_dev, 0, (size_t)n_key * nbytes, st));
  if (N == 0 || n_cam == 0) return FDGS_OK;
  fdgs_render_opts o{};
  o.use_mask = 0;   // the masks are built from unfiltered renders
  o.tile_sets = 1;  // same blend decisions as the 3-sigma squares, shorter lists
  const int total = n_key * n_cam;
  if (total > 1 && N < (1u << kBatchIdBits)) {
    // every (key-frame, view) render through the batched pipeline, 16 per batch, with the
    // weighted persistent blend marking its contributors in the key-frame's word row; a
    // last, partial batch is padded with repeats that mark nothing, so every batch has the
    // same geometry and reuses one plan
    TRY(grow(s->aux[5], (size_t)n_key * words * 4));
    uint32_t *rows = s->aux[5].as<uint32_t>();
    CK(cudaMemsetAsync(rows, 0, (size_t)n_key * words * 4, st));
    std::vector<fdgs_camera> bc;
    std::vector<float> bt;
    std::vector<float *> outs;
    const int per = std::min(16, total);
    for (int i0 = 0; i0 < total; i0 += per) {
      const int n = per;
      bc.clear();
      bt.clear();
      size_t pix = 0;
      for (int j = i0; j < i0 + n; ++j) {
        const int i = std::min(j, total - 1);
        bc.push_back(cams[i % n_cam]);
        bt.push_back(key_times[i / n_cam]);
        pix += (size_t)cams[i % n_cam].width * cams[i % n_cam].height;
      }
      TRY(grow(s->aux[4], pix * 12));
      outs.clear();
      size_t off = 0;
      for (int i = 0; i < n; ++i) {
        outs.push_back(s->aux[4].as<float>() + off);
        off += (size_t)bc[i].width * bc[i].height * 3;
      }
      TRY(batch_args_ok(s, bc.data(), bt.data(), n, outs.data()));
      TRY(plan_prepare(s, bc.data(), n, false));
      BatchPlan &p = *s->plan;
      TRY(plan_fill(s, p, bc.data(), bt.data(), &o, outs.data()));
      for (int i = 0; i < n; ++i)
        p.h_reqs[i].mark_row =
            i0 + i < total ? rows + (size_t)((i0 + i) / n_cam) * words : nullptr;
      TRY(grow(p.wsum, std::max<uint64_t>(p.rn, 1) * 4));
      TRY(grow(p.stop, std::max<uint64_t>(p.rn, 1) * 4));
      p.weighted = true;
      p.mark = true;
      const int rc = plan_run(s, p, st);
      p.weighted = false;
      p.mark = false;
      TRY(rc);
    }
    for (int k = 0; k < n_key; ++k)
      launch_pack_mask_row(rows + (size_t)k * words, nbytes, bits_out_dev + (size_t)k * nbytes,
                           st);
    CK(cudaGetLastError());
    return FDGS_OK;
  }
  TRY(grow(s->aux[5], (size_t)words * 4));
  uint32_t *row = s->aux[5].as<uint32_t>();
  for (int k = 0; k < n_key; ++k) {
    CK(cudaMemsetAsync(row, 0, (size_t)words * 4, st));
    for (int ic = 0; ic < n_cam; ++ic) {
      Workspace &ws = s->main;
      TRY(grow(s->aux[4], (size_t)cams[ic].width * cams[ic].height * 12));
      FrameMeta m;
      TRY(render_impl(s, ws, &cams[ic], key_times[k], &o, s->aux[4].as<float>(), false, true,
                      false, m, st));
      launch_mark_contributors(m.sorted, ws.ctr.as<uint32_t>() + C_NVIS, m.nv,
                               ws.wsum.as<float>(), ws.stopmark.as<uint32_t>(), row, st);
    }
    launch_pack_mask_row(row, nbytes, bits_out_dev + (size_t)k * nbytes, st);
  }
  CK(cudaGetLastError());
  return FDGS_OK;
}

int fdgs_set_sh_codebook(fdgs_scene *s, const float *codebook_dev, int n_code,
                         const uint16_t *codes_dev) {
  if (!s) return fail(FDGS_ERR_INVALID, "null scene");
  if (!codebook_dev) {
    s->sh_cb = nullptr;
    s->sh_code = nullptr;
    s->n_code = 0;
    return FDGS_OK;
  }
  if (s->d.sh_degree < 1) return fail(FDGS_ERR_INVALID, "a codebook needs sh_degree >= 1");
  if (n_code < 1 || n_code > 65536 || (s->d.n > 0 && !codes_dev))
    return fail(FDGS_ERR_INVALID, "n_code must be 1..65536 and codes non-null");
  s->sh_cb = codebook_dev;
  s->sh_code = codes_dev;
  s->n_code = n_code;
  return FDGS_OK;
}

int fdgs_set_batch_list_capacity(fdgs_scene *s, uint64_t entries) {
  if (!s) return fail(FDGS_ERR_INVALID, "null scene");
  s->list_cap_hint = entries;
  if (s->plan && entries) {
    BatchPlan &p = *s->plan;
    p.key_cap = entries;
    TRY(plan_alloc_lists(p));
    if (p.exec) {                 // the captured graph holds the old capacity
      cudaGraphExecDestroy(p.exec);
      p.exec = nullptr;
    }
  }
  return FDGS_OK;
}

int fdgs_batch_counts(fdgs_scene *s, uint64_t *n_visible, uint64_t *n_keys,
                      uint64_t *n_block_entries) {
  if (!s) return fail(FDGS_ERR_INVALID, "null scene");
  if (!s->plan) return fail(FDGS_ERR_STATE, "no batch has been rendered");
  const BatchPlan &p = *s->plan;
  if (n_visible) *n_visible = p.h_ctr[BC_NVIS];
  if (n_keys) *n_keys = (uint64_t)p.h_ctr[BC_NKEYS_LO] | ((uint64_t)p.h_ctr[BC_NKEYS_HI] << 32);
  if (n_block_entries)
    *n_block_entries =
        (uint64_t)p.h_ctr[BC_NBKEYS_LO] | ((uint64_t)p.h_ctr[BC_NBKEYS_HI] << 32);
  return FDGS_OK;
}

int fdgs_batch_tile_lists(fdgs_scene *s, int req, uint32_t *tile_ranges_host,
                          uint32_t *tile_ids_host, uint64_t ids_cap, uint64_t *n_tiles,
                          uint64_t *n_ids) {
  if (!s) return fail(FDGS_ERR_INVALID, "null scene");
  if (!s->plan || !s->plan->vis_sorted) return fail(FDGS_ERR_STATE, "no batch has been rendered");
  const BatchPlan &p = *s->plan;
  if (req < 0 || req >= p.nreq) return fail(FDGS_ERR_INVALID, "request index out of range");
  CK(cudaDeviceSynchronize());
  const ReqDesc &q = p.h_reqs[req];
  const size_t tiles = (size_t)q.cam.gx * q.cam.gy;
  std::vector<uint2> rg(tiles);
  CK(cudaMemcpy(rg.data(), p.ranges.as<uint2>() + q.tile_base, tiles * 8,
                cudaMemcpyDeviceToHost));
  // the device holds each tile's list length as [0, length); laid out tile-major, the
  // request's lists start where the previous tile's end
  uint64_t n = 0;
  for (size_t t = 0; t < tiles; ++t) {
    const uint32_t len = rg[t].y - rg[t].x;
    rg[t] = make_uint2((uint32_t)n, (uint32_t)(n + len));
    n += len;
  }
  const uint32_t lo = 0;
  if (n_tiles) *n_tiles = tiles;
  if (n_ids) *n_ids = n;
  if (tile_ranges_host)
    for (size_t t = 0; t < tiles; ++t) {
      tile_ranges_host[2 * t] = rg[t].x;
      tile_ranges_host[2 * t + 1] = rg[t].y;
    }
  if (!tile_ids_host || n == 0) return FDGS_OK;
  if (ids_cap < n) return fail(FDGS_ERR_INVALID, "tile_ids buffer holds %llu of %llu ids",
                                (unsigned long long)ids_cap, (unsigned long long)n);
  // the request's block lists, then each tile's list: its block's entries holding its bit
  const int gx = q.cam.gx;
  const int bgx = (gx + kListBlock - 1) / kListBlock, bgy = (q.cam.gy + kListBlock - 1) / kListBlock;
  const size_t nb = (size_t)bgx * bgy;
  std::vector<uint2> br(nb);
  CK(cudaMemcpy(br.data(), p.branges.as<uint2>() + q.block_base, nb * 8,
                cudaMemcpyDeviceToHost));
  const uint32_t blo = br[0].x, bhi = br[nb - 1].y;
  std::vector<uint32_t> ents(std::max<uint32_t>(bhi - blo, 1));
  std::vector<uint16_t> tms(std::max<uint32_t>(bhi - blo, 1));
  if (bhi > blo) {
    CK(cudaMemcpy(ents.data(), p.lists.as<uint32_t>() + blo, (size_t)(bhi - blo) * 4,
                  cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(tms.data(), p.ltm.as<uint16_t>() + blo, (size_t)(bhi - blo) * 2,
                  cudaMemcpyDeviceToHost));
  }
  // entries are record indices req x n + id
  const uint64_t N = (uint64_t)p.d.n, rbase = (uint64_t)req * N;
  for (size_t t = 0; t < tiles; ++t) {
    const int tx = (int)(t % gx), ty = (int)(t / gx);
    const uint2 b2 = br[(ty / kListBlock) * bgx + tx / kListBlock];
    const int bit = (ty % kListBlock) * kListBlock + tx % kListBlock;
    uint64_t o = rg[t].x - lo;
    for (uint32_t e = b2.x; e < b2.y; ++e) {
      if (!((tms[e - blo] >> bit) & 1u)) continue;
      const uint64_t ri = ents[e - blo];
      if (ri < rbase || ri >= rbase + N || o >= rg[t].y - lo)
        return fail(FDGS_ERR_STATE, "block lists disagree with the tile counts");
      tile_ids_host[o++] = (uint32_t)(ri - rbase);
    }
    if (o != rg[t].y - lo) return fail(FDGS_ERR_STATE, "block lists disagree with the tile counts");
  }
  return FDGS_OK;
}

int fdgs_variation_score(fdgs_scene *s, const fdgs_camera *cams, int n_cam, const float *ts,
                         int n_t, int batch, float *score_out_dev, fdgs_stream stream) {
  return fdgs_variation_score_variant(s, cams, n_cam, ts, n_t, batch, FDGS_SCORE_FULL,
                                      score_out_dev, stream);
}

}  // extern "C"
namespace {
int score_impl(fdgs_scene *s, const fdgs_camera *cams, int n_cam, const float *ts, int n_t,
               int batch, int variant, float *score_out_dev, bool zero, fdgs_stream stream);
}  // namespace
extern "C" {
  NvtxRange nvtx_range_("fdgs_variation_score");

int fdgs_variation_score_variant(fdgs_scene *s, const fdgs_camera *cams, int n_cam,
                                 const float *ts, int n_t, int batch, int variant,
                                 float *score_out_dev, fdgs_stream stream) {
  return score_impl(s, cams, n_cam, ts, n_t, batch, variant, score_out_dev, true, stream);
}

int fdgs_variation_score_add(fdgs_scene *s, const fdgs_camera *cams, int n_cam, const float *ts,
                             int n_t, int batch, int variant, float *score_inout_dev,
                             fdgs_stream stream) {
  return score_impl(s, cams, n_cam, ts, n_t, batch, variant, score_inout_dev, false, stream);
}

}  // extern "C"

namespace {

// The score pass; zero: overwrite score_out_dev, else add to it (a pass split into parts).
int score_impl(fdgs_scene *s, const fdgs_camera *cams, int n_cam, const float *ts, int n_t,
               int batch, int variant, float *score_out_dev, bool zero, fdgs_stream stream) {
  if (!s) return fail(FDGS_ERR_INVALID, "null scene");
  if (n_cam < 0 || n_t < 0 || batch < 1 || !score_out_dev ||
      (n_cam > 0 && !cams) || (n_t > 0 && !ts))
    return fail(FDGS_ERR_INVALID, "bad score arguments");
  if (variant < FDGS_SCORE_FULL || variant > FDGS_SCORE_SIGMA_T)
    return fail(FDGS_ERR_INVALID, "unknown score variant %d", variant);
  cudaStream_t st = (cudaStream_t)stream;
  const uint32_t N = (uint32_t)s->d.n;
  if (zero) CK(cudaMemsetAsync(score_out_dev, 0, (size_t)N * 4, st));
  if (N == 0) return FDGS_OK;
  // gamma = clamp(V / V_p90, 0, 1)^0.1, V_p90 the nearest-rank 90th percentile
  TRY(grow(s->aux[0], (size_t)N * 4 * 2 + 16));   // volume bits, ping-pong
  const size_t goff = ((size_t)N * 4 + 255) & ~(size_t)255;
  TRY(grow(s->aux[1], goff + (size_t)N * 8));     // gamma, then Sigma_t (FP64)
  TRY(grow(s->aux[2], sort_scratch_bytes(N, 32)));
  TRY(grow(s->aux[3], 16));
  uint32_t *vb = s->aux[0].as<uint32_t>();
  CK(cudaMemcpyAsync(s->aux[3].p, &N, 4, cudaMemcpyHostToDevice, st));
  launch_volume_bits((const float4 *)s->d.logscale4, N, vb, st);
  uint32_t *vs = radix_sort<uint32_t>(vb, vb + N, s->aux[3].as<uint32_t>(), N, 0, 32,
                                      s->aux[2].p, st, s->status.as<uint32_t>());
  const uint32_t k = (uint32_t)std::max<int64_t>(1, (int64_t)ceil(0.9 * (double)N)) - 1;
  float *gamma = s->aux[1].as<float>();
  double *sig_t = (double *)((char *)s->aux[1].p + goff);
  launch_score_consts((const float4 *)s->d.logscale4, (const float4 *)s->d.q_left,
                      (const float4 *)s->d.q_right, N, vs, k, gamma, sig_t, st);
  if (variant == FDGS_SCORE_TEMPORAL) {
    // no render: S_i = sum over t of f_i(t) gamma_i
    for (int it = 0; it < n_t; ++it)
      launch_score_temporal((const float4 *)s->d.mean4, sig_t, gamma, N, ts[it],
                            score_out_dev, st);
    CK(cudaGetLastError());
    return FDGS_OK;
  }
  fdgs_render_opts o{};
  o.use_mask = 0;
  o.tile_sets = 1;   // same weights as the 3-sigma squares, shorter lists
  if (batch > 1 && n_cam > 0 && n_t > 0 && N < (1u << kBatchIdBits)) {
    // batches of up to `batch` (t, camera) renders through the batched pipeline, each with
    // the weighted persistent blend and the batched accumulation
    const int per = std::min(batch, 128);
    std::vector<fdgs_camera> bc;
    std::vector<float> bt;
    std::vector<float *> outs;
    const int total = n_t * n_cam;
    for (int i0 = 0; i0 < total; i0 += per) {
      const int n = std::min(per, total - i0);
      bc.clear();
      bt.clear();
      size_t pix = 0;
      for (int i = i0; i < i0 + n; ++i) {
        bc.push_back(cams[i % n_cam]);
        bt.push_back(ts[i / n_cam]);
        pix += (size_t)cams[i % n_cam].width * cams[i % n_cam].height;
      }
      TRY(grow(s->aux[4], pix * 12));
      outs.clear();
      size_t off = 0;
      for (int i = 0; i < n; ++i) {
        outs.push_back(s->aux[4].as<float>() + off);
        off += (size_t)bc[i].width * bc[i].height * 3;
      }
      TRY(batch_args_ok(s, bc.data(), bt.data(), n, outs.data()));
      TRY(plan_prepare(s, bc.data(), n, false));
      BatchPlan &p = *s->plan;
      TRY(plan_fill(s, p, bc.data(), bt.data(), &o, outs.data()));
      TRY(grow(p.wsum, std::max<uint64_t>(p.rn, 1) * 4));
      TRY(grow(p.stop, std::max<uint64_t>(p.rn, 1) * 4));
      p.weighted = true;
      p.score_out = score_out_dev;
      p.score_variant = variant;
      p.gamma = gamma;
      p.sig_t = sig_t;
      const int rc = plan_run(s, p, st);
      p.weighted = false;
      p.score_out = nullptr;
      p.score_variant = 0;
      p.gamma = nullptr;
      p.sig_t = nullptr;
      TRY(rc);
    }
    return FDGS_OK;
  }
  int done = 0;
  for (int it = 0; it < n_t; ++it)
    for (int ic = 0; ic < n_cam; ++ic) {
      Workspace &ws = s->main;
      TRY(grow(s->aux[4], (size_t)cams[ic].width * cams[ic].height * 12));
      FrameMeta m;
      TRY(render_impl(s, ws, &cams[ic], ts[it], &o, s->aux[4].as<float>(), false, true, false,
                      m, st));
      launch_score_accumulate(m.sorted, ws.ctr.as<uint32_t>() + C_NVIS, m.nv, ws.wsum.as<float>(),
                              (const float4 *)s->d.mean4, sig_t, gamma, ts[it], score_out_dev,
                              variant, st);
      if (++done % batch == 0) CK(cudaGetLastError());
    }
  CK(cudaGetLastError());
  return FDGS_OK;
}

}  // namespace

extern "C" {

int fdgs_select_keep(fdgs_scene *s, const float *score_dev, int64_t n, float prune_ratio,
                     uint8_t *keep_out_dev, fdgs_stream stream) {
  NvtxRange nvtx_range_("fdgs_select_keep");
  if (!s || !score_dev || !keep_out_dev || n < 0 || n >= (1ll << 30))
    return fail(FDGS_ERR_INVALID, "bad keep-set arguments");
  if (!(prune_ratio >= 0.f && prune_ratio <= 1.f))
    return fail(FDGS_ERR_INVALID, "prune_ratio must be in [0, 1]");
  if (n == 0) return FDGS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const uint32_t N = (uint32_t)n;
  TRY(grow(s->aux[0], (size_t)N * 16 + 16));
  TRY(grow(s->aux[2], sort_scratch_bytes(N, 32)));
  TRY(grow(s->aux[3], 16));
  uint64_t *keys = s->aux[0].as<uint64_t>();
  CK(cudaMemcpyAsync(s->aux[3].p, &N, 4, cudaMemcpyHostToDevice, st));
  launch_score_keys(score_dev, N, keys, st);
  uint64_t *srt = radix_sort<uint64_t>(keys, keys + N, s->aux[3].as<uint32_t>(), N, 32, 32,
                                       s->aux[2].p, st, s->status.as<uint32_t>());
  const uint32_t n_drop = (uint32_t)floor((double)prune_ratio * (double)N);
  launch_keep_from_sorted(srt, N, n_drop, keep_out_dev, st);
  CK(cudaGetLastError());
  return FDGS_OK;
}

int fdgs_set_list_builder(int mode) {
  if (mode < 0 || mode > 2)
    return fail(FDGS_ERR_INVALID, "mode must be 0 (auto), 1 (sort) or 2 (bitmask)");
  g_list_mode = mode;
  return FDGS_OK;
}

int fdgs_finetune_reset(fdgs_scene *s) {
  if (!s) return fail(FDGS_ERR_INVALID, "null scene");
  s->ft_step = 0;
  s->ft_total = 0;     // the next step zeroes the moments
  return FDGS_OK;
}

int fdgs_finetune_step(fdgs_scene *s, const fdgs_camera *cam, float t,
                       const fdgs_render_opts *opts, const float *target_dev,
                       const fdgs_adam_opts *adam, float *loss_accum_dev, fdgs_stream stream) {
  NvtxRange nvtx_range_("fdgs_finetune_step");
  if (!s) return fail(FDGS_ERR_INVALID, "null scene");
  if (!cam || !target_dev || !adam) return fail(FDGS_ERR_INVALID, "null argument");
  if (!(adam->beta1 >= 0.f && adam->beta1 < 1.f && adam->beta2 >= 0.f && adam->beta2 < 1.f &&
        adam->eps >= 0.f))
    return fail(FDGS_ERR_INVALID, "Adam needs 0 <= beta < 1 and eps >= 0");
  cudaStream_t st = (cudaStream_t)stream;
  const uint64_t N = (uint64_t)s->d.n;
  if (N == 0) return FDGS_OK;
  const uint64_t K = (uint64_t)(s->d.sh_degree + 1) * (s->d.sh_degree + 1);
  // the attribute arrays as one parameter space: mean4, logscale4, q_left, q_right, opacity,
  // the SH DC plane and the higher SH bands (the SH array is [K][3][N], DC plane first)
  const uint64_t len[7] = {4 * N, 4 * N, 4 * N, 4 * N, N, 3 * N, 3 * N * (K - 1)};
  float *par[7] = {const_cast<float *>(s->d.mean4), const_cast<float *>(s->d.logscale4),
                   const_cast<float *>(s->d.q_left), const_cast<float *>(s->d.q_right),
                   const_cast<float *>(s->d.opacity_logit), const_cast<float *>(s->d.sh),
                   const_cast<float *>(s->d.sh) + 3 * N};
  uint64_t off[8] = {0};
  for (int i = 0; i < 7; ++i) off[i + 1] = off[i] + len[i];
  const uint64_t total = off[7];
  TRY(grow(s->ft_grad, total * 4));
  TRY(grow(s->ft_m, total * 4));
  TRY(grow(s->ft_v, total * 4));
  TRY(grow(s->ft_loss, 16));
  if (s->ft_total != total) {
    CK(cudaMemsetAsync(s->ft_m.p, 0, total * 4, st));
    CK(cudaMemsetAsync(s->ft_v.p, 0, total * 4, st));
    s->ft_total = total;
    s->ft_step = 0;
  }
  const uint64_t pix = (uint64_t)cam->width * cam->height;
  if (cam->width <= 0 || cam->height <= 0) return fail(FDGS_ERR_INVALID, "bad camera size");
  TRY(grow(s->ft_img, pix * 12));
  TRY(grow(s->ft_dL, pix * 12));
  // forward with a frame kept for the reverse replay
  fdgs_frame *f = nullptr;
  TRY(fdgs_render(s, cam, t, opts, s->ft_img.as<float>(), &f, stream));
  float *loss = loss_accum_dev ? loss_accum_dev : s->ft_loss.as<float>();
  launch_l1_grad(s->ft_img.as<float>(), target_dev, (uint32_t)(3 * pix), s->ft_dL.as<float>(),
                 loss, st);
  float *g = s->ft_grad.as<float>();
  CK(cudaMemsetAsync(g, 0, total * 4, st));
  const int rc = fdgs_render_backward(s, f, s->ft_dL.as<float>(), g + off[0], g + off[1],
                                      g + off[2], g + off[3], g + off[4], g + off[5], stream);
  fdgs_frame_release(f);
  TRY(rc);
  // Adam with PyTorch's bias corrections
  ++s->ft_step;
  const double bc1 = 1.0 - pow((double)adam->beta1, (double)s->ft_step);
  const double bc2 = 1.0 - pow((double)adam->beta2, (double)s->ft_step);
  AdamArgs a{};
  a.nseg = 0;
  for (int i = 0; i < 7; ++i) {
    if (len[i] == 0) continue;
    a.off[a.nseg] = off[i];
    a.param[a.nseg] = par[i];
    a.step_size[a.nseg] = (float)(adam->lr[i] / bc1);
    ++a.nseg;
  }
  a.off[a.nseg] = total;
  a.grad = g;
  a.m = s->ft_m.as<float>();
  a.v = s->ft_v.as<float>();
  a.b1 = adam->beta1;
  a.b2 = adam->beta2;
  a.eps = adam->eps;
  a.sqrt_bc2 = (float)sqrt(bc2);
  launch_adam(a, st);
  CK(cudaGetLastError());
  return FDGS_OK;
}

int fdgs_set_batch_shape(fdgs_scene *s, int footprint, int ctas_per_sm) {
  if (!s) return fail(FDGS_ERR_INVALID, "null scene");
  if (footprint < 0 || footprint >= kBlendShapes)
    return fail(FDGS_ERR_INVALID, "blend shape must be in [0, %d)", kBlendShapes);
  if (ctas_per_sm < 0 || ctas_per_sm > 64)
    return fail(FDGS_ERR_INVALID, "CTAs per SM must be in [0, 64]");
  s->batch_footprint = footprint;
  s->batch_ctas = ctas_per_sm;
  if (s->plan) {
    BatchPlan &p = *s->plan;
    p.footprint = footprint;
    p.ctas = ctas_per_sm ? ctas_per_sm : batch_blend_max_ctas_per_sm(footprint);
    p.tuned = false;
    if (p.exec) {            // the next batch runs eagerly and captures the new shape
      cudaGraphExecDestroy(p.exec);
      p.exec = nullptr;
    }
  }
  return FDGS_OK;
}

int fdgs_set_batch_staging(int mode) {
  if (mode < 0 || mode > 1)
    return fail(FDGS_ERR_INVALID, "staging must be 0 (cp.async) or 1 (TMA gather4)");
  g_batch_staging = mode;
  return FDGS_OK;
}

int fdgs_set_blend_shape(int footprint) {
  if (footprint < -1 || footprint >= kBlendShapes)
    return fail(FDGS_ERR_INVALID, "blend shape must be -1 (the defaults), 0 (16x2), 1 (8x4), "
                "2 (4x8), 3 (8x8), 4 (16x8), 5 (8x16) or 6 (16x16)");
  g_blend_shape = footprint < 0 ? kBlendShapeDefault : footprint;
  g_blend_shape_fwd = footprint < 0 ? kBlendShapeFwdDefault : footprint;
  return FDGS_OK;
}

int fdgs_profile_enable(fdgs_scene *s, int flags) {
  if (!s) return fail(FDGS_ERR_INVALID, "null scene");
  if ((flags & 1) && !s->ev[0])
    for (auto &e : s->ev) CK(cudaEventCreate(&e));
  if (flags & 2) TRY(grow(s->evals, 24));
  s->prof = flags;
  return FDGS_OK;
}

int fdgs_profile_read(fdgs_scene *s, float *stage_ms, uint64_t *blend_counts) {
  if (!s) return fail(FDGS_ERR_INVALID, "null scene");
  CK(cudaDeviceSynchronize());
  if (stage_ms) {
    // forward stages from events 0..8, backward stages from events 9..11; zeros for a stage
    // whose events were never recorded
    for (int i = 0; i < FDGS_PROFILE_STAGES; ++i) {
      stage_ms[i] = 0.f;
      if (!s->ev[0]) continue;
      const int a = i < 8 ? i : i + 1;
      if (cudaEventElapsedTime(&stage_ms[i], s->ev[a], s->ev[a + 1]) != cudaSuccess) {
        cudaGetLastError();
        stage_ms[i] = 0.f;
      }
    }
  }
  if (blend_counts) {
    blend_counts[0] = blend_counts[1] = blend_counts[2] = 0;
    if (s->evals.p) CK(cudaMemcpy(blend_counts, s->evals.p, 24, cudaMemcpyDeviceToHost));
  }
  return FDGS_OK;
}

int fdgs_debug_inject(int kind, int64_t value) {
  switch (kind) {
    case FDGS_INJECT_NONE:
      fdgs::g_debug_spin_limit = 0;
      fdgs::g_debug_withhold = ~0u;
      fdgs::g_debug_tma_skip = 0;
      g_fail_allocs = 0;
      return FDGS_OK;
    case FDGS_INJECT_SPIN_LIMIT:
      if (value < 0 || value > (int64_t)kSpinLimit)
        return fail(FDGS_ERR_INVALID, "spin limit must be in [0, %u]", kSpinLimit);
      fdgs::g_debug_spin_limit = (uint32_t)value;
      return FDGS_OK;
    case FDGS_INJECT_WITHHOLD_PUBLISH:
      if (value < 0 || value >= (1ll << 30))
        return fail(FDGS_ERR_INVALID, "partition index out of range");
      fdgs::g_debug_withhold = (uint32_t)value;
      return FDGS_OK;
    case FDGS_INJECT_FAIL_ALLOCS:
      if (value < 0 || value > (1 << 20)) return fail(FDGS_ERR_INVALID, "bad allocation count");
      g_fail_allocs = (int)value;
      return FDGS_OK;
    case FDGS_INJECT_TMA_MISSING_ARRIVAL:
      fdgs::g_debug_tma_skip = 1;
      return FDGS_OK;
    default:
      return fail(FDGS_ERR_INVALID, "unknown injection kind %d", kind);
  }
}

int fdgs_status_sync(fdgs_scene *s) {
  if (!s) return fail(FDGS_ERR_INVALID, "null scene");
  CK(cudaDeviceSynchronize());
  return check_device_errors(s, nullptr);
}

}  // extern "C"
