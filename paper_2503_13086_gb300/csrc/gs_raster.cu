// gs_raster.cu -- the rasterizer engine: workspaces, capacity management, the K1-K10 launch
// sequence, per-kernel timing, and the stateless gs_raster_* / gs_adam_step entry points.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "gs_engine.h"

namespace gs {

thread_local std::string g_last_error;

// Device allocations and frees (which may synchronise the device) never run while another
// session captures a step into a CUDA graph: both take this lock.
std::mutex& alloc_capture_mutex() {
  static std::mutex mu;
  return mu;
}

gs_status fail(gs_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

gs_status DevBuf::reserve(size_t want, size_t* account) {
  if (want <= bytes) return GS_OK;
  std::lock_guard<std::mutex> lock(alloc_capture_mutex());
  if (p) {
    // steps enqueued earlier may still use the old buffer
    cudaDeviceSynchronize();
    cudaFree(p);
    if (account) *account -= bytes + kCanaryBytes;
    p = nullptr;
    bytes = 0;
  }
  if (want == 0) return GS_OK;
  const size_t rounded = (want + 255) & ~size_t(255);
  cudaError_t e = cudaMalloc(&p, rounded + kCanaryBytes);
  if (e != cudaSuccess) {
    p = nullptr;
    cudaGetLastError();
    return fail(GS_ERR_OOM, std::string("cudaMalloc(") + std::to_string(rounded) + "): " + cudaGetErrorString(e));
  }
  // guard words behind the usable bytes, complete before any stream can use the buffer
  e = cudaMemset(static_cast<char*>(p) + rounded, 0xA5, kCanaryBytes);
  if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
  if (e != cudaSuccess) {
    cudaFree(p);
    p = nullptr;
    return fail(GS_ERR_CUDA, std::string("guard words: ") + cudaGetErrorString(e));
  }
  bytes = rounded;
  if (account) *account += bytes + kCanaryBytes;
  return GS_OK;
}

void DevBuf::release(size_t* account) {
  if (!p) {
    bytes = 0;
    return;
  }
  std::lock_guard<std::mutex> lock(alloc_capture_mutex());
  if (p) {
    cudaDeviceSynchronize();
    cudaFree(p);
    if (account) *account -= bytes + kCanaryBytes;
  }
  p = nullptr;
  bytes = 0;
}

// Guard-word check: one CTA of 64 threads per buffer (64 x 4 B = kCanaryBytes).
constexpr int kCanaryBatch = 64;
struct CanaryList {
  const unsigned* p[kCanaryBatch];
  int n;
};
static_assert(kCanaryBytes == 64 * 4, "one thread per guard word");

__global__ void k_canary_check(CanaryList L, int first, unsigned* __restrict__ flags) {
  const int b = blockIdx.x;
  if (b >= L.n) return;
  if (L.p[b][threadIdx.x] != kCanaryWord) atomicOr(&flags[(first + b) >> 5], 1u << ((first + b) & 31));
}

gs_status check_canaries(const CanaryRef* refs, int n, unsigned* flags, cudaStream_t s) {
  const int words = (n + 31) / 32;
  cudaError_t e = words > 0 ? cudaMemsetAsync(flags, 0, (size_t)words * 4, s) : cudaSuccess;
  // one launch per run of up to kCanaryBatch consecutive allocated buffers; flag bit = position in refs
  int k = 0;
  while (k < n && e == cudaSuccess) {
    if (!refs[k].buf || !refs[k].buf->p) {
      ++k;
      continue;
    }
    CanaryList L{};
    const int first = k;
    while (k < n && L.n < kCanaryBatch && refs[k].buf && refs[k].buf->p) {
      const DevBuf* d = refs[k].buf;
      L.p[L.n++] = reinterpret_cast<const unsigned*>(static_cast<const char*>(d->p) + d->bytes);
      ++k;
    }
    k_canary_check<<<L.n, 64, 0, s>>>(L, first, flags);
    e = cudaGetLastError();
  }
  std::vector<unsigned> h((size_t)words, 0u);
  if (e == cudaSuccess && words > 0) e = cudaMemcpyAsync(h.data(), flags, (size_t)words * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(GS_ERR_CUDA, std::string("guard-word check: ") + cudaGetErrorString(e));
  for (int j = 0; j < n; ++j)
    if ((h[(size_t)j >> 5] >> (j & 31)) & 1u)
      return fail(GS_ERR_INTERNAL, std::string("device buffer '") + refs[j].name +
                                       "' was written past its end (its guard words changed)");
  return GS_OK;
}

static int bits_for(long long x) {  // bits needed to represent values 0..x
  int b = 0;
  while (x > 0) {
    ++b;
    x >>= 1;
  }
  return b;
}

// Kernel attributes, occupancy figures and the loss window's constants, set once per process
// (sessions may be created from several host threads at once).
static void init_attributes_once() {
  static std::once_flag once;
  std::call_once(once, [] {
    init_sort_attributes();
    init_blend_attributes();
    init_loss_attributes();
  });
}

Raster::Raster() {
  init_attributes_once();
  Tiling first;
  if (tiling_candidates(&first, 1) > 0) tiling = first;  // the default is the first compiled tiling
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (num_sms <= 0) num_sms = 1;
  cudaMallocHost(&sp_h, sizeof(StepParams));
  cudaMallocHost(&views_h, sizeof(ViewDev) * kMaxViews);
  cudaMallocHost(&ctl_h, sizeof(Control));
  cudaMallocHost(&ledger_h, sizeof(Ledger));
  std::memset(sp_h, 0, sizeof(StepParams));
  std::memset(ctl_h, 0, sizeof(Control));
  std::memset(ledger_h, 0, sizeof(Ledger));
  cudaEventCreateWithFlags(&staged, cudaEventDisableTiming);
  for (int k = 0; k < kNumEvents; ++k) cudaEventCreate(&ev[k]);
  sp_d.reserve(sizeof(StepParams), &bytes_in_use);
  views_d.reserve(sizeof(ViewDev) * kMaxViews, &bytes_in_use);
  ledger_d.reserve(sizeof(Ledger), &bytes_in_use);
  cudaMemset(ledger_d.p, 0, sizeof(Ledger));
}

Raster::~Raster() {
  DevBuf* all[] = {&sp_d, &views_d, &ledger_d, &zeroA, &zeroB, &xyo, &conic, &rgb, &depth, &radius, &rect, &count, &offsets,
                   &clamp, &g2s, &keys0, &keys1, &vals0, &vals1, &ginst, &inst_rec, &carry, &ckpt, &cmask, &order, &tile_chunks, &partials, &block_sums, &own_image,
                   &own_last, &own_dimage};
  for (DevBuf* b : all) b->release(&bytes_in_use);
  if (sp_h) cudaFreeHost(sp_h);
  if (views_h) cudaFreeHost(views_h);
  if (ctl_h) cudaFreeHost(ctl_h);
  if (ledger_h) cudaFreeHost(ledger_h);
  cudaEventDestroy(staged);
  for (int k = 0; k < kNumEvents; ++k) cudaEventDestroy(ev[k]);
}

Control* Raster::ctl() const { return reinterpret_cast<Control*>(zeroA.p); }
unsigned long long* Raster::scan_state() const {
  return reinterpret_cast<unsigned long long*>(static_cast<char*>(zeroA.p) + kCtlBytes);
}
unsigned* Raster::hist() const { return reinterpret_cast<unsigned*>(zeroB.p); }
unsigned* Raster::sort_state() const {
  return reinterpret_cast<unsigned*>(static_cast<char*>(zeroB.p) + kHistBytes);
}
uint2* Raster::ranges() const {
  return reinterpret_cast<uint2*>(static_cast<char*>(zeroB.p) + kHistBytes + sort_state_bytes);
}
int* Raster::chunk_tile() const {
  return reinterpret_cast<int*>(static_cast<char*>(zeroB.p) + kHistBytes + sort_state_bytes + ranges_bytes);
}
unsigned* Raster::tile_done() const {
  return reinterpret_cast<unsigned*>(static_cast<char*>(zeroB.p) + kHistBytes + sort_state_bytes + ranges_bytes +
                                     chunk_bytes);
}
ProjBuffers Raster::proj() const {
  ProjBuffers p;
  p.xyo = static_cast<float4*>(xyo.p);
  p.conic = static_cast<float4*>(conic.p);
  p.rgb = static_cast<float4*>(rgb.p);
  p.depth = static_cast<float*>(depth.p);
  p.radius = static_cast<int*>(radius.p);
  p.rect = static_cast<uint2*>(rect.p);
  p.count = static_cast<unsigned*>(count.p);
  p.offsets = static_cast<unsigned*>(offsets.p);
  p.clamp = static_cast<unsigned char*>(clamp.p);
  return p;
}

gs_status Raster::set_views(const gs_camera* cams, int nv, const float* const* targets) {
  if (nv <= 0 || nv > kMaxViews) return fail(GS_ERR_CAPACITY, "n_views must be in 1.." + std::to_string(kMaxViews));
  views.assign(nv, ViewDev{});
  long long tb = 0, pb = 0, lb = 0;
  for (int v = 0; v < nv; ++v) {
    const gs_camera& c = cams[v];
    if (c.width <= 0 || c.height <= 0 || c.width > 65535 * tiling.tw || c.height > 65535 * tiling.th)
      return fail(GS_ERR_INVALID_ARG, "camera size out of range");
    if (!(c.fx > 0.f) || !(c.fy > 0.f)) return fail(GS_ERR_INVALID_ARG, "focal lengths must be positive");
    ViewDev& V = views[v];
    std::memcpy(V.R, c.R, sizeof(V.R));
    std::memcpy(V.t, c.t, sizeof(V.t));
    V.fx = c.fx;
    V.fy = c.fy;
    V.cx = c.cx;
    V.cy = c.cy;
    for (int a = 0; a < 3; ++a)
      V.campos[a] = -(c.R[0 * 3 + a] * c.t[0] + c.R[1 * 3 + a] * c.t[1] + c.R[2 * 3 + a] * c.t[2]);
    V.limx = kFovLim * ((float)c.width / (2.f * c.fx));
    V.limy = kFovLim * ((float)c.height / (2.f * c.fy));
    V.W = c.width;
    V.H = c.height;
    V.tw = tiling.tw;
    V.th = tiling.th;
    V.gx = (c.width + tiling.tw - 1) / tiling.tw;
    V.gy = (c.height + tiling.th - 1) / tiling.th;
    V.tile_base = tb;
    V.pix_base = pb;
    V.loss_block_base = lb;
    V.target = targets ? targets[v] : nullptr;
    tb += (long long)V.gx * V.gy;
    pb += (long long)c.width * c.height;
    lb += loss_blocks(c.width, c.height);
  }
  n_views = nv;
  n_tiles = tb;
  n_pix = pb;
  n_loss_blocks = lb;
  tile_bits = bits_for(n_tiles - 1);
  passes = (32 + tile_bits + kSortBits - 1) / kSortBits;  // at most; the step may need fewer
  if (passes > kMaxSortPasses) return fail(GS_ERR_CAPACITY, "too many tiles");
  return GS_OK;
}

gs_status Raster::ensure_records(int stride_) {
  const long long recs = (long long)n_views * stride_;
  if ((unsigned long long)recs >= (1ull << 32)) return fail(GS_ERR_CAPACITY, "views x stride exceeds 2^32 records");
  gs_status s;
  if ((s = xyo.reserve(recs * 16, &bytes_in_use)) || (s = conic.reserve(recs * 16, &bytes_in_use)) ||
      (s = rgb.reserve(recs * 16, &bytes_in_use)) || (s = depth.reserve(recs * 4, &bytes_in_use)) ||
      (s = radius.reserve(recs * 4, &bytes_in_use)) || (s = rect.reserve(recs * 8, &bytes_in_use)) ||
      (s = count.reserve(recs * 4, &bytes_in_use)) || (s = offsets.reserve(recs * 4, &bytes_in_use)) ||
      (s = clamp.reserve(recs, &bytes_in_use)) || (s = g2s.reserve(recs * 36, &bytes_in_use)))
    return s;
  const long long scan_tiles = (recs + kScanTile - 1) / kScanTile;
  if ((s = zeroA.reserve(kCtlBytes + scan_tiles * 8, &bytes_in_use))) return s;
  zeroA_bytes = kCtlBytes + scan_tiles * 8;
  if ((s = partials.reserve(n_pix * 10 * 4, &bytes_in_use)) || (s = block_sums.reserve(n_loss_blocks * 16, &bytes_in_use)))
    return s;
  return GS_OK;
}

gs_status Raster::ensure_instances(unsigned long long m) {
  if (m < 1024) m = 1024;
  if (m > m_cap) {
    unsigned long long want = m;
    if (want > (1ull << 31)) return fail(GS_ERR_CAPACITY, "more than 2^31 Gaussian-tile instances");
    gs_status s;
    // free first so the peak does not hold old and new copies
    DevBuf* bufs[] = {&keys0, &keys1, &vals0, &vals1, &ginst, &ckpt, &inst_rec, &carry};
    for (DevBuf* b : bufs) b->release(&bytes_in_use);
    const unsigned long long chunks = (want >> 5) + 1;
    m_cap = 0;  // until every buffer below exists (a failed reserve leaves them released)
    if ((s = keys0.reserve(want * 8, &bytes_in_use)) || (s = keys1.reserve(want * 8, &bytes_in_use)) ||
        (s = vals0.reserve(want * 4, &bytes_in_use)) || (s = vals1.reserve(want * 4, &bytes_in_use)) ||
        (s = ginst.reserve(want * 48, &bytes_in_use)) || (s = inst_rec.reserve(want * 4, &bytes_in_use)) ||
        (s = carry.reserve(2 * 9 * 4 * ((want + 31) / 32 + 1), &bytes_in_use)))
      return s;
    (void)chunks;
    m_cap = want;
  }
  // checkpoints and chunk map depend on tiles as well
  const unsigned long long n_ids = (m_cap >> 5) + (unsigned long long)n_tiles + 1;
  gs_status s;
  const unsigned long long tile_pix = (unsigned long long)tiling.tw * tiling.th;
  if ((s = ckpt.reserve(n_ids * tile_pix * sizeof(float4), &bytes_in_use)) ||
      (s = cmask.reserve(n_ids * tile_pix * 4, &bytes_in_use)) || (s = order.reserve((size_t)n_tiles * 4, &bytes_in_use)) ||
      (s = tile_chunks.reserve((size_t)n_tiles * 4, &bytes_in_use)))
    return s;
  const unsigned long long sort_tiles = (m_cap + kSortTile - 1) / kSortTile;
  sort_state_bytes = (size_t)passes * sort_tiles * kSortBins * 4;
  ranges_bytes = (size_t)n_tiles * 8;
  chunk_bytes = (size_t)n_ids * 4;
  zeroB_bytes = kHistBytes + sort_state_bytes + ranges_bytes + chunk_bytes + (size_t)n_tiles * 4;
  if ((s = zeroB.reserve(zeroB_bytes, &bytes_in_use))) return s;
  return GS_OK;
}

static bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &st);
  return st != cudaStreamCaptureStatusNone;
}

void Raster::mark(cudaStream_t s, int k) {
  if (!timing) return;
  // inside a capture the record becomes an event node of the graph
  if (capturing(s)) cudaEventRecordWithFlags(ev[k], s, cudaEventRecordExternal);
  else cudaEventRecord(ev[k], s);
}

gs_status Raster::stage(cudaStream_t s) {
  // The pinned staging buffers are read by an async copy; wait for the previous copy before
  // overwriting them (cheap: the copy runs at the head of the previous step).
  cudaError_t e = cudaEventSynchronize(staged);
  if (e != cudaSuccess) return fail(GS_ERR_CUDA, std::string("staging wait: ") + cudaGetErrorString(e));
  std::memcpy(views_h, views.data(), sizeof(ViewDev) * views.size());
  return GS_OK;
}

gs_status Raster::upload(cudaStream_t s) {
  cudaMemcpyAsync(sp_d.p, sp_h, sizeof(StepParams), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(views_d.p, views_h, sizeof(ViewDev) * n_views, cudaMemcpyHostToDevice, s);
  // Mark when the staging buffers may be overwritten for the next step: right after these
  // copies, also inside a captured step (an event node of the graph).
  if (capturing(s)) cudaEventRecordWithFlags(staged, s, cudaEventRecordExternal);
  else cudaEventRecord(staged, s);
  return GS_OK;
}

gs_status Raster::enqueue_forward_head(cudaStream_t s, const float* params, int stride_, bool size_exactly) {
  cudaMemsetAsync(zeroA.p, 0, zeroA_bytes, s);
  // zeroB is cleared here too unless the sizing below may reallocate it, so that the kernels from
  // K1 on follow one another with no other node between them (programmatic dependent launch)
  zeroB_pending = size_exactly;
  if (!size_exactly) cudaMemsetAsync(zeroB.p, 0, zeroB_bytes, s);
  mark(s, 0);
  launch_project(params, stride_, n_views, sp(), vd(), proj(), s);
  mark(s, 1);
  const long long n_items = (long long)n_views * stride_;
  launch_scan(proj().count, proj().offsets, n_items, scan_state(), ctl(), size_exactly ? ~0ull : m_cap, ledger(), s,
              proj().depth);
  mark(s, 2);
  if (size_exactly) {
    cudaMemcpyAsync(ctl_h, ctl(), sizeof(Control), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(GS_ERR_CUDA, std::string("forward: ") + cudaGetErrorString(e));
    const unsigned long long m = ctl_h->m_total;
    if (m > m_cap) {
      gs_status st = ensure_instances(m + m / 4 + 1024);
      if (st) return st;
    }
  }
  return GS_OK;
}

gs_status Raster::enqueue_forward_tail(cudaStream_t s, float* image, float* T, unsigned* last, unsigned* gp) {
  last_gp = gp;
  if (zeroB_pending) cudaMemsetAsync(zeroB.p, 0, zeroB_bytes, s);
  zeroB_pending = false;
  const long long n_items = (long long)n_views * stride;
  unsigned long long* k0 = static_cast<unsigned long long*>(keys0.p);
  unsigned long long* k1 = static_cast<unsigned long long*>(keys1.p);
  unsigned* v0 = static_cast<unsigned*>(vals0.p);
  unsigned* v1 = static_cast<unsigned*>(vals1.p);
  launch_emit(proj(), vd(), stride, n_items, k0, v0, k1, v1, static_cast<unsigned*>(inst_rec.p),
              hist(), tile_bits, (long long)m_cap, num_sms, ctl(), s);
  mark(s, 3);
  const unsigned long long sort_tiles = (m_cap + kSortTile - 1) / kSortTile;
  for (int p = 0; p < passes; ++p)  // passes the step does not need return at once; the list ends in buffer 0
    launch_sort_pass(k0, v0, k1, v1, hist(), sort_state() + (size_t)p * sort_tiles * kSortBins, p, tile_bits,
                     (long long)m_cap, ctl(), s);
  mark(s, 4);
  launch_ranges(k0, ranges(), tile_bits, (long long)m_cap, ctl(), s);
  launch_tile_order(ranges(), n_tiles, static_cast<int*>(order.p), ctl(), s);
  mark(s, 5);
  launch_blend_forward(tiling, vd(), n_views, n_tiles, ranges(), v0, proj(), sp(), ctl(),
                       static_cast<const int*>(order.p), image, T, last, gp, static_cast<float4*>(ckpt.p),
                       static_cast<unsigned*>(cmask.p), chunk_tile(), static_cast<int*>(tile_chunks.p), tile_done(),
                       num_sms, s);
  mark(s, 6);
  return GS_OK;
}

void Raster::enqueue_loss(cudaStream_t s, const float* image, float* dimage, bool after_forward) {
  launch_loss(vd(), n_views, n_loss_blocks, image, sp(), static_cast<float*>(partials.p),
              static_cast<double*>(block_sums.p), ctl(), ledger(), dimage, after_forward ? tile_done() : nullptr,
              forward_warps(tiling, n_tiles, num_sms), s);
  mark(s, 7);
}

void Raster::enqueue_blend_backward(cudaStream_t s, const float* image, const float* dimage) {
  launch_blend_backward(tiling, vd(), n_views, n_tiles, ranges(), static_cast<unsigned*>(vals0.p), proj(),
                        ctl(), image, dimage, static_cast<float4*>(ckpt.p), static_cast<unsigned*>(cmask.p),
                        chunk_tile(), static_cast<int*>(tile_chunks.p), static_cast<float4*>(ginst.p), last_gp, sp(),
                        num_sms, s);
  mark(s, 8);
}

void Raster::enqueue_backward(cudaStream_t s, float* params, const float* image, const unsigned* last,
                              const float* dimage, float* grads, float* m, float* v, float* grad2d) {
  (void)last;  // the backward reads the forward's per-chunk masks instead of the last index
  enqueue_blend_backward(s, image, dimage);
  launch_project_backward(params, stride, n_views, sp(), vd(), proj(), static_cast<float4*>(ginst.p),
                          static_cast<const unsigned*>(inst_rec.p), static_cast<float*>(carry.p), (long long)m_cap,
                          static_cast<float*>(g2s.p), ctl(), grads, m, v, grad2d, num_sms, s);
  if (dstat)
    launch_densify_stats(n, stride, n_views, vd(), proj().count, static_cast<const float*>(g2s.p), ctl(), dstat, s);
  mark(s, 9);
}

void Raster::enqueue_readback(cudaStream_t s) {
  cudaMemcpyAsync(ctl_h, ctl(), sizeof(Control), cudaMemcpyDeviceToHost, s);
}

gs_status Raster::collect_times() {
  if (!timing) return GS_OK;
  for (int k = 0; k < kNumKernels; ++k) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ev[k], ev[k + 1]) == cudaSuccess) acc_ms[k] += ms;
    else cudaGetLastError();
  }
  ++timed_steps;
  return GS_OK;
}

gs_status Raster::check_control() {
  if (ctl_h->error & kErrTimeout) return fail(GS_ERR_TIMEOUT, "a device-side wait (decoupled look-back) timed out");
  return GS_OK;
}

}  // namespace gs

using gs::fail;

extern "C" {

const char* gs_last_error(void) { return gs::g_last_error.c_str(); }
const char* gs_version(void) { return "gs-onthefly-gb300 0.1 (sm_103a)"; }

gs_status gs_wait_probe(uint32_t spin_limit, uint32_t out_error[2], float out_ms[2]) {
  if (!out_error) return fail(GS_ERR_INVALID_ARG, "out_error is NULL");
  out_error[0] = out_error[1] = 0u;
  return gs::run_wait_probe(spin_limit, out_error, out_ms);
}

gs_status gs_loss_wait_probe(uint32_t spin_limit, uint32_t* out_error, float* out_ms) {
  if (!out_error) return fail(GS_ERR_INVALID_ARG, "out_error is NULL");
  *out_error = 0u;
  return gs::run_loss_wait_probe(spin_limit, out_error, out_ms);
}

gs_status gs_raster_create(gs_raster** out) {
  if (!out) return fail(GS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  gs::Raster* r = new (std::nothrow) gs::Raster();
  if (!r) return fail(GS_ERR_OOM, "host allocation failed");
  if (!r->sp_h || !r->views_h || !r->ctl_h || !r->sp_d.p || !r->views_d.p) {
    delete r;
    return fail(GS_ERR_OOM, "pinned/device allocation of the raster failed");
  }
  *out = reinterpret_cast<gs_raster*>(r);
  return GS_OK;
}

gs_status gs_raster_destroy(gs_raster* r) {
  if (!r) return GS_OK;
  cudaDeviceSynchronize();
  delete reinterpret_cast<gs::Raster*>(r);
  return GS_OK;
}

gs_status gs_raster_forward(gs_raster* rr, void* stream, const float* params, int64_t n, int64_t stride,
                            const gs_camera* cams, int n_views, const float bg[3], float* out_image, float* out_T,
                            uint32_t* out_last, uint32_t* out_gp, uint64_t* out_pairs) {
  gs::Raster* r = reinterpret_cast<gs::Raster*>(rr);
  if (!r || !params || !cams || !out_image || !out_last) return fail(GS_ERR_INVALID_ARG, "NULL argument");
  if (n < 0 || stride <= 0 || n > stride || stride % 32 != 0 || stride > (1 << 30))
    return fail(GS_ERR_INVALID_ARG, "need 0 <= n <= stride, stride a positive multiple of 32");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  gs_status st;
  if ((st = r->set_views(cams, n_views, nullptr))) return st;
  r->stride = (int)stride;
  r->n = (int)n;
  if ((st = r->ensure_records((int)stride))) return st;
  if ((st = r->ensure_instances(r->m_cap))) return st;
  if ((st = r->stage(s))) return st;
  gs::StepParams& P = *r->sp_h;
  P.n = (int)n;
  P.n_views = n_views;
  for (int k = 0; k < 3; ++k) P.bg[k] = bg ? bg[k] : 0.f;
  P.adam = 0;
  r->reset_ledger(s);
  r->upload(s);
  if ((st = r->enqueue_forward_head(s, params, (int)stride, true))) return st;
  if ((st = r->ensure_instances(r->m_cap))) return st;
  if ((st = r->enqueue_forward_tail(s, out_image, out_T, out_last, out_gp))) return st;
  r->have_forward = true;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(GS_ERR_CUDA, std::string("forward launch: ") + cudaGetErrorString(e));
  if (out_pairs) {
    r->enqueue_readback(s);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(GS_ERR_CUDA, std::string("forward: ") + cudaGetErrorString(e));
    *out_pairs = r->ctl_h->pairs;
    if ((st = r->check_control())) return st;
  }
  return GS_OK;
}

gs_status gs_raster_loss(gs_raster* rr, void* stream, const float* image, const float* target,
                         const gs_loss_weights* w, float* out_dimage, double* out_loss) {
  gs::Raster* r = reinterpret_cast<gs::Raster*>(rr);
  if (!r || !image || !target) return fail(GS_ERR_INVALID_ARG, "NULL argument");
  if (!r->have_forward) return fail(GS_ERR_STATE, "gs_raster_loss needs a forward first");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (auto& V : r->views) V.target = target + 3 * V.pix_base;
  gs_status st;
  if ((st = r->stage(s))) return st;
  const gs_loss_weights lw = w ? *w : gs_loss_weights{0.8f, 0.2f, 0.f};
  if (!(lw.lambda_l1 >= 0.f) || !(lw.lambda_ssim >= 0.f) || !(lw.lambda_load >= 0.f))
    return fail(GS_ERR_INVALID_ARG, "loss weights must be >= 0");
  r->sp_h->lambda_ssim = lw.lambda_ssim;
  r->sp_h->lambda_l1 = lw.lambda_l1;
  r->sp_h->lambda_load = lw.lambda_load;
  r->upload(s);
  // the loss may run again on the same forward (other weights): its CTA counter starts at 0
  cudaMemsetAsync(&r->ctl()->loss_done, 0, sizeof(unsigned), s);
  r->enqueue_loss(s, image, out_dimage, false);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(GS_ERR_CUDA, std::string("loss launch: ") + cudaGetErrorString(e));
  if (out_loss) {
    r->enqueue_readback(s);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(GS_ERR_CUDA, std::string("loss: ") + cudaGetErrorString(e));
    *out_loss = r->ctl_h->loss;
  }
  return GS_OK;
}

gs_status gs_raster_backward(gs_raster* rr, void* stream, const float* params, const float* image,
                             const uint32_t* last, const float* dimage, float* out_grads, float* out_grad2d) {
  gs::Raster* r = reinterpret_cast<gs::Raster*>(rr);
  if (!r || !params || !image || !last || !dimage || !out_grads) return fail(GS_ERR_INVALID_ARG, "NULL argument");
  if (!r->have_forward) return fail(GS_ERR_STATE, "gs_raster_backward needs a forward first");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (r->sp_h->lambda_load > 0.f && !r->last_gp)
    return fail(GS_ERR_STATE, "the load term (lambda_load > 0) needs the forward's out_gp");
  gs_status st;
  if ((st = r->stage(s))) return st;
  r->sp_h->adam = 0;
  r->upload(s);
  // the backward may run again on the same forward (another dL/dimage): its work counter starts at 0
  cudaMemsetAsync(&r->ctl()->bwd_work, 0, sizeof(unsigned), s);
  r->enqueue_backward(s, const_cast<float*>(params), image, last, dimage, out_grads, nullptr, nullptr, out_grad2d);
  r->enqueue_readback(s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(GS_ERR_CUDA, std::string("backward: ") + cudaGetErrorString(e));
  r->collect_times();
  return r->check_control();
}

gs_status gs_adam_step(void* stream, float* params, const float* grads, float* m, float* v, int64_t n, int64_t stride,
                       const float lr[6], float beta1, float beta2, float eps, int64_t step) {
  if (!params || !grads || !m || !v || !lr) return fail(GS_ERR_INVALID_ARG, "NULL argument");
  if (n < 0 || stride <= 0 || n > stride || stride % 32 != 0 || step < 1)
    return fail(GS_ERR_INVALID_ARG, "need 0 <= n <= stride (multiple of 32) and step >= 1");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // small private staging for the scalars
  static thread_local gs::DevBuf spd;
  static thread_local gs::StepParams* sph = nullptr;
  static thread_local cudaEvent_t done = nullptr;
  if (!sph) {
    if (cudaMallocHost(&sph, sizeof(gs::StepParams)) != cudaSuccess) return fail(GS_ERR_OOM, "pinned alloc");
    cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
    gs_status st = spd.reserve(sizeof(gs::StepParams), nullptr);
    if (st) return st;
  } else {
    cudaEventSynchronize(done);
  }
  std::memset(sph, 0, sizeof(gs::StepParams));
  for (int k = 0; k < 6; ++k) sph->lr[k] = lr[k];
  sph->beta1 = beta1;
  sph->beta2 = beta2;
  sph->eps = eps;
  sph->step_size_scale = (float)(1.0 / (1.0 - std::pow((double)beta1, (double)step)));
  sph->bc2_sqrt = (float)std::sqrt(1.0 - std::pow((double)beta2, (double)step));
  sph->n = (int)n;
  cudaMemcpyAsync(spd.p, sph, sizeof(gs::StepParams), cudaMemcpyHostToDevice, s);
  cudaEventRecord(done, s);
  gs::launch_adam(params, grads, m, v, (int)n, (int)stride, static_cast<gs::StepParams*>(spd.p), s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(GS_ERR_CUDA, std::string("adam launch: ") + cudaGetErrorString(e));
  return GS_OK;
}

gs_status gs_raster_read(gs_raster* rr, int which, void* host_dst, size_t capacity, size_t* out_bytes) {
  gs::Raster* r = reinterpret_cast<gs::Raster*>(rr);
  if (!r) return fail(GS_ERR_INVALID_ARG, "NULL raster");
  if (!r->have_forward) return fail(GS_ERR_STATE, "no forward to read");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(GS_ERR_CUDA, cudaGetErrorString(e));
  cudaMemcpy(r->ctl_h, r->ctl(), sizeof(gs::Control), cudaMemcpyDeviceToHost);
  const unsigned long long M = r->ctl_h->m_total;
  const size_t recs = (size_t)r->n_views * r->stride;
  const void* src = nullptr;
  size_t bytes = 0;
  switch (which) {
    case 0: src = r->xyo.p; bytes = recs * 16; break;
    case 1: src = r->conic.p; bytes = recs * 16; break;
    case 2: src = r->rgb.p; bytes = recs * 16; break;
    case 3: src = r->depth.p; bytes = recs * 4; break;
    case 4: src = r->radius.p; bytes = recs * 4; break;
    case 5: src = r->rect.p; bytes = recs * 8; break;
    case 6: src = r->count.p; bytes = recs * 4; break;
    case 7: src = r->offsets.p; bytes = recs * 4; break;
    case 8: bytes = M * 8; break;  // assembled below: the sort keeps only the depth bits that vary
    case 9: src = r->vals0.p; bytes = M * 4; break;
    case 10: src = r->ranges(); bytes = (size_t)r->n_tiles * 8; break;
    case 11: src = r->clamp.p; bytes = recs; break;
    case 12: src = r->ginst.p; bytes = M * 48; break;
    default: return fail(GS_ERR_INVALID_ARG, "unknown buffer id");
  }
  if (out_bytes) *out_bytes = bytes;
  if (!host_dst) return GS_OK;
  if (capacity < bytes) return fail(GS_ERR_INVALID_ARG, "host buffer too small");
  if (which == 8) {
    // the sorted (global tile << 32 | fp32 depth bits) keys, in list order
    std::vector<unsigned> v(M);
    std::vector<uint2> rg((size_t)r->n_tiles);
    std::vector<float> depth(recs);
    if ((M && cudaMemcpy(v.data(), r->vals0.p, M * 4, cudaMemcpyDeviceToHost) != cudaSuccess) ||
        (r->n_tiles && cudaMemcpy(rg.data(), r->ranges(), rg.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess) ||
        (recs && cudaMemcpy(depth.data(), r->depth.p, recs * 4, cudaMemcpyDeviceToHost) != cudaSuccess))
      return fail(GS_ERR_CUDA, "reading the tile lists failed");
    unsigned long long* out = static_cast<unsigned long long*>(host_dst);
    for (size_t t = 0; t < rg.size(); ++t)
      for (unsigned i = rg[t].x; i < rg[t].y && i < M; ++i) {
        unsigned bits = 0;
        std::memcpy(&bits, &depth[v[i]], 4);
        out[i] = ((unsigned long long)t << 32) | bits;
      }
    return GS_OK;
  }
  if (bytes) {
    e = cudaMemcpy(host_dst, src, bytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(GS_ERR_CUDA, cudaGetErrorString(e));
  }
  return GS_OK;
}

gs_status gs_raster_set_timing(gs_raster* rr, int enable) {
  gs::Raster* r = reinterpret_cast<gs::Raster*>(rr);
  if (!r) return fail(GS_ERR_INVALID_ARG, "NULL raster");
  r->timing = enable != 0;
  std::memset(r->acc_ms, 0, sizeof(r->acc_ms));
  r->timed_steps = 0;
  return GS_OK;
}

gs_status gs_tiling_candidates(gs_tiling* out, int32_t capacity, int32_t* out_n) {
  gs::Tiling t[GS_MAX_TILINGS];
  const int n = gs::tiling_candidates(t, GS_MAX_TILINGS);
  if (out_n) *out_n = n;
  if (!out) return GS_OK;
  if (capacity < 0) return fail(GS_ERR_INVALID_ARG, "negative capacity");
  for (int k = 0; k < n && k < capacity && k < GS_MAX_TILINGS; ++k) out[k] = gs_tiling{t[k].tw, t[k].th, t[k].batch};
  return GS_OK;
}

gs_status gs_raster_set_tiling(gs_raster* rr, const gs_tiling* t) {
  gs::Raster* r = reinterpret_cast<gs::Raster*>(rr);
  if (!r || !t) return fail(GS_ERR_INVALID_ARG, "NULL argument");
  const gs::Tiling tl{t->tile_w, t->tile_h, t->batch};
  if (!gs::tiling_supported(tl)) return fail(GS_ERR_INVALID_ARG, "tiling not among gs_tiling_candidates");
  r->tiling = tl;
  return GS_OK;
}

gs_status gs_raster_kernel_times(gs_raster* rr, float out_ms[9]) {
  gs::Raster* r = reinterpret_cast<gs::Raster*>(rr);
  if (!r || !out_ms) return fail(GS_ERR_INVALID_ARG, "NULL argument");
  for (int k = 0; k < gs::kNumKernels; ++k) out_ms[k] = (float)r->acc_ms[k];
  return GS_OK;
}

}  // extern "C"
