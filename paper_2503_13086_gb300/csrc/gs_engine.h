// gs_engine.h -- host-side engine objects behind the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/gs.h"
#include "gs_device.cuh"
#include "gs_kernels.h"

namespace gs {

extern thread_local std::string g_last_error;
gs_status fail(gs_status s, const std::string& msg);
// K2's and K4's look-back waits run once each with a predecessor that never starts (gs_wait_probe).
gs_status run_wait_probe(unsigned spin_limit, unsigned out_error[2], float out_ms[2]);
gs_status run_loss_wait_probe(unsigned spin_limit, unsigned* out_error, float* out_ms);
std::mutex& alloc_capture_mutex();

// A named NVTX range over a scope (host-side phases of the session: steps, field update, graph
// capture, densification...), for profilers that read NVTX (ncu --nvtx).  Costs nothing when no
// tool is attached.
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

void init_sort_attributes();
void init_blend_attributes();
void init_loss_attributes();

// Every DevBuf allocation carries kCanaryBytes of guard words (bytes 0xA5) behind its usable
// `bytes`; no kernel writes them, so a changed word means a write past the end of the buffer.
constexpr size_t kCanaryBytes = 256;
constexpr unsigned kCanaryWord = 0xA5A5A5A5u;

// A device allocation that only grows.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  gs_status reserve(size_t want, size_t* account);
  void release(size_t* account);
};

// One buffer whose guard words a check covers.
struct CanaryRef {
  const char* name;
  const DevBuf* buf;
};
// Checks the guard words of `refs` (buffers without an allocation are skipped) on stream s and
// waits for the result; `flags` is a device scratch of at least (n + 31) / 32 words.  On a changed
// word returns GS_ERR_INTERNAL naming the first such buffer.
gs_status check_canaries(const CanaryRef* refs, int n, unsigned* flags, cudaStream_t s);

constexpr int kMaxViews = 32;
// kernel launches of one optimisation step besides the sort passes: K1, K2, K3 x 2, K5 x 2, K6,
// K7 x 2, K8, K9a x 2, K9
constexpr int kStepLaunchesBase = 13;
constexpr int kNumKernels = 9;
constexpr int kNumEvents = kNumKernels + 1;
constexpr size_t kCtlBytes = 1024;                                   // Control, padded
constexpr size_t kHistBytes = (size_t)kMaxSortPasses * kSortBins * 4;  // digit histograms

// Workspaces and launch sequence of one rasterizer instance.
struct Raster {
  Raster();
  ~Raster();

  // problem of the current step
  int n = 0, stride = 0, n_views = 0, passes = 0, tile_bits = 0;
  long long n_tiles = 0, n_pix = 0, n_loss_blocks = 0;
  std::vector<ViewDev> views;
  bool have_forward = false;
  int num_sms = 1;
  Tiling tiling;   // tile shape and K6 batch of the next step
  float* dstat = nullptr;  // densification statistics (2 rows of stride floats), nullptr: off
  const unsigned* last_gp = nullptr;  // G_p of the last forward (the load term's input), nullptr: none

  // device buffers
  DevBuf sp_d, views_d;
  DevBuf zeroA;  // Control + scan look-back state (cleared before K1)
  DevBuf zeroB;  // histograms + sort look-back state + ranges + chunk map + tile counts (cleared before K3)
  size_t zeroA_bytes = 0, zeroB_bytes = 0, sort_state_bytes = 0, ranges_bytes = 0, chunk_bytes = 0;
  bool zeroB_pending = true;  // zeroB still to be cleared by the forward tail
  DevBuf xyo, conic, rgb, depth, radius, rect, count, offsets, clamp, g2s;
  DevBuf keys0, keys1, vals0, vals1, ginst, ckpt, cmask, order, tile_chunks;
  DevBuf inst_rec, carry;  // instance -> record, K9a partials
  DevBuf partials, block_sums;
  DevBuf ledger_d;  // Ledger of the current run of steps
  DevBuf own_image, own_last, own_dimage;  // used by sessions
  unsigned long long m_cap = 0;
  size_t bytes_in_use = 0;

  // pinned staging
  StepParams* sp_h = nullptr;
  ViewDev* views_h = nullptr;
  Control* ctl_h = nullptr;
  Ledger* ledger_h = nullptr;
  cudaEvent_t staged = nullptr;

  // timing
  bool timing = false;
  cudaEvent_t ev[kNumEvents];
  double acc_ms[kNumKernels] = {0};
  long long timed_steps = 0;

  Control* ctl() const;
  unsigned long long* scan_state() const;
  unsigned* hist() const;
  unsigned* sort_state() const;
  uint2* ranges() const;
  int* chunk_tile() const;
  unsigned* tile_done() const;  // per tile: 1 once the blend forward finished it
  ProjBuffers proj() const;
  const StepParams* sp() const { return static_cast<const StepParams*>(sp_d.p); }
  const ViewDev* vd() const { return static_cast<const ViewDev*>(views_d.p); }

  gs_status set_views(const gs_camera* cams, int nv, const float* const* targets);
  gs_status ensure_records(int stride_);
  gs_status ensure_instances(unsigned long long m);
  gs_status stage(cudaStream_t s);
  gs_status upload(cudaStream_t s);
  void mark(cudaStream_t s, int k);
  gs_status enqueue_forward_head(cudaStream_t s, const float* params, int stride_, bool size_exactly);
  gs_status enqueue_forward_tail(cudaStream_t s, float* image, float* T, unsigned* last, unsigned* gp);
  // after_forward: the loss follows this step's blend forward directly in the stream (its blocks then
  // start as the forward completes the tiles under them)
  void enqueue_loss(cudaStream_t s, const float* image, float* dimage, bool after_forward);
  void enqueue_blend_backward(cudaStream_t s, const float* image, const float* dimage);
  void enqueue_backward(cudaStream_t s, float* params, const float* image, const unsigned* last, const float* dimage,
                        float* grads, float* m, float* v, float* grad2d);
  void enqueue_readback(cudaStream_t s);
  Ledger* ledger() const { return static_cast<Ledger*>(ledger_d.p); }
  void reset_ledger(cudaStream_t s) { cudaMemsetAsync(ledger_d.p, 0, sizeof(Ledger), s); }
  void read_ledger(cudaStream_t s) { cudaMemcpyAsync(ledger_h, ledger_d.p, sizeof(Ledger), cudaMemcpyDeviceToHost, s); }
  gs_status collect_times();
  gs_status check_control();
};

}  // namespace gs
