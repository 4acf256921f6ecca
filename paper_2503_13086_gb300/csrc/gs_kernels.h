// gs_kernels.h -- launch wrappers of the rasterizer kernels (host-visible declarations).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "gs_device.cuh"

namespace gs {

// Per-record outputs of K1 (record = view * stride + Gaussian id).
struct ProjBuffers {
  float4* xyo;           // (u, v, ex, ey): mean and half extents of the 1/255 cutoff box
  float4* conic;         // pre-scaled conic (-a/2, -b, -c/2) and thr = -ln(255 opacity)
  float4* rgb;           // (r, g, b, opacity)
  float* depth;          // camera-space z
  int* radius;           // 0 = culled
  uint2* rect;           // (x0 | x1 << 16, y0 | y1 << 16) tile rectangle
  unsigned* count;       // tiles touched, 0 = culled
  unsigned* offsets;     // exclusive scan of count
  unsigned char* clamp;  // bit ch set: colour channel ch was clamped at 0
};

// Sort geometry.
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr int kSortThreads = 512;
constexpr int kSortItems = 8;
constexpr int kSortMinBlocks = 2;  // resident onesweep CTAs per SM the registers must allow
constexpr int kSortTile = kSortThreads * kSortItems;  // keys per onesweep CTA
constexpr int kSortBits = 8;
constexpr int kSortBins = 1 << kSortBits;
constexpr int kMaxSortPasses = 8;

// Tile shape of the binning and blending, and the number of sorted Gaussians K6 stages in shared
// memory per round.  Only the shapes/batches in tiling_candidates() are compiled.
struct Tiling {
  int tw = 16, th = 16, batch = 256;
  bool operator==(const Tiling& o) const { return tw == o.tw && th == o.th && batch == o.batch; }
};
int tiling_candidates(Tiling* out, int cap);  // returns how many; fills up to cap
bool tiling_supported(const Tiling& t);

void launch_project(const float* params, int stride, int n_views, const StepParams* sp, const ViewDev* views,
                    const ProjBuffers& out, cudaStream_t s);
// K9a (per-record sums of the instance gradients, into g2s: 9 planes of views x stride floats) and
// K9 + K10.
void launch_project_backward(float* params, int stride, int n_views, const StepParams* sp, const ViewDev* views,
                             const ProjBuffers& pb, const float4* ginst, const unsigned* inst_rec, float* carry,
                             long long m_cap, float* g2s, const Control* ctl, float* grads_out, float* m, float* v,
                             float* grad2d_out, int num_sms, cudaStream_t s);
void launch_adam(float* params, const float* grads, float* m, float* v, int n, int stride, const StepParams* sp,
                 cudaStream_t s);

void launch_scan(const unsigned* in, unsigned* out, long long n_items, unsigned long long* state, Control* ctl,
                 unsigned long long m_cap, Ledger* ledger, cudaStream_t s, const float* depth = nullptr);
void launch_emit(const ProjBuffers& pb, const ViewDev* views, int stride, long long n_items, unsigned long long* keys0,
                 unsigned* vals0, unsigned long long* keys1, unsigned* vals1, unsigned* inst_rec, unsigned* hist,
                 int tile_bits, long long m_cap, int num_sms, const Control* ctl, cudaStream_t s);
void launch_sort_pass(unsigned long long* keys0, unsigned* vals0, unsigned long long* keys1, unsigned* vals1,
                      const unsigned* hist, unsigned* state, int pass, int tile_bits, long long m_cap, Control* ctl,
                      cudaStream_t s);
void launch_ranges(const unsigned long long* keys, uint2* ranges, int tile_bits, long long m_cap, const Control* ctl,
                   cudaStream_t s);

void launch_tile_order(const uint2* ranges, long long n_tiles, int* order, const Control* ctl, cudaStream_t s);
void launch_blend_forward(const Tiling& tl, const ViewDev* views, int n_views, long long n_tiles, const uint2* ranges,
                          const unsigned* vals, const ProjBuffers& pb, const StepParams* sp, Control* ctl,
                          const int* order, float* image, float* T, unsigned* last, unsigned* gp, float4* ckpt,
                          unsigned* cmask, int* chunk_tile, int* tile_chunks, unsigned* tile_done, int num_sms,
                          cudaStream_t s);
// Warps the blend forward launches for this problem (each adds 1 to Control::fwd_done at its end).
long long forward_warps(const Tiling& tl, long long n_tiles, int num_sms);
void launch_blend_backward(const Tiling& tl, const ViewDev* views, int n_views, long long n_tiles, const uint2* ranges,
                           const unsigned* vals, const ProjBuffers& pb, Control* ctl, const float* image,
                           const float* dimage, const float4* ckpt, const unsigned* cmask, const int* chunk_tile,
                           const int* tile_chunks, float4* ginst, const unsigned* gp, const StepParams* sp,
                           int num_sms, cudaStream_t s);

// Field update (Sec. IV-B): the registered sparse points, hashed by cubic cells.
constexpr float kCoarseCells = 4.f;  // coarse grid cell edge in fine cells (3-NN search)
struct PointGridDev {
  const float* xyz;           // 3 floats per point
  unsigned long long* keys;   // per slot: cell key, ~0 = empty
  int* head;                  // per slot: first point of the cell, -1 = none
  const int* next;            // per point: next point of its cell, -1 = end
  unsigned mask;              // slots - 1 (slots a power of two, at least twice the points)
  float cell;                 // cell edge
};
void launch_hwc_to_chw(const float* src, float* dst, long long npix, cudaStream_t s);
// src: the device address of page-locked host memory (read by the kernel over the host link).
void launch_hwc_to_chw_host(const float* src, float* dst, long long npix, cudaStream_t s);
void launch_far_points(const PointGridDev& g, const float* xyz, int n_new, float thr2, int ring, unsigned* far,
                       cudaStream_t s);
void launch_insert_points(const PointGridDev& g, int* next, long long first, long long count, cudaStream_t s);
void launch_scan_flags(const unsigned* far, int n, unsigned* offsets, unsigned* count, cudaStream_t s);
void launch_init_gaussians(const PointGridDev& g, const PointGridDev& gc, const float* xyz, const float* rgb, int n_new, long long self0,
                           const unsigned* far, const unsigned* offsets, float* params, float* m, float* v, int stride,
                           int n0, float opacity_logit, double sh_c0, cudaStream_t s);

// 3DGS adaptive density control (k_densify.cu).
struct DensifyThresholds {
  float grad;       // mean view-space gradient norm that makes a Gaussian clone or split
  float ls_dense;   // log(percent_dense x extent): clone at or below, split above
  float ls_big;     // log(max_scale x extent): pruned above
  float logit_min;  // logit(min_opacity): pruned below
  float ls_shrink;  // log(1.6): what a split lowers every log-scale by
  unsigned long long seed_base;  // seed ^ (round x 0x9E3779B97F4A7C15)
};
void launch_densify_stats(int n, int stride, int n_views, const ViewDev* views, const unsigned* count,
                          const float* g2s, const Control* ctl, float* dstat, cudaStream_t s);
void launch_densify_count(int n, int stride, const float* params, const float* dstat, const DensifyThresholds& th,
                          unsigned* ca, unsigned* cb, unsigned* cc, unsigned* cand, cudaStream_t s);
void launch_densify_write(int n, int stride, const float* params, const float* m, const float* v, const float* dstat,
                          const DensifyThresholds& th, const unsigned* oa, const unsigned* ob, const unsigned* oc,
                          const unsigned* totals, int stride2, float* p2, float* m2, float* v2, cudaStream_t s);

// Loss: per-view partial maps, the loss value in ctl->loss, dL/dimage.
long long loss_blocks(int W, int H);
// tile_done (nullable): the blend forward's per-tile completion flags; with it the loss forward follows
// the blend forward directly and starts each block once the tiles under its window are complete (and
// its last CTA once fwd_warps warps have counted themselves in Control::fwd_done) instead of waiting
// for the whole forward.  Null: the image is complete before the launch (it waits for its predecessor).
void launch_loss(const ViewDev* views, int n_views, long long n_blocks, const float* image, const StepParams* sp,
                 float* partials, double* block_sums, Control* ctl, Ledger* ledger, float* dimage,
                 const unsigned* tile_done, long long fwd_warps, cudaStream_t s);

}  // namespace gs
