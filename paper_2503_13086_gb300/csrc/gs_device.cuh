// gs_device.cuh -- device-side definitions shared by the rasterizer kernels (sm_103a).
//
// The hot path of On-the-Fly GS (every Local & Semi-Global iteration, Sec. IV-C) is the 3DGS
// rasterizer of Sec. III (Eq. 1-2) with the constants of the original 3DGS (Sec. V-A), its
// L1 + D-SSIM loss (Eq. 10), a splatting-parallel backward (Sec. IV-D) and Adam with the
// per-image learning rate of Eq. 6-8.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gs {

constexpr int kNumParams = 59;      // mean 3, log-scale 3, quaternion 4, opacity 1, SH 48
constexpr int kMaxTilePix = 256;    // largest tile (pixels = threads of one blend CTA)
constexpr int kChunk = 32;          // Gaussians per backward work item and checkpoint period
constexpr int kMaxStepViews = 32;   // views of one step
constexpr float kNearZ = 0.2f;      // cull at camera z <= 0.2
constexpr float kDilate = 0.3f;     // low-pass term added to the 2D covariance diagonal
constexpr float kFovLim = 1.3f;     // x/z, y/z clamped to 1.3 x half-FOV tangent inside J
constexpr float kAlphaMax = 0.99f;  // alpha clamp
constexpr float kAlphaMin = 1.0f / 255.0f;  // alpha cutoff
constexpr float kTransMin = 1e-4f;  // stop before T would drop below this

// Programmatic dependent launch.  The step's kernels are launched with programmatic stream
// serialisation (launch_dep): a kernel's CTAs may be scheduled while its predecessor is still
// running, so every such kernel first waits, in every thread, until the predecessor grid has
// completed and its writes are visible (dep_wait, before reading anything), then lets its own
// successor be scheduled (dep_release).  Outside such a launch both are no-ops.
__device__ __forceinline__ void dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void dep_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline void launch_dep(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...);
}

// Error bits of Control::error.
constexpr unsigned kErrTimeout = 1u;     // a bounded spin-wait gave up
constexpr unsigned kErrOverflow = 2u;    // instance capacity exceeded (step skipped)

// One camera of a step, in device memory.
struct ViewDev {
  float R[9];      // world -> camera rotation, row-major
  float t[3];
  float fx, fy, cx, cy;
  float campos[3];  // camera centre in world space, -R^T t
  float limx, limy;
  int W, H;        // image size in pixels
  int tw, th;      // tile size in pixels (the same for every view of a step)
  int gx, gy;      // tile grid
  long long tile_base;   // first global tile id of this view
  long long pix_base;    // first pixel of this view in the packed per-pixel buffers
  long long loss_block_base;  // first loss CTA of this view
  const float* target;   // target image (3 x H x W) for the loss
};

// Step control block in device memory, cleared at the start of every step.
struct Control {
  unsigned long long m_total;   // instances emitted by the key emission
  unsigned long long pairs;     // Gaussian-pixel pairs (entries evaluated up to termination)
  unsigned long long blended;   // Gaussian-pixel pairs blended (sum of G_p)
  unsigned long long gp_pixels; // pixels with G_p > 0 (the "visible range" of Eq. 9)
  unsigned long long gp_sq;     // sum of G_p^2 over those pixels
  unsigned int overflow;        // instance capacity exceeded
  unsigned int error;           // kErr* bits
  unsigned int dmax;            // largest fp32 depth bits of a record with instances
  unsigned int dnot;            // ~ smallest such bits (so that the cleared 0 is neutral)
  unsigned int scan_ticket;
  unsigned int sort_ticket[8];
  unsigned int bwd_work;
  unsigned int fwd_work;
  unsigned int loss_done;
  unsigned int fwd_done;        // blend-forward warps past their last counter update
  unsigned int order_count[32];  // tiles per list-length bucket (long-first schedule)
  double loss_view[32];         // per-view loss of the last step
  double loss;                  // batch loss (mean over views)
};

// Running totals over a run of steps enqueued without host synchronisation (not cleared per
// step).  A step whose instances overflow the buffers latches `skip`; every later step of the run
// then does nothing, so the host can re-run the skipped tail in order after growing the buffers.
struct Ledger {
  double loss_sum;
  unsigned long long pairs, blended, instances;
  unsigned long long m_need;  // largest instance count a skipped step needed
  unsigned long long last_gp_sum, last_gp_pixels, last_gp_sq;  // G_p moments of the last completed step
  unsigned int steps_ok;      // steps completed (a prefix of the run)
  unsigned int skip;
  unsigned int error;
  unsigned int pad;
};

// Scalars of one step in device memory (so a captured graph picks up new values).
struct StepParams {
  int n;                 // live Gaussians
  int n_views;
  float bg[3];
  float lambda_ssim;     // D-SSIM weight of the loss
  float lambda_l1;       // L1 weight of the loss
  float lambda_load;     // weight of L_load (Eq. 9): added to the loss; its gradient through the soft count
  float lr[6];           // learning rate per parameter group
  float beta1, beta2, eps;
  float step_size_scale; // 1 / (1 - beta1^t)
  float bc2_sqrt;        // sqrt(1 - beta2^t)
  int adam;              // 1: apply Adam, 0: write gradients, 2: write nothing (autotuner timing)
  int sparse;            // with adam == 1: only Gaussians with instances in a view of the step
};

// Exponent of the 2D Gaussian at offset (dx, dy) from its centre.  The conic is stored
// pre-scaled as (A, B, C) = (-a/2, -b, -c/2) so that power = A dx^2 + B dx dy + C dy^2.  The
// rounding is fixed with explicit intrinsics: the forward and the backward kernels evaluate the
// identical instruction sequence and therefore take identical cutoff decisions.
__device__ __forceinline__ float splat_power(float A, float B, float C, float dx, float dy) {
  return __fmaf_rn(dx, __fmaf_rn(A, dx, __fmul_rn(B, dy)), __fmul_rn(__fmul_rn(C, dy), dy));
}

__device__ __forceinline__ float splat_exp(float power) { return __expf(power); }

// Sort key layout of a step: (global tile << D) | (fp32 depth bits - smallest depth bits of the
// step), D the bits that difference needs (positive floats order like their bits, so the
// difference keeps the order); and the 8-bit passes the tile_bits + D key bits need.
struct KeyLayout {
  int D;
  int passes;
  unsigned dmin;
};
__device__ __forceinline__ KeyLayout key_layout(const Control* ctl, int tile_bits) {
  KeyLayout k;
  const unsigned dmax = ctl->dmax, dnot = ctl->dnot;
  k.dmin = ~dnot;
  const unsigned span = (dmax | dnot) ? dmax - k.dmin : 0u;
  k.D = span ? 32 - __clz(span) : 0;
  k.passes = (tile_bits + k.D + 7) / 8;
  return k;
}

// Bounded spin limit for inter-CTA waits (decoupled look-back).  On expiry the waiting CTA sets
// kErrTimeout and proceeds; the host reports GS_ERR_TIMEOUT.  A round of the scan's look-back takes
// about 0.29 us on a GB300 and one of a sort pass's about 0.37 us, so a wait that nothing ends gives
// up after about 1.2 / 1.6 s; a predecessor that is running publishes within microseconds.
constexpr unsigned kSpinLimit = 1u << 22;

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Relaxed loads and stores for look-back status words: a word carries its flag and value
// together and nothing else is read through it, so several loads can be in flight at once and a
// store needs no fence.
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_u32(unsigned* p, unsigned v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_release_add_u32(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

}  // namespace gs
