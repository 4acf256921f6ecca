// k_densify.cu -- the adaptive density control of the original 3DGS (clone, split, prune), kept by
// On-the-Fly GS among "all other settings" of 3DGS (Sec. V-A), as an optional step, sm_103a.
//
//   KD1 (every optimisation step, when enabled): per Gaussian and per view in which it has
//       instances, the norm of its view-space mean gradient -- the per-view pixel-space sum of K9a
//       scaled by (W / 2, H / 2) -- accumulated with a count;
//   KD2: per Gaussian, whether it is kept, cloned, split (2 children) and which results survive the
//       prune (opacity, world-space size), as counts for three scans;
//   KD3: the new columns -- kept originals (with their Adam moments), then clones, then children
//       (mean + R(q) (s * z), log-scales lowered by log 1.6), moments of the new ones 0.
// Decisions compare log-scales and opacity logits with thresholds the host takes to those domains,
// so they are taken on the exact float32 parameters.  The normals z come from a counter-based
// generator (SplitMix64 outputs of a per-(round, Gaussian, child, axis) counter, Box-Muller in
// double precision), so a split is reproducible and independent of the launch configuration.
#include "gs_engine.h"

namespace gs {

namespace {

__device__ __forceinline__ unsigned long long sm64(unsigned long long x) {
  unsigned long long z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ float child_normal(unsigned long long base, unsigned long long i, int c, int a) {
  const unsigned long long k = (2ull * i + (unsigned long long)c) * 3ull + (unsigned long long)a;
  const unsigned long long h1 = sm64(base + 2ull * k), h2 = sm64(base + 2ull * k + 1ull);
  const double u1 = (double)((h1 >> 11) + 1ull) * 0x1.0p-53;
  const double u2 = (double)(h2 >> 11) * 0x1.0p-53;
  return (float)(sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2));
}

struct Decision {
  bool clone, split, prune_orig, prune_child;
};

__device__ __forceinline__ Decision decide(const float* __restrict__ params, int stride, int i,
                                           const float* __restrict__ dstat, const DensifyThresholds& th) {
  const float acc = dstat[i], cnt = dstat[stride + i];
  const float g = cnt > 0.f ? __fdiv_rn(acc, cnt) : 0.f;
  const float maxls = fmaxf(fmaxf(params[3 * stride + i], params[4 * stride + i]), params[5 * stride + i]);
  const float logit = params[10 * stride + i];
  Decision d;
  const bool hot = g >= th.grad;
  d.clone = hot && maxls <= th.ls_dense;
  d.split = hot && maxls > th.ls_dense;
  d.prune_orig = logit < th.logit_min || maxls > th.ls_big;
  d.prune_child = logit < th.logit_min || __fsub_rn(maxls, th.ls_shrink) > th.ls_big;
  return d;
}

}  // namespace

// KD1
__global__ void __launch_bounds__(256) k_densify_stats(int n, int stride, int n_views, const ViewDev* __restrict__ views,
                                                       const unsigned* __restrict__ count,
                                                       const float* __restrict__ g2s, const Control* __restrict__ ctl,
                                                       float* __restrict__ dstat) {
  dep_wait();
  dep_release();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || ctl->overflow) return;
  const long long n_rec = (long long)n_views * stride;
  float acc = dstat[i], cnt = dstat[stride + i];
  for (int v = 0; v < n_views; ++v) {
    const long long rec = (long long)v * stride + i;
    if (!count[rec]) continue;
    const float gx = __fmul_rn(g2s[rec], 0.5f * (float)views[v].W);
    const float gy = __fmul_rn(g2s[n_rec + rec], 0.5f * (float)views[v].H);
    acc = __fadd_rn(acc, __fsqrt_rn(__fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy))));
    cnt += 1.f;
  }
  dstat[i] = acc;
  dstat[stride + i] = cnt;
}

// KD2: counts of kept originals (a), surviving clones (b) and surviving children (c) per Gaussian,
// and the candidate totals (clones, splits) in cand[0..1].
__global__ void __launch_bounds__(256) k_densify_count(int n, int stride, const float* __restrict__ params,
                                                       const float* __restrict__ dstat, DensifyThresholds th,
                                                       unsigned* __restrict__ ca, unsigned* __restrict__ cb,
                                                       unsigned* __restrict__ cc, unsigned* __restrict__ cand) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Decision d = decide(params, stride, i, dstat, th);
  ca[i] = (!d.split && !d.prune_orig) ? 1u : 0u;
  cb[i] = (d.clone && !d.prune_orig) ? 1u : 0u;
  cc[i] = (d.split && !d.prune_child) ? 2u : 0u;
  if (d.clone) atomicAdd(&cand[0], 1u);
  if (d.split) atomicAdd(&cand[1], 1u);
}

// KD3
__global__ void __launch_bounds__(256) k_densify_write(int n, int stride, const float* __restrict__ params,
                                                       const float* __restrict__ m, const float* __restrict__ v,
                                                       const float* __restrict__ dstat, DensifyThresholds th,
                                                       const unsigned* __restrict__ oa, const unsigned* __restrict__ ob,
                                                       const unsigned* __restrict__ oc,
                                                       const unsigned* __restrict__ totals, int stride2,
                                                       float* __restrict__ p2, float* __restrict__ m2,
                                                       float* __restrict__ v2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Decision d = decide(params, stride, i, dstat, th);
  const unsigned A = totals[0], B = totals[1];
  if (!d.split && !d.prune_orig) {
    const long long j = oa[i];
    for (int r = 0; r < kNumParams; ++r) {
      p2[(long long)r * stride2 + j] = params[(long long)r * stride + i];
      m2[(long long)r * stride2 + j] = m[(long long)r * stride + i];
      v2[(long long)r * stride2 + j] = v[(long long)r * stride + i];
    }
  }
  if (d.clone && !d.prune_orig) {
    const long long j = (long long)A + ob[i];
    for (int r = 0; r < kNumParams; ++r) {
      p2[(long long)r * stride2 + j] = params[(long long)r * stride + i];
      m2[(long long)r * stride2 + j] = 0.f;
      v2[(long long)r * stride2 + j] = 0.f;
    }
  }
  if (d.split && !d.prune_child) {
    // rotation of the normalised quaternion (w, x, y, z)
    float qw = params[6 * stride + i], qx = params[7 * stride + i], qy = params[8 * stride + i],
          qz = params[9 * stride + i];
    const float qi = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
    qw *= qi;
    qx *= qi;
    qy *= qi;
    qz *= qi;
    const float R[9] = {1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - qw * qz), 2.f * (qx * qz + qw * qy),
                        2.f * (qx * qy + qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - qw * qx),
                        2.f * (qx * qz - qw * qy), 2.f * (qy * qz + qw * qx), 1.f - 2.f * (qx * qx + qy * qy)};
    float s[3];
    for (int a = 0; a < 3; ++a) s[a] = expf(params[(3 + a) * stride + i]);
    for (int c = 0; c < 2; ++c) {
      const long long j = (long long)A + B + oc[i] + c;
      float z[3];
      for (int a = 0; a < 3; ++a) z[a] = s[a] * child_normal(th.seed_base, (unsigned long long)i, c, a);
      for (int r = 0; r < kNumParams; ++r) {
        float val = params[(long long)r * stride + i];
        if (r < 3) val += R[3 * r] * z[0] + R[3 * r + 1] * z[1] + R[3 * r + 2] * z[2];
        else if (r < 6) val = __fsub_rn(val, th.ls_shrink);
        p2[(long long)r * stride2 + j] = val;
        m2[(long long)r * stride2 + j] = 0.f;
        v2[(long long)r * stride2 + j] = 0.f;
      }
    }
  }
}

void launch_densify_stats(int n, int stride, int n_views, const ViewDev* views, const unsigned* count,
                          const float* g2s, const Control* ctl, float* dstat, cudaStream_t s) {
  if (n <= 0) return;
  launch_dep(k_densify_stats, dim3((n + 255) / 256), dim3(256), 0, s, n, stride, n_views, views, count, g2s, ctl,
      dstat);
}

void launch_densify_count(int n, int stride, const float* params, const float* dstat, const DensifyThresholds& th,
                          unsigned* ca, unsigned* cb, unsigned* cc, unsigned* cand, cudaStream_t s) {
  if (n <= 0) return;
  k_densify_count<<<(n + 255) / 256, 256, 0, s>>>(n, stride, params, dstat, th, ca, cb, cc, cand);
}

void launch_densify_write(int n, int stride, const float* params, const float* m, const float* v, const float* dstat,
                          const DensifyThresholds& th, const unsigned* oa, const unsigned* ob, const unsigned* oc,
                          const unsigned* totals, int stride2, float* p2, float* m2, float* v2, cudaStream_t s) {
  if (n <= 0) return;
  k_densify_write<<<(n + 255) / 256, 256, 0, s>>>(n, stride, params, m, v, dstat, th, oa, ob, oc, totals, stride2, p2,
                                                  m2, v2);
}

}  // namespace gs
