// k_project.cu -- K1 (EWA projection + SH colour) and the fused K9 + K10 (projection backward
// chained straight into Adam), sm_103a.
//
// K1 evaluates, per (view, Gaussian), Eq. 1 (Sigma = R S S^T R^T) and its EWA splat into the
// image as used by the 3DGS rasterizer (Sec. III; constants of the original 3DGS, Sec. V-A), the
// degree-3 SH colour and the tile rectangle.  K9 chains the per-instance 2D gradients from the
// blend backward into the 59 parameters of each Gaussian, summed over the views of the step,
// and K10 applies Adam with the per-group learning rate (the mean-position rate is the per-image
// rate of Eq. 6-8) in the same pass, so no gradient buffer is written or read.
//
// Data layout: parameters component-major, params[c * stride + i] (see gs.h).  Per-record
// outputs (record = view * stride + Gaussian) are structure-of-arrays of 16-byte records so the
// blend kernels gather a Gaussian with three 16-byte loads.
#include "gs_device.cuh"
#include "gs_kernels.h"

namespace gs {

// Real SH up to degree 3 (Condon-Shortley phase, 3DGS ordering).  The constants are the
// normalisation factors sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!): 1/(2 sqrt(pi)), sqrt(3/(4 pi)),
// sqrt(15/pi)/2, sqrt(5/pi)/4, sqrt(15/pi)/4, sqrt(35/(2 pi))/4, sqrt(105/pi)/2,
// sqrt(21/(2 pi))/4, sqrt(7/pi)/4, sqrt(105/pi)/4.
constexpr float kSH0 = 0.28209479177387814f;
constexpr float kSH1 = 0.48860251190291992f;
constexpr float kSH2a = 1.09254843059207907f;
constexpr float kSH2b = 0.31539156525252005f;
constexpr float kSH2c = 0.54627421529603953f;
constexpr float kSH3a = 0.59004358992664352f;
constexpr float kSH3b = 2.89061144264055405f;
constexpr float kSH3c = 0.45704579946446573f;
constexpr float kSH3d = 0.37317633259011540f;
constexpr float kSH3e = 1.44530572132027702f;

__device__ __forceinline__ void sh_basis(float x, float y, float z, float Y[16]) {
  const float xx = x * x, yy = y * y, zz = z * z;
  Y[0] = kSH0;
  Y[1] = -kSH1 * y;
  Y[2] = kSH1 * z;
  Y[3] = -kSH1 * x;
  Y[4] = kSH2a * x * y;
  Y[5] = -kSH2a * y * z;
  Y[6] = kSH2b * (2.f * zz - xx - yy);
  Y[7] = -kSH2a * x * z;
  Y[8] = kSH2c * (xx - yy);
  Y[9] = -kSH3a * y * (3.f * xx - yy);
  Y[10] = kSH3b * x * y * z;
  Y[11] = -kSH3c * y * (4.f * zz - xx - yy);
  Y[12] = kSH3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
  Y[13] = -kSH3c * x * (4.f * zz - xx - yy);
  Y[14] = kSH3e * z * (xx - yy);
  Y[15] = -kSH3a * x * (xx - 3.f * yy);
}

// Accumulate into d[3] the gradient with respect to (x, y, z) of sum_k Y_k(x, y, z) * w[k].
__device__ __forceinline__ void sh_basis_vjp(float x, float y, float z, const float w[16], float d[3]) {
  const float xx = x * x, yy = y * y, zz = z * z;
  float gx = 0.f, gy = 0.f, gz = 0.f;
  gy += -kSH1 * w[1];
  gz += kSH1 * w[2];
  gx += -kSH1 * w[3];
  gx += kSH2a * y * w[4];
  gy += kSH2a * x * w[4];
  gy += -kSH2a * z * w[5];
  gz += -kSH2a * y * w[5];
  gx += -2.f * kSH2b * x * w[6];
  gy += -2.f * kSH2b * y * w[6];
  gz += 4.f * kSH2b * z * w[6];
  gx += -kSH2a * z * w[7];
  gz += -kSH2a * x * w[7];
  gx += 2.f * kSH2c * x * w[8];
  gy += -2.f * kSH2c * y * w[8];
  gx += -6.f * kSH3a * x * y * w[9];
  gy += -kSH3a * (3.f * xx - 3.f * yy) * w[9];
  gx += kSH3b * y * z * w[10];
  gy += kSH3b * x * z * w[10];
  gz += kSH3b * x * y * w[10];
  gx += 2.f * kSH3c * x * y * w[11];
  gy += -kSH3c * (4.f * zz - xx - 3.f * yy) * w[11];
  gz += -8.f * kSH3c * y * z * w[11];
  gx += -6.f * kSH3d * x * z * w[12];
  gy += -6.f * kSH3d * y * z * w[12];
  gz += kSH3d * (6.f * zz - 3.f * xx - 3.f * yy) * w[12];
  gx += -kSH3c * (4.f * zz - 3.f * xx - yy) * w[13];
  gy += 2.f * kSH3c * x * y * w[13];
  gz += -8.f * kSH3c * x * z * w[13];
  gx += 2.f * kSH3e * x * z * w[14];
  gy += -2.f * kSH3e * y * z * w[14];
  gz += kSH3e * (xx - yy) * w[14];
  gx += -kSH3a * (3.f * xx - 3.f * yy) * w[15];
  gy += 6.f * kSH3a * x * y * w[15];
  d[0] += gx;
  d[1] += gy;
  d[2] += gz;
}

// Geometry of one Gaussian seen from one view: what K1 computes and K9 recomputes.
struct Geo {
  float p[3];          // camera-space mean
  float qn[4], qinv;   // normalised quaternion, 1/|q|
  float Rq[9], s[3];
  float M[9];          // Rq diag(s)
  float Sig[6];        // 3D covariance (xx, xy, xz, yy, yz, zz)
  float Tm[6];         // J R_cam
  float txz, tyz;
  bool xin, yin;
  float cov[3];        // dilated 2D covariance (a', b', c')
  float det;
};

__device__ __forceinline__ bool geo_forward(const ViewDev& V, const float mu[3], const float ls[3],
                                            const float q[4], Geo& g) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
    g.p[r] = V.R[3 * r] * mu[0] + V.R[3 * r + 1] * mu[1] + V.R[3 * r + 2] * mu[2] + V.t[r];
  if (!(g.p[2] > kNearZ)) return false;
  const float qq = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
  if (!(qq > 0.f)) return false;
  g.qinv = rsqrtf(qq);
#pragma unroll
  for (int k = 0; k < 4; ++k) g.qn[k] = q[k] * g.qinv;
  const float w = g.qn[0], x = g.qn[1], y = g.qn[2], z = g.qn[3];
  g.Rq[0] = 1.f - 2.f * (y * y + z * z);
  g.Rq[1] = 2.f * (x * y - w * z);
  g.Rq[2] = 2.f * (x * z + w * y);
  g.Rq[3] = 2.f * (x * y + w * z);
  g.Rq[4] = 1.f - 2.f * (x * x + z * z);
  g.Rq[5] = 2.f * (y * z - w * x);
  g.Rq[6] = 2.f * (x * z - w * y);
  g.Rq[7] = 2.f * (y * z + w * x);
  g.Rq[8] = 1.f - 2.f * (x * x + y * y);
#pragma unroll
  for (int k = 0; k < 3; ++k) g.s[k] = __expf(ls[k]);
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) g.M[3 * r + c] = g.Rq[3 * r + c] * g.s[c];
  auto dotrow = [&](int a, int b) {
    return g.M[3 * a] * g.M[3 * b] + g.M[3 * a + 1] * g.M[3 * b + 1] + g.M[3 * a + 2] * g.M[3 * b + 2];
  };
  g.Sig[0] = dotrow(0, 0);
  g.Sig[1] = dotrow(0, 1);
  g.Sig[2] = dotrow(0, 2);
  g.Sig[3] = dotrow(1, 1);
  g.Sig[4] = dotrow(1, 2);
  g.Sig[5] = dotrow(2, 2);

  const float pz = g.p[2];
  const float iz = 1.f / pz;
  const float xz = g.p[0] * iz, yz = g.p[1] * iz;
  g.xin = (xz >= -V.limx) && (xz <= V.limx);
  g.yin = (yz >= -V.limy) && (yz <= V.limy);
  g.txz = fminf(V.limx, fmaxf(-V.limx, xz));
  g.tyz = fminf(V.limy, fmaxf(-V.limy, yz));
  const float J00 = V.fx * iz, J02 = -V.fx * g.txz * iz;
  const float J11 = V.fy * iz, J12 = -V.fy * g.tyz * iz;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    g.Tm[c] = J00 * V.R[c] + J02 * V.R[6 + c];
    g.Tm[3 + c] = J11 * V.R[3 + c] + J12 * V.R[6 + c];
  }
  // Sigma full-matrix accessor
  const float S[9] = {g.Sig[0], g.Sig[1], g.Sig[2], g.Sig[1], g.Sig[3], g.Sig[4], g.Sig[2], g.Sig[4], g.Sig[5]};
  float st0[3], st1[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    st0[r] = S[3 * r] * g.Tm[0] + S[3 * r + 1] * g.Tm[1] + S[3 * r + 2] * g.Tm[2];
    st1[r] = S[3 * r] * g.Tm[3] + S[3 * r + 1] * g.Tm[4] + S[3 * r + 2] * g.Tm[5];
  }
  g.cov[0] = g.Tm[0] * st0[0] + g.Tm[1] * st0[1] + g.Tm[2] * st0[2] + kDilate;
  g.cov[1] = g.Tm[0] * st1[0] + g.Tm[1] * st1[1] + g.Tm[2] * st1[2];
  g.cov[2] = g.Tm[3] * st1[0] + g.Tm[4] * st1[1] + g.Tm[5] * st1[2] + kDilate;
  g.det = g.cov[0] * g.cov[2] - g.cov[1] * g.cov[1];
  return g.det > 0.f;
}

// ---------------------------------------------------------------------------------------------
// K1: projection forward.  grid = (ceil(stride / 256), views); one thread per (view, Gaussian).
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 6) k_project(const float* __restrict__ params, int stride,
                                                 const StepParams* __restrict__ sp,
                                                 const ViewDev* __restrict__ views, ProjBuffers out) {
  dep_wait();
  dep_release();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int v = blockIdx.y;
  if (i >= stride) return;
  const long long rec = (long long)v * stride + i;
  const int n = sp->n;
  auto cull = [&]() {
    out.count[rec] = 0u;
    out.radius[rec] = 0;
  };
  if (i >= n) {
    cull();
    return;
  }
  const ViewDev& V = views[v];
  const float mu[3] = {__ldg(params + i), __ldg(params + stride + i), __ldg(params + 2 * stride + i)};
  const float ls[3] = {__ldg(params + 3 * stride + i), __ldg(params + 4 * stride + i), __ldg(params + 5 * stride + i)};
  const float q[4] = {__ldg(params + 6 * stride + i), __ldg(params + 7 * stride + i), __ldg(params + 8 * stride + i),
                      __ldg(params + 9 * stride + i)};
  Geo g;
  if (!geo_forward(V, mu, ls, q, g)) {
    cull();
    return;
  }
  const float det = g.det;
  const float ca = g.cov[2] / det, cb = -g.cov[1] / det, cc = g.cov[0] / det;
  const float u = V.fx * g.p[0] / g.p[2] + V.cx;
  const float vv = V.fy * g.p[1] / g.p[2] + V.cy;
  const float mid = 0.5f * (g.cov[0] + g.cov[2]);
  const float lam = mid + sqrtf(fmaxf(0.1f, mid * mid - det));
  const int r = (int)ceilf(3.f * sqrtf(lam));
  // Tile rectangle: [floor((u - r)/tw), floor((u + r + tw - 1)/tw)) clamped to the grid, same for
  // y with th, in fp32 (the expression the key emission and its checks use).
  const float rf = (float)r;
  const float twf = (float)V.tw, thf = (float)V.th;
  int x0 = (int)floorf(__fdiv_rn(__fsub_rn(u, rf), twf));
  int y0 = (int)floorf(__fdiv_rn(__fsub_rn(vv, rf), thf));
  int x1 = (int)floorf(__fdiv_rn(__fadd_rn(__fadd_rn(u, rf), (float)(V.tw - 1)), twf));
  int y1 = (int)floorf(__fdiv_rn(__fadd_rn(__fadd_rn(vv, rf), (float)(V.th - 1)), thf));
  x0 = min(V.gx, max(0, x0));
  x1 = min(V.gx, max(0, x1));
  y0 = min(V.gy, max(0, y0));
  y1 = min(V.gy, max(0, y1));
  const unsigned cnt = (unsigned)((x1 - x0) * (y1 - y0));
  if (cnt == 0u || !isfinite(u) || !isfinite(vv) || !isfinite(ca) || !isfinite(cb) || !isfinite(cc)) {
    cull();
    return;
  }
  // Colour: degree-3 SH at the unit direction from the camera centre to the mean, + 0.5, >= 0.
  float d0 = mu[0] - V.campos[0], d1 = mu[1] - V.campos[1], d2 = mu[2] - V.campos[2];
  const float dl = rsqrtf(d0 * d0 + d1 * d1 + d2 * d2);
  d0 *= dl;
  d1 *= dl;
  d2 *= dl;
  // the 48 SH coefficient rows and the opacity logit on their way to L2 at once (no register held):
  // the loads below, which the compiler issues a few at a time (40 registers keep six CTAs per SM,
  // so a 200k-Gaussian view is one wave), then find them there instead of making one DRAM round
  // trip per batch
  {
    const float* pf = params + 10ll * stride + i;
#pragma unroll 1
    for (int k = 0; k < 49; ++k, pf += stride) asm volatile("prefetch.global.L2 [%0];" ::"l"(pf));
  }
  float Y[16];
  sh_basis(d0, d1, d2, Y);
  float col[3];
  unsigned clampbits = 0u;
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < 16; ++k) acc += Y[k] * __ldg(params + (11 + 3 * k + ch) * stride + i);
    acc += 0.5f;
    if (acc < 0.f) clampbits |= 1u << ch;
    col[ch] = fmaxf(acc, 0.f);
  }
  const float opac = 1.f / (1.f + __expf(-__ldg(params + 10 * stride + i)));
  // alpha = opacity * exp(power) reaches 1/255 only where power >= thr = -ln(255 opacity), i.e.
  // inside the ellipse d^T conic d <= 2 ln(255 opacity); its axis-aligned half extents are
  // sqrt(2 ln(255 opacity) cov_xx), sqrt(.. cov_yy).  Widened by 0.1 % + 0.01 px so no pixel the
  // blend would accept lies outside (a culling bound only; it decides nothing by itself).
  const float thr = -logf(255.f * opac);
  float ex = -1e30f, ey = -1e30f;
  if (thr < 0.f) {
    ex = sqrtf(-2.f * thr * g.cov[0]) * 1.001f + 0.01f;
    ey = sqrtf(-2.f * thr * g.cov[2]) * 1.001f + 0.01f;
  }
  out.xyo[rec] = make_float4(u, vv, ex, ey);
  out.conic[rec] = make_float4(-0.5f * ca, -cb, -0.5f * cc, thr);
  out.rgb[rec] = make_float4(col[0], col[1], col[2], opac);
  out.depth[rec] = g.p[2];
  out.radius[rec] = r;
  out.rect[rec] = make_uint2((unsigned)x0 | ((unsigned)x1 << 16), (unsigned)y0 | ((unsigned)y1 << 16));
  out.count[rec] = cnt;
  out.clamp[rec] = (unsigned char)clampbits;
}

// ---------------------------------------------------------------------------------------------
// K9 + K10: per Gaussian, sum the instance gradients of every view, chain them to the 59
// parameters and either apply Adam (hot path) or write the gradient (parity / autograd).
// Streaming layout: the geometry is chained view by view; what the 48 SH coefficients need
// (view direction, masked colour gradient, 1/|mu - camera|) is kept per view, and the SH rows
// are then updated one coefficient at a time, so a thread never holds all 59 gradients.
// ---------------------------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ void sh_term(float x, float y, float z, float& Y, float& gx, float& gy, float& gz) {
  const float xx = x * x, yy = y * y, zz = z * z;
  switch (K) {
    case 0: Y = kSH0; gx = gy = gz = 0.f; break;
    case 1: Y = -kSH1 * y; gx = 0.f; gy = -kSH1; gz = 0.f; break;
    case 2: Y = kSH1 * z; gx = 0.f; gy = 0.f; gz = kSH1; break;
    case 3: Y = -kSH1 * x; gx = -kSH1; gy = 0.f; gz = 0.f; break;
    case 4: Y = kSH2a * x * y; gx = kSH2a * y; gy = kSH2a * x; gz = 0.f; break;
    case 5: Y = -kSH2a * y * z; gx = 0.f; gy = -kSH2a * z; gz = -kSH2a * y; break;
    case 6: Y = kSH2b * (2.f * zz - xx - yy); gx = -2.f * kSH2b * x; gy = -2.f * kSH2b * y; gz = 4.f * kSH2b * z; break;
    case 7: Y = -kSH2a * x * z; gx = -kSH2a * z; gy = 0.f; gz = -kSH2a * x; break;
    case 8: Y = kSH2c * (xx - yy); gx = 2.f * kSH2c * x; gy = -2.f * kSH2c * y; gz = 0.f; break;
    case 9: Y = -kSH3a * y * (3.f * xx - yy); gx = -6.f * kSH3a * x * y; gy = -kSH3a * (3.f * xx - 3.f * yy); gz = 0.f; break;
    case 10: Y = kSH3b * x * y * z; gx = kSH3b * y * z; gy = kSH3b * x * z; gz = kSH3b * x * y; break;
    case 11:
      Y = -kSH3c * y * (4.f * zz - xx - yy);
      gx = 2.f * kSH3c * x * y; gy = -kSH3c * (4.f * zz - xx - 3.f * yy); gz = -8.f * kSH3c * y * z;
      break;
    case 12:
      Y = kSH3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
      gx = -6.f * kSH3d * x * z; gy = -6.f * kSH3d * y * z; gz = kSH3d * (6.f * zz - 3.f * xx - 3.f * yy);
      break;
    case 13:
      Y = -kSH3c * x * (4.f * zz - xx - yy);
      gx = -kSH3c * (4.f * zz - 3.f * xx - yy); gy = 2.f * kSH3c * x * y; gz = -8.f * kSH3c * x * z;
      break;
    case 14: Y = kSH3e * z * (xx - yy); gx = 2.f * kSH3e * x * z; gy = -2.f * kSH3e * y * z; gz = kSH3e * (xx - yy); break;
    default: Y = -kSH3a * x * (xx - 3.f * yy); gx = -kSH3a * (3.f * xx - 3.f * yy); gy = 6.f * kSH3a * x * y; gz = 0.f; break;
  }
}

struct AdamArgs {
  float* params;
  float* m;
  float* v;
  float* grads_out;
  int stride;
  int adam;
  float b1, b2, eps, ssc, bc2s;
  float lr[6];
};

template <int N>
__device__ __forceinline__ void apply_rows_mv(const AdamArgs& A, int c0, const int* grp, int i, const float* g,
                                              const float* pcur, const float* m, const float* v);

// Adam (or gradient write) for n consecutive component rows c0..c0+n-1 of Gaussian i, with
// every load issued before the first store so the rows stream concurrently.
template <int N>
__device__ __forceinline__ void apply_rows(const AdamArgs& A, int c0, const int* grp, int i, const float* g,
                                           const float* pcur) {
  if (A.adam == 2) return;  // timing run of the autotuner: gradients computed, nothing written
  if (!A.adam) {
#pragma unroll
    for (int r = 0; r < N; ++r) A.grads_out[(long long)(c0 + r) * A.stride + i] = g[r];
    return;
  }
  float m[N], v[N];
#pragma unroll
  for (int r = 0; r < N; ++r) {
    const long long k = (long long)(c0 + r) * A.stride + i;
    m[r] = A.m[k];
    v[r] = A.v[k];
  }
  apply_rows_mv<N>(A, c0, grp, i, g, pcur, m, v);
}

// The update of apply_rows with the rows' moments already loaded (m, v).
template <int N>
__device__ __forceinline__ void apply_rows_mv(const AdamArgs& A, int c0, const int* grp, int i, const float* g,
                                              const float* pcur, const float* m, const float* v) {
  const float ibc2s = 1.f / A.bc2s;
#pragma unroll
  for (int r = 0; r < N; ++r) {
    const long long k = (long long)(c0 + r) * A.stride + i;
    const float mm = A.b1 * m[r] + (1.f - A.b1) * g[r];
    const float vv = A.b2 * v[r] + (1.f - A.b2) * g[r] * g[r];
    A.m[k] = mm;
    A.v[k] = vv;
    // lr m_hat / (sqrt(v_hat) + eps) with a 2-ulp divide (the IEEE divide and sqrt sequences cost
    // more than the whole rest of the update)
    A.params[k] = pcur[r] - __fdividef((A.lr[grp[r]] * A.ssc) * mm, __fsqrt_rn(vv) * ibc2s + A.eps);
  }
}

// L2 prefetch of rows c0 .. c0 + nrows - 1 of Gaussian i (the parameters too if pmv), so that their
// DRAM reads are under way while the thread works on the rows before them.  Holds no register.
__device__ __forceinline__ void l2_prefetch(const float* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }
__device__ __forceinline__ void l2_prefetch_rows(const AdamArgs& A, int c0, int nrows, int i, bool pmv) {
  for (int r = 0; r < nrows; ++r) {
    const long long k = (long long)(c0 + r) * A.stride + i;
    if (pmv) l2_prefetch(A.params + k);
    l2_prefetch(A.m + k);
    l2_prefetch(A.v + k);
  }
}

// Four SH coefficients (12 rows) K0..K0+3: gradient sum over the visible views, the direction
// gradient they feed, and the update.
template <int K0, int MAXV>
__device__ __forceinline__ void sh_group(const AdamArgs& A, int i, int nvis, unsigned vmask, float (&vdir)[MAXV][3],
                                         float (&vcol)[MAXV][3], float (&vdd)[MAXV][3]) {
  constexpr bool kSmall = MAXV <= 4;
  if (A.adam == 1) {  // the next group's rows (after the last group, the mean's moments)
    if (K0 < 12) l2_prefetch_rows(A, 11 + 3 * (K0 + 4), 12, i, true);
    else l2_prefetch_rows(A, 0, 3, i, false);
  }
  // the group's parameter rows and (for Adam) their moments, all loads issued at once
  float p[12], m[12], v[12];
#pragma unroll
  for (int r = 0; r < 12; ++r) {
    const long long k = (long long)(11 + 3 * K0 + r) * A.stride + i;
    p[r] = A.params[k];
    m[r] = A.adam == 1 ? A.m[k] : 0.f;
    v[r] = A.adam == 1 ? A.v[k] : 0.f;
  }
  float g[12];
#pragma unroll
  for (int r = 0; r < 12; ++r) g[r] = 0.f;
#pragma unroll(kSmall ? MAXV : 1)
  for (int j = 0; j < (kSmall ? MAXV : nvis); ++j) {
    if (kSmall && !((vmask >> j) & 1u)) continue;
    const float x = vdir[j][0], y = vdir[j][1], z = vdir[j][2];
    const float c0 = vcol[j][0], c1 = vcol[j][1], c2 = vcol[j][2];
    float Y[4], gx[4], gy[4], gz[4];
    sh_term<K0 + 0>(x, y, z, Y[0], gx[0], gy[0], gz[0]);
    sh_term<K0 + 1>(x, y, z, Y[1], gx[1], gy[1], gz[1]);
    sh_term<K0 + 2>(x, y, z, Y[2], gx[2], gy[2], gz[2]);
    sh_term<K0 + 3>(x, y, z, Y[3], gx[3], gy[3], gz[3]);
    float ddx = 0.f, ddy = 0.f, ddz = 0.f;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      g[3 * kk + 0] += Y[kk] * c0;
      g[3 * kk + 1] += Y[kk] * c1;
      g[3 * kk + 2] += Y[kk] * c2;
      const float w = p[3 * kk] * c0 + p[3 * kk + 1] * c1 + p[3 * kk + 2] * c2;
      ddx += gx[kk] * w;
      ddy += gy[kk] * w;
      ddz += gz[kk] * w;
    }
    vdd[j][0] += ddx;
    vdd[j][1] += ddy;
    vdd[j][2] += ddz;
  }
  int grp[12];
#pragma unroll
  for (int r = 0; r < 12; ++r) grp[r] = (K0 == 0 && r < 3) ? 4 : 5;
  if (A.adam == 1) apply_rows_mv<12>(A, 11 + 3 * K0, grp, i, g, p, m, v);
  else apply_rows<12>(A, 11 + 3 * K0, grp, i, g, p);
}

// A warp whose 32 Gaussians had no instance in any view of the step (none past n): their gradients
// are all zero.  In the streaming fields Gaussians are appended per arriving image, so a view's
// visible set comes in long runs and most warps outside it qualify.
__device__ __forceinline__ bool warp_unseen(const unsigned* __restrict__ count, int n_views, int stride, int i, int n) {
  bool seen = i >= n;
  for (int v = 0; v < n_views && !seen; ++v) seen = count[(long long)v * stride + i] != 0u;
  return __all_sync(0xffffffffu, !seen);
}

// Adam with a zero gradient (or the zero gradient itself) over the 59 rows of such a warp's Gaussians
// i0 .. i0 + 31, in 16-byte accesses: eight lanes per 32-Gaussian row segment, four rows per pass.
// The update is the expression apply_rows_mv evaluates, with g = 0, so the result is the same bits.
__device__ __forceinline__ void unseen_rows(const AdamArgs& A, int i0, int lane) {
  if (A.adam == 2) return;
  const int sub = lane >> 3, c4 = (lane & 7) * 4;
  if (!A.adam) {
    for (int r = sub; r < kNumParams; r += 4)
      *reinterpret_cast<float4*>(A.grads_out + (long long)r * A.stride + i0 + c4) = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  const float ibc2s = 1.f / A.bc2s;
  const float g = 0.f;
  // rows sub, sub + 4, ..., five at a time with every load issued before the first store (the
  // stores could alias the next rows' loads as far as the compiler knows, so it would not hoist them)
  constexpr int kU = 5;
  for (int r0 = sub; r0 < kNumParams; r0 += 4 * kU) {
    float4 p[kU], m[kU], v[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int r = r0 + 4 * u;
      if (r < kNumParams) {
        const long long k = (long long)r * A.stride + i0 + c4;
        p[u] = *reinterpret_cast<const float4*>(A.params + k);
        m[u] = *reinterpret_cast<const float4*>(A.m + k);
        v[u] = *reinterpret_cast<const float4*>(A.v + k);
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int r = r0 + 4 * u;
      if (r >= kNumParams) continue;
      // the row's group rate, selected among registers (a computed index would put A.lr in local memory)
      const float lr = r < 3 ? A.lr[0] : (r < 6 ? A.lr[1] : (r < 10 ? A.lr[2] : (r < 11 ? A.lr[3] : (r < 14 ? A.lr[4] : A.lr[5]))));
      auto upd = [&](float& pp, float& mm, float& vv) {
        mm = A.b1 * mm + (1.f - A.b1) * g;
        vv = A.b2 * vv + (1.f - A.b2) * g * g;
        pp = pp - __fdividef((lr * A.ssc) * mm, __fsqrt_rn(vv) * ibc2s + A.eps);
      };
      upd(p[u].x, m[u].x, v[u].x);
      upd(p[u].y, m[u].y, v[u].y);
      upd(p[u].z, m[u].z, v[u].z);
      upd(p[u].w, m[u].w, v[u].w);
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int r = r0 + 4 * u;
      if (r >= kNumParams) continue;
      const long long k = (long long)r * A.stride + i0 + c4;
      *reinterpret_cast<float4*>(A.m + k) = m[u];
      *reinterpret_cast<float4*>(A.v + k) = v[u];
      *reinterpret_cast<float4*>(A.params + k) = p[u];
    }
  }
}

// K9a: per record (view, Gaussian), the sum of its instances' nine gradients (a reduce by key over
// the instances, whose records are non-decreasing in emission order).  Warps take 32-instance
// chunks (coalesced) and sum each record's run inside the chunk by a segmented scan over the
// lanes.  A run that lies inside one chunk is the record's sum; a run cut by a chunk boundary is
// a partial: the chunk's first run (record started earlier) goes to head[chunk], its last run
// (record continues) to tail[chunk]; k_inst_carry adds, per record that spans chunks, its tail
// partial, the middle chunks' heads and the last chunk's head, in chunk order (deterministic).
// Output: g2s, 9 planes of n_rec floats; grad2d (nullable) the same as 9 floats per record.
__global__ void __launch_bounds__(256) k_inst_reduce(const unsigned* __restrict__ inst_rec,
                                                     const float4* __restrict__ ginst,
                                                     const unsigned* __restrict__ count,
                                                     const unsigned* __restrict__ offsets, long long n_rec,
                                                     const Control* __restrict__ ctl, float* __restrict__ g2s,
                                                     float* __restrict__ grad2d, float* __restrict__ head,
                                                     float* __restrict__ tail) {
  dep_wait();
  dep_release();
  if (ctl->overflow) return;
  const int lane = threadIdx.x & 31;
  const unsigned long long M = ctl->m_total;
  const unsigned long long n_chunks = (M + 31) >> 5;
  const unsigned long long w0 = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long n_warps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  for (unsigned long long c = w0; c < n_chunks; c += n_warps) {
    const unsigned long long e = (c << 5) + lane;
    const bool valid = e < M;
    const unsigned r = valid ? inst_rec[e] : 0xffffffffu;
    float x[9];
    if (valid) {
      const float4 a = ginst[3ull * e], b = ginst[3ull * e + 1], cc = ginst[3ull * e + 2];
      x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
      x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
      x[8] = cc.x;
    } else {
#pragma unroll
      for (int k = 0; k < 9; ++k) x[k] = 0.f;
    }
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned rd = __shfl_up_sync(0xffffffffu, r, d);
      const bool same = lane >= d && rd == r;
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const float y = __shfl_up_sync(0xffffffffu, x[k], d);
        if (same) x[k] += y;
      }
    }
    const unsigned r_next = __shfl_down_sync(0xffffffffu, r, 1);
    if (valid && (lane == 31 || r_next != r)) {
      const unsigned long long off = offsets[r], cnt = count[r];
      const bool begins = off >= (c << 5);
      const bool ends = off + cnt - 1 == e;
      if (begins && ends) {
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          g2s[k * n_rec + r] = x[k];
          if (grad2d) grad2d[9ull * r + k] = x[k];
        }
      } else {
        float* dst = (begins ? tail : head) + 9 * c;
#pragma unroll
        for (int k = 0; k < 9; ++k) dst[k] = x[k];
      }
    }
  }
}

__global__ void __launch_bounds__(256) k_inst_carry(const unsigned* __restrict__ count,
                                                    const unsigned* __restrict__ offsets, long long n_rec,
                                                    const Control* __restrict__ ctl, const float* __restrict__ head,
                                                    const float* __restrict__ tail, float* __restrict__ g2s,
                                                    float* __restrict__ grad2d) {
  dep_wait();
  dep_release();
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (ctl->overflow || r >= n_rec) return;
  const unsigned long long cnt = count[r];
  if (!cnt) return;
  const unsigned long long off = offsets[r];
  const unsigned long long c0 = off >> 5, c1 = (off + cnt - 1) >> 5;
  if (c0 == c1) return;  // summed inside one chunk
  float x[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) x[k] = tail[9 * c0 + k];
  for (unsigned long long c = c0 + 1; c <= c1; ++c)
#pragma unroll
    for (int k = 0; k < 9; ++k) x[k] += head[9 * c + k];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    g2s[k * n_rec + r] = x[k];
    if (grad2d) grad2d[9ull * r + k] = x[k];
  }
}

// Chain rule of one view's 2D gradient (d mean2d, d pre-scaled conic; g2[0..4]) back to the mean,
// the log-scales and the quaternion (accumulated into gmu, gls, gq).
__device__ __forceinline__ void geo_backward(const ViewDev& V, const Geo& g, const float g2[9], float gmu[3],
                                             float gls[3], float gq[4]) {
  // Pre-scaled conic gradient back to the conic (a, b, c): power = -a/2 dx^2 - b dx dy - c/2 dy^2.
  const float dA = g2[2], dB = g2[3], dC = g2[4];
  const float A_ = g.cov[0], B_ = g.cov[1], C_ = g.cov[2], det = g.det;
  const float id = 1.f / det, id2 = id * id;
  const float da = dA * (-C_ * C_ * id2) + dB * (B_ * C_ * id2) + dC * (id - A_ * C_ * id2);
  const float db = dA * (2.f * B_ * C_ * id2) + dB * (-id - 2.f * B_ * B_ * id2) + dC * (2.f * A_ * B_ * id2);
  const float dc = dA * (id - A_ * C_ * id2) + dB * (A_ * B_ * id2) + dC * (-A_ * A_ * id2);

  // (a, b, c) = entries of Tm Sigma Tm^T
  const float* T0 = g.Tm;
  const float* T1 = g.Tm + 3;
  const float S[9] = {g.Sig[0], g.Sig[1], g.Sig[2], g.Sig[1], g.Sig[3], g.Sig[4], g.Sig[2], g.Sig[4], g.Sig[5]};
  float Gs[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      Gs[3 * r + c] = da * T0[r] * T0[c] + 0.5f * db * (T0[r] * T1[c] + T1[r] * T0[c]) + dc * T1[r] * T1[c];
  float dT0[3], dT1[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const float s0 = S[3 * r] * T0[0] + S[3 * r + 1] * T0[1] + S[3 * r + 2] * T0[2];
    const float s1 = S[3 * r] * T1[0] + S[3 * r + 1] * T1[1] + S[3 * r + 2] * T1[2];
    dT0[r] = 2.f * da * s0 + db * s1;
    dT1[r] = 2.f * dc * s1 + db * s0;
  }
  const float dJ00 = dT0[0] * V.R[0] + dT0[1] * V.R[1] + dT0[2] * V.R[2];
  const float dJ02 = dT0[0] * V.R[6] + dT0[1] * V.R[7] + dT0[2] * V.R[8];
  const float dJ11 = dT1[0] * V.R[3] + dT1[1] * V.R[4] + dT1[2] * V.R[5];
  const float dJ12 = dT1[0] * V.R[6] + dT1[1] * V.R[7] + dT1[2] * V.R[8];
  const float px = g.p[0], py = g.p[1], pz = g.p[2];
  const float iz = 1.f / pz, iz2 = iz * iz, iz3 = iz2 * iz;
  float dp[3] = {0.f, 0.f, 0.f};
  dp[2] += dJ00 * (-V.fx * iz2) + dJ11 * (-V.fy * iz2);
  if (g.xin) {
    dp[0] += dJ02 * (-V.fx * iz2);
    dp[2] += dJ02 * (2.f * V.fx * px * iz3);
  } else {
    dp[2] += dJ02 * (V.fx * g.txz * iz2);
  }
  if (g.yin) {
    dp[1] += dJ12 * (-V.fy * iz2);
    dp[2] += dJ12 * (2.f * V.fy * py * iz3);
  } else {
    dp[2] += dJ12 * (V.fy * g.tyz * iz2);
  }
  dp[0] += g2[0] * V.fx * iz;
  dp[2] += g2[0] * (-V.fx * px * iz2);
  dp[1] += g2[1] * V.fy * iz;
  dp[2] += g2[1] * (-V.fy * py * iz2);
#pragma unroll
  for (int a = 0; a < 3; ++a) gmu[a] += V.R[a] * dp[0] + V.R[3 + a] * dp[1] + V.R[6 + a] * dp[2];

  float dM[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      dM[3 * r + c] = 2.f * (Gs[3 * r] * g.M[c] + Gs[3 * r + 1] * g.M[3 + c] + Gs[3 * r + 2] * g.M[6 + c]);
  float dRq[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) dRq[3 * r + c] = dM[3 * r + c] * g.s[c];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float ds = dM[c] * g.Rq[c] + dM[3 + c] * g.Rq[3 + c] + dM[6 + c] * g.Rq[6 + c];
    gls[c] += ds * g.s[c];
  }
  const float w = g.qn[0], x = g.qn[1], y = g.qn[2], z = g.qn[3];
  float dqn[4];
  dqn[0] = 2.f * (-z * dRq[1] + y * dRq[2] + z * dRq[3] - x * dRq[5] - y * dRq[6] + x * dRq[7]);
  dqn[1] = 2.f * (y * dRq[1] + z * dRq[2] + y * dRq[3] - 2.f * x * dRq[4] - w * dRq[5] + z * dRq[6] +
                  w * dRq[7] - 2.f * x * dRq[8]);
  dqn[2] = 2.f * (-2.f * y * dRq[0] + x * dRq[1] + w * dRq[2] + x * dRq[3] + z * dRq[5] - w * dRq[6] +
                  z * dRq[7] - 2.f * y * dRq[8]);
  dqn[3] = 2.f * (-2.f * z * dRq[0] - w * dRq[1] + x * dRq[2] + w * dRq[3] - 2.f * z * dRq[4] + y * dRq[5] +
                  x * dRq[6] + y * dRq[7]);
  const float qd = g.qn[0] * dqn[0] + g.qn[1] * dqn[1] + g.qn[2] * dqn[2] + g.qn[3] * dqn[3];
#pragma unroll
  for (int k = 0; k < 4; ++k) gq[k] += (dqn[k] - g.qn[k] * qd) * g.qinv;
}

template <int MAXV>
__global__ void __launch_bounds__(256, 2) k_project_backward(
    float* __restrict__ params, int stride, const StepParams* __restrict__ sp,
    const ViewDev* __restrict__ views, int n_views, const unsigned* __restrict__ count,
    const unsigned char* __restrict__ clampbits, const float* __restrict__ g2s, const Control* __restrict__ ctl,
    float* __restrict__ grads_out, float* __restrict__ adam_m, float* __restrict__ adam_v, int vec_ok) {
  dep_wait();
  dep_release();
  const long long n_rec = (long long)n_views * stride;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (ctl->overflow) return;  // the step was skipped; the host re-runs it with more capacity
  const bool unseen = vec_ok && warp_unseen(count, n_views, stride, i, sp->n);
  if (i >= sp->n) return;

  AdamArgs A;
  A.params = params;
  A.m = adam_m;
  A.v = adam_v;
  A.grads_out = grads_out;
  A.stride = stride;
  A.adam = sp->adam;
  A.b1 = sp->beta1;
  A.b2 = sp->beta2;
  A.eps = sp->eps;
  A.ssc = sp->step_size_scale;
  A.bc2s = sp->bc2_sqrt;
#pragma unroll
  for (int k = 0; k < 6; ++k) A.lr[k] = sp->lr[k];
  if (unseen) {  // sparse Adam leaves such Gaussians as they are
    if (!(A.adam == 1 && sp->sparse)) unseen_rows(A, i - (int)(threadIdx.x & 31), threadIdx.x & 31);
    return;
  }

  float mu[3], ls[3], q[4];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    mu[k] = params[k * stride + i];
    ls[k] = params[(3 + k) * stride + i];
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) q[k] = params[(6 + k) * stride + i];
  const float logit = params[10 * stride + i];
  if (A.adam == 1 && !sp->sparse) l2_prefetch_rows(A, 3, 8, i, false);  // moments of the rows after the chain

  float gmu[3] = {0.f, 0.f, 0.f}, gls[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f};
  float gop = 0.f;
  // per visible view: direction, masked colour gradient, 1/|d|, and the direction gradient.
  // Up to 4 views these live in registers (slot = view, vmask = visible slots); beyond that in a
  // compacted local array (slot = nvis).
  constexpr bool kSmall = MAXV <= 4;
  float vdir[MAXV][3], vcol[MAXV][3], vinv[MAXV], vdd[MAXV][3];
  int nvis = 0;
  unsigned vmask = 0u;
  float o = 0.f;
  bool have_o = false;
#pragma unroll(kSmall ? MAXV : 1)
  for (int v = 0; v < (kSmall ? MAXV : n_views); ++v) {
    if (kSmall && v >= n_views) break;
    const long long rec = (long long)v * stride + i;
    const unsigned cnt = count[rec];
    // the record's sums are loaded with its count (read but unused for a record without instances)
    float g2[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) g2[k] = g2s[k * n_rec + rec];
    if (cnt == 0u) continue;
    const int slot = kSmall ? v : nvis;
    const ViewDev& V = views[v];
    Geo g;
    if (!geo_forward(V, mu, ls, q, g)) continue;

    if (!have_o) {
      o = 1.f / (1.f + __expf(-logit));
      have_o = true;
    }
    gop += g2[5] * o * (1.f - o);

    // view direction and the colour gradient of the unclamped channels, kept for the SH rows
    const float d0 = mu[0] - V.campos[0], d1 = mu[1] - V.campos[1], d2 = mu[2] - V.campos[2];
    const float dinv = rsqrtf(d0 * d0 + d1 * d1 + d2 * d2);
    const unsigned cb = clampbits[rec];
    vdir[slot][0] = d0 * dinv;
    vdir[slot][1] = d1 * dinv;
    vdir[slot][2] = d2 * dinv;
    vcol[slot][0] = (cb & 1u) ? 0.f : g2[6];
    vcol[slot][1] = (cb & 2u) ? 0.f : g2[7];
    vcol[slot][2] = (cb & 4u) ? 0.f : g2[8];
    vinv[slot] = dinv;
    vdd[slot][0] = vdd[slot][1] = vdd[slot][2] = 0.f;
    vmask |= 1u << slot;
    ++nvis;

    geo_backward(V, g, g2, gmu, gls, gq);
  }
  if (nvis == 0 && A.adam == 1 && sp->sparse) return;  // sparse Adam: not seen by the step
  if (A.adam == 1) l2_prefetch_rows(A, 11, 12, i, true);  // the first SH group

  // log-scales, quaternion and opacity are complete here: update them before the SH rows so their
  // gradients and values are not held through them (only the mean takes the direction gradient)
  {
    const float gg[8] = {gls[0], gls[1], gls[2], gq[0], gq[1], gq[2], gq[3], gop};
    const float pc[8] = {ls[0], ls[1], ls[2], q[0], q[1], q[2], q[3], logit};
    const int grp[8] = {1, 1, 1, 2, 2, 2, 2, 3};
    apply_rows<8>(A, 3, grp, i, gg, pc);
  }

  // SH rows, four coefficients (12 rows) at a time; accumulates the direction gradient.
  sh_group<0>(A, i, nvis, vmask, vdir, vcol, vdd);
  sh_group<4>(A, i, nvis, vmask, vdir, vcol, vdd);
  sh_group<8>(A, i, nvis, vmask, vdir, vcol, vdd);
  sh_group<12>(A, i, nvis, vmask, vdir, vcol, vdd);

  // direction = (mu - c)/|mu - c|  ->  mean
#pragma unroll(kSmall ? MAXV : 1)
  for (int j = 0; j < (kSmall ? MAXV : nvis); ++j) {
    if (kSmall && !((vmask >> j) & 1u)) continue;
    const float dd = vdir[j][0] * vdd[j][0] + vdir[j][1] * vdd[j][1] + vdir[j][2] * vdd[j][2];
#pragma unroll
    for (int a = 0; a < 3; ++a) gmu[a] += (vdd[j][a] - vdir[j][a] * dd) * vinv[j];
  }
  const int grp[3] = {0, 0, 0};
  apply_rows<3>(A, 0, grp, i, gmu, mu);
}

// One SH coefficient K of one view: its three gradient rows (colour gradient x Y_K(dir)) into
// shared memory, and its share of the direction gradient (grad Y_K . (coefficient . colour grad)).
template <int K>
__device__ __forceinline__ void sh_view(const float* __restrict__ params, int stride, int i, float x, float y, float z,
                                        const float c[3], float* __restrict__ gsh, float dd[3]) {
  float Y, gx, gy, gz;
  sh_term<K>(x, y, z, Y, gx, gy, gz);
  float w = 0.f;
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    gsh[(3 * K + ch) * 256] += Y * c[ch];
    w += __ldg(params + (long long)(11 + 3 * K + ch) * stride + i) * c[ch];
  }
  dd[0] += gx * w;
  dd[1] += gy * w;
  dd[2] += gz * w;
}

template <int K>
__device__ __forceinline__ void sh_views(const float* __restrict__ params, int stride, int i, float x, float y, float z,
                                         const float c[3], float* __restrict__ gsh, float dd[3]) {
  sh_view<K>(params, stride, i, x, y, z, c, gsh, dd);
  if constexpr (K + 1 < 16) sh_views<K + 1>(params, stride, i, x, y, z, c, gsh, dd);
}

// K9 + K10 for steps over several views: the views are taken one at a time, each one's SH rows
// summed straight into per-thread shared-memory accumulators (48 rows) and its direction gradient
// folded into the mean at once, so no per-view state is kept in registers or local memory.
__global__ void __launch_bounds__(256, 2) k_project_backward_views(
    float* __restrict__ params, int stride, const StepParams* __restrict__ sp,
    const ViewDev* __restrict__ views, int n_views, const unsigned* __restrict__ count,
    const unsigned char* __restrict__ clampbits, const float* __restrict__ g2s, const Control* __restrict__ ctl,
    float* __restrict__ grads_out, float* __restrict__ adam_m, float* __restrict__ adam_v, int vec_ok) {
  dep_wait();
  dep_release();
  const long long n_rec = (long long)n_views * stride;
  __shared__ float s_gsh[48 * 256];  // [row][thread]
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (ctl->overflow) return;
  const bool unseen = vec_ok && warp_unseen(count, n_views, stride, i, sp->n);
  if (i >= sp->n) return;
  float* gsh = s_gsh + threadIdx.x;

  AdamArgs A;
  A.params = params;
  A.m = adam_m;
  A.v = adam_v;
  A.grads_out = grads_out;
  A.stride = stride;
  A.adam = sp->adam;
  A.b1 = sp->beta1;
  A.b2 = sp->beta2;
  A.eps = sp->eps;
  A.ssc = sp->step_size_scale;
  A.bc2s = sp->bc2_sqrt;
#pragma unroll
  for (int k = 0; k < 6; ++k) A.lr[k] = sp->lr[k];
  if (unseen) {  // sparse Adam leaves such Gaussians as they are
    if (!(A.adam == 1 && sp->sparse)) unseen_rows(A, i - (int)(threadIdx.x & 31), threadIdx.x & 31);
    return;
  }
#pragma unroll
  for (int r = 0; r < 48; ++r) gsh[r * 256] = 0.f;

  float mu[3], ls[3], q[4];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    mu[k] = params[k * stride + i];
    ls[k] = params[(3 + k) * stride + i];
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) q[k] = params[(6 + k) * stride + i];
  const float logit = params[10 * stride + i];
  const float o = 1.f / (1.f + __expf(-logit));
  if (A.adam == 1 && !sp->sparse) l2_prefetch_rows(A, 0, 11, i, false);  // moments of the geometry rows

  float gmu[3] = {0.f, 0.f, 0.f}, gls[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f};
  float gop = 0.f;
  bool seen = false;
  for (int v = 0; v < n_views; ++v) {
    const long long rec = (long long)v * stride + i;
    const unsigned cnt = count[rec];
    if (cnt == 0u) continue;
    seen = true;
    float g2[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) g2[k] = g2s[k * n_rec + rec];
    const ViewDev& V = views[v];
    // colour: SH rows and the direction gradient of this view
    const float d0 = mu[0] - V.campos[0], d1 = mu[1] - V.campos[1], d2 = mu[2] - V.campos[2];
    const float dinv = rsqrtf(d0 * d0 + d1 * d1 + d2 * d2);
    const float x = d0 * dinv, y = d1 * dinv, z = d2 * dinv;
    const unsigned cb = clampbits[rec];
    const float col[3] = {(cb & 1u) ? 0.f : g2[6], (cb & 2u) ? 0.f : g2[7], (cb & 4u) ? 0.f : g2[8]};
    float dd[3] = {0.f, 0.f, 0.f};
    sh_views<0>(params, stride, i, x, y, z, col, gsh, dd);
    const float ddot = x * dd[0] + y * dd[1] + z * dd[2];
    gmu[0] += (dd[0] - x * ddot) * dinv;
    gmu[1] += (dd[1] - y * ddot) * dinv;
    gmu[2] += (dd[2] - z * ddot) * dinv;
    // geometry
    Geo g;
    if (!geo_forward(V, mu, ls, q, g)) continue;
    gop += g2[5] * o * (1.f - o);
    geo_backward(V, g, g2, gmu, gls, gq);
  }
  if (!seen && A.adam == 1 && sp->sparse) return;  // sparse Adam: not seen by the step
  if (A.adam == 1) l2_prefetch_rows(A, 11, 12, i, false);  // the first SH group's moments
  const float gg[11] = {gmu[0], gmu[1], gmu[2], gls[0], gls[1], gls[2], gq[0], gq[1], gq[2], gq[3], gop};
  const float pc[11] = {mu[0], mu[1], mu[2], ls[0], ls[1], ls[2], q[0], q[1], q[2], q[3], logit};
  const int grp[11] = {0, 0, 0, 1, 1, 1, 2, 2, 2, 2, 3};
  apply_rows<11>(A, 0, grp, i, gg, pc);
#pragma unroll
  for (int g0 = 0; g0 < 48; g0 += 12) {
    if (A.adam == 1 && g0 + 12 < 48) l2_prefetch_rows(A, 11 + g0 + 12, 12, i, false);  // the next group's
    float p12[12], g12[12];
    int grp12[12];
#pragma unroll
    for (int r = 0; r < 12; ++r) {
      p12[r] = params[(long long)(11 + g0 + r) * stride + i];
      g12[r] = gsh[(g0 + r) * 256];
      grp12[r] = (g0 + r) < 3 ? 4 : 5;
    }
    apply_rows<12>(A, 11 + g0, grp12, i, g12, p12);
  }
}

// Plain Adam over a gradient buffer (parity of K10 on its own; dense, vectorised by 4).
__global__ void __launch_bounds__(256) k_adam(float* __restrict__ params, const float* __restrict__ grads,
                                              float* __restrict__ m, float* __restrict__ v, int n, int stride,
                                              const StepParams* __restrict__ sp) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // float4 index
  const long long per_row = stride / 4;
  if (q >= per_row * kNumParams) return;
  const int c = (int)(q / per_row);
  const int i0 = (int)(q - (long long)c * per_row) * 4;
  if (i0 >= n) return;
  const int grp = c < 3 ? 0 : (c < 6 ? 1 : (c < 10 ? 2 : (c < 11 ? 3 : (c < 14 ? 4 : 5))));
  const float lr = sp->lr[grp] * sp->step_size_scale;
  const float b1 = sp->beta1, b2 = sp->beta2, eps = sp->eps, bc2s = sp->bc2_sqrt;
  float4 p = reinterpret_cast<float4*>(params)[q];
  const float4 g = reinterpret_cast<const float4*>(grads)[q];
  float4 mm = reinterpret_cast<float4*>(m)[q];
  float4 vv = reinterpret_cast<float4*>(v)[q];
  auto upd = [&](float& pp, float gg, float& m1, float& v1, int lane) {
    if (i0 + lane >= n) return;
    m1 = b1 * m1 + (1.f - b1) * gg;
    v1 = b2 * v1 + (1.f - b2) * gg * gg;
    pp -= lr * m1 / (sqrtf(v1) / bc2s + eps);
  };
  upd(p.x, g.x, mm.x, vv.x, 0);
  upd(p.y, g.y, mm.y, vv.y, 1);
  upd(p.z, g.z, mm.z, vv.z, 2);
  upd(p.w, g.w, mm.w, vv.w, 3);
  reinterpret_cast<float4*>(params)[q] = p;
  reinterpret_cast<float4*>(m)[q] = mm;
  reinterpret_cast<float4*>(v)[q] = vv;
}

void launch_project(const float* params, int stride, int n_views, const StepParams* sp, const ViewDev* views,
                    const ProjBuffers& out, cudaStream_t s) {
  dim3 grid((stride + 255) / 256, n_views);
  launch_dep(k_project, dim3(grid), dim3(256), 0, s, params, stride, sp, views, out);
}

void launch_project_backward(float* params, int stride, int n_views, const StepParams* sp, const ViewDev* views,
                             const ProjBuffers& pb, const float4* ginst, const unsigned* inst_rec, float* carry,
                             long long m_cap, float* g2s, const Control* ctl, float* grads_out, float* m, float* v,
                             float* grad2d_out, int num_sms, cudaStream_t s) {
  const long long n_rec = (long long)n_views * stride;
  if (n_rec > 0) {
    float* head = carry;
    float* tail = carry + 9 * ((m_cap + 31) / 32 + 1);
    launch_dep(k_inst_reduce, dim3((unsigned)(num_sms * 8)), dim3(256), 0, s, inst_rec, ginst, pb.count, pb.offsets,
        n_rec, ctl, g2s, grad2d_out, head, tail);
    launch_dep(k_inst_carry, dim3((unsigned)((n_rec + 255) / 256)), dim3(256), 0, s, pb.count, pb.offsets, n_rec, ctl,
        head, tail, g2s, grad2d_out);
  }
  const unsigned grid = (unsigned)((stride + 255) / 256);
  // 16-byte row accesses for warps no view saw: rows of a multiple-of-4 stride from 16-byte aligned bases
  const auto al16 = [](const void* p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  const int vec_ok = (stride % 4 == 0) && al16(params) && al16(m) && al16(v) && al16(grads_out);
  if (n_views <= 1)
    launch_dep(k_project_backward<1>, dim3(grid), dim3(256), 0, s, params, stride, sp, views, n_views, pb.count,
        pb.clamp, g2s, ctl, grads_out, m, v, vec_ok);
  else
    launch_dep(k_project_backward_views, dim3(grid), dim3(256), 0, s, params, stride, sp, views, n_views, pb.count,
        pb.clamp, g2s, ctl, grads_out, m, v, vec_ok);
}

void launch_adam(float* params, const float* grads, float* m, float* v, int n, int stride, const StepParams* sp,
                 cudaStream_t s) {
  const long long quads = (long long)(stride / 4) * kNumParams;
  k_adam<<<(unsigned)((quads + 255) / 256), 256, 0, s>>>(params, grads, m, v, n, stride, sp);
}

}  // namespace gs
