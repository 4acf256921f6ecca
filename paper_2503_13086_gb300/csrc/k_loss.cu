// k_loss.cu -- K7: L = (1 - lambda) L1 + lambda (1 - SSIM) of Eq. 10 (its L1 and SSIM terms),
// and dL/d(render), sm_103a.
//
// SSIM uses the 11 x 11 Gaussian window (sigma 1.5) of 3DGS, zero padding and "same" output
// size, C1 = 0.01^2, C2 = 0.03^2, per colour channel; means run over 3 H W and, for a batch of
// views, the loss is the mean of the per-view losses.  The window is separable: each CTA stages
// a 32 x 16 output block plus a 5-pixel halo in shared memory, blurs rows then columns.
//   pass 1 (k_loss_forward): the five window moments -> SSIM map, the three partial derivatives
//          of SSIM with respect to (mu_x, E[x^2], E[xy]) per pixel, and per-CTA sums;
//   pass 2 (k_loss_backward): the same window applied to those partials (the window is
//          symmetric, so the adjoint of the blur is the blur) gives dL/dx.
// The last CTA of pass 1 reduces the per-CTA sums in a fixed order: the loss is deterministic.
#include "gs_device.cuh"
#include "gs_kernels.h"

namespace gs {

namespace {
constexpr int kBX = 32, kBY = 16, kR = 5;
constexpr int kSX = kBX + 2 * kR, kSY = kBY + 2 * kR;  // 42 x 26 staged block
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;

__device__ __forceinline__ void window(float w[11]) {
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 11; ++k) {
    const float d = (float)(k - kR);
    w[k] = expf(-d * d / (2.f * 1.5f * 1.5f));
    s += w[k];
  }
#pragma unroll
  for (int k = 0; k < 11; ++k) w[k] /= s;
}

__device__ __forceinline__ int view_of_block(const ViewDev* __restrict__ views, int n_views, long long b) {
  int v = 0;
  while (v + 1 < n_views && views[v + 1].loss_block_base <= b) ++v;
  return v;
}
}  // namespace

long long loss_blocks(int W, int H) { return (long long)((W + kBX - 1) / kBX) * ((H + kBY - 1) / kBY); }

__global__ void __launch_bounds__(256) k_loss_forward(const ViewDev* __restrict__ views, int n_views,
                                                      long long n_blocks, const float* __restrict__ image,
                                                      const StepParams* __restrict__ sp,
                                                      float* __restrict__ partials, double* __restrict__ block_sums,
                                                      Control* __restrict__ ctl) {
  __shared__ float sx[kSY][kSX], sy[kSY][kSX];
  __shared__ float hm[5][kSY][kBX];
  __shared__ double s_red[2][8];
  __shared__ bool s_last;
  if (ctl->overflow) return;
  float w[11];
  window(w);
  const long long b = blockIdx.x;
  const int v = view_of_block(views, n_views, b);
  const ViewDev& V = views[v];
  const int bxn = (V.W + kBX - 1) / kBX;
  const long long lb = b - V.loss_block_base;
  const int bx = (int)(lb % bxn), by = (int)(lb / bxn);
  const int ox = bx * kBX, oy = by * kBY;
  const long long HW = (long long)V.W * V.H;
  const float* X = image + 3 * V.pix_base;
  const float* Yt = V.target;
  float* P = partials + 9 * V.pix_base;
  double l1 = 0.0, ss = 0.0;
  for (int ch = 0; ch < 3; ++ch) {
    for (int k = threadIdx.x; k < kSX * kSY; k += blockDim.x) {
      const int r = k / kSX, c = k % kSX;
      const int gy = oy + r - kR, gx = ox + c - kR;
      const bool in = gx >= 0 && gx < V.W && gy >= 0 && gy < V.H;
      const long long pix = (long long)gy * V.W + gx;
      sx[r][c] = in ? X[ch * HW + pix] : 0.f;
      sy[r][c] = in ? Yt[ch * HW + pix] : 0.f;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kSY * kBX; k += blockDim.x) {
      const int r = k / kBX, c = k % kBX;
      float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f, m4 = 0.f;
#pragma unroll
      for (int t = 0; t < 11; ++t) {
        const float xv = sx[r][c + t], yv = sy[r][c + t];
        m0 += w[t] * xv;
        m1 += w[t] * yv;
        m2 += w[t] * xv * xv;
        m3 += w[t] * yv * yv;
        m4 += w[t] * xv * yv;
      }
      hm[0][r][c] = m0;
      hm[1][r][c] = m1;
      hm[2][r][c] = m2;
      hm[3][r][c] = m3;
      hm[4][r][c] = m4;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kBY * kBX; k += blockDim.x) {
      const int r = k / kBX, c = k % kBX;
      const int gy = oy + r, gx = ox + c;
      if (gx >= V.W || gy >= V.H) continue;
      float mx = 0.f, my = 0.f, exx = 0.f, eyy = 0.f, exy = 0.f;
#pragma unroll
      for (int t = 0; t < 11; ++t) {
        mx += w[t] * hm[0][r + t][c];
        my += w[t] * hm[1][r + t][c];
        exx += w[t] * hm[2][r + t][c];
        eyy += w[t] * hm[3][r + t][c];
        exy += w[t] * hm[4][r + t][c];
      }
      const float N1 = 2.f * mx * my + kC1, N2 = 2.f * (exy - mx * my) + kC2;
      const float D1 = mx * mx + my * my + kC1, D2 = (exx - mx * mx) + (eyy - my * my) + kC2;
      const float N = N1 * N2, D = D1 * D2;
      const float iD = 1.f / D;
      const float S = N * iD;
      ss += (double)S;
      const float dN = 2.f * my * N2 - 2.f * my * N1;
      const float dD = 2.f * mx * D2 - 2.f * mx * D1;
      const long long pix = (long long)gy * V.W + gx;
      P[(3 * ch + 0) * HW + pix] = (dN * D - N * dD) * iD * iD;  // dS/dmu_x
      P[(3 * ch + 1) * HW + pix] = -N * D1 * iD * iD;             // dS/dE[x^2]
      P[(3 * ch + 2) * HW + pix] = 2.f * N1 * iD;                 // dS/dE[xy]
      l1 += (double)fabsf(sx[r + kR][c + kR] - sy[r + kR][c + kR]);
    }
    __syncthreads();
  }
  // per-CTA sums (fixed-order tree), then the last CTA reduces all CTAs in index order
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    l1 += __shfl_down_sync(0xffffffffu, l1, o);
    ss += __shfl_down_sync(0xffffffffu, ss, o);
  }
  if ((threadIdx.x & 31) == 0) {
    s_red[0][threadIdx.x >> 5] = l1;
    s_red[1][threadIdx.x >> 5] = ss;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0;
    for (int k = 0; k < 8; ++k) {
      a += s_red[0][k];
      c += s_red[1][k];
    }
    block_sums[2 * b] = a;
    block_sums[2 * b + 1] = c;
    __threadfence();
    s_last = atomicAdd(&ctl->loss_done, 1u) == (unsigned)(n_blocks - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const double lam = (double)sp->lambda_ssim;
  double total = 0.0;
  for (int vv = 0; vv < n_views; ++vv) {
    const ViewDev& U = views[vv];
    const long long b0 = U.loss_block_base;
    const long long b1 = (vv + 1 < n_views) ? views[vv + 1].loss_block_base : n_blocks;
    double a = 0.0, c = 0.0;
    for (long long k = b0 + threadIdx.x; k < b1; k += blockDim.x) {
      a += ((volatile double*)block_sums)[2 * k];
      c += ((volatile double*)block_sums)[2 * k + 1];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      c += __shfl_down_sync(0xffffffffu, c, o);
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
      s_red[0][threadIdx.x >> 5] = a;
      s_red[1][threadIdx.x >> 5] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double A = 0.0, Cs = 0.0;
      for (int k = 0; k < 8; ++k) {
        A += s_red[0][k];
        Cs += s_red[1][k];
      }
      const double cntp = 3.0 * (double)U.W * (double)U.H;
      const double lv = (1.0 - lam) * (A / cntp) + lam * (1.0 - Cs / cntp);
      if (vv < 32) ctl->loss_view[vv] = lv;
      total += lv;
    }
  }
  if (threadIdx.x == 0) ctl->loss = total / (double)n_views;
}

__global__ void __launch_bounds__(256) k_loss_backward(const ViewDev* __restrict__ views, int n_views,
                                                       const float* __restrict__ image,
                                                       const StepParams* __restrict__ sp,
                                                       const float* __restrict__ partials,
                                                       const Control* __restrict__ ctl, float* __restrict__ dimage) {
  __shared__ float sp3[3][kSY][kSX];
  __shared__ float hb[3][kSY][kBX];
  if (ctl->overflow) return;
  float w[11];
  window(w);
  const long long b = blockIdx.x;
  const int v = view_of_block(views, n_views, b);
  const ViewDev& V = views[v];
  const int bxn = (V.W + kBX - 1) / kBX;
  const long long lb = b - V.loss_block_base;
  const int bx = (int)(lb % bxn), by = (int)(lb / bxn);
  const int ox = bx * kBX, oy = by * kBY;
  const long long HW = (long long)V.W * V.H;
  const float* X = image + 3 * V.pix_base;
  const float* Yt = V.target;
  const float* P = partials + 9 * V.pix_base;
  float* dX = dimage + 3 * V.pix_base;
  const float lam = sp->lambda_ssim;
  const float scale = 1.f / (3.f * (float)V.W * (float)V.H * (float)n_views);
  const float gl1 = (1.f - lam) * scale, gs = -lam * scale;
  for (int ch = 0; ch < 3; ++ch) {
    for (int k = threadIdx.x; k < kSX * kSY; k += blockDim.x) {
      const int r = k / kSX, c = k % kSX;
      const int gy = oy + r - kR, gx = ox + c - kR;
      const bool in = gx >= 0 && gx < V.W && gy >= 0 && gy < V.H;
      const long long pix = (long long)gy * V.W + gx;
#pragma unroll
      for (int m = 0; m < 3; ++m) sp3[m][r][c] = in ? P[(3 * ch + m) * HW + pix] : 0.f;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kSY * kBX; k += blockDim.x) {
      const int r = k / kBX, c = k % kBX;
      float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
      for (int t = 0; t < 11; ++t) {
        a0 += w[t] * sp3[0][r][c + t];
        a1 += w[t] * sp3[1][r][c + t];
        a2 += w[t] * sp3[2][r][c + t];
      }
      hb[0][r][c] = a0;
      hb[1][r][c] = a1;
      hb[2][r][c] = a2;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kBY * kBX; k += blockDim.x) {
      const int r = k / kBX, c = k % kBX;
      const int gy = oy + r, gx = ox + c;
      if (gx >= V.W || gy >= V.H) continue;
      float b0 = 0.f, b1 = 0.f, b2 = 0.f;
#pragma unroll
      for (int t = 0; t < 11; ++t) {
        b0 += w[t] * hb[0][r + t][c];
        b1 += w[t] * hb[1][r + t][c];
        b2 += w[t] * hb[2][r + t][c];
      }
      const long long pix = (long long)gy * V.W + gx;
      const float xv = X[ch * HW + pix], yv = Yt[ch * HW + pix];
      const float diff = xv - yv;
      const float sgn = diff > 0.f ? 1.f : (diff < 0.f ? -1.f : 0.f);
      dX[ch * HW + pix] = gl1 * sgn + gs * (b0 + 2.f * xv * b1 + yv * b2);
    }
    __syncthreads();
  }
}

void launch_loss(const ViewDev* views, int n_views, long long n_blocks, const float* image, const StepParams* sp,
                 float* partials, double* block_sums, Control* ctl, float* dimage, cudaStream_t s) {
  if (n_blocks <= 0) return;
  k_loss_forward<<<(unsigned)n_blocks, 256, 0, s>>>(views, n_views, n_blocks, image, sp, partials, block_sums, ctl);
  if (dimage)
    k_loss_backward<<<(unsigned)n_blocks, 256, 0, s>>>(views, n_views, image, sp, partials, ctl, dimage);
}

}  // namespace gs
