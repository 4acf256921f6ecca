// k_loss.cu -- K7: L = lambda_1 L1 + lambda_ssim (1 - SSIM) (+ lambda_load L_load) of Eq. 10, and
// dL/d(render), sm_103a (the load term's gradient enters the blend backward, K8).
//
// SSIM uses the 11 x 11 Gaussian window (sigma 1.5) of 3DGS, zero padding and "same" output
// size, C1 = 0.01^2, C2 = 0.03^2, per colour channel; means run over 3 H W and, for a batch of
// views, the loss is the mean of the per-view losses.  The window is separable: each CTA stages
// a 32 x 48 output block plus a 5-pixel halo in shared memory, blurs rows then columns.  The
// staging is asynchronous (cp.async, zero-filled outside the image) into one buffer, so that three
// CTAs share an SM and overlap one another's staging (a second buffer with the next channel in
// flight left room for two).
//   pass 1 (k_loss_forward): the five window moments -> SSIM map, the three partial derivatives
//          of SSIM with respect to (mu_x, E[x^2], E[xy]) per pixel, and per-CTA sums;
//   pass 2 (k_loss_backward): the same window applied to those partials (the window is
//          symmetric, so the adjoint of the blur is the blur) gives dL/dx.
// The last CTA of pass 1 reduces the per-CTA sums in a fixed order: the loss is deterministic.
#include <cmath>

#include "gs_device.cuh"
#include "gs_engine.h"

namespace gs {

namespace {
constexpr int kBX = 32, kBY = 48, kR = 5;
constexpr int kSX = kBX + 2 * kR, kSY = kBY + 2 * kR;  // staged block with the halo
constexpr int kVR = kBY / 8;  // column pass: 32 columns x 8 segments of kVR rows (256 threads)
static_assert(kVR % 2 == 0, "column outputs are paired for the packed single-map blur");
constexpr int kStageBufs = 1;  // staging buffers: 2 = the next channel in flight, 1 = more CTAs per SM
constexpr int kSXP = 44;                               // padded row: 16-byte aligned float4 reads
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;

// The normalised window w[k] = exp(-d^2 / (2 1.5^2)) / sum, d = k - 5, set once by the host (in
// double, rounded to float), held twice for the packed FP32x2 FMAs: c_w2[k] = (w[k], w[k]).
__constant__ float2 c_w2[11];
// (w[t], w[t - 1]) for t = 0..11 (0 outside the window): the weights of one input at two adjacent
// outputs, for blurring a single map two outputs per packed FMA
__constant__ float2 c_wp[12];

__device__ __forceinline__ int view_of_block(const ViewDev* __restrict__ views, int n_views, long long b) {
  int v = 0;
  while (v + 1 < n_views && views[v + 1].loss_block_base <= b) ++v;
  return v;
}

// 4-byte asynchronous copy global -> shared; ok == false writes 0 (reads nothing).
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool ok) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = ok ? 4 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Stage MAPS planes (W x H each) of the 42 x 58 block at (ox - 5, oy - 5) into dst[m] (rows of
// kSXP floats); outside the image (and the pad columns) become 0.  A task is 4 consecutive
// columns of one row (the rows of an image of any width are not 16-byte aligned, so the copies
// are 4-byte ones; the row and bounds arithmetic is shared by the four).
template <int MAPS>
__device__ __forceinline__ void stage_block(float (*dst)[kSY][kSXP], const float* const (&src)[MAPS], int ox, int oy,
                                            int W, int H) {
  constexpr int kGroups = kSXP / 4;
  for (int task = threadIdx.x; task < kSY * kGroups; task += blockDim.x) {
    const int r = task / kGroups, c0 = (task - r * kGroups) * 4;
    const int gy = oy + r - kR, gx0 = ox + c0 - kR;
    const bool row_ok = gy >= 0 && gy < H;
    const long long rowbase = row_ok ? (long long)gy * W : 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int gx = gx0 + i;
      const bool ok = row_ok && c0 + i < kSX && gx >= 0 && gx < W;
      const long long pix = ok ? rowbase + gx : 0;
#pragma unroll
      for (int m = 0; m < MAPS; ++m) cp_async4(&dst[m][r][c0 + i], src[m] + pix, ok);
    }
  }
  cp_async_commit();
}

}  // namespace

long long loss_blocks(int W, int H) { return (long long)((W + kBX - 1) / kBX) * ((H + kBY - 1) / kBY); }

// The row pass blurs 8 adjacent outputs per thread from 18 staged values per map, the column pass
// 4 from 14, so a staged value is read once per 8 (4) outputs.
struct LossFwdSmem {
  float in[kStageBufs][2][kSY][kSXP];  // [buffer][x / y][row][col]
  float2 hxy[kSY][kBX + 1];   // row-blurred (E[x], E[y])
  float2 hq[kSY][kBX + 1];    // row-blurred (E[x^2], E[y^2])
  float hc[kSY][kBX + 1];     // row-blurred E[xy]
};
struct LossBwdSmem {
  float in[kStageBufs][3][kSY][kSXP];  // [buffer][partial][row][col]
  float2 hab[kSY][kBX + 1];   // row-blurred (dS/dmu_x, dS/dE[x^2])
  float hc[kSY][kBX + 1];     // row-blurred dS/dE[xy]
};

__global__ void __launch_bounds__(256, 3) k_loss_forward(const ViewDev* __restrict__ views, int n_views,
                                                      long long n_blocks, const float* __restrict__ image,
                                                      const StepParams* __restrict__ sp,
                                                      float* __restrict__ partials, double* __restrict__ block_sums,
                                                      Control* __restrict__ ctl, Ledger* __restrict__ ledger) {
  dep_wait();
  dep_release();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  LossFwdSmem& S = *reinterpret_cast<LossFwdSmem*>(smem_raw);
  __shared__ double s_red[2][8];
  __shared__ bool s_last;
  if (ctl->overflow) return;
  const long long b = blockIdx.x;
  const int v = view_of_block(views, n_views, b);
  const ViewDev& V = views[v];
  const int bxn = (V.W + kBX - 1) / kBX;
  const long long lb = b - V.loss_block_base;
  const int bx = (int)(lb % bxn), by = (int)(lb / bxn);
  const int ox = bx * kBX, oy = by * kBY;
  const long long HW = (long long)V.W * V.H;
  const float* X = image + 3 * V.pix_base;
  float* P = partials + 9 * V.pix_base;
  const float* Yt = V.target;
  double l1 = 0.0, ss = 0.0;
  if (kStageBufs == 2) {
    const float* const src[2] = {X, Yt};
    stage_block<2>(S.in[0], src, ox, oy, V.W, V.H);
  }
  for (int ch = 0; ch < 3; ++ch) {
    const int cur = kStageBufs == 2 ? (ch & 1) : 0;
    if (kStageBufs == 1) {
      const float* const src[2] = {X + ch * HW, Yt + ch * HW};
      stage_block<2>(S.in[0], src, ox, oy, V.W, V.H);
      cp_async_wait<0>();
    } else if (ch < 2) {
      const float* const src[2] = {X + (ch + 1) * HW, Yt + (ch + 1) * HW};
      stage_block<2>(S.in[(cur + 1) % kStageBufs], src, ox, oy, V.W, V.H);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    float (*sx)[kSXP] = S.in[cur][0];
    float (*sy)[kSXP] = S.in[cur][1];
    // horizontal: 42 rows x 4 segments of 8 columns, one per thread.  x and y (and x^2 and y^2)
    // share the window weights, so they are blurred as pairs with the packed FP32x2 FMA of sm_100+;
    // xy is blurred two adjacent outputs per packed FMA.
    for (int task = threadIdx.x; task < kSY * (kBX / 8); task += blockDim.x) {
      const int r = task >> 2, c0 = (task & 3) * 8;
      const float* rx = sx[r] + c0;
      const float* ry = sy[r] + c0;
      float2 axy[8], aq[8], ac[4];
#pragma unroll
      for (int o = 0; o < 8; ++o) {
        axy[o] = make_float2(0.f, 0.f);
        aq[o] = make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) ac[k] = make_float2(0.f, 0.f);
#pragma unroll
      for (int j4 = 0; j4 < 20; j4 += 4) {  // inputs c0 .. c0 + 17 (+ 2 zero pad columns)
        const float4 X4 = *reinterpret_cast<const float4*>(rx + j4);
        const float4 Y4 = *reinterpret_cast<const float4*>(ry + j4);
        const float xs[4] = {X4.x, X4.y, X4.z, X4.w}, ys[4] = {Y4.x, Y4.y, Y4.z, Y4.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = j4 + u;
          if (j >= 18) break;
          const float2 v = make_float2(xs[u], ys[u]);
          const float2 v2 = __fmul2_rn(v, v);
          const float c = xs[u] * ys[u];
          const float2 cc = make_float2(c, c);
#pragma unroll
          for (int o = 0; o < 8; ++o) {
            const int t = j - o;
            if (t >= 0 && t < 11) {
              axy[o] = __ffma2_rn(c_w2[t], v, axy[o]);
              aq[o] = __ffma2_rn(c_w2[t], v2, aq[o]);
            }
          }
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int t = j - 2 * k;
            if (t >= 0 && t <= 11) ac[k] = __ffma2_rn(c_wp[t], cc, ac[k]);
          }
        }
      }
#pragma unroll
      for (int o = 0; o < 8; ++o) {
        S.hxy[r][c0 + o] = axy[o];
        S.hq[r][c0 + o] = aq[o];
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        S.hc[r][c0 + 2 * k] = ac[k].x;
        S.hc[r][c0 + 2 * k + 1] = ac[k].y;
      }
    }
    __syncthreads();
    // vertical: 32 columns x 8 segments of kVR rows
    {
      const int c = threadIdx.x % kBX, r0 = (threadIdx.x / kBX) * kVR;
      float2 mxy[kVR], mq[kVR], mc2[kVR / 2];
#pragma unroll
      for (int o = 0; o < kVR; ++o) {
        mxy[o] = make_float2(0.f, 0.f);
        mq[o] = make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int k = 0; k < kVR / 2; ++k) mc2[k] = make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < kVR + 10; ++j) {
        const float2 hxy = S.hxy[r0 + j][c], hq = S.hq[r0 + j][c];
        const float hc = S.hc[r0 + j][c];
        const float2 hcc = make_float2(hc, hc);
#pragma unroll
        for (int o = 0; o < kVR; ++o) {
          const int t = j - o;
          if (t >= 0 && t < 11) {
            mxy[o] = __ffma2_rn(c_w2[t], hxy, mxy[o]);
            mq[o] = __ffma2_rn(c_w2[t], hq, mq[o]);
          }
        }
#pragma unroll
        for (int k = 0; k < kVR / 2; ++k) {
          const int t = j - 2 * k;
          if (t >= 0 && t <= 11) mc2[k] = __ffma2_rn(c_wp[t], hcc, mc2[k]);
        }
      }
      float l1c = 0.f, ssc = 0.f;  // at most kVR terms per thread and channel: float is exact enough
#pragma unroll
      for (int o = 0; o < kVR; ++o) {
        const int gy = oy + r0 + o, gx = ox + c;
        if (gx >= V.W || gy >= V.H) continue;
        const float mx = mxy[o].x, my = mxy[o].y, exx = mq[o].x, eyy = mq[o].y;
        const float exy = (o & 1) ? mc2[o / 2].y : mc2[o / 2].x;
        const float N1 = 2.f * mx * my + kC1, N2 = 2.f * (exy - mx * my) + kC2;
        const float D1 = mx * mx + my * my + kC1, D2 = (exx - mx * mx) + (eyy - my * my) + kC2;
        const float N = N1 * N2, D = D1 * D2;
        const float iD = 1.f / D;
        ssc += N * iD;
        const float dN = 2.f * my * N2 - 2.f * my * N1;
        const float dD = 2.f * mx * D2 - 2.f * mx * D1;
        const long long pix = (long long)gy * V.W + gx;
        P[(3 * ch + 0) * HW + pix] = (dN * D - N * dD) * iD * iD;  // dS/dmu_x
        P[(3 * ch + 1) * HW + pix] = -N * D1 * iD * iD;             // dS/dE[x^2]
        P[(3 * ch + 2) * HW + pix] = 2.f * N1 * iD;                 // dS/dE[xy]
        l1c += fabsf(sx[r0 + o + kR][c + kR] - sy[r0 + o + kR][c + kR]);
      }
      l1 += (double)l1c;
      ss += (double)ssc;
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
  const double lam = (double)sp->lambda_ssim, lam1 = (double)sp->lambda_l1;
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
      const double lv = lam1 * (A / cntp) + lam * (1.0 - Cs / cntp);
      if (vv < 32) ctl->loss_view[vv] = lv;
      total += lv;
    }
  }
  if (threadIdx.x == 0) {
    double loss = total / (double)n_views;
    // Eq. 9-10: + lambda_load L_load over the pixels some Gaussian reaches (all views of the step;
    // K6's moments of G_p); its gradient enters the blend backward through the soft count
    if (sp->lambda_load != 0.f && ctl->gp_pixels) {  // std of G_p
      const double np = (double)ctl->gp_pixels, mean = (double)ctl->blended / np;
      const double var = (double)ctl->gp_sq / np - mean * mean;
      loss += (double)sp->lambda_load * sqrt(var > 0.0 ? var : 0.0);
    }
    ctl->loss = loss;
    if (ledger) {  // this step is complete up to Adam, which cannot fail any more
      ledger->loss_sum += ctl->loss;
      ledger->pairs += ctl->pairs;
      ledger->blended += ctl->blended;
      ledger->instances += ctl->m_total;
      ledger->steps_ok += 1u;
      ledger->error |= ctl->error;
      ledger->last_gp_sum = ctl->blended;
      ledger->last_gp_pixels = ctl->gp_pixels;
      ledger->last_gp_sq = ctl->gp_sq;
    }
  }
}

__global__ void __launch_bounds__(256, 3) k_loss_backward(const ViewDev* __restrict__ views, int n_views,
                                                       const float* __restrict__ image,
                                                       const StepParams* __restrict__ sp,
                                                       const float* __restrict__ partials,
                                                       const Control* __restrict__ ctl, float* __restrict__ dimage) {
  dep_wait();
  dep_release();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  LossBwdSmem& S = *reinterpret_cast<LossBwdSmem*>(smem_raw);
  if (ctl->overflow) return;
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
  const float gl1 = sp->lambda_l1 * scale, gs = -lam * scale;
  if (kStageBufs == 2) {
    const float* const src[3] = {P, P + HW, P + 2 * HW};
    stage_block<3>(S.in[0], src, ox, oy, V.W, V.H);
  }
  for (int ch = 0; ch < 3; ++ch) {
    const int cur = kStageBufs == 2 ? (ch & 1) : 0;
    if (kStageBufs == 1) {
      const float* const src[3] = {P + (3 * ch) * HW, P + (3 * ch + 1) * HW, P + (3 * ch + 2) * HW};
      stage_block<3>(S.in[0], src, ox, oy, V.W, V.H);
      cp_async_wait<0>();
    } else if (ch < 2) {
      const float* const src[3] = {P + (3 * ch + 3) * HW, P + (3 * ch + 4) * HW, P + (3 * ch + 5) * HW};
      stage_block<3>(S.in[(cur + 1) % kStageBufs], src, ox, oy, V.W, V.H);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    // this thread's four output pixels: fetch the render and target now, used after the blur
    const int vc = threadIdx.x % kBX, vr0 = (threadIdx.x / kBX) * kVR;
    float xo[kVR], yo[kVR];
#pragma unroll
    for (int o = 0; o < kVR; ++o) {
      const int gy = oy + vr0 + o, gx = ox + vc;
      const bool in = gx < V.W && gy < V.H;
      const long long pix = in ? (long long)gy * V.W + gx : 0;
      xo[o] = in ? X[ch * HW + pix] : 0.f;
      yo[o] = in ? Yt[ch * HW + pix] : 0.f;
    }
    for (int task = threadIdx.x; task < kSY * (kBX / 8); task += blockDim.x) {
      const int r = task >> 2, c0 = (task & 3) * 8;
      const float* ra = S.in[cur][0][r] + c0;
      const float* rb = S.in[cur][1][r] + c0;
      const float* rc = S.in[cur][2][r] + c0;
      float2 aab[8], ac[4];
#pragma unroll
      for (int o = 0; o < 8; ++o) aab[o] = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < 4; ++k) ac[k] = make_float2(0.f, 0.f);
#pragma unroll
      for (int j4 = 0; j4 < 20; j4 += 4) {
        const float4 A4 = *reinterpret_cast<const float4*>(ra + j4);
        const float4 B4 = *reinterpret_cast<const float4*>(rb + j4);
        const float4 C4 = *reinterpret_cast<const float4*>(rc + j4);
        const float as[4] = {A4.x, A4.y, A4.z, A4.w}, bs[4] = {B4.x, B4.y, B4.z, B4.w};
        const float cs[4] = {C4.x, C4.y, C4.z, C4.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = j4 + u;
          if (j >= 18) break;
          const float2 v = make_float2(as[u], bs[u]);
          const float2 cc = make_float2(cs[u], cs[u]);
#pragma unroll
          for (int o = 0; o < 8; ++o) {
            const int t = j - o;
            if (t >= 0 && t < 11) aab[o] = __ffma2_rn(c_w2[t], v, aab[o]);
          }
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int t = j - 2 * k;
            if (t >= 0 && t <= 11) ac[k] = __ffma2_rn(c_wp[t], cc, ac[k]);
          }
        }
      }
#pragma unroll
      for (int o = 0; o < 8; ++o) S.hab[r][c0 + o] = aab[o];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        S.hc[r][c0 + 2 * k] = ac[k].x;
        S.hc[r][c0 + 2 * k + 1] = ac[k].y;
      }
    }
    __syncthreads();
    {
      const int c = vc, r0 = vr0;
      float2 bab[kVR], bc2[kVR / 2];
#pragma unroll
      for (int o = 0; o < kVR; ++o) bab[o] = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < kVR / 2; ++k) bc2[k] = make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < kVR + 10; ++j) {
        const float2 h = S.hab[r0 + j][c];
        const float hc = S.hc[r0 + j][c];
        const float2 hcc = make_float2(hc, hc);
#pragma unroll
        for (int o = 0; o < kVR; ++o) {
          const int t = j - o;
          if (t >= 0 && t < 11) bab[o] = __ffma2_rn(c_w2[t], h, bab[o]);
        }
#pragma unroll
        for (int k = 0; k < kVR / 2; ++k) {
          const int t = j - 2 * k;
          if (t >= 0 && t <= 11) bc2[k] = __ffma2_rn(c_wp[t], hcc, bc2[k]);
        }
      }
#pragma unroll
      for (int o = 0; o < kVR; ++o) {
        const int gy = oy + r0 + o, gx = ox + c;
        if (gx >= V.W || gy >= V.H) continue;
        const long long pix = (long long)gy * V.W + gx;
        const float xv = xo[o], yv = yo[o];
        const float diff = xv - yv;
        const float sgn = diff > 0.f ? 1.f : (diff < 0.f ? -1.f : 0.f);
        const float bc = (o & 1) ? bc2[o / 2].y : bc2[o / 2].x;
        dX[ch * HW + pix] = gl1 * sgn + gs * (bab[o].x + 2.f * xv * bab[o].y + yv * bc);
      }
    }
    __syncthreads();
  }
}

void init_loss_attributes() {
  float w[11];
  float2 w2[11];
  double sum = 0.0, e[11];
  for (int k = 0; k < 11; ++k) {
    const double d = (double)(k - kR);
    e[k] = std::exp(-d * d / (2.0 * 1.5 * 1.5));
    sum += e[k];
  }
  for (int k = 0; k < 11; ++k) {
    w[k] = (float)(e[k] / sum);
    w2[k] = make_float2(w[k], w[k]);
  }
  float2 wp[12];
  for (int t = 0; t < 12; ++t) wp[t] = make_float2(t <= 10 ? w[t] : 0.f, t >= 1 ? w[t - 1] : 0.f);
  cudaMemcpyToSymbol(c_w2, w2, sizeof(w2));
  cudaMemcpyToSymbol(c_wp, wp, sizeof(wp));
  cudaFuncSetAttribute(k_loss_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(LossFwdSmem));
  cudaFuncSetAttribute(k_loss_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(LossBwdSmem));
}

void launch_loss(const ViewDev* views, int n_views, long long n_blocks, const float* image, const StepParams* sp,
                 float* partials, double* block_sums, Control* ctl, Ledger* ledger, float* dimage, cudaStream_t s) {
  if (n_blocks <= 0) return;
  launch_dep(k_loss_forward, dim3((unsigned)n_blocks), dim3(256), sizeof(LossFwdSmem), s, views, n_views, n_blocks,
      image, sp, partials, block_sums, ctl, ledger);
  if (dimage)
    launch_dep(k_loss_backward, dim3((unsigned)n_blocks), dim3(256), sizeof(LossBwdSmem), s, views, n_views, image, sp,
        partials, ctl, dimage);
}

}  // namespace gs
