// k_loss.cu -- K7: L = lambda_1 L1 + lambda_ssim (1 - SSIM) (+ lambda_load L_load) of Eq. 10, and
// dL/d(render), sm_103a (the load term's gradient enters the blend backward, K8).
//
// SSIM uses the 11 x 11 Gaussian window (sigma 1.5) of 3DGS, zero padding and "same" output
// size, C1 = 0.01^2, C2 = 0.03^2, per colour channel; means run over 3 H W and, for a batch of
// views, the loss is the mean of the per-view losses.  E[x^2] and E[y^2] enter SSIM only through
// sigma_x^2 + sigma_y^2, so their window means are taken as one map E[x^2 + y^2] (the window is
// linear): the forward blurs two pair maps, (x, y) and (x^2 + y^2, xy), with the packed FP32x2 FMA
// of sm_100+ and no register shuffling, and the backward the pair (dS/dmu_x, dS/dE[x^2 + y^2]) and
// the single map dS/dE[xy], two adjacent outputs per packed FMA.  The window is separable and
// symmetric (six distinct weights).  Each CTA stages a 32 x 48 output block plus a 5-pixel halo in
// shared memory (cp.async, zero-filled outside the image, consecutive threads on consecutive
// columns; blocks inside the image skip the bounds tests) and blurs rows, then columns:
//   pass 1 (k_loss_forward): the window moments -> SSIM map, the three partial derivatives of SSIM
//          per pixel (an (a, b) pair plane and a c plane per channel), and per-CTA sums;
//   pass 2 (k_loss_backward): the same window applied to those partials (the window is
//          symmetric, so the adjoint of the blur is the blur) gives dL/dx.
// In a step, pass 1 follows the blend forward without waiting for it to complete: each block waits
// for the completion flags of the tiles under its window and reads the render through L2.
// Both passes run three 256-thread CTAs per SM (80 registers): their shared memory would fit four,
// but at four (64 registers) the optimisation step that contains them measured 20 us slower.  The
// last CTA of pass 1 reduces the per-CTA sums in a fixed order: the loss is deterministic.
#include <cmath>

#include "gs_device.cuh"
#include "gs_engine.h"

namespace gs {

namespace {
constexpr int kBX = 32, kBY = 48, kR = 5;
constexpr int kSX = kBX + 2 * kR, kSY = kBY + 2 * kR;  // staged block with the halo (42 x 58)
constexpr int kVR = kBY / 8;                           // column pass: 32 columns x 8 segments of 6 rows
constexpr int kSXP = 42;                               // staged pair rows (336 B)
constexpr int kSCP = 44;                               // staged single-map rows (176 B)
constexpr int kHP = kBX + 1;                           // row-blurred rows, padded
constexpr int kThreads = 256;
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;

// (w[t], w[t]) for t = 0..5 of the normalised window w[k] = exp(-(k - 5)^2 / (2 1.5^2)) / sum, set
// once by the host (in double, rounded to float); w[t] = w[10 - t].
__constant__ float2 c_w6[6];
__device__ __forceinline__ float2 wgt(int t) { return c_w6[t <= kR ? t : 2 * kR - t]; }

__device__ __forceinline__ int view_of_block(const ViewDev* __restrict__ views, int n_views, long long b) {
  int v = 0;
  while (v + 1 < n_views && views[v + 1].loss_block_base <= b) ++v;
  return v;
}

// The staged block: element e -> (row e / 42, column e % 42), image pixel (ox - 5 + col, oy - 5 +
// row), 0 outside the image.
constexpr int kStageN = kSY * kSX;

__device__ __forceinline__ bool block_inside(int ox, int oy, int W, int H) {
  return ox >= kR && oy >= kR && ox + kBX + kR <= W && oy + kBY + kR <= H;
}

__device__ __forceinline__ void cp_async4(void* dst, const void* src, bool ok) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(ok ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src, bool ok) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(ok ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Asynchronous staging: thread t takes elements t, t + 256, ...; element e is (row e / 42,
// column e % 42), so consecutive threads take consecutive columns.  A block whose staged window
// lies inside the image (most of them) skips the bounds tests.
template <typename Copy>
__device__ __forceinline__ void stage_async(int ox, int oy, int W, int H, Copy copy) {
  int r = threadIdx.x / kSX, col = threadIdx.x - r * kSX;
  constexpr int kDr = kThreads / kSX, kDc = kThreads % kSX;
  if (block_inside(ox, oy, W, H)) {
    int pix = (oy + r - kR) * W + (ox + col - kR);
#pragma unroll 2
    for (int e = threadIdx.x; e < kStageN; e += kThreads) {
      copy(r, col, pix, true);
      col += kDc;
      r += kDr;
      pix += kDr * W + kDc;
      if (col >= kSX) {
        col -= kSX;
        ++r;
        pix += W - kSX;
      }
    }
  } else {
#pragma unroll 2
    for (int e = threadIdx.x; e < kStageN; e += kThreads) {
      const int gy = oy + r - kR, gx = ox + col - kR;
      const bool ok = (unsigned)gy < (unsigned)H && (unsigned)gx < (unsigned)W;
      copy(r, col, ok ? gy * W + gx : 0, ok);
      col += kDc;
      r += kDr;
      if (col >= kSX) {
        col -= kSX;
        ++r;
      }
    }
  }
  cp_async_commit();
}

// Synchronous staging of the render through L2 (ld.global.cg) for a block that starts while the blend
// forward still runs: a neighbour tile may have been incomplete when this SM's L1 last held a sector
// of it, so the render must not be read through L1.  All of a thread's loads are in flight together.
__device__ __forceinline__ void stage_render_l2(float2 (*xy)[kSXP], const float* __restrict__ Xc, int ox, int oy,
                                                int W, int H) {
  constexpr int kPer = (kStageN + kThreads - 1) / kThreads;
  float v[kPer];
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const int e = threadIdx.x + k * kThreads;
    const int r = e / kSX, col = e - r * kSX;
    const int gy = oy + r - kR, gx = ox + col - kR;
    const bool ok = e < kStageN && (unsigned)gy < (unsigned)H && (unsigned)gx < (unsigned)W;
    v[k] = ok ? __ldcg(Xc + (long long)gy * W + gx) : 0.f;
  }
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const int e = threadIdx.x + k * kThreads;
    if (e < kStageN) {
      const int r = e / kSX;
      xy[r][e - r * kSX].x = v[k];
    }
  }
}

// Bounded wait (one thread) until *p >= need, at most `limit` polls; false when it gave up.
__device__ __forceinline__ bool wait_count(const unsigned* p, unsigned need, unsigned limit) {
  for (unsigned k = 0; k < limit; ++k) {
    if (ld_acquire_u32(p) >= need) return true;
    __nanosleep(128);
  }
  return false;
}

}  // namespace

long long loss_blocks(int W, int H) { return (long long)((W + kBX - 1) / kBX) * ((H + kBY - 1) / kBY); }

// Forward 50.1 KB, backward 52.7 KB.
struct LossFwdSmem {
  float2 xy[kSY][kSXP];  // staged (x, y)
  float2 hA[kSY][kHP];   // row-blurred (E[x], E[y])
  float2 hB[kSY][kHP];   // row-blurred (E[x^2 + y^2], E[xy])
};
struct LossBwdSmem {
  float2 ab[kSY][kSXP];  // staged (dS/dmu_x, dS/dE[x^2 + y^2])
  float c[kSY][kSCP];    // staged dS/dE[xy]
  float2 hab[kSY][kHP];
  float hc[kSY][kHP];
};

__global__ void __launch_bounds__(kThreads, 3) k_loss_forward(const ViewDev* __restrict__ views, int n_views,
                                                           long long n_blocks, const float* __restrict__ image,
                                                           const StepParams* __restrict__ sp,
                                                           float* __restrict__ partials,
                                                           double* __restrict__ block_sums,
                                                           Control* __restrict__ ctl, Ledger* __restrict__ ledger,
                                                           const unsigned* __restrict__ tile_done,
                                                           unsigned long long fwd_warps, unsigned spin_limit) {
  // Directly after the blend forward (tile_done given) this grid does not wait for the forward to
  // complete: its CTAs are scheduled once every forward CTA is running (the forward is persistent,
  // so every one of them is resident and makes progress), and each block waits only for the tiles
  // under its window.  What the forward writes (render, counters) is then read through L2.
  if (!tile_done) dep_wait();
  dep_release();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  LossFwdSmem& S = *reinterpret_cast<LossFwdSmem*>(smem_raw);
  __shared__ double s_red[2][8];
  __shared__ bool s_last;
  if (ld_relaxed_u32(&ctl->overflow)) return;
  const long long b = blockIdx.x;
  const int v = view_of_block(views, n_views, b);
  const ViewDev& V = views[v];
  const int bxn = (V.W + kBX - 1) / kBX;
  const long long lb = b - V.loss_block_base;
  const int bx = (int)(lb % bxn), by = (int)(lb / bxn);
  const int ox = bx * kBX, oy = by * kBY;
  if (tile_done) {
    if (threadIdx.x < 32) {
      // the tiles under the staged window (clipped to the image), one lane per tile
      const int tx0 = max(0, ox - kR) / V.tw, tx1 = min(V.W - 1, ox + kBX + kR - 1) / V.tw;
      const int ty0 = max(0, oy - kR) / V.th, ty1 = min(V.H - 1, oy + kBY + kR - 1) / V.th;
      const int ntx = tx1 - tx0 + 1, nt = ntx * (ty1 - ty0 + 1);
      bool ok = true;
      for (int k = threadIdx.x; k < nt && ok; k += 32)
        ok = wait_count(tile_done + V.tile_base + (long long)(ty0 + k / ntx) * V.gx + (tx0 + k % ntx), 1u, spin_limit);
      if (!ok) atomicOr(&ctl->error, kErrTimeout);
    }
    __syncthreads();
  }
  const long long HW = (long long)V.W * V.H;
  const float* X = image + 3 * V.pix_base;
  // per view 10 floats per pixel (so that every view's pair planes are 8-byte aligned): the three
  // channels' (a, b) pair planes, then their c planes
  float* Q = partials + 10 * V.pix_base;
  float2* Pab = reinterpret_cast<float2*>(Q);
  float* Pc = Q + 6 * HW;
  const float* Yt = V.target;
  double l1 = 0.0, ss = 0.0;
  for (int ch = 0; ch < 3; ++ch) {
    {
      const float* Xc = X + ch * HW;
      const float* Yc = Yt + ch * HW;
      if (tile_done) {
        stage_async(ox, oy, V.W, V.H,
                    [&](int r, int col, int pix, bool ok) { cp_async4(&S.xy[r][col].y, Yc + pix, ok); });
        stage_render_l2(S.xy, Xc, ox, oy, V.W, V.H);
      } else {
        stage_async(ox, oy, V.W, V.H, [&](int r, int col, int pix, bool ok) {
          cp_async4(&S.xy[r][col].x, Xc + pix, ok);
          cp_async4(&S.xy[r][col].y, Yc + pix, ok);
        });
      }
    }
    cp_async_wait<0>();
    __syncthreads();
    // row pass: 58 rows x 4 segments of 8 outputs, consecutive threads on consecutive rows (so the
    // 16-byte reads of a quarter warp hit distinct banks)
    for (int task = threadIdx.x; task < kSY * (kBX / 8); task += kThreads) {
      const int seg = task / kSY, r = task - seg * kSY, c0 = seg * 8;
      float2 a1[8], a2[8];
#pragma unroll
      for (int o = 0; o < 8; ++o) a1[o] = a2[o] = make_float2(0.f, 0.f);
      const float4* s4 = reinterpret_cast<const float4*>(&S.xy[r][c0]);
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        const float4 f = s4[q];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int j = 2 * q + h;
          const float x = h ? f.z : f.x, y = h ? f.w : f.y;
          const float2 v1 = make_float2(x, y);
          const float2 v2 = make_float2(fmaf(x, x, y * y), x * y);
#pragma unroll
          for (int o = 0; o < 8; ++o) {
            const int t = j - o;
            if (t >= 0 && t <= 2 * kR) {
              a1[o] = __ffma2_rn(wgt(t), v1, a1[o]);
              a2[o] = __ffma2_rn(wgt(t), v2, a2[o]);
            }
          }
        }
      }
#pragma unroll
      for (int o = 0; o < 8; ++o) {
        S.hA[r][c0 + o] = a1[o];
        S.hB[r][c0 + o] = a2[o];
      }
    }
    __syncthreads();
    {
      const int c = threadIdx.x % kBX, r0 = (threadIdx.x / kBX) * kVR;
      float2 mA[kVR], mB[kVR];
#pragma unroll
      for (int o = 0; o < kVR; ++o) mA[o] = mB[o] = make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < kVR + 2 * kR; ++j) {
        const float2 hA = S.hA[r0 + j][c], hB = S.hB[r0 + j][c];
#pragma unroll
        for (int o = 0; o < kVR; ++o) {
          const int t = j - o;
          if (t >= 0 && t <= 2 * kR) {
            mA[o] = __ffma2_rn(wgt(t), hA, mA[o]);
            mB[o] = __ffma2_rn(wgt(t), hB, mB[o]);
          }
        }
      }
      float l1c = 0.f, ssc = 0.f;
      const int gx = ox + c;
#pragma unroll
      for (int o = 0; o < kVR; ++o) {
        const int gy = oy + r0 + o;
        if (gx >= V.W || gy >= V.H) continue;
        const float mx = mA[o].x, my = mA[o].y, eq = mB[o].x, exy = mB[o].y;
        const float mxmy = mx * my, m2 = fmaf(mx, mx, my * my);
        const float N1 = 2.f * mxmy + kC1, N2 = 2.f * (exy - mxmy) + kC2;
        const float D1 = m2 + kC1, D2 = (eq - m2) + kC2;
        const float N = N1 * N2, D = D1 * D2;
        const float iD = __fdividef(1.f, D);  // C1 C2 <= D < 4: within 2 ulp
        const float Sv = N * iD;
        ssc += Sv;
        const float dN = 2.f * my * (N2 - N1), dD = 2.f * mx * (D2 - D1);
        const long long pix = ch * HW + (long long)gy * V.W + gx;
        Pab[pix] = make_float2((dN - Sv * dD) * iD,  // dS/dmu_x
                               -(Sv * D1) * iD);     // dS/dE[x^2 + y^2]
        Pc[pix] = 2.f * N1 * iD;                     // dS/dE[xy]
        const float2 xy = S.xy[r0 + o + kR][c + kR];
        l1c += fabsf(xy.x - xy.y);
      }
      l1 += (double)l1c;
      ss += (double)ssc;
    }
    __syncthreads();
  }
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
    for (long long k = b0 + threadIdx.x; k < b1; k += kThreads) {
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
    // the forward's counters: complete once every forward warp has counted itself (when this grid
    // did not wait for the forward), read through L2
    if (tile_done && !wait_count(&ctl->fwd_done, (unsigned)fwd_warps, spin_limit)) atomicOr(&ctl->error, kErrTimeout);
    const unsigned long long gp_pixels = ld_relaxed_u64(&ctl->gp_pixels), blended = ld_relaxed_u64(&ctl->blended);
    const unsigned long long gp_sq = ld_relaxed_u64(&ctl->gp_sq), pairs = ld_relaxed_u64(&ctl->pairs);
    double loss = total / (double)n_views;
    if (sp->lambda_load != 0.f && gp_pixels) {
      const double np = (double)gp_pixels, mean = (double)blended / np;
      const double var = (double)gp_sq / np - mean * mean;
      loss += (double)sp->lambda_load * sqrt(var > 0.0 ? var : 0.0);
    }
    ctl->loss = loss;
    if (ledger) {
      ledger->loss_sum += loss;
      ledger->pairs += pairs;
      ledger->blended += blended;
      ledger->instances += ld_relaxed_u64(&ctl->m_total);
      ledger->steps_ok += 1u;
      ledger->error |= ld_relaxed_u32(&ctl->error);
      ledger->last_gp_sum = blended;
      ledger->last_gp_pixels = gp_pixels;
      ledger->last_gp_sq = gp_sq;
    }
  }
}

__global__ void __launch_bounds__(kThreads, 3) k_loss_backward(const ViewDev* __restrict__ views, int n_views,
                                                            const float* __restrict__ image,
                                                            const StepParams* __restrict__ sp,
                                                            const float* __restrict__ partials,
                                                            const Control* __restrict__ ctl,
                                                            float* __restrict__ dimage) {
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
  const float* Q = partials + 10 * V.pix_base;
  const float2* Pab = reinterpret_cast<const float2*>(Q);
  const float* Pc = Q + 6 * HW;
  float* dX = dimage + 3 * V.pix_base;
  const float lam = sp->lambda_ssim;
  const float scale = 1.f / (3.f * (float)V.W * (float)V.H * (float)n_views);
  const float gl1 = sp->lambda_l1 * scale, gs = -lam * scale;
  for (int ch = 0; ch < 3; ++ch) {
    {
      const float2* ABc = Pab + ch * HW;
      const float* Cc = Pc + ch * HW;
      stage_async(ox, oy, V.W, V.H, [&](int r, int col, int pix, bool ok) {
        cp_async8(&S.ab[r][col], ABc + pix, ok);
        cp_async4(&S.c[r][col], Cc + pix, ok);
      });
    }
    cp_async_wait<0>();
    __syncthreads();
    for (int task = threadIdx.x; task < kSY * (kBX / 8); task += kThreads) {
      const int seg = task / kSY, r = task - seg * kSY, c0 = seg * 8;
      float2 aab[8], ac[4];
#pragma unroll
      for (int o = 0; o < 8; ++o) aab[o] = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < 4; ++k) ac[k] = make_float2(0.f, 0.f);
      const float4* s4 = reinterpret_cast<const float4*>(&S.ab[r][c0]);
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        const float4 f = s4[q];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int j = 2 * q + h;
          const float2 v1 = h ? make_float2(f.z, f.w) : make_float2(f.x, f.y);
#pragma unroll
          for (int o = 0; o < 8; ++o) {
            const int t = j - o;
            if (t >= 0 && t <= 2 * kR) aab[o] = __ffma2_rn(wgt(t), v1, aab[o]);
          }
        }
      }
      // the single map: output pairs (2k, 2k + 1) from input pairs (c[m], c[m + 1]), m = 2k + t
      const float4* c4 = reinterpret_cast<const float4*>(&S.c[r][c0]);
      float cv[20];
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        const float4 f = c4[q];
        cv[4 * q] = f.x;
        cv[4 * q + 1] = f.y;
        cv[4 * q + 2] = f.z;
        cv[4 * q + 3] = f.w;
      }
#pragma unroll
      for (int m = 0; m <= 16; ++m) {
        const float2 p = make_float2(cv[m], cv[m + 1]);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int t = m - 2 * k;
          if (t >= 0 && t <= 2 * kR) ac[k] = __ffma2_rn(wgt(t), p, ac[k]);
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
      const int c = threadIdx.x % kBX, r0 = (threadIdx.x / kBX) * kVR;
      const int gx = ox + c;
      float xo[kVR], yo[kVR];
#pragma unroll
      for (int o = 0; o < kVR; ++o) {
        const int gy = oy + r0 + o;
        const bool in = gx < V.W && gy < V.H;
        const long long pix = in ? ch * HW + (long long)gy * V.W + gx : 0;
        xo[o] = in ? X[pix] : 0.f;
        yo[o] = in ? Yt[pix] : 0.f;
      }
      float2 bab[kVR], bc[kVR / 2];
#pragma unroll
      for (int o = 0; o < kVR; ++o) bab[o] = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < kVR / 2; ++k) bc[k] = make_float2(0.f, 0.f);
      float hv[kVR + 2 * kR];
#pragma unroll
      for (int j = 0; j < kVR + 2 * kR; ++j) {
        const float2 h = S.hab[r0 + j][c];
        hv[j] = S.hc[r0 + j][c];
#pragma unroll
        for (int o = 0; o < kVR; ++o) {
          const int t = j - o;
          if (t >= 0 && t <= 2 * kR) bab[o] = __ffma2_rn(wgt(t), h, bab[o]);
        }
      }
#pragma unroll
      for (int m = 0; m <= kVR - 2 + 2 * kR; ++m) {
        const float2 p = make_float2(hv[m], hv[m + 1]);
#pragma unroll
        for (int k = 0; k < kVR / 2; ++k) {
          const int t = m - 2 * k;
          if (t >= 0 && t <= 2 * kR) bc[k] = __ffma2_rn(wgt(t), p, bc[k]);
        }
      }
#pragma unroll
      for (int o = 0; o < kVR; ++o) {
        const int gy = oy + r0 + o;
        if (gx >= V.W || gy >= V.H) continue;
        const float xv = xo[o], yv = yo[o];
        const float diff = xv - yv;
        const float sgn = diff > 0.f ? 1.f : (diff < 0.f ? -1.f : 0.f);
        const float bcv = (o & 1) ? bc[o / 2].y : bc[o / 2].x;
        dX[ch * HW + (long long)gy * V.W + gx] = gl1 * sgn + gs * (bab[o].x + 2.f * xv * bab[o].y + yv * bcv);
      }
    }
    __syncthreads();
  }
}

void init_loss_attributes() {
  double sum = 0.0, e[11];
  for (int k = 0; k < 11; ++k) {
    const double d = (double)(k - kR);
    e[k] = std::exp(-d * d / (2.0 * 1.5 * 1.5));
    sum += e[k];
  }
  float2 w6[6];
  for (int t = 0; t <= kR; ++t) {
    const float w = (float)(e[t] / sum);
    w6[t] = make_float2(w, w);
  }
  cudaMemcpyToSymbol(c_w6, w6, sizeof(w6));
  cudaFuncSetAttribute(k_loss_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(LossFwdSmem));
  cudaFuncSetAttribute(k_loss_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(LossBwdSmem));
}

void launch_loss(const ViewDev* views, int n_views, long long n_blocks, const float* image, const StepParams* sp,
                 float* partials, double* block_sums, Control* ctl, Ledger* ledger, float* dimage,
                 const unsigned* tile_done, long long fwd_warps, cudaStream_t s) {
  if (n_blocks <= 0) return;
  launch_dep(k_loss_forward, dim3((unsigned)n_blocks), dim3(kThreads), sizeof(LossFwdSmem), s, views, n_views,
      n_blocks, image, sp, partials, block_sums, ctl, ledger, tile_done, (unsigned long long)fwd_warps, kSpinLimit);
  if (dimage)
    launch_dep(k_loss_backward, dim3((unsigned)n_blocks), dim3(kThreads), sizeof(LossBwdSmem), s, views, n_views,
        image, sp, partials, ctl, dimage);
}

// Failure detection for the loss forward's waits when it runs under the blend forward: a one-block
// view (32 x 48 pixels, six 16 x 16 tiles) whose tiles are never flagged and whose forward warps never
// count themselves, so the tile wait and the last CTA's wait can only end by giving up.
gs_status run_loss_wait_probe(unsigned spin_limit, unsigned* out_error, float* out_ms) {
  if (spin_limit == 0u) spin_limit = kSpinLimit;
  init_loss_attributes();
  constexpr int W = kBX, H = kBY;
  const size_t npix = (size_t)W * H;
  const size_t off_views = 0, off_sp = 1024, off_ctl = 2048, off_sums = off_ctl + kCtlBytes;
  const size_t off_done = off_sums + 64, off_img = off_done + 64;
  const size_t off_tgt = off_img + 3 * npix * 4, off_part = off_tgt + 3 * npix * 4;
  const size_t bytes = off_part + 10 * npix * 4;
  char* d = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  gs_status status = GS_OK;
  auto check = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && status == GS_OK) status = fail(GS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaSuccess;
  };
  if (check(cudaMalloc(&d, bytes), "cudaMalloc") && check(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "stream") &&
      check(cudaEventCreate(&ev[0]), "event") && check(cudaEventCreate(&ev[1]), "event") &&
      check(cudaMemsetAsync(d, 0, bytes, st), "cudaMemsetAsync")) {
    ViewDev v{};
    v.W = W;
    v.H = H;
    v.tw = 16;
    v.th = 16;
    v.gx = 2;
    v.gy = 3;
    v.target = reinterpret_cast<const float*>(d + off_tgt);
    StepParams sp{};
    sp.n_views = 1;
    sp.lambda_ssim = 0.2f;
    sp.lambda_l1 = 0.8f;
    if (check(cudaMemcpyAsync(d + off_views, &v, sizeof(v), cudaMemcpyHostToDevice, st), "cudaMemcpyAsync") &&
        check(cudaMemcpyAsync(d + off_sp, &sp, sizeof(sp), cudaMemcpyHostToDevice, st), "cudaMemcpyAsync")) {
      Control* ctl = reinterpret_cast<Control*>(d + off_ctl);
      cudaEventRecord(ev[0], st);
      k_loss_forward<<<1, kThreads, sizeof(LossFwdSmem), st>>>(
          reinterpret_cast<const ViewDev*>(d + off_views), 1, 1, reinterpret_cast<const float*>(d + off_img),
          reinterpret_cast<const StepParams*>(d + off_sp), reinterpret_cast<float*>(d + off_part),
          reinterpret_cast<double*>(d + off_sums), ctl, nullptr, reinterpret_cast<const unsigned*>(d + off_done), 1ull,
          spin_limit);
      cudaEventRecord(ev[1], st);
      check(cudaGetLastError(), "loss wait probe launch");
      Control r{};
      if (check(cudaMemcpyAsync(&r, ctl, sizeof(Control), cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync") &&
          check(cudaStreamSynchronize(st), "cudaStreamSynchronize")) {
        *out_error = r.error;
        if (out_ms) cudaEventElapsedTime(out_ms, ev[0], ev[1]);
      }
    }
  }
  for (cudaEvent_t e : ev)
    if (e) cudaEventDestroy(e);
  if (st) cudaStreamDestroy(st);
  if (d) cudaFree(d);
  return status;
}

}  // namespace gs
