// k_blend.cu -- K6 (front-to-back alpha blending, Eq. 2) and K8 (its splatting-parallel
// backward, Sec. IV-D), sm_103a.
//
// K6: one CTA per 16 x 16 tile (all views' tiles in one grid), one pixel per thread.  The
// tile's sorted Gaussians are staged through shared memory in batches; a pixel stops before the
// Gaussian that would take its transmittance below 1e-4 and the CTA leaves the batch loop as
// soon as every pixel has stopped (__syncthreads_count).  Every 32 list entries each live pixel
// stores a checkpoint (T, accumulated colour) so the backward can start any 32-entry chunk
// without re-walking the list.
//
// K8: splatting-parallel gradient accumulation (the paper adopts it from Taming 3DGS to remove
// the serialized per-pixel atomics of the original backward).  A persistent warp takes one
// (tile, 32-entry chunk) at a time.  Lane l owns Gaussian l of the chunk and keeps its nine
// gradient sums in registers; the tile's live pixels stream through the warp as a skewed
// pipeline (at step s lane l works on pixel s - l), the running (T, colour-in-front) state of a
// pixel passing from lane to lane by one shuffle.  Each instance's gradient is written once,
// to its own slot, with no atomics, so the result is deterministic.
#include "gs_device.cuh"
#include "gs_engine.h"

namespace gs {

namespace {
constexpr int kBlendBatch = 256;

__device__ __forceinline__ int view_of_tile(const ViewDev* __restrict__ views, int n_views, long long t) {
  int v = 0;
  while (v + 1 < n_views && views[v + 1].tile_base <= t) ++v;
  return v;
}

__device__ __forceinline__ long long chunk_base(unsigned start, long long tile) {
  return (long long)(start >> 5) + tile;
}
}  // namespace

// ---------------------------------------------------------------------------------------------
// K6
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kTilePix) k_blend_forward(
    const ViewDev* __restrict__ views, int n_views, const uint2* __restrict__ ranges,
    const unsigned* __restrict__ vals, const ProjBuffers pb, const StepParams* __restrict__ sp,
    Control* __restrict__ ctl, float* __restrict__ image, float* __restrict__ Tout, unsigned* __restrict__ last_out,
    unsigned* __restrict__ gp_out, float4* __restrict__ ckpt, int* __restrict__ chunk_tile) {
  __shared__ float4 s_xyo[kBlendBatch];
  __shared__ float4 s_con[kBlendBatch];
  __shared__ float4 s_rgb[kBlendBatch];
  __shared__ unsigned long long s_pairs[kTilePix / 32];
  if (ctl->overflow) return;
  const long long t = blockIdx.x;
  const int v = view_of_tile(views, n_views, t);
  const ViewDev& V = views[v];
  const long long local = t - V.tile_base;
  const int tx = (int)(local % V.gx), ty = (int)(local / V.gx);
  const int tid = threadIdx.x;
  const int px = tx * kTile + (tid & (kTile - 1));
  const int py = ty * kTile + (tid / kTile);
  const bool inside = px < V.W && py < V.H;
  const float pxf = (float)px, pyf = (float)py;

  const uint2 rg = ranges[t];
  const unsigned start = rg.x;
  const int L = (int)(rg.y - rg.x);
  const long long cb = chunk_base(start, t);
  for (int k = tid; k < (L + kChunk - 1) / kChunk; k += kTilePix) chunk_tile[cb + k] = (int)(t + 1);

  float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
  unsigned last = 0u, gp = 0u;
  unsigned neval = (unsigned)L;
  bool done = !inside;
  for (int b0 = 0; b0 < L; b0 += kBlendBatch) {
    if (__syncthreads_count(done) == kTilePix) break;
    const int j = b0 + tid;
    if (j < L) {
      const unsigned rec = vals[start + j];
      s_xyo[tid] = pb.xyo[rec];
      s_con[tid] = pb.conic[rec];
      s_rgb[tid] = pb.rgb[rec];
    }
    __syncthreads();
    if (!done) {
      const int nb = min(kBlendBatch, L - b0);
      for (int jj = 0; jj < nb; ++jj) {
        const int jg = b0 + jj;
        if ((jg & (kChunk - 1)) == 0 && jg > 0)
          ckpt[(cb + (jg >> 5)) * kTilePix + tid] = make_float4(T, C0, C1, C2);
        const float4 xy = s_xyo[jj];
        const float4 co = s_con[jj];
        const float dx = __fsub_rn(xy.x, pxf), dy = __fsub_rn(xy.y, pyf);
        const float power = splat_power(co.x, co.y, co.z, dx, dy);
        if (power > 0.f) continue;
        const float alpha = fminf(kAlphaMax, __fmul_rn(xy.z, splat_exp(power)));
        if (alpha < kAlphaMin) continue;
        const float testT = __fmul_rn(T, __fsub_rn(1.f, alpha));
        if (testT < kTransMin) {
          done = true;
          neval = (unsigned)jg + 1u;
          break;
        }
        const float4 c = s_rgb[jj];
        const float w = __fmul_rn(alpha, T);
        C0 = __fmaf_rn(c.x, w, C0);
        C1 = __fmaf_rn(c.y, w, C1);
        C2 = __fmaf_rn(c.z, w, C2);
        T = testT;
        last = (unsigned)jg + 1u;
        ++gp;
      }
    }
  }
  unsigned long long my_pairs = 0;
  if (inside) {
    const long long HW = (long long)V.W * V.H;
    const long long pix = (long long)py * V.W + px;
    float* img = image + 3 * V.pix_base;
    img[pix] = C0 + T * sp->bg[0];
    img[HW + pix] = C1 + T * sp->bg[1];
    img[2 * HW + pix] = C2 + T * sp->bg[2];
    const long long gpix = V.pix_base + pix;
    if (Tout) Tout[gpix] = T;
    last_out[gpix] = last;
    if (gp_out) gp_out[gpix] = gp;
    my_pairs = neval;
  }
  // Gaussian-pixel pairs by definition: entries evaluated per pixel up to its termination.
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) my_pairs += __shfl_down_sync(0xffffffffu, my_pairs, o);
  if ((tid & 31) == 0) s_pairs[tid >> 5] = my_pairs;
  __syncthreads();
  if (tid == 0) {
    unsigned long long s = 0;
#pragma unroll
    for (int w = 0; w < kTilePix / 32; ++w) s += s_pairs[w];
    atomicAdd(&ctl->pairs, s);
  }
}

void launch_blend_forward(const ViewDev* views, int n_views, long long n_tiles, const uint2* ranges,
                          const unsigned* vals, const ProjBuffers& pb, const StepParams* sp, Control* ctl,
                          float* image, float* T, unsigned* last, unsigned* gp, float4* ckpt, int* chunk_tile,
                          cudaStream_t s) {
  if (n_tiles <= 0) return;
  k_blend_forward<<<(unsigned)n_tiles, kTilePix, 0, s>>>(views, n_views, ranges, vals, pb, sp, ctl, image, T, last,
                                                          gp, ckpt, chunk_tile);
}

// ---------------------------------------------------------------------------------------------
// K8
// ---------------------------------------------------------------------------------------------
constexpr int kBwdWarps = 8;

struct BwdWarpSmem {
  float4 a[kTilePix];   // (dL/dC r, g, b, bits: pixel index | (entries of this chunk it reaches) << 8)
  float4 b[kTilePix];   // (rendered C r, g, b incl. background, 0)
  float4 c[kTilePix];   // checkpoint (T, colour in front) at the chunk start
};

__global__ void __launch_bounds__(kBwdWarps * 32) k_blend_backward(
    const ViewDev* __restrict__ views, int n_views, long long n_tiles, const uint2* __restrict__ ranges,
    const unsigned* __restrict__ vals, const ProjBuffers pb, Control* __restrict__ ctl,
    const float* __restrict__ image, const unsigned* __restrict__ last_in, const float* __restrict__ dimage,
    const float4* __restrict__ ckpt, const int* __restrict__ chunk_tile, float4* __restrict__ ginst) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  BwdWarpSmem& S = reinterpret_cast<BwdWarpSmem*>(smem_raw)[warp];
  if (ctl->overflow) return;
  const unsigned long long M = ctl->m_total;
  const long long n_ids = (long long)(M >> 5) + n_tiles + 1;
  const unsigned lt = (1u << lane) - 1u;

  for (;;) {
    long long id = 0;
    if (lane == 0) id = (long long)atomicAdd(&ctl->bwd_work, 1u);
    id = __shfl_sync(0xffffffffu, id, 0);
    if (id >= n_ids) break;
    const int tp1 = chunk_tile[id];
    if (tp1 == 0) continue;
    const long long t = tp1 - 1;
    const uint2 rg = ranges[t];
    const unsigned start = rg.x;
    const int L = (int)(rg.y - rg.x);
    const int k = (int)(id - chunk_base(start, t));
    const int base = k * kChunk;
    const int cnt = min(kChunk, L - base);
    const int v = view_of_tile(views, n_views, t);
    const ViewDev& V = views[v];
    const long long local = t - V.tile_base;
    const int tx = (int)(local % V.gx), ty = (int)(local / V.gx);

    // Lane l's Gaussian and the slot of its instance gradient.
    float4 xy = make_float4(0.f, 0.f, 0.f, 0.f), co = xy, col = xy;
    unsigned long long e = 0;
    if (lane < cnt) {
      const unsigned rec = vals[start + base + lane];
      xy = pb.xyo[rec];
      co = pb.conic[rec];
      col = pb.rgb[rec];
      const uint2 rc = pb.rect[rec];
      const unsigned x0 = rc.x & 0xffffu, x1 = rc.x >> 16, y0 = rc.y & 0xffffu;
      e = (unsigned long long)pb.offsets[rec] + (unsigned long long)((ty - (int)y0) * (int)(x1 - x0) + (tx - (int)x0));
    }

    // Stage the pixels of the tile that reach this chunk (last contributor beyond its start).
    const long long HW = (long long)V.W * V.H;
    const float* img = image + 3 * V.pix_base;
    const float* dimg = dimage + 3 * V.pix_base;
    int n_act = 0;
    for (int p0 = 0; p0 < kTilePix; p0 += 32) {
      const int p = p0 + lane;
      const int px = tx * kTile + (p & (kTile - 1)), py = ty * kTile + p / kTile;
      const bool inside = px < V.W && py < V.H;
      const long long pix = (long long)py * V.W + px;
      const unsigned lp = inside ? last_in[V.pix_base + pix] : 0u;
      const bool act = lp > (unsigned)base;
      const unsigned ball = __ballot_sync(0xffffffffu, act);
      if (act) {
        const int slot = n_act + __popc(ball & lt);
        const unsigned reach = min(lp - (unsigned)base, (unsigned)kChunk);
        S.a[slot] = make_float4(dimg[pix], dimg[HW + pix], dimg[2 * HW + pix],
                                __uint_as_float((unsigned)p | (reach << 8)));
        S.b[slot] = make_float4(img[pix], img[HW + pix], img[2 * HW + pix], 0.f);
        S.c[slot] = k == 0 ? make_float4(1.f, 0.f, 0.f, 0.f) : ckpt[(chunk_base(start, t) + k) * kTilePix + p];
      }
      n_act += __popc(ball);
    }
    __syncwarp();

    float g_u = 0.f, g_v = 0.f, g_a = 0.f, g_b = 0.f, g_c = 0.f, g_o = 0.f, g_r = 0.f, g_g = 0.f, g_bl = 0.f;
    float T = 1.f, F0 = 0.f, F1 = 0.f, F2 = 0.f;  // state of the pixel this lane holds
    const float A2 = co.x, B2 = co.y, C2 = co.z;   // pre-scaled conic (-a/2, -b, -c/2)
    const float opac = xy.z;
    for (int s = 0; s < n_act + kChunk - 1; ++s) {
      // Shift the pipeline by one lane; lane 0 takes the next pixel's checkpoint.
      float iT = __shfl_up_sync(0xffffffffu, T, 1);
      float i0 = __shfl_up_sync(0xffffffffu, F0, 1);
      float i1 = __shfl_up_sync(0xffffffffu, F1, 1);
      float i2 = __shfl_up_sync(0xffffffffu, F2, 1);
      const int q = s - lane;
      if (lane == 0 && q < n_act) {
        const float4 c = S.c[q];
        iT = c.x;
        i0 = c.y;
        i1 = c.z;
        i2 = c.w;
      }
      T = iT;
      F0 = i0;
      F1 = i1;
      F2 = i2;
      if (q < 0 || q >= n_act || lane >= cnt) continue;
      const float4 pa = S.a[q];
      const unsigned bits = __float_as_uint(pa.w);
      const int p = (int)(bits & 0xffu);
      if (lane >= (int)(bits >> 8)) continue;  // this pixel stopped before Gaussian `lane`
      const float pxf = (float)(tx * kTile + (p & (kTile - 1)));
      const float pyf = (float)(ty * kTile + p / kTile);
      const float dx = __fsub_rn(xy.x, pxf), dy = __fsub_rn(xy.y, pyf);
      const float power = splat_power(A2, B2, C2, dx, dy);
      if (power > 0.f) continue;
      const float G = splat_exp(power);
      const float oG = __fmul_rn(opac, G);
      const float alpha = fminf(kAlphaMax, oG);
      if (alpha < kAlphaMin) continue;
      const float w = __fmul_rn(alpha, T);
      const float n0 = __fmaf_rn(col.x, w, F0);
      const float n1 = __fmaf_rn(col.y, w, F1);
      const float n2 = __fmaf_rn(col.z, w, F2);
      const float4 pbv = S.b[q];
      // colour behind this Gaussian (later Gaussians plus background): C_pixel - front incl.
      const float inv = __fdividef(1.f, 1.f - alpha);
      const float dalpha = pa.x * (col.x * T - (pbv.x - n0) * inv) + pa.y * (col.y * T - (pbv.y - n1) * inv) +
                           pa.z * (col.z * T - (pbv.z - n2) * inv);
      g_r += w * pa.x;
      g_g += w * pa.y;
      g_bl += w * pa.z;
      if (!(oG > kAlphaMax)) {
        g_o += dalpha * G;
        const float dpow = dalpha * alpha;
        g_u += dpow * (2.f * A2 * dx + B2 * dy);
        g_v += dpow * (B2 * dx + 2.f * C2 * dy);
        g_a += dpow * (-0.5f * dx * dx);
        g_b += dpow * (-dx * dy);
        g_c += dpow * (-0.5f * dy * dy);
      }
      T = __fmul_rn(T, __fsub_rn(1.f, alpha));
      F0 = n0;
      F1 = n1;
      F2 = n2;
    }
    if (lane < cnt) {
      ginst[3 * e] = make_float4(g_u, g_v, g_a, g_b);
      ginst[3 * e + 1] = make_float4(g_c, g_o, g_r, g_g);
      ginst[3 * e + 2] = make_float4(g_bl, 0.f, 0.f, 0.f);
    }
    __syncwarp();
  }
}

void init_blend_attributes() {
  cudaFuncSetAttribute(k_blend_backward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)(sizeof(BwdWarpSmem) * kBwdWarps));
}

void launch_blend_backward(const ViewDev* views, int n_views, long long n_tiles, const uint2* ranges,
                           const unsigned* vals, const ProjBuffers& pb, Control* ctl, const float* image,
                           const unsigned* last, const float* dimage, const float4* ckpt, const int* chunk_tile,
                           float4* ginst, int num_sms, cudaStream_t s) {
  const int smem = (int)(sizeof(BwdWarpSmem) * kBwdWarps);
  k_blend_backward<<<num_sms * 2, kBwdWarps * 32, smem, s>>>(views, n_views, n_tiles, ranges, vals, pb, ctl, image,
                                                              last, dimage, ckpt, chunk_tile, ginst);
}

}  // namespace gs
