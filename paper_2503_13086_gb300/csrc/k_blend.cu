// k_blend.cu -- K6 (front-to-back alpha blending, Eq. 2) and K8 (its splatting-parallel
// backward, Sec. IV-D), sm_103a.
//
// Both are templates over the tile shape TW x TH (a multiple of the 8 x 4 warp block, at most 256
// pixels) and K6 over the staged batch; the autotuner of the session picks the instance.
//
// K6: persistent CTAs of TW x TH threads (one pixel per thread, each warp an 8 x 4 pixel block)
// take tiles longest-list first, so the few very long tiles do not end up as the tail of the
// launch.  A tile's sorted Gaussians come through shared memory as jobs of up to BATCH entries, two
// jobs resident at a time: the warp that finishes a job first stages the next one (the next batch
// of the same tile while a warp of it still blends, else the next tile) with asynchronous copies,
// and publishes it on an mbarrier, so staging overlaps the other warps' walk and a fast warp can run
// a job ahead of the tile's slowest block instead of waiting for it at a CTA barrier.  Jobs are
// walked in chunks of 32.  A warp skips a Gaussian outright when the bounding box of its 1/255 cutoff
// ellipse misses the warp's block (warp-uniform); for the others each pixel tests its exponent
// against -ln(255 opacity) and only then evaluates exp, alpha, the early stop and the blending.  (A
// separate, pipelined candidate pass before the sequential walk computed the exponent twice for
// every candidate: equal on sparse views, 6-10 % slower on dense ones.)
// Per (pixel, chunk) K6 stores the transmittance and colour at the chunk start and a 32-bit mask
// of the Gaussians actually blended; a tile gets no more batches once every warp's pixels stopped.
// When the last of a tile's warps leaves it, the tile is flagged complete (a GPU-scope release), so
// the loss that follows can start on the image blocks over finished tiles while K6 still runs.
//
// K8: gradient accumulation per Gaussian (the splatting-based parallelism the paper adopts from
// Taming 3DGS to remove the serialized per-pixel atomics of the original backward).  Work item =
// (tile, 32-entry chunk), one warp each, taken from a global counter.  The warp compacts the
// tile's pixels whose mask for this chunk is non-empty and takes them 128 at a time, four per
// lane held as the halves of two packed FP32x2 values (sm_100's FFMA2 / FMUL2 / FADD2 work on both
// halves at once).  First each lane restarts its pixels from the checkpoint.  The lanes then walk the union
// of their pixels' blended Gaussians in list order, three Gaussians at a time: a lane computes its
// pixels' nine gradient terms for each (a pixel that did not blend it takes G = 0, which leaves
// its state unchanged and its terms zero) and advances transmittance and front colour exactly as
// the forward did (the colour behind a Gaussian is the rendered colour minus the colour
// accumulated in front of it); it adds its pixels' terms, and the 27 terms are summed over the
// lanes through shared memory in a fixed order and added to the Gaussians' running sums.  A round's pixels share
// few Gaussians (about 9 of 32), each blended by many of them, so this keeps more lanes busy than
// one lane per Gaussian.  No atomics: the gradient is deterministic, and each instance's gradient
// is written once, to its own slot.
#include "gs_device.cuh"
#include "gs_engine.h"

namespace gs {

namespace {

// Pixel layout of a TW x TH tile: warp w covers the 8 x 4 block (w % BX, w / BX) of the tile,
// lane l its pixel (l % 8, l / 8).  K6 and K8 share this mapping.
template <int TW, int TH>
struct Shape {
  static constexpr int kPix = TW * TH;
  static constexpr int kWarps = kPix / 32;
  static constexpr int kBX = TW / 8;
  static constexpr int kBY = TH / 4;
  static_assert(TW % 8 == 0 && TH % 4 == 0 && kPix >= 32 && kPix <= kMaxTilePix, "unsupported tile shape");
  static_assert(kWarps <= 8, "the per-entry warp-block mask is 8 bits");
  __device__ static __forceinline__ void slot_xy(int s, int& ox, int& oy) {
    const int w = s >> 5, l = s & 31;
    ox = ((w % kBX) << 3) + (l & 7);
    oy = ((w / kBX) << 2) + (l >> 3);
  }
};

__device__ __forceinline__ int view_of_tile(const ViewDev* __restrict__ views, int n_views, long long t) {
  int v = 0;
  while (v + 1 < n_views && views[v + 1].tile_base <= t) ++v;
  return v;
}

// Chunk id of a tile's chunk 0: unique over tiles and < (instances / 32) + tiles + 1.
__device__ __forceinline__ long long chunk_base(unsigned start, long long tile) {
  return (long long)(start >> 5) + tile;
}
}  // namespace

// ---------------------------------------------------------------------------------------------
// Tile order for K6: buckets by floor(log2(list length)), longest bucket first (one CTA).
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_tile_order(const uint2* __restrict__ ranges, long long n_tiles,
                                                     int* __restrict__ order, const Control* __restrict__ ctl) {
  dep_wait();
  dep_release();
  __shared__ unsigned s_cnt[32];
  __shared__ unsigned s_base[32];
  if (ctl->overflow) return;
  if (threadIdx.x < 32) s_cnt[threadIdx.x] = 0u;
  __syncthreads();
  for (long long t = threadIdx.x; t < n_tiles; t += blockDim.x) {
    const unsigned L = ranges[t].y - ranges[t].x;
    const int b = L ? 32 - __clz(L) : 0;  // 0 = empty, else 1 + floor(log2 L), at most 31
    atomicAdd(&s_cnt[min(b, 31)], 1u);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned run = 0;
    for (int b = 31; b >= 0; --b) {
      s_base[b] = run;
      run += s_cnt[b];
    }
  }
  __syncthreads();
  for (long long t = threadIdx.x; t < n_tiles; t += blockDim.x) {
    const unsigned L = ranges[t].y - ranges[t].x;
    const int b = L ? 32 - __clz(L) : 0;
    order[atomicAdd(&s_base[min(b, 31)], 1u)] = (int)t;
  }
}

// ---------------------------------------------------------------------------------------------
// K6
// ---------------------------------------------------------------------------------------------
// Work flows through the CTA as jobs: a job is one staged batch (up to BATCH sorted entries) of one
// tile, and kFwdBufs jobs are in shared memory at a time.  Each warp walks every job in order (its 8 x 4
// block of the job's tile); the warp that finishes job j first stages job j + 1 into the other
// buffer of job j + 1 - kFwdBufs once every warp is through that job -- the next batch of the same tile while any warp of it still blends, else the first batch
// of the next tile in the longest-first order -- so staging overlaps the slower warps' walk and a
// warp waits only when it has caught up with the staging, not for the tile's slowest block.  A job
// is published by an mbarrier (`full`, 32 arrivals: the staging warp's lanes) and released by
// another (`empty`, one arrival per warp).  Every wait is bounded: a wait that gives up sets
// kErrTimeout and its warp leaves (the host reports GS_ERR_TIMEOUT; the outputs are then unspecified).
namespace {
constexpr int kFwdBufs = 2;  // jobs in shared memory at a time (3 measured 112 against 107 us)

struct FwdJob {
  long long t;      // global tile
  unsigned start;   // first entry of the tile's list
  int L;            // list length
  int b0;           // first entry of this batch
  int seq;          // tile sequence number within the CTA
  int end;          // 1: no more work
};

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
// 16-byte asynchronous copy global -> shared (both 16-byte aligned)
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(smem_u32(bar)) : "memory");
}
// Bounded wait for the phase of the given parity to complete; false when it gave up.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, unsigned limit) {
  for (unsigned k = 0; k < limit; ++k) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}
}  // namespace

template <int TW, int TH, int BATCH>
__global__ void __launch_bounds__(TW * TH, 1024 / (TW * TH)) k_blend_forward(
    const ViewDev* __restrict__ views, int n_views, long long n_tiles, const uint2* __restrict__ ranges,
    const unsigned* __restrict__ vals, const ProjBuffers pb, const StepParams* __restrict__ sp,
    Control* __restrict__ ctl, const int* __restrict__ order, float* __restrict__ image, float* __restrict__ Tout,
    unsigned* __restrict__ last_out, unsigned* __restrict__ gp_out, float4* __restrict__ ckpt,
    unsigned* __restrict__ cmask, int* __restrict__ chunk_tile, int* __restrict__ tile_chunks,
    unsigned* __restrict__ tile_done) {
  dep_wait();
  dep_release();
  using S = Shape<TW, TH>;
  constexpr int kPix = S::kPix;
  static_assert(BATCH % kChunk == 0, "batches hold whole chunks");
  __shared__ float4 s_xyo[kFwdBufs][BATCH];
  __shared__ float4 s_con[kFwdBufs][BATCH];
  __shared__ float4 s_rgb[kFwdBufs][BATCH];
  __shared__ unsigned char s_bm[kFwdBufs][BATCH];  // per entry: the warp blocks its cutoff box reaches
  __shared__ FwdJob s_job[kFwdBufs];
  __shared__ __align__(8) unsigned long long s_full[kFwdBufs], s_empty[kFwdBufs];
  __shared__ int s_next;     // the next job to be staged (the stager of job j + 1 is elected on it)
  __shared__ int s_live[kFwdBufs];  // per tile (sequence mod kFwdBufs): warps with pixels still blending
  __shared__ unsigned s_fin[4];     // per tile (sequence mod 4): warps that left it (at most 3 tiles open)
  // the stager's progress through the tiles (only the warp staging the next job reads or writes it;
  // jobs are staged one after another)
  __shared__ long long s_cur_t;
  __shared__ unsigned s_cur_start;
  __shared__ int s_cur_L, s_cur_nb, s_cur_seq;
  if (ctl->overflow) return;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const float bg0 = sp->bg[0], bg1 = sp->bg[1], bg2 = sp->bg[2];
  unsigned my_pairs = 0, my_blend = 0, my_gpn = 0, my_gpsq = 0;  // this thread's pixels (fit 32 bits)

  // Stage job j (one warp): decide what it is, then load its entries into buffer j % kFwdBufs.
  auto stage = [&](int j) -> bool {
    const int buf = j % kFwdBufs;
    if (j >= kFwdBufs && !mbar_wait(&s_empty[buf], ((j - kFwdBufs) / kFwdBufs) & 1, kSpinLimit)) return false;
    if (lane == 0) {
      FwdJob jb;
      jb.end = 0;
      if (s_cur_seq >= 0 && s_cur_nb * BATCH < s_cur_L && s_live[s_cur_seq % kFwdBufs] > 0) {
        jb.t = s_cur_t;  // the tile's next batch
        jb.start = s_cur_start;
        jb.L = s_cur_L;
        jb.b0 = s_cur_nb * BATCH;
        jb.seq = s_cur_seq;
        ++s_cur_nb;
      } else {
        // chunks whose masks every pixel of the finished tile received (the backward reads those)
        if (s_cur_seq >= 0)
          tile_chunks[s_cur_t] = min((s_cur_L + kChunk - 1) / kChunk, s_cur_nb * (BATCH / kChunk));
        const int item = (int)atomicAdd(&ctl->fwd_work, 1u);
        if (item >= n_tiles) {
          jb.end = 1;
          jb.t = 0;
          jb.start = 0;
          jb.L = 0;
          jb.b0 = 0;
          jb.seq = s_cur_seq + 1;
        } else {
          const long long t = order[item];
          const uint2 rg = ranges[t];
          s_cur_t = t;
          s_cur_start = rg.x;
          s_cur_L = (int)(rg.y - rg.x);
          s_cur_nb = 1;
          s_cur_seq += 1;
          s_live[s_cur_seq % kFwdBufs] = S::kWarps;
          jb.t = t;
          jb.start = rg.x;
          jb.L = s_cur_L;
          jb.b0 = 0;
          jb.seq = s_cur_seq;
        }
      }
      s_job[buf] = jb;
    }
    __syncwarp();
    const FwdJob jb = s_job[buf];
    if (!jb.end) {
      if (jb.b0 == 0) {  // a new tile: map its chunks back to it for the backward
        const long long cb = chunk_base(jb.start, jb.t);
        for (int k = lane; k < (jb.L + kChunk - 1) / kChunk; k += 32) chunk_tile[cb + k] = (int)(jb.t + 1);
      }
      const int v = view_of_tile(views, n_views, jb.t);
      const ViewDev& V = views[v];
      const long long local = jb.t - V.tile_base;
      const float tx0 = (float)((int)(local % V.gx) * TW), ty0 = (float)((int)(local / V.gx) * TH);
      const int nb = min(BATCH, jb.L - jb.b0);
      // all of the lane's record indices in flight at once, then its records copied straight into
      // shared memory by asynchronous 16-byte copies (no registers held), then the block masks
      constexpr int kPer = BATCH / 32;
      unsigned recs[kPer];
#pragma unroll
      for (int k = 0; k < kPer; ++k) {
        const int jj = lane + 32 * k;
        recs[k] = jj < nb ? __ldg(vals + jb.start + jb.b0 + jj) : 0u;
      }
#pragma unroll
      for (int k = 0; k < kPer; ++k) {
        const int jj = lane + 32 * k;
        if (jj < nb) {
          cp_async16(&s_xyo[buf][jj], pb.xyo + recs[k]);
          cp_async16(&s_con[buf][jj], pb.conic + recs[k]);
          cp_async16(&s_rgb[buf][jj], pb.rgb + recs[k]);
        }
      }
      asm volatile("cp.async.wait_all;" ::: "memory");
#pragma unroll
      for (int k = 0; k < kPer; ++k) {
        const int jj = lane + 32 * k;
        if (jj >= nb) break;
        const float4 xy = s_xyo[buf][jj];
        // which 8 x 4 warp blocks (warp w at (8 (w % BX), 4 (w / BX))) the cutoff box of this
        // Gaussian reaches; block centres are 3.5 / 1.5 px from their edge pixels
        unsigned xm = 0u, ym = 0u;
#pragma unroll
        for (int bx = 0; bx < S::kBX; ++bx)
          if (fabsf(xy.x - (tx0 + 8.f * bx + 3.5f)) <= xy.z + 3.5f) xm |= 1u << bx;
#pragma unroll
        for (int by = 0; by < S::kBY; ++by)
          if (fabsf(xy.y - (ty0 + 4.f * by + 1.5f)) <= xy.w + 1.5f) ym |= 1u << by;
        unsigned bm = 0u;
#pragma unroll
        for (int by = 0; by < S::kBY; ++by)
          if (ym & (1u << by)) bm |= xm << (S::kBX * by);
        s_bm[buf][jj] = (unsigned char)bm;
      }
    }
    mbar_arrive(&s_full[buf]);  // every lane: its own writes are published with it
    return true;
  };

  if (tid == 0) {
    for (int b = 0; b < kFwdBufs; ++b) {
      mbar_init(&s_full[b], 32);
      mbar_init(&s_empty[b], S::kWarps);
    }
    s_next = 1;
    s_cur_seq = -1;
    s_cur_nb = 0;
    s_cur_L = 0;
    for (int b = 0; b < kFwdBufs; ++b) s_live[b] = 0;
    for (int b = 0; b < 4; ++b) s_fin[b] = 0u;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  bool ok = warp != 0 || stage(0);

  // this thread's pixel of the current tile
  int my_seq = -1;
  long long my_t = 0;
  long long pix_base = 0;
  int px = 0, py = 0, Wv = 0;
  long long HWv = 0, cb = 0;
  bool inside = false, done = true, counted = true;
  float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
  unsigned last = 0u, gp = 0u, neval = 0u;
  float pxf = 0.f, pyf = 0.f;
  // (warp-uniform: every lane of the warp leaves the tile at the same job)
  auto finish_tile = [&]() {
    if (my_seq < 0) return;
    if (inside) {
      const long long pix = (long long)py * Wv + px;
      float* img = image + 3 * pix_base;
      img[pix] = C0 + T * bg0;
      img[HWv + pix] = C1 + T * bg1;
      img[2 * HWv + pix] = C2 + T * bg2;
      const long long gpix = pix_base + pix;
      if (Tout) Tout[gpix] = T;
      last_out[gpix] = last;
      if (gp_out) gp_out[gpix] = gp;
      my_pairs += neval;
      my_blend += gp;
      if (gp) {
        my_gpn += 1;
        my_gpsq += gp * gp;
      }
    }
    // this warp's pixels of the tile are final.  The warp barrier orders its lanes' writes before
    // lane 0's CTA-scope release on the tile's arrival count; the last warp to arrive acquires them
    // all and publishes the tile with one GPU-scope release, so a reader that acquires the flag sees
    // every pixel of the tile (the loss forward starts a block once the tiles under it are flagged).
    // Job j + 1 is staged only once every warp is through job j - 1, so the warps that have not left
    // a tile are on the tiles of three consecutive jobs at most: four counters are never shared.
    __syncwarp();
    if (lane == 0) {
      unsigned* fin = &s_fin[my_seq & 3];
      unsigned old;
      asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], 1;" : "=r"(old) : "r"(smem_u32(fin)) : "memory");
      if (old == (unsigned)(S::kWarps - 1)) {
        *fin = 0u;
        red_release_add_u32(tile_done + my_t, 1u);
      }
    }
  };

  for (int j = 0; ok; ++j) {
    const int buf = j % kFwdBufs;
    if (!mbar_wait(&s_full[buf], (j / kFwdBufs) & 1, kSpinLimit)) {
      ok = false;
      break;
    }
    const FwdJob jb = s_job[buf];
    if (jb.seq != my_seq) {  // a new tile (or the end)
      finish_tile();
      if (jb.end) break;
      my_seq = jb.seq;
      my_t = jb.t;
      const int v = view_of_tile(views, n_views, jb.t);
      const ViewDev& V = views[v];
      const long long local = jb.t - V.tile_base;
      const int tx = (int)(local % V.gx), ty = (int)(local / V.gx);
      int ox, oy;
      S::slot_xy(tid, ox, oy);
      px = tx * TW + ox;
      py = ty * TH + oy;
      Wv = V.W;
      HWv = (long long)V.W * V.H;
      pix_base = V.pix_base;
      inside = px < V.W && py < V.H;
      pxf = (float)px;
      pyf = (float)py;
      cb = chunk_base(jb.start, jb.t);
      T = 1.f;
      C0 = C1 = C2 = 0.f;
      last = gp = 0u;
      neval = (unsigned)jb.L;
      done = !inside;
      counted = false;
    }
    // walk this job's chunks (a warp whose pixels have all stopped still records empty masks)
    const int nb = min(BATCH, jb.L - jb.b0);
    for (int c0 = 0; c0 < nb; c0 += kChunk) {
      const int jg0 = jb.b0 + c0;
      const long long chunk = cb + (jg0 >> 5);
      const int ce = min(kChunk, nb - c0);
      // entries of this chunk whose cutoff box reaches this warp's block (warp-uniform)
      const unsigned rel = __ballot_sync(0xffffffffu, lane < ce && ((s_bm[buf][c0 + lane] >> warp) & 1u));
      if (done) {
        cmask[chunk * kPix + tid] = 0u;
        continue;
      }
      if (jg0 > 0) ckpt[chunk * kPix + tid] = make_float4(T, C0, C1, C2);
      unsigned cand = rel;
      unsigned mask = 0u;
      while (cand) {
        const int q = __ffs(cand) - 1;
        cand &= cand - 1u;
        const float4 xy = s_xyo[buf][c0 + q];
        const float4 co = s_con[buf][c0 + q];
        const float power = splat_power(co.x, co.y, co.z, __fsub_rn(xy.x, pxf), __fsub_rn(xy.y, pyf));
        if (power > 0.f || !(power >= co.w)) continue;
        const float4 c = s_rgb[buf][c0 + q];
        const float alpha = fminf(kAlphaMax, __fmul_rn(c.w, splat_exp(power)));
        if (alpha < kAlphaMin) continue;
        const float testT = __fmul_rn(T, __fsub_rn(1.f, alpha));
        if (testT < kTransMin) {
          done = true;
          neval = (unsigned)(jg0 + q) + 1u;
          break;
        }
        const float w = __fmul_rn(alpha, T);
        C0 = __fmaf_rn(c.x, w, C0);
        C1 = __fmaf_rn(c.y, w, C1);
        C2 = __fmaf_rn(c.z, w, C2);
        T = testT;
        last = (unsigned)(jg0 + q) + 1u;
        ++gp;
        mask |= 1u << q;
      }
      cmask[chunk * kPix + tid] = mask;
    }
    // this warp's pixels have all stopped: the stager need not stage more of the tile for it
    if (!counted && __all_sync(0xffffffffu, done)) {
      counted = true;
      if (lane == 0) atomicSub(&s_live[my_seq % kFwdBufs], 1);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&s_empty[buf]);
    // the first warp to finish job j stages job j + 1
    int mine = 0;
    if (lane == 0) mine = atomicCAS(&s_next, j + 1, j + 2) == j + 1;
    if (__shfl_sync(0xffffffffu, mine, 0) && !stage(j + 1)) ok = false;
  }
  if (!ok && lane == 0) atomicOr(&ctl->error, kErrTimeout);
  // Gaussian-pixel pairs by definition: entries evaluated per pixel up to its termination.
  unsigned long long sp_ = my_pairs, sb = my_blend, sn = my_gpn, sq = my_gpsq;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sp_ += __shfl_down_sync(0xffffffffu, sp_, o);
    sb += __shfl_down_sync(0xffffffffu, sb, o);
    sn += __shfl_down_sync(0xffffffffu, sn, o);
    sq += __shfl_down_sync(0xffffffffu, sq, o);
  }
  if (lane == 0) {
    if (sp_) atomicAdd(&ctl->pairs, sp_);
    if (sb) atomicAdd(&ctl->blended, sb);
    if (sn) {
      atomicAdd(&ctl->gp_pixels, sn);
      atomicAdd(&ctl->gp_sq, sq);
    }
    red_release_add_u32(&ctl->fwd_done, 1u);  // after this warp's counters (the loss's last CTA waits)
  }
}

void launch_tile_order(const uint2* ranges, long long n_tiles, int* order, const Control* ctl, cudaStream_t s) {
  if (n_tiles <= 0) return;
  launch_dep(k_tile_order, dim3(1), dim3(1024), 0, s, ranges, n_tiles, order, ctl);
}

namespace {
// Resident CTAs per SM of one K6 instance (persistent grid = that x SMs), set at start-up.
template <int TW, int TH, int BATCH>
int& fwd_occupancy() {
  static int occ = 0;
  return occ;
}

template <int TW, int TH, int BATCH>
void init_forward_instance() {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_blend_forward<TW, TH, BATCH>, TW * TH, 0) != cudaSuccess) {
    cudaGetLastError();
    occ = 0;
  }
  fwd_occupancy<TW, TH, BATCH>() = occ > 0 ? occ : 1;
}

// Persistent grid of one K6 instance: every resident CTA, at most one per tile.
template <int TW, int TH, int BATCH>
long long forward_grid(long long n_tiles, int num_sms) {
  long long grid = (long long)num_sms * fwd_occupancy<TW, TH, BATCH>();
  return grid > n_tiles ? n_tiles : grid;
}

template <int TW, int TH, int BATCH>
void launch_forward_instance(const ViewDev* views, int n_views, long long n_tiles, const uint2* ranges,
                             const unsigned* vals, const ProjBuffers& pb, const StepParams* sp, Control* ctl,
                             const int* order, float* image, float* T, unsigned* last, unsigned* gp, float4* ckpt,
                             unsigned* cmask, int* chunk_tile, int* tile_chunks, unsigned* tile_done, int num_sms,
                             cudaStream_t s) {
  launch_dep(k_blend_forward<TW, TH, BATCH>, dim3((unsigned)forward_grid<TW, TH, BATCH>(n_tiles, num_sms)),
      dim3(TW * TH), 0, s, views, n_views, n_tiles, ranges, vals, pb, sp, ctl, order, image, T, last, gp, ckpt, cmask,
      chunk_tile, tile_chunks, tile_done);
}
}  // namespace

// The compiled (tile shape, batch) instances; the first is the default.
#define GS_TILINGS(X) X(16, 16, 256) X(16, 16, 128) X(16, 8, 256) X(16, 8, 128) X(8, 8, 128) X(8, 8, 64) X(32, 8, 256)

int tiling_candidates(Tiling* out, int cap) {
  int n = 0;
#define GS_LIST(W, H, B)            \
  if (n < cap && out) out[n] = Tiling{W, H, B}; \
  ++n;
  GS_TILINGS(GS_LIST)
#undef GS_LIST
  return n;
}

bool tiling_supported(const Tiling& t) {
#define GS_SUP(W, H, B) \
  if (t.tw == W && t.th == H && t.batch == B) return true;
  GS_TILINGS(GS_SUP)
#undef GS_SUP
  return false;
}

void launch_blend_forward(const Tiling& tl, const ViewDev* views, int n_views, long long n_tiles, const uint2* ranges,
                          const unsigned* vals, const ProjBuffers& pb, const StepParams* sp, Control* ctl,
                          const int* order, float* image, float* T, unsigned* last, unsigned* gp, float4* ckpt,
                          unsigned* cmask, int* chunk_tile, int* tile_chunks, unsigned* tile_done, int num_sms,
                          cudaStream_t s) {
  if (n_tiles <= 0) return;
#define GS_FWD(W, H, B)                                                                                              \
  if (tl.tw == W && tl.th == H && tl.batch == B) {                                                                  \
    launch_forward_instance<W, H, B>(views, n_views, n_tiles, ranges, vals, pb, sp, ctl, order, image, T, last, gp, \
                                     ckpt, cmask, chunk_tile, tile_chunks, tile_done, num_sms, s);                \
    return;                                                                                                        \
  }
  GS_TILINGS(GS_FWD)
#undef GS_FWD
}

long long forward_warps(const Tiling& tl, long long n_tiles, int num_sms) {
  if (n_tiles <= 0) return 0;
#define GS_FWDW(W, H, B) \
  if (tl.tw == W && tl.th == H && tl.batch == B) return forward_grid<W, H, B>(n_tiles, num_sms) * (W * H / 32);
  GS_TILINGS(GS_FWDW)
#undef GS_FWDW
  return 0;
}

// ---------------------------------------------------------------------------------------------
// K8
// ---------------------------------------------------------------------------------------------
constexpr int kBwdWarps = 4;
constexpr int kGroup = 3;  // Gaussians whose gradient terms are summed together (3 x 9 <= 32 lanes)
constexpr int kBwdPairs = 2;  // packed pixel pairs per lane (4 pixels, 128 per round)

template <int PIX>
struct BwdWarp {
  float4 a[kChunk], b[kChunk], c[kChunk];  // the chunk's Gaussians (records A, B, C)
  uint2 act[PIX];                          // compacted (slot, mask) of the pixels to visit
  float red[kGroup * 9][36];               // per term of a group of 3 Gaussians: the 32 lanes' values
                                           // (rows padded to 16-byte multiples for vector reads)
  float acc[kChunk][9];                    // per Gaussian of the chunk: running gradient sums
};

template <int TW, int TH>
__global__ void __launch_bounds__(kBwdWarps * 32) k_blend_backward(
    const ViewDev* __restrict__ views, int n_views, long long n_tiles, const uint2* __restrict__ ranges,
    const unsigned* __restrict__ vals, const ProjBuffers pb, Control* __restrict__ ctl,
    const float* __restrict__ image, const float* __restrict__ dimage, const float4* __restrict__ ckpt,
    const unsigned* __restrict__ cmask, const int* __restrict__ chunk_tile, const int* __restrict__ tile_chunks,
    float4* __restrict__ ginst, const unsigned* __restrict__ gp, const StepParams* __restrict__ sp) {
  dep_wait();
  dep_release();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  using Sh = Shape<TW, TH>;
  constexpr int kPix = Sh::kPix;
  BwdWarp<kPix>& S = reinterpret_cast<BwdWarp<kPix>*>(smem_raw)[warp];
  if (ctl->overflow) return;
  // Eq. 9-10: dL/dG_p = lambda_load (G_p - mean) / (N std) over the N pixels with G_p > 0 (K6's
  // moments of all the step's views); it reaches alpha through the soft count, the sum of the
  // blended Gaussians' alphas.  load_a = lambda_load / (N std), load_mu = mean; off without G_p.
  float load_a = 0.f, load_mu = 0.f;
  if (gp != nullptr && sp->lambda_load > 0.f && ctl->gp_pixels > 0ull) {
    const double np = (double)ctl->gp_pixels, mean = (double)ctl->blended / np;
    const double var = (double)ctl->gp_sq / np - mean * mean;
    if (var > 0.0) {
      load_a = (float)((double)sp->lambda_load / (np * sqrt(var)));
      load_mu = (float)mean;
    }
  }
  const bool load = load_a != 0.f;
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
    const long long cid = chunk_base(start, t) + k;

    unsigned long long e = 0;
    if (lane < cnt) {
      const unsigned rec = vals[start + base + lane];
      S.a[lane] = pb.xyo[rec];
      S.b[lane] = pb.conic[rec];
      S.c[lane] = pb.rgb[rec];
      const uint2 rc = pb.rect[rec];
      const unsigned x0 = rc.x & 0xffffu, x1 = rc.x >> 16, y0 = rc.y & 0xffffu;
      e = (unsigned long long)pb.offsets[rec] + (unsigned long long)((ty - (int)y0) * (int)(x1 - x0) + (tx - (int)x0));
    }
#pragma unroll
    for (int c = 0; c < 9; ++c) S.acc[lane][c] = 0.f;
    // Chunks past tile_chunks[t] were never reached by any pixel: all gradients are zero.
    int n_act = 0;
    if (k < tile_chunks[t]) {
      // compact the pixels that blended at least one Gaussian of this chunk
#pragma unroll
      for (int r = 0; r < kPix / 32; ++r) {
        const int slot = r * 32 + lane;
        const unsigned mask = cmask[cid * kPix + slot];
        const unsigned ball = __ballot_sync(0xffffffffu, mask != 0u);
        if (mask) S.act[n_act + __popc(ball & lt)] = make_uint2((unsigned)slot, mask);
        n_act += __popc(ball);
      }
    }
    __syncwarp();
    const long long HW = (long long)V.W * V.H;
    const float* img = image + 3 * V.pix_base;
    const float* dimg = dimage + 3 * V.pix_base;
    for (int r0 = 0; r0 < n_act; r0 += 64 * kBwdPairs) {
      // this lane's pixels act[r0 + 32 h + lane], h = 0 .. 2 kBwdPairs - 1, pair p holding pixels
      // 2p (.x) and 2p + 1 (.y): dL/dC, the rendered colour, the state at the chunk start, minus
      // the pixel coordinates
      unsigned mk[2 * kBwdPairs];
      float2 d0[kBwdPairs], d1[kBwdPairs], d2[kBwdPairs], P0[kBwdPairs], P1[kBwdPairs], P2[kBwdPairs];
      float2 T[kBwdPairs], F0[kBwdPairs], F1[kBwdPairs], F2[kBwdPairs], npx[kBwdPairs], npy[kBwdPairs];
      float2 LW[kBwdPairs];  // dL/dG_p of the load term per pixel (0 without it)
      unsigned any = 0u;
#pragma unroll
      for (int pp = 0; pp < kBwdPairs; ++pp) {
        float st[2][13];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int i = r0 + 32 * (2 * pp + h) + lane;
          const uint2 pm = i < n_act ? S.act[i] : make_uint2(0u, 0u);
          mk[2 * pp + h] = pm.y;
          any |= pm.y;
          float* q = st[h];
          q[0] = q[1] = q[2] = q[3] = q[4] = q[5] = 0.f;
          q[6] = 1.f;
          q[7] = q[8] = q[9] = q[10] = q[11] = q[12] = 0.f;
          if (pm.y) {
            int ox, oy;
            Sh::slot_xy((int)pm.x, ox, oy);
            const int px = tx * TW + ox, py = ty * TH + oy;
            const long long pix = (long long)py * V.W + px;
            q[0] = dimg[pix];
            q[1] = dimg[HW + pix];
            q[2] = dimg[2 * HW + pix];
            q[3] = img[pix];
            q[4] = img[HW + pix];
            q[5] = img[2 * HW + pix];
            if (k > 0) {
              const float4 ck = ckpt[cid * kPix + pm.x];
              q[6] = ck.x;
              q[7] = ck.y;
              q[8] = ck.z;
              q[9] = ck.w;
            }
            q[10] = -(float)px;
            q[11] = -(float)py;
            if (load) q[12] = load_a * ((float)gp[V.pix_base + pix] - load_mu);
          }
        }
        d0[pp] = make_float2(st[0][0], st[1][0]);
        d1[pp] = make_float2(st[0][1], st[1][1]);
        d2[pp] = make_float2(st[0][2], st[1][2]);
        P0[pp] = make_float2(st[0][3], st[1][3]);
        P1[pp] = make_float2(st[0][4], st[1][4]);
        P2[pp] = make_float2(st[0][5], st[1][5]);
        T[pp] = make_float2(st[0][6], st[1][6]);
        F0[pp] = make_float2(st[0][7], st[1][7]);
        F1[pp] = make_float2(st[0][8], st[1][8]);
        F2[pp] = make_float2(st[0][9], st[1][9]);
        npx[pp] = make_float2(st[0][10], st[1][10]);
        npy[pp] = make_float2(st[0][11], st[1][11]);
        LW[pp] = make_float2(st[0][12], st[1][12]);
      }
      const float2 one2 = make_float2(1.f, 1.f), neg2 = make_float2(-1.f, -1.f);
      // The round's pixels walk the union of their Gaussians in list order, three at a time.  A
      // pixel that did not blend a Gaussian takes it with G = 0: alpha = 0 leaves its
      // transmittance and front colour exactly as they were and zeroes its nine terms, so the walk
      // has no per-pixel branch.  Each lane adds its pixels' terms; the 27 terms of a group are
      // then summed over the lanes through shared memory (fixed order).
      unsigned uni = __reduce_or_sync(0xffffffffu, any);
      while (uni) {
        int qs[kGroup];
        int ng = 0;
#pragma unroll
        for (int gi = 0; gi < kGroup; ++gi) {
          qs[gi] = 0;
          // the nine terms summed over this lane's pixel pairs, both halves kept apart until the end
          float2 g2[9];
#pragma unroll
          for (int j = 0; j < 9; ++j) g2[j] = make_float2(0.f, 0.f);
          if (uni) {
            const int q = __ffs(uni) - 1;
            uni &= uni - 1u;
            qs[gi] = q;
            ng = gi + 1;
            const float4 xy = S.a[q], co = S.b[q], c = S.c[q];
            const float2 A2 = make_float2(co.x, co.x), B2 = make_float2(co.y, co.y), C2 = make_float2(co.z, co.z);
            const float2 cx = make_float2(c.x, c.x), cy = make_float2(c.y, c.y), cz = make_float2(c.z, c.z);
            const float2 A2x2 = make_float2(2.f * co.x, 2.f * co.x), C2x2 = make_float2(2.f * co.z, 2.f * co.z);
#pragma unroll
            for (int pp = 0; pp < kBwdPairs; ++pp) {
              const bool ba = (mk[2 * pp] >> q) & 1u, bb = (mk[2 * pp + 1] >> q) & 1u;
              if (!(ba || bb)) continue;
              const float2 dx = __fadd2_rn(make_float2(xy.x, xy.x), npx[pp]);
              const float2 dy = __fadd2_rn(make_float2(xy.y, xy.y), npy[pp]);
              // the forward's exponent, rounding step for rounding step (splat_power)
              const float2 pw =
                  __ffma2_rn(dx, __ffma2_rn(A2, dx, __fmul2_rn(B2, dy)), __fmul2_rn(__fmul2_rn(C2, dy), dy));
              const float2 G = make_float2(ba ? splat_exp(pw.x) : 0.f, bb ? splat_exp(pw.y) : 0.f);
              const float2 oG = __fmul2_rn(make_float2(c.w, c.w), G);
              const float2 alpha = make_float2(fminf(kAlphaMax, oG.x), fminf(kAlphaMax, oG.y));
              const float2 w = __fmul2_rn(alpha, T[pp]);
              const float2 n0 = __ffma2_rn(cx, w, F0[pp]);
              const float2 n1 = __ffma2_rn(cy, w, F1[pp]);
              const float2 n2 = __ffma2_rn(cz, w, F2[pp]);
              // colour behind = rendered colour (incl. background) - colour in front incl. this one
              const float2 behind2 = __fmul2_rn(d2[pp], __ffma2_rn(n2, neg2, P2[pp]));
              const float2 DS = __ffma2_rn(d0[pp], __ffma2_rn(n0, neg2, P0[pp]),
                                           __ffma2_rn(d1[pp], __ffma2_rn(n1, neg2, P1[pp]), behind2));
              // dL/dalpha = sum_ch dL/dC_ch (c_ch T - behind_ch / (1 - alpha)); no gradient to the
              // opacity and footprint where alpha was clamped
              const float2 cd = __ffma2_rn(cx, d0[pp], __ffma2_rn(cy, d1[pp], __fmul2_rn(cz, d2[pp])));
              const float2 ninv = make_float2(-__fdividef(1.f, 1.f - alpha.x), -__fdividef(1.f, 1.f - alpha.y));
              float2 dal = __ffma2_rn(DS, ninv, __fmul2_rn(T[pp], cd));
              if (load) dal = __fadd2_rn(dal, LW[pp]);  // + dL/dG_p x d alpha / d alpha
              dal.x = oG.x > kAlphaMax ? 0.f : dal.x;
              dal.y = oG.y > kAlphaMax ? 0.f : dal.y;
              const float2 dpow = __fmul2_rn(dal, alpha);
              const float2 ex = __ffma2_rn(A2x2, dx, __fmul2_rn(B2, dy));
              const float2 ey = __ffma2_rn(B2, dx, __fmul2_rn(C2x2, dy));
              const float2 pdx = __fmul2_rn(dpow, dx), pdy = __fmul2_rn(dpow, dy);
              g2[0] = __ffma2_rn(dpow, ex, g2[0]);
              g2[1] = __ffma2_rn(dpow, ey, g2[1]);
              g2[2] = __ffma2_rn(pdx, dx, g2[2]);
              g2[3] = __ffma2_rn(pdx, dy, g2[3]);
              g2[4] = __ffma2_rn(pdy, dy, g2[4]);
              g2[5] = __ffma2_rn(dal, G, g2[5]);
              g2[6] = __ffma2_rn(w, d0[pp], g2[6]);
              g2[7] = __ffma2_rn(w, d1[pp], g2[7]);
              g2[8] = __ffma2_rn(w, d2[pp], g2[8]);
              T[pp] = __fmul2_rn(T[pp], __ffma2_rn(alpha, neg2, one2));
              F0[pp] = n0;
              F1[pp] = n1;
              F2[pp] = n2;
            }
          }
          // terms 2-4 of the conic: -1/2, -1, -1/2 times the accumulated products
          S.red[9 * gi + 0][lane] = g2[0].x + g2[0].y;
          S.red[9 * gi + 1][lane] = g2[1].x + g2[1].y;
          S.red[9 * gi + 2][lane] = -0.5f * (g2[2].x + g2[2].y);
          S.red[9 * gi + 3][lane] = -(g2[3].x + g2[3].y);
          S.red[9 * gi + 4][lane] = -0.5f * (g2[4].x + g2[4].y);
#pragma unroll
          for (int j = 5; j < 9; ++j) S.red[9 * gi + j][lane] = g2[j].x + g2[j].y;
        }
        __syncwarp();
        if (lane < 9 * ng) {
          // the term's 32 values: eight 16-byte reads, four running sums (fixed order)
          const float4* row = reinterpret_cast<const float4*>(S.red[lane]);
          float4 s4 = row[0];
#pragma unroll
          for (int k = 1; k < 8; ++k) {
            const float4 x = row[k];
            s4.x += x.x;
            s4.y += x.y;
            s4.z += x.z;
            s4.w += x.w;
          }
          const float sum = (s4.x + s4.y) + (s4.z + s4.w);
          const int gi = lane / 9;
          const int q = gi == 0 ? qs[0] : (gi == 1 ? qs[1] : qs[2]);
          S.acc[q][lane - 9 * gi] += sum;
        }
        __syncwarp();
      }
    }
    __syncwarp();
    if (lane < cnt) {
      const float* a = S.acc[lane];
      ginst[3 * e] = make_float4(a[0], a[1], a[2], a[3]);
      ginst[3 * e + 1] = make_float4(a[4], a[5], a[6], a[7]);
      ginst[3 * e + 2] = make_float4(a[8], 0.f, 0.f, 0.f);
    }
    __syncwarp();
  }
}

namespace {
template <int TW, int TH>
int& bwd_occupancy() {
  static int occ = 0;
  return occ;
}

template <int TW, int TH>
void init_backward_instance() {
  const int smem = (int)(sizeof(BwdWarp<TW * TH>) * kBwdWarps);
  cudaFuncSetAttribute(k_blend_backward<TW, TH>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_blend_backward<TW, TH>, kBwdWarps * 32, smem) !=
      cudaSuccess) {
    cudaGetLastError();
    occ = 0;
  }
  bwd_occupancy<TW, TH>() = occ > 0 ? occ : 1;
}

template <int TW, int TH>
void launch_backward_instance(const ViewDev* views, int n_views, long long n_tiles, const uint2* ranges,
                              const unsigned* vals, const ProjBuffers& pb, Control* ctl, const float* image,
                              const float* dimage, const float4* ckpt, const unsigned* cmask, const int* chunk_tile,
                              const int* tile_chunks, float4* ginst, const unsigned* gp, const StepParams* sp,
                              int num_sms, cudaStream_t s) {
  launch_dep(k_blend_backward<TW, TH>, dim3(num_sms * bwd_occupancy<TW, TH>()), dim3(kBwdWarps * 32),
      sizeof(BwdWarp<TW * TH>) * kBwdWarps, s, views, n_views, n_tiles, ranges, vals, pb, ctl, image, dimage, ckpt,
      cmask, chunk_tile, tile_chunks, ginst, gp, sp);
}
}  // namespace

void init_blend_attributes() {
#define GS_INIT(W, H, B)              \
  init_forward_instance<W, H, B>();   \
  init_backward_instance<W, H>();
  GS_TILINGS(GS_INIT)
#undef GS_INIT
}

void launch_blend_backward(const Tiling& tl, const ViewDev* views, int n_views, long long n_tiles, const uint2* ranges,
                           const unsigned* vals, const ProjBuffers& pb, Control* ctl, const float* image,
                           const float* dimage, const float4* ckpt, const unsigned* cmask, const int* chunk_tile,
                           const int* tile_chunks, float4* ginst, const unsigned* gp, const StepParams* sp,
                           int num_sms, cudaStream_t s) {
  // the backward depends on the tile shape only
#define GS_BWD(W, H, B)                                                                                          \
  if (tl.tw == W && tl.th == H) {                                                                               \
    launch_backward_instance<W, H>(views, n_views, n_tiles, ranges, vals, pb, ctl, image, dimage, ckpt, cmask, \
                                   chunk_tile, tile_chunks, ginst, gp, sp, num_sms, s);                        \
    return;                                                                                                    \
  }
  GS_TILINGS(GS_BWD)
#undef GS_BWD
}

}  // namespace gs
