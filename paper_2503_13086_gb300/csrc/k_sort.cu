// k_sort.cu -- K2 (exclusive scan of tiles touched), K3 (duplication into (tile, depth) keys),
// K4 (stable LSD radix sort, one onesweep pass per 8-bit digit) and K5 (per-tile ranges), sm_103a.
//
// These implement the tile-binning of the 3DGS rasterizer the paper builds on (Sec. III; the
// "original 3DGS" settings of Sec. V-A).  Canonical order: (global tile, fp32 depth bits,
// record index).  Instances are emitted in record order and every sort pass is stable, so the
// record index breaks depth ties.  The key holds only the depth bits that vary within the step
// (their range comes out of the scan), so a step usually needs 5 passes of 8 bits instead of 6; the
// number of passes is decided on the device and the passes always end in buffer 0.  Every count lives in device memory: no kernel here needs the
// host to know how many instances were emitted, so the whole chain can be graph-captured.
// The inter-CTA waits (decoupled look-back) spin at most kSpinLimit times, then flag
// kErrTimeout and carry on rather than hang.
#include "gs_device.cuh"
#include "gs_engine.h"

namespace gs {

namespace {
constexpr unsigned long long kScanAgg = 1ull << 62;
constexpr unsigned long long kScanPrefix = 2ull << 62;
constexpr unsigned long long kScanValMask = (1ull << 62) - 1;
constexpr unsigned kSortAgg = 1u << 30;
constexpr unsigned kSortPrefix = 2u << 30;
constexpr unsigned kSortValMask = (1u << 30) - 1;

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}
}  // namespace

// ---------------------------------------------------------------------------------------------
// K2: single-pass exclusive scan with decoupled look-back.  Tiles are taken in launch order via
// an atomic ticket, so every tile a CTA waits on belongs to a CTA that is already running.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kScanThreads) k_scan(const unsigned* __restrict__ in, unsigned* __restrict__ out,
                                                       long long n_items, unsigned long long* __restrict__ state,
                                                       Control* __restrict__ ctl, unsigned long long m_cap,
                                                       Ledger* __restrict__ ledger, const float* __restrict__ depth,
                                                       unsigned spin_limit) {
  dep_wait();
  dep_release();
  __shared__ unsigned s_tile;
  __shared__ unsigned s_warp[kScanThreads / 32];
  __shared__ unsigned long long s_excl;
  if (threadIdx.x == 0) s_tile = atomicAdd(&ctl->scan_ticket, 1u);
  __syncthreads();
  const unsigned tile = s_tile;
  const long long num_tiles = (n_items + kScanTile - 1) / kScanTile;
  const long long base = (long long)tile * kScanTile + (long long)threadIdx.x * kScanItems;
  unsigned x[kScanItems];
  if (base + kScanItems <= n_items) {
    const uint4 a = *reinterpret_cast<const uint4*>(in + base);
    const uint4 b = *reinterpret_cast<const uint4*>(in + base + 4);
    x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
    x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
  } else {
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) x[k] = (base + k < n_items) ? in[base + k] : 0u;
  }
  unsigned tsum = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) tsum += x[k];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (depth) {  // range of the depth bits of the records with instances (the sort key layout)
    unsigned dmax = 0u, dnot = 0u;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
      if (x[k]) {
        const unsigned b = __float_as_uint(depth[base + k]);
        dmax = max(dmax, b);
        dnot = max(dnot, ~b);
      }
    dmax = __reduce_max_sync(0xffffffffu, dmax);
    dnot = __reduce_max_sync(0xffffffffu, dnot);
    if (lane == 0 && (dmax | dnot)) {
      atomicMax(&ctl->dmax, dmax);
      atomicMax(&ctl->dnot, dnot);
    }
  }
  // block-wide exclusive scan of the per-thread sums
  unsigned incl = tsum;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += y;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    unsigned w = lane < kScanThreads / 32 ? s_warp[lane] : 0u;
    unsigned wi = w;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, wi, d);
      if (lane >= d) wi += y;
    }
    if (lane < kScanThreads / 32) s_warp[lane] = wi - w;  // exclusive warp offsets
    const unsigned total = __shfl_sync(0xffffffffu, wi, kScanThreads / 32 - 1);
    // decoupled look-back by the whole warp: lane l reads the status of tile j - l, so one round
    // trip covers up to 32 predecessors
    unsigned long long excl = 0;
    if (tile == 0) {
      if (lane == 0) st_relaxed_u64(&state[0], kScanPrefix | (unsigned long long)total);
    } else {
      if (lane == 0) st_relaxed_u64(&state[tile], kScanAgg | (unsigned long long)total);
      long long j = (long long)tile - 1;
      unsigned spins = 0;
      for (;;) {
        const long long idx = j - lane;
        const unsigned long long sv = idx >= 0 ? ld_relaxed_u64(&state[idx]) : kScanPrefix;
        const unsigned long long flag = sv & ~kScanValMask;
        const unsigned notready = __ballot_sync(0xffffffffu, flag == 0ull);
        const unsigned isprefix = __ballot_sync(0xffffffffu, flag == kScanPrefix);
        const unsigned stop = notready | isprefix;
        const int first = stop ? __ffs(stop) - 1 : 32;  // lanes below it hold aggregates
        const bool take = lane < first || (lane == first && ((isprefix >> lane) & 1u));
        unsigned long long v = take ? (sv & kScanValMask) : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        excl += v;
        if (first < 32 && ((isprefix >> first) & 1u)) break;
        j -= first;
        if (first < 32 && ++spins > spin_limit) {
          if (lane == 0) atomicOr(&ctl->error, kErrTimeout);
          break;
        }
      }
      if (lane == 0) st_relaxed_u64(&state[tile], kScanPrefix | (excl + total));
    }
    if (lane == 0) {
      s_excl = excl;
      if ((long long)tile == num_tiles - 1) {
        const unsigned long long m = excl + total;
        ctl->m_total = m;
        // an overflow skips this step; an earlier skipped step of the run skips it too
        if (m > m_cap || (ledger && ledger->skip)) {
          ctl->overflow = 1u;
          atomicOr(&ctl->error, kErrOverflow);
          if (ledger) {
            ledger->skip = 1u;
            if (m > ledger->m_need) ledger->m_need = m;
          }
        }
      }
    }
  }
  __syncthreads();
  unsigned run = (unsigned)s_excl + s_warp[warp] + (incl - tsum);
  if (base + kScanItems <= n_items) {
    unsigned y[kScanItems];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      y[k] = run;
      run += x[k];
    }
    *reinterpret_cast<uint4*>(out + base) = make_uint4(y[0], y[1], y[2], y[3]);
    *reinterpret_cast<uint4*>(out + base + 4) = make_uint4(y[4], y[5], y[6], y[7]);
  } else {
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      if (base + k < n_items) out[base + k] = run;
      run += x[k];
    }
  }
}

void launch_scan(const unsigned* in, unsigned* out, long long n_items, unsigned long long* state, Control* ctl,
                 unsigned long long m_cap, Ledger* ledger, cudaStream_t s, const float* depth) {
  const long long tiles = (n_items + kScanTile - 1) / kScanTile;
  launch_dep(k_scan, dim3((unsigned)tiles), dim3(kScanThreads), 0, s, in, out, n_items, state, ctl, m_cap, ledger,
      depth, kSpinLimit);
}

// ---------------------------------------------------------------------------------------------
// K3: duplication into (tile, depth) keys, one thread per instance.  First every record writes
// its index over its instances' slots of inst_rec (a record with more than kFillAlone instances is
// written by its whole warp, so one large Gaussian does not serialise a warp); then each instance reads
// its owner from there (one coalesced load) and writes its key.  Also histograms every radix digit
// for the sort (the passes whose digit lies in the depth part of the key once per record, through
// the thread of its first instance).
// ---------------------------------------------------------------------------------------------
constexpr unsigned kFillAlone = 4;  // larger records are written by their whole warp
__global__ void __launch_bounds__(256) k_fill_owner(const unsigned* __restrict__ count,
                                                    const unsigned* __restrict__ offsets, long long n_items,
                                                    unsigned* __restrict__ inst_rec, const Control* __restrict__ ctl) {
  dep_wait();
  dep_release();
  if (ctl->overflow) return;
  const int lane = threadIdx.x & 31;
  const long long rec = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned cnt = rec < n_items ? count[rec] : 0u;
  const unsigned off = cnt ? offsets[rec] : 0u;
  if (cnt <= kFillAlone) {
    for (unsigned k = 0; k < cnt; ++k) inst_rec[(unsigned long long)off + k] = (unsigned)rec;
  }
  unsigned big = __ballot_sync(0xffffffffu, cnt > kFillAlone);
  while (big) {
    const int l = __ffs(big) - 1;
    big &= big - 1u;
    const unsigned r = __shfl_sync(0xffffffffu, (unsigned)rec, l);
    const unsigned o = __shfl_sync(0xffffffffu, off, l);
    const unsigned c = __shfl_sync(0xffffffffu, cnt, l);
    for (unsigned k = lane; k < c; k += 32u) inst_rec[(unsigned long long)o + k] = r;
  }
}

__global__ void __launch_bounds__(1024) k_emit(const ProjBuffers pb, const ViewDev* __restrict__ views, int stride,
                                              unsigned long long* __restrict__ keys0, unsigned* __restrict__ vals0,
                                              unsigned long long* __restrict__ keys1, unsigned* __restrict__ vals1,
                                              const unsigned* __restrict__ inst_rec, unsigned* __restrict__ hist,
                                              int tile_bits, const Control* __restrict__ ctl) {
  dep_wait();
  dep_release();
  __shared__ unsigned s_hist[kMaxSortPasses][kSortBins];
  for (int k = threadIdx.x; k < kMaxSortPasses * kSortBins; k += blockDim.x) (&s_hist[0][0])[k] = 0u;
  __syncthreads();
  // the passes end in buffer 0: start in buffer (passes & 1)
  const KeyLayout kl = key_layout(ctl, tile_bits);
  const int passes = kl.passes;
  const int depth_passes = min(passes, kl.D / kSortBits);
  unsigned long long* __restrict__ keys = (passes & 1) ? keys1 : keys0;
  unsigned* __restrict__ vals = (passes & 1) ? vals1 : vals0;
  if (!ctl->overflow) {
    const unsigned long long M = ctl->m_total;
    for (unsigned long long e = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; e < M;
         e += (unsigned long long)gridDim.x * blockDim.x) {
      const unsigned rec = inst_rec[e];
      const unsigned k = (unsigned)(e - pb.offsets[rec]);
      const uint2 rc = pb.rect[rec];
      const unsigned db = __float_as_uint(pb.depth[rec]);
      const ViewDev& V = views[rec / (unsigned)stride];
      const unsigned x0 = rc.x & 0xffffu, x1 = rc.x >> 16, y0 = rc.y & 0xffffu;
      const unsigned w = x1 - x0;
      const unsigned ty = y0 + k / w, tx = x0 + k % w;
      const unsigned long long tile = (unsigned long long)(V.tile_base + (long long)ty * V.gx + tx);
      const unsigned long long key = (tile << kl.D) | (unsigned long long)(db - kl.dmin);
      keys[e] = key;
      vals[e] = rec;
      for (int p = depth_passes; p < passes; ++p)
        atomicAdd(&s_hist[p][(key >> (p * kSortBits)) & (kSortBins - 1)], 1u);
      if (k == 0) {  // every instance of the record has the record's depth digits
        const unsigned cnt = pb.count[rec];
        for (int p = 0; p < depth_passes; ++p)
          atomicAdd(&s_hist[p][((db - kl.dmin) >> (p * kSortBits)) & (kSortBins - 1)], cnt);
      }
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < passes * kSortBins; k += blockDim.x) {
    const unsigned c = (&s_hist[0][0])[k];
    if (c) atomicAdd(hist + k, c);
  }
}

void launch_emit(const ProjBuffers& pb, const ViewDev* views, int stride, long long n_items, unsigned long long* keys0,
                 unsigned* vals0, unsigned long long* keys1, unsigned* vals1, unsigned* inst_rec, unsigned* hist,
                 int tile_bits, long long m_cap, int num_sms, const Control* ctl, cudaStream_t s) {
  if (n_items <= 0) return;
  launch_dep(k_fill_owner, dim3((unsigned)((n_items + 255) / 256)), dim3(256), 0, s, pb.count, pb.offsets, n_items,
      inst_rec, ctl);
  // The same threads per SM either way.  Each CTA adds its shared histograms (up to 8 x 256 bins)
  // into the global ones with one atomic per non-empty bin: with few instances those flushes
  // dominate, so fewer, larger CTAs (0.42M instances: 22.6 -> 14.8 us); with many, the CTA's
  // threads contend on its shared bins instead, so more, smaller CTAs (7M instances: 0.129 ms
  // with 1024-thread CTAs, 0.108 ms with 512).
  const bool small = m_cap <= (1ll << 22);
  launch_dep(k_emit, dim3((unsigned)(num_sms * (small ? 2 : 4))), dim3(small ? 1024 : 512), 0, s, pb, views, stride,
      keys0, vals0, keys1, vals1, inst_rec, hist, tile_bits, ctl);
}

// ---------------------------------------------------------------------------------------------
// K4: one stable counting pass over an 8-bit digit (onesweep: digit offsets from the upfront
// histogram, per-CTA offsets by decoupled look-back per digit).  Within a CTA the keys are
// ranked warp by warp with match.any so the pass is stable, staged in shared memory in digit
// order, and written out as contiguous runs.
// ---------------------------------------------------------------------------------------------
struct SortSmem {
  unsigned long long keys[kSortTile];
  unsigned vals[kSortTile];
  unsigned cnt[kSortThreads / 32][kSortBins];
  unsigned bstart[kSortBins];
  unsigned gbase[kSortBins];
  unsigned tile;
};

__global__ void __launch_bounds__(kSortThreads, kSortMinBlocks) k_sort_pass(unsigned long long* __restrict__ keys0,
                                                            unsigned* __restrict__ vals0,
                                                            unsigned long long* __restrict__ keys1,
                                                            unsigned* __restrict__ vals1,
                                                            const unsigned* __restrict__ hist,
                                                            unsigned* __restrict__ state, int pass, int tile_bits,
                                                            Control* __restrict__ ctl, unsigned spin_limit) {
  dep_wait();
  dep_release();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SortSmem& S = *reinterpret_cast<SortSmem*>(smem_raw);
  if (ctl->overflow) return;
  // passes beyond the step's key bits do nothing; pass j reads buffer (passes - j) & 1
  const int passes = key_layout(ctl, tile_bits).passes;
  if (pass >= passes) return;
  const bool from1 = ((passes - pass) & 1) != 0;
  const unsigned long long* __restrict__ kin = from1 ? keys1 : keys0;
  const unsigned* __restrict__ vin = from1 ? vals1 : vals0;
  unsigned long long* __restrict__ kout = from1 ? keys0 : keys1;
  unsigned* __restrict__ vout = from1 ? vals0 : vals1;
  const unsigned long long M = ctl->m_total;
  if (threadIdx.x == 0) S.tile = atomicAdd(&ctl->sort_ticket[pass], 1u);
  for (int k = threadIdx.x; k < (kSortThreads / 32) * kSortBins; k += kSortThreads) (&S.cnt[0][0])[k] = 0u;
  __syncthreads();
  const unsigned tile = S.tile;
  const unsigned long long tile0 = (unsigned long long)tile * kSortTile;
  if (tile0 >= M) return;
  const int shift = pass * kSortBits;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = lanemask_lt();

  unsigned long long key[kSortItems];
  unsigned val[kSortItems];
  unsigned rank[kSortItems];
  const unsigned long long wbase = tile0 + (unsigned long long)warp * (kSortItems * 32);
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const unsigned long long idx = wbase + (unsigned)(r * 32 + lane);
    const bool valid = idx < M;
    key[r] = valid ? kin[idx] : ~0ull;
    val[r] = valid ? vin[idx] : 0u;
  }
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const unsigned long long idx = wbase + (unsigned)(r * 32 + lane);
    const bool valid = idx < M;
    const unsigned d = (unsigned)(key[r] >> shift) & (kSortBins - 1);
    const unsigned peers = __match_any_sync(0xffffffffu, valid ? d : (kSortBins + d));
    const unsigned pre = valid ? S.cnt[warp][d] : 0u;
    __syncwarp();
    if (valid && (peers & lt) == 0u) S.cnt[warp][d] = pre + __popc(peers);
    __syncwarp();
    rank[r] = pre + __popc(peers & lt);
  }
  __syncthreads();
  // Per digit (thread d < 256; whole warps): warp-exclusive prefix in place, CTA total, decoupled
  // look-back across CTAs, then the digit bases by a block-wide scan over the 256 digits.
  static_assert(kSortThreads % kSortBins == 0, "the digit threads are whole warps");
  __shared__ unsigned s_wa[kSortBins / 32], s_wb[kSortBins / 32];
  const int d = threadIdx.x;
  const bool digit = d < kSortBins;
  unsigned total = 0u, excl = 0u, h = 0u, a = 0u, b = 0u;
  if (digit) {
    unsigned run = 0;
#pragma unroll
    for (int w = 0; w < kSortThreads / 32; ++w) {
      const unsigned c = S.cnt[w][d];
      S.cnt[w][d] = run;
      run += c;
    }
    total = run;
    unsigned* st = state + (unsigned long long)tile * kSortBins + d;
    if (tile == 0) {
      st_relaxed_u32(st, kSortPrefix | total);
    } else {
      st_relaxed_u32(st, kSortAgg | total);
      // look-back over windows of kLookBack predecessors (their loads in flight together)
      constexpr int kLookBack = 8;
      long long j = (long long)tile - 1;
      unsigned spins = 0;
      bool done = false;
      while (!done) {
        unsigned sv[kLookBack];
#pragma unroll
        for (int w = 0; w < kLookBack; ++w)
          sv[w] = j - w >= 0 ? ld_relaxed_u32(state + (unsigned long long)(j - w) * kSortBins + d) : kSortPrefix;
        int used = 0;
        bool wait = false;
#pragma unroll
        for (int w = 0; w < kLookBack; ++w) {
          if (done || wait) continue;
          const unsigned flag = sv[w] & ~kSortValMask;
          if (flag == 0u) {
            wait = true;
            continue;
          }
          excl += sv[w] & kSortValMask;
          ++used;
          if (flag == kSortPrefix) done = true;
        }
        j -= used;
        if (wait && ++spins > spin_limit) {
          atomicOr(&ctl->error, kErrTimeout);
          break;
        }
      }
      st_relaxed_u32(st, kSortPrefix | (excl + total));
    }
    // digit base = exclusive scan of the global histogram; CTA digit start = exclusive scan of
    // the CTA totals
    h = hist[pass * kSortBins + d];
    a = h;
    b = total;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned ya = __shfl_up_sync(0xffffffffu, a, o);
      const unsigned yb = __shfl_up_sync(0xffffffffu, b, o);
      if (lane >= o) {
        a += ya;
        b += yb;
      }
    }
    if (lane == 31) {
      s_wa[warp] = a;
      s_wb[warp] = b;
    }
  }
  __syncthreads();
  if (digit) {
    unsigned pa = 0, pb = 0;
    for (int w = 0; w < warp; ++w) {
      pa += s_wa[w];
      pb += s_wb[w];
    }
    S.gbase[d] = pa + a - h + excl;
    S.bstart[d] = pb + b - total;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const unsigned long long idx = wbase + (unsigned)(r * 32 + lane);
    if (idx < M) {
      const unsigned d = (unsigned)(key[r] >> shift) & (kSortBins - 1);
      const unsigned pos = S.bstart[d] + S.cnt[warp][d] + rank[r];
      S.keys[pos] = key[r];
      S.vals[pos] = val[r];
    }
  }
  __syncthreads();
  const unsigned tile_count = (unsigned)min((unsigned long long)kSortTile, M - tile0);
  for (unsigned k = threadIdx.x; k < tile_count; k += kSortThreads) {
    const unsigned long long kk = S.keys[k];
    const unsigned d = (unsigned)(kk >> shift) & (kSortBins - 1);
    const unsigned gpos = S.gbase[d] + (k - S.bstart[d]);
    kout[gpos] = kk;
    vout[gpos] = S.vals[k];
  }
}

void init_sort_attributes() {
  cudaFuncSetAttribute(k_sort_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SortSmem));
}

void launch_sort_pass(unsigned long long* keys0, unsigned* vals0, unsigned long long* keys1, unsigned* vals1,
                      const unsigned* hist, unsigned* state, int pass, int tile_bits, long long m_cap, Control* ctl,
                      cudaStream_t s) {
  const long long tiles = (m_cap + kSortTile - 1) / kSortTile;
  launch_dep(k_sort_pass, dim3((unsigned)(tiles > 0 ? tiles : 1)), dim3(kSortThreads), sizeof(SortSmem), s, keys0,
      vals0, keys1, vals1, hist, state, pass, tile_bits, ctl, kSpinLimit);
}

// ---------------------------------------------------------------------------------------------
// K5: per-tile [start, end) of the sorted list.  Empty tiles keep the [0, 0) the step's clear
// left them.  Grid-stride over the device-resident instance count.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_ranges(const unsigned long long* __restrict__ keys, uint2* __restrict__ ranges,
                                                int tile_bits, const Control* __restrict__ ctl) {
  dep_wait();
  dep_release();
  if (ctl->overflow) return;
  const unsigned long long M = ctl->m_total;
  const int D = key_layout(ctl, tile_bits).D;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < M;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned tile = (unsigned)(keys[i] >> D);
    if (i == 0 || (unsigned)(keys[i - 1] >> D) != tile) ranges[tile].x = (unsigned)i;
    if (i == M - 1 || (unsigned)(keys[i + 1] >> D) != tile) ranges[tile].y = (unsigned)(i + 1);
  }
}

void launch_ranges(const unsigned long long* keys, uint2* ranges, int tile_bits, long long m_cap, const Control* ctl,
                   cudaStream_t s) {
  long long blocks = (m_cap + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  launch_dep(k_ranges, dim3((unsigned)blocks), dim3(256), 0, s, keys, ranges, tile_bits, ctl);
}

// ---------------------------------------------------------------------------------------------
// Failure detection for the two inter-CTA waits.  Each wait is run once on a two-tile problem by a
// single CTA that holds ticket 1: tile 0 is never started, so its status word stays 0 and the wait
// can only end by giving up.  The problems are laid out so that the CTA's remaining work after
// giving up (with a partial prefix of 0) stays inside its own buffers.
// ---------------------------------------------------------------------------------------------
gs_status run_wait_probe(unsigned spin_limit, unsigned out_error[2], float out_ms[2]) {
  if (spin_limit == 0u) spin_limit = kSpinLimit;
  init_sort_attributes();
  const size_t n_scan = 2 * (size_t)kScanTile, n_sort = 2 * (size_t)kSortTile;
  const size_t off_ctl_b = kCtlBytes, off_state_a = 2 * kCtlBytes;
  const size_t off_state_b = off_state_a + 2 * sizeof(unsigned long long);
  const size_t off_hist = off_state_b + 2 * kSortBins * sizeof(unsigned);
  const size_t off_in = off_hist + (size_t)kMaxSortPasses * kSortBins * sizeof(unsigned);
  const size_t off_out = off_in + n_scan * sizeof(unsigned);
  const size_t off_k0 = off_out + n_scan * sizeof(unsigned);
  const size_t off_k1 = off_k0 + n_sort * sizeof(unsigned long long);
  const size_t off_v0 = off_k1 + n_sort * sizeof(unsigned long long);
  const size_t off_v1 = off_v0 + n_sort * sizeof(unsigned);
  const size_t bytes = off_v1 + n_sort * sizeof(unsigned);
  char* d = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  gs_status status = GS_OK;
  auto check = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && status == GS_OK) status = fail(GS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaSuccess;
  };
  if (check(cudaMalloc(&d, bytes), "cudaMalloc") && check(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "stream") &&
      check(cudaEventCreate(&ev[0]), "event") && check(cudaEventCreate(&ev[1]), "event") &&
      check(cudaEventCreate(&ev[2]), "event") && check(cudaMemsetAsync(d, 0, bytes, st), "cudaMemsetAsync")) {
    Control ca{}, cb{};
    ca.scan_ticket = 1u;       // the CTA takes tile 1 of the scan
    cb.sort_ticket[0] = 1u;    // and tile 1 of pass 0 of the sort
    cb.m_total = n_sort;       // all keys 0: one pass, every key in digit 0
    const unsigned h0 = (unsigned)n_sort;
    Control* ctl_a = reinterpret_cast<Control*>(d);
    Control* ctl_b = reinterpret_cast<Control*>(d + off_ctl_b);
    unsigned* hist = reinterpret_cast<unsigned*>(d + off_hist);
    if (check(cudaMemcpyAsync(ctl_a, &ca, sizeof(Control), cudaMemcpyHostToDevice, st), "cudaMemcpyAsync") &&
        check(cudaMemcpyAsync(ctl_b, &cb, sizeof(Control), cudaMemcpyHostToDevice, st), "cudaMemcpyAsync") &&
        check(cudaMemcpyAsync(hist, &h0, sizeof(unsigned), cudaMemcpyHostToDevice, st), "cudaMemcpyAsync")) {
      cudaEventRecord(ev[0], st);
      k_scan<<<1, kScanThreads, 0, st>>>(reinterpret_cast<const unsigned*>(d + off_in),
                                         reinterpret_cast<unsigned*>(d + off_out), (long long)n_scan,
                                         reinterpret_cast<unsigned long long*>(d + off_state_a), ctl_a, ~0ull,
                                         nullptr, nullptr, spin_limit);
      cudaEventRecord(ev[1], st);
      k_sort_pass<<<1, kSortThreads, sizeof(SortSmem), st>>>(
          reinterpret_cast<unsigned long long*>(d + off_k0), reinterpret_cast<unsigned*>(d + off_v0),
          reinterpret_cast<unsigned long long*>(d + off_k1), reinterpret_cast<unsigned*>(d + off_v1), hist,
          reinterpret_cast<unsigned*>(d + off_state_b), 0, 8, ctl_b, spin_limit);
      cudaEventRecord(ev[2], st);
      check(cudaGetLastError(), "wait probe launch");
      Control ra{}, rb{};
      if (check(cudaMemcpyAsync(&ra, ctl_a, sizeof(Control), cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync") &&
          check(cudaMemcpyAsync(&rb, ctl_b, sizeof(Control), cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync") &&
          check(cudaStreamSynchronize(st), "cudaStreamSynchronize")) {
        out_error[0] = ra.error;
        out_error[1] = rb.error;
        if (out_ms) {
          cudaEventElapsedTime(&out_ms[0], ev[0], ev[1]);
          cudaEventElapsedTime(&out_ms[1], ev[1], ev[2]);
        }
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
