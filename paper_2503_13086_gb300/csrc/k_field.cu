// k_field.cu -- the field update of Sec. IV-B on the device: which of an arriving image's sparse
// points become new Gaussians, and their initialisation, sm_103a.
//
// Every sparse point registered so far lives in device memory, indexed by a uniform grid of cubic
// cells stored as an open-addressing hash table (cell key -> head of a linked list of the cell's
// points).  The paper searches a tree; any exact neighbour structure gives the same answers.
//   K11a  new point k is "far" when no earlier point lies within the threshold (the cells within
//         ceil(threshold / cell) rings are searched, so none is missed);
//   K11b  all of the image's points join the grid;
//   K11c  exclusive scan of the far flags (new Gaussians keep the points' order);
//   K11d  each far point becomes a Gaussian with the 3DGS initialisation: isotropic log-scale from
//         the mean squared distance to its 3 nearest other points (shells of cells, stopping once
//         the third nearest is closer than the searched reach), identity rotation, opacity 0.1,
//         DC colour from the point colour, higher SH zero; its Adam moments are zeroed.
// The points are hashed twice: in cells of the threshold (the far test, and the 3-NN search for
// its first shells) and in cells kCoarseCells times larger, where the 3-NN search restarts when
// the first shells do not settle it, so a sparse neighbourhood costs a few coarse shells instead
// of thousands of empty fine cells.
// Squared distances are formed with explicit round-to-nearest operations (no contraction), so
// the decisions are the same on every host and device.
#include "gs_engine.h"

namespace gs {

namespace {

constexpr unsigned long long kEmptyCell = ~0ull;
constexpr int kMaxShells = 64;   // kNN search bound (coarse cells); beyond it the points found are used
constexpr int kFineShells = 3;   // fine-grid shells tried first

__device__ __forceinline__ long long cell_of(float v, float cell) {
  return (long long)floorf(__fdiv_rn(v, cell));
}

__device__ __forceinline__ unsigned long long cell_key(long long ix, long long iy, long long iz) {
  return ((unsigned long long)(ix & 0x1FFFFF) << 42) | ((unsigned long long)(iy & 0x1FFFFF) << 21) |
         (unsigned long long)(iz & 0x1FFFFF);
}

__device__ __forceinline__ unsigned slot_of(unsigned long long key, unsigned mask) {
  unsigned long long z = key * 0x9E3779B97F4A7C15ull;
  z ^= z >> 29;
  return (unsigned)z & mask;
}

__device__ __forceinline__ float dist2(const float* __restrict__ a, float x, float y, float z) {
  const float dx = __fsub_rn(a[0], x), dy = __fsub_rn(a[1], y), dz = __fsub_rn(a[2], z);
  return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

__device__ __forceinline__ bool finite3(const float* p) {
  return isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2]);
}

// Head of the list of a cell, -1 if the cell holds no point.  The table is never full (its
// capacity is at least twice the number of points), so the probe ends at an empty slot.
__device__ __forceinline__ int cell_head(const PointGridDev& g, unsigned long long key) {
  unsigned s = slot_of(key, g.mask);
  for (unsigned probe = 0; probe <= g.mask; ++probe) {
    const unsigned long long k = g.keys[s];
    if (k == key) return g.head[s];
    if (k == kEmptyCell) return -1;
    s = (s + 1u) & g.mask;
  }
  return -1;
}

// The three smallest squared distances from p to the grid's points other than `self` (b0 <= b1 <=
// b2, INFINITY where fewer), searching shells 0..max_shells-1 of cells around p's cell and stopping
// once the third is within the searched reach.  Returns the number of points seen, or -(seen + 1)
// when the shells ran out before the answer was settled.
__device__ __forceinline__ int knn3(const PointGridDev& g, const float* p, long long self, int max_shells, float& b0,
                                    float& b1, float& b2) {
  const long long cx = cell_of(p[0], g.cell), cy = cell_of(p[1], g.cell), cz = cell_of(p[2], g.cell);
  b0 = b1 = b2 = INFINITY;
  int found = 0;
  for (int r = 0; r < max_shells; ++r) {
    for (int a = -r; a <= r; ++a)
      for (int b = -r; b <= r; ++b) {
        const bool face = (a == -r || a == r || b == -r || b == r);
        const int cstep = face ? 1 : (r > 0 ? 2 * r : 1);  // inside the square only the two caps
        for (int c = -r; c <= r; c += cstep)
          for (int id = cell_head(g, cell_key(cx + a, cy + b, cz + c)); id >= 0; id = g.next[id]) {
            if (id == self) continue;
            const float d = dist2(g.xyz + 3ll * id, p[0], p[1], p[2]);
            ++found;
            if (d < b2) {
              if (d < b1) {
                b2 = b1;
                if (d < b0) {
                  b1 = b0;
                  b0 = d;
                } else {
                  b1 = d;
                }
              } else {
                b2 = d;
              }
            }
          }
      }
    const float reach = __fmul_rn((float)r, g.cell);  // every point this close has been seen
    if (found >= 3 && b2 <= __fmul_rn(reach, reach)) return found;
  }
  return -found - 1;
}

}  // namespace

// K11a
__global__ void __launch_bounds__(256) k_far_points(PointGridDev g, const float* __restrict__ xyz, int n_new,
                                                    float thr2, int ring, unsigned* __restrict__ far) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_new) return;
  const float* p = xyz + 3ll * k;
  unsigned is_far = 0u;
  if (finite3(p)) {
    is_far = 1u;
    const long long cx = cell_of(p[0], g.cell), cy = cell_of(p[1], g.cell), cz = cell_of(p[2], g.cell);
    for (int a = -ring; a <= ring && is_far; ++a)
      for (int b = -ring; b <= ring && is_far; ++b)
        for (int c = -ring; c <= ring && is_far; ++c)
          for (int id = cell_head(g, cell_key(cx + a, cy + b, cz + c)); id >= 0; id = g.next[id])
            if (dist2(g.xyz + 3ll * id, p[0], p[1], p[2]) <= thr2) {
              is_far = 0u;
              break;
            }
  }
  far[k] = is_far;
}

// K11b (and the rebuild after the table grows): insert points first..first+count-1.
__global__ void __launch_bounds__(256) k_insert_points(PointGridDev g, int* __restrict__ next, long long first,
                                                       long long count) {
  const long long i = first + (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= first + count) return;
  const float* p = g.xyz + 3 * i;
  if (!finite3(p)) {
    next[i] = -1;
    return;
  }
  const unsigned long long key = cell_key(cell_of(p[0], g.cell), cell_of(p[1], g.cell), cell_of(p[2], g.cell));
  unsigned s = slot_of(key, g.mask);
  for (unsigned probe = 0; probe <= g.mask; ++probe) {
    const unsigned long long old = atomicCAS(&g.keys[s], kEmptyCell, key);
    if (old == kEmptyCell || old == key) {
      next[i] = atomicExch(&g.head[s], (int)i);
      return;
    }
    s = (s + 1u) & g.mask;
  }
}

// K11c: exclusive scan of n flags by one CTA of 1024 threads; total in *count.
__global__ void __launch_bounds__(1024) k_scan_flags(const unsigned* __restrict__ far, int n,
                                                     unsigned* __restrict__ offsets, unsigned* __restrict__ count) {
  __shared__ unsigned s_warp[32];
  __shared__ unsigned s_carry;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_carry = 0u;
  __syncthreads();
  for (int base = 0; base < n; base += 1024) {
    const int i = base + tid;
    const unsigned f = i < n ? far[i] : 0u;
    unsigned x = f;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
      unsigned w = s_warp[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      s_warp[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    const unsigned carry = s_carry;
    const unsigned before = (warp ? s_warp[warp - 1] : 0u) + x - f;
    if (i < n) offsets[i] = carry + before;
    __syncthreads();
    if (tid == 0) s_carry = carry + s_warp[31];
    __syncthreads();
  }
  if (tid == 0) *count = s_carry;
}

// K11d
__global__ void __launch_bounds__(128) k_init_gaussians(PointGridDev g, PointGridDev gc, const float* __restrict__ xyz,
                                                        const float* __restrict__ rgb, int n_new, long long self0,
                                                        const unsigned* __restrict__ far,
                                                        const unsigned* __restrict__ offsets, float* __restrict__ params,
                                                        float* __restrict__ adam_m, float* __restrict__ adam_v,
                                                        int stride, int n0, float opacity_logit, double sh_c0) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_new || !far[k]) return;
  const float* p = xyz + 3ll * k;
  const long long self = self0 + k;
  float b0, b1, b2;
  int found = knn3(g, p, self, kFineShells, b0, b1, b2);
  if (found < 0) found = knn3(gc, p, self, kMaxShells, b0, b1, b2);
  if (found < 0) found = -found - 1;  // shell limit reached: the points found are used
  float d2 = 1e-7f;
  if (found > 0) {
    const int m = found < 3 ? found : 3;
    float s = b0;
    if (m > 1) s = __fadd_rn(s, b1);
    if (m > 2) s = __fadd_rn(s, b2);
    d2 = fmaxf(__fdiv_rn(s, (float)m), 1e-7f);
  }
  const float ls = logf(sqrtf(d2));
  const long long j = (long long)n0 + offsets[k];
  float col[kNumParams];
#pragma unroll
  for (int q = 0; q < kNumParams; ++q) col[q] = 0.f;
  col[0] = p[0];
  col[1] = p[1];
  col[2] = p[2];
  col[3] = col[4] = col[5] = ls;
  col[6] = 1.f;
  col[10] = opacity_logit;
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) col[11 + ch] = (float)(((double)rgb[3ll * k + ch] - 0.5) / sh_c0);
#pragma unroll
  for (int q = 0; q < kNumParams; ++q) {
    params[(long long)q * stride + j] = col[q];
    adam_m[(long long)q * stride + j] = 0.f;
    adam_v[(long long)q * stride + j] = 0.f;
  }
}

// An arriving image in the interleaved layout callers decode to (H x W x 3) into the planar layout
// the loss reads (3 x H x W): one thread per pixel, 12 contiguous bytes read, three coalesced
// planes written.
__global__ void __launch_bounds__(256) k_hwc_to_chw(const float* __restrict__ src, float* __restrict__ dst,
                                                    long long npix) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npix) return;
  const float r = src[3 * p], g = src[3 * p + 1], b = src[3 * p + 2];
  dst[p] = r;
  dst[npix + p] = g;
  dst[2 * npix + p] = b;
}

// The same from page-locked host memory read directly over the host link (a 16-byte aligned source):
// a CTA moves 1024 pixels (12 KB of the interleaved stream) with consecutive 16-byte loads into
// shared memory, then writes its part of the three planes, so the link sees whole contiguous
// requests and no staging copy is made.
constexpr int kHostPix = 1024;
__global__ void __launch_bounds__(256) k_hwc_to_chw_host(const float* __restrict__ src, float* __restrict__ dst,
                                                         long long npix) {
  __shared__ float4 s[kHostPix * 3 / 4];
  const long long p0 = (long long)blockIdx.x * kHostPix;
  const long long f0 = 3 * p0;  // first float of the CTA's span (a multiple of 4: 16-byte aligned)
  const long long nf = 3 * min((long long)kHostPix, npix - p0);
  const float4* s4 = reinterpret_cast<const float4*>(src + f0);
  for (int k = threadIdx.x; k < kHostPix * 3 / 4; k += blockDim.x) {
    if (4ll * k + 4 <= nf) {
      s[k] = s4[k];
    } else {
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (4ll * k < nf) v.x = src[f0 + 4 * k];
      if (4ll * k + 1 < nf) v.y = src[f0 + 4 * k + 1];
      if (4ll * k + 2 < nf) v.z = src[f0 + 4 * k + 2];
      s[k] = v;
    }
  }
  __syncthreads();
  const float* sf = reinterpret_cast<const float*>(s);
  for (int q = threadIdx.x; q < kHostPix; q += blockDim.x) {
    const long long p = p0 + q;
    if (p < npix) {
      dst[p] = sf[3 * q];
      dst[npix + p] = sf[3 * q + 1];
      dst[2 * npix + p] = sf[3 * q + 2];
    }
  }
}

void launch_hwc_to_chw(const float* src, float* dst, long long npix, cudaStream_t s) {
  if (npix <= 0) return;
  k_hwc_to_chw<<<(unsigned)((npix + 255) / 256), 256, 0, s>>>(src, dst, npix);
}

void launch_hwc_to_chw_host(const float* src, float* dst, long long npix, cudaStream_t s) {
  if (npix <= 0) return;
  if ((reinterpret_cast<uintptr_t>(src) & 15u) == 0)
    k_hwc_to_chw_host<<<(unsigned)((npix + kHostPix - 1) / kHostPix), 256, 0, s>>>(src, dst, npix);
  else
    k_hwc_to_chw<<<(unsigned)((npix + 255) / 256), 256, 0, s>>>(src, dst, npix);
}

void launch_far_points(const PointGridDev& g, const float* xyz, int n_new, float thr2, int ring, unsigned* far,
                       cudaStream_t s) {
  if (n_new <= 0) return;
  k_far_points<<<(n_new + 255) / 256, 256, 0, s>>>(g, xyz, n_new, thr2, ring, far);
}

void launch_insert_points(const PointGridDev& g, int* next, long long first, long long count, cudaStream_t s) {
  if (count <= 0) return;
  k_insert_points<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(g, next, first, count);
}

void launch_scan_flags(const unsigned* far, int n, unsigned* offsets, unsigned* count, cudaStream_t s) {
  k_scan_flags<<<1, 1024, 0, s>>>(far, n, offsets, count);
}

void launch_init_gaussians(const PointGridDev& g, const PointGridDev& gc, const float* xyz, const float* rgb, int n_new, long long self0,
                           const unsigned* far, const unsigned* offsets, float* params, float* m, float* v, int stride,
                           int n0, float opacity_logit, double sh_c0, cudaStream_t s) {
  if (n_new <= 0) return;
  k_init_gaussians<<<(n_new + 127) / 128, 128, 0, s>>>(g, gc, xyz, rgb, n_new, self0, far, offsets, params, m, v, stride,
                                                       n0, opacity_logit, sh_c0);
}

}  // namespace gs
