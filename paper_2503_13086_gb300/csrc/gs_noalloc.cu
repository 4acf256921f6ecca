// gs_noalloc.cu -- gs_scan_noalloc: the tile-count scan (K2) for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs while another component owns the
// allocator (a memory pool that forbids outside allocations, a host that has reserved all device
// memory up front), or code on a path where an allocation's implicit synchronisation is not
// allowed.  For them this entry point runs the same single-pass scan kernel as the rasterizer,
// with its scratch (the look-back state of the CTAs and the control word) in a file-scope device
// array instead of a workspace: it calls no cudaMalloc, cudaFree or allocating library routine.
#include <mutex>
#include <string>

#include "gs_engine.h"

namespace gs {
namespace {

// At most 2^24 counts per call: 8192 scan tiles of 2048 counts, 8 bytes of look-back state each,
// after a 1 KiB control block.  Every GPU that loads the library holds these 65 KiB until exit.
constexpr long long kNoAllocMaxItems = 1ll << 24;
constexpr long long kNoAllocTiles = kNoAllocMaxItems / kScanTile;
constexpr size_t kNoAllocBytes = kCtlBytes + (size_t)kNoAllocTiles * 8;

static __device__ __align__(256) unsigned char g_scan_scratch[kNoAllocBytes];

// Device address of g_scan_scratch per device.  In host code the array's name only stands in for
// the symbol; the address comes from cudaGetSymbolAddress with that device current.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// The total, or UINT64_MAX when a look-back wait of the scan gave up (its offsets are then not
// valid): the one result a caller reads, so a timeout is visible without a host readback.
__global__ void k_noalloc_total(const Control* __restrict__ ctl, unsigned long long* __restrict__ out_total) {
  *out_total = (ctl->error & kErrTimeout) ? ~0ull : ctl->m_total;
}

}  // namespace
}  // namespace gs

extern "C" GS_API gs_status gs_scan_noalloc(void* stream, const uint32_t* counts, int64_t n, uint32_t* out_offsets,
                                            uint64_t* out_total) {
  using namespace gs;
  if (n < 0 || n > kNoAllocMaxItems)
    return fail(GS_ERR_CAPACITY, "gs_scan_noalloc: n must be in 0.." + std::to_string(kNoAllocMaxItems));
  if ((n > 0 && (!counts || !out_offsets)) ||
      ((reinterpret_cast<uintptr_t>(counts) | reinterpret_cast<uintptr_t>(out_offsets)) & 15u))
    return fail(GS_ERR_INVALID_ARG, "gs_scan_noalloc: counts and out_offsets must be non-NULL and 16-byte aligned");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(GS_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(GS_ERR_CAPACITY, "gs_scan_noalloc: device index too large");
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
      // one-time set-up on this device (must not happen inside a stream capture)
      e = cudaGetSymbolAddress(&g_addr[dev], g_scan_scratch);
      if (e != cudaSuccess) {
        g_addr[dev] = nullptr;
        return fail(GS_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      }
    }
    base = g_addr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Control* ctl = static_cast<Control*>(base);
  unsigned long long* state = reinterpret_cast<unsigned long long*>(static_cast<char*>(base) + kCtlBytes);
  const long long tiles = (n + kScanTile - 1) / kScanTile;
  // the previous call's tickets, totals and look-back flags must not leak into this one
  e = cudaMemsetAsync(base, 0, kCtlBytes + (size_t)tiles * 8, s);
  if (e != cudaSuccess) return fail(GS_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  if (n > 0) launch_scan(counts, out_offsets, n, state, ctl, ~0ull, nullptr, s);
  if (out_total) k_noalloc_total<<<1, 1, 0, s>>>(ctl, reinterpret_cast<unsigned long long*>(out_total));
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(GS_ERR_CUDA, std::string("gs_scan_noalloc launch: ") + cudaGetErrorString(e));
  return GS_OK;
}
