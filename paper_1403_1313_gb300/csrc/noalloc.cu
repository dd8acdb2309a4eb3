// Sorting codes without allocating device memory.
//
// Some callers cannot allocate device memory at the point where they need their codes ordered:
// code that runs inside a framework whose allocator owns all free device memory, and
// latency-critical loops that must never block on an allocator or on the implicit device
// synchronisation of cudaMalloc / cudaFree.  motif_sort_codes_noalloc serves them: it runs the
// library's sort/dedup kernels with their scratch taken from a fixed array compiled into the
// library.
//
// The array below is a static __device__ allocation: every GPU that loads the library holds it
// (about 2.6 MB) until the process exits.  Host code cannot pass the symbol itself to a kernel —
// on the host, g_noalloc_scratch names a host-side shadow, not device memory — so the first call
// on each device looks up the array's device address with cudaGetSymbolAddress (with that device
// current) and caches it, together with the device's current context: a call from another
// context (after cudaDeviceReset, for instance) looks the address up again.  Every call shares
// the array, so calls that overlap on the GPU (two streams, or two host threads on one device)
// race on it and must be serialised by the caller.
#include <cuda.h>

#include <mutex>

#include "plan.h"

namespace {

constexpr long long kNoallocMaxCodes = 1ll << 18;  // codes per call
constexpr int kNoallocMaxSms = 256;                // radix CTAs are sized by min(SMs, this)
// Radix scratch for kNoallocMaxCodes codes at kNoallocMaxSms SMs (alternate key buffer,
// per-CTA digit histograms, per-CTA keep counts), then one 256-byte cell for the element count.
constexpr size_t kNoallocSortBytes = (size_t)kNoallocMaxCodes * 8 +
                                     (size_t)256 * 2 * kNoallocMaxSms * 4 +
                                     (size_t)2 * 2 * kNoallocMaxSms * 4 + 64;
constexpr size_t kNoallocCellOffset = (kNoallocSortBytes + 255) / 256 * 256;
constexpr size_t kNoallocBytes = kNoallocCellOffset + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// Per-device set-up: the scratch array's device address and the SM count, and the context the
// address belongs to.
std::mutex g_mu;
unsigned char* g_addr[64] = {};
int g_sms[64] = {};
CUcontext g_ctx[64] = {};

// The calling thread's current context, through the driver entry point the runtime exposes (no
// link against the driver library); null if it cannot be had.
CUcontext current_context() {
  typedef CUresult (*GetCurrent)(CUcontext*);
  static GetCurrent fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return (GetCurrent) nullptr;
    }
    return reinterpret_cast<GetCurrent>(f);
  }();
  CUcontext c = nullptr;
  if (fn && fn(&c) != CUDA_SUCCESS) c = nullptr;
  return c;
}

int noalloc_setup(int dev, unsigned char** base, int* sms) {
  if (dev < 0 || dev >= 64) return MOTIF_ERR_ARG;
  std::lock_guard<std::mutex> g(g_mu);
  const CUcontext ctx = current_context();
  if (!g_addr[dev] || g_ctx[dev] != ctx) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return MOTIF_ERR_CUDA;
    }
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
      return MOTIF_ERR_CUDA;
    g_addr[dev] = static_cast<unsigned char*>(p);
    g_sms[dev] = n < kNoallocMaxSms ? n : kNoallocMaxSms;
    g_ctx[dev] = ctx;
  }
  *base = g_addr[dev];
  *sms = g_sms[dev];
  return MOTIF_OK;
}

__global__ void set_count_kernel(unsigned long long* cell, unsigned long long v) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *cell = v;
}

__global__ void get_count_kernel(const unsigned long long* cell, int64_t* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *out = (int64_t)*cell;
}

}  // namespace

extern "C" int motif_sort_codes_noalloc(uint64_t* d_codes, int64_t count, int32_t key_bits,
                                        int64_t* d_unique_count, void* stream) {
  if (count < 0 || key_bits < 1 || key_bits > 64 || !d_unique_count || (count > 0 && !d_codes))
    return MOTIF_ERR_ARG;
  if (count > kNoallocMaxCodes) return MOTIF_ERR_CAPACITY;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return MOTIF_ERR_CUDA;
  }
  unsigned char* base = nullptr;
  int sms = 0;
  int rc = noalloc_setup(dev, &base, &sms);
  if (rc) return rc;
  if (motif::sort_scratch_bytes(count, sms) > kNoallocSortBytes) return MOTIF_ERR_CAPACITY;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // The count cell keeps the previous call's value: set it for this call.
  unsigned long long* cell = reinterpret_cast<unsigned long long*>(base + kNoallocCellOffset);
  set_count_kernel<<<1, 32, 0, s>>>(cell, (unsigned long long)count);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = motif::launch_sort_unique(d_codes, cell, count, key_bits, base, sms, (long long)count, s);
  if (e == cudaSuccess) {
    get_count_kernel<<<1, 32, 0, s>>>(cell, d_unique_count);
    e = cudaGetLastError();
  }
  motif::note_launches(2);
  return motif::status_from_cuda(e);
}
