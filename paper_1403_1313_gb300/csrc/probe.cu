// K4: issue-rate probes for the integer instructions the window compare is built from.
//
// The compare step (Hamming distance of an l-mer against a window, tested against d) is pure
// integer work: XOR / LOP3, a shift, POPC and a min.  Its roofline is therefore an issue-rate
// roofline, and the per-SM, per-clock rate of each of those instructions has to be measured on
// the part rather than taken from documentation of older compute capabilities.  Each probe runs
// one CTA of 1024 threads per SM (dynamic shared memory sized so that no second CTA fits), times
// itself with the SM cycle counter, and reports operations per SM per clock.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <algorithm>
#include <vector>

#include "motif_internal.h"

namespace {

constexpr int kProbeThreads = 1024;
constexpr int kProbeSmemWords = 4096;  // 16 KB of window-like words for the LDS probes

template <int KIND>
__global__ void __launch_bounds__(kProbeThreads, 1)
probe_kernel(uint32_t seed, int iters, long long* cycles, uint32_t* sink) {
  __shared__ uint4 win[kProbeSmemWords / 4];
  const int tid = threadIdx.x;
  for (int i = tid; i < kProbeSmemWords / 4; i += blockDim.x) {
    uint32_t a = seed * 2654435761u + 4u * i;
    win[i] = make_uint4(a & 0x15555555u, (a >> 1) & 0x15555555u, (a * 7u) & 0x15555555u,
                        (a * 13u) & 0x15555555u);
  }
  uint32_t r[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) r[c] = seed ^ (uint32_t)(tid * 8 + c) * 0x9E3779B9u;
  uint32_t a = seed * 3u + 1u, b = seed * 5u + 7u;
  uint32_t mn[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) mn[c] = 31u;
  __syncthreads();
  long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
    if (KIND == MOTIF_PROBE_POPC) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int c = 0; c < 8; ++c) asm volatile("popc.b32 %0, %0;" : "+r"(r[c]));
    } else if (KIND == MOTIF_PROBE_LOP3) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int c = 0; c < 8; ++c)
          asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(r[c]) : "r"(a), "r"(b));
    } else if (KIND == MOTIF_PROBE_IMNMX) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int c = 0; c < 8; ++c) asm volatile("min.u32 %0, %0, %1;" : "+r"(r[c]) : "r"(a));
    } else if (KIND == MOTIF_PROBE_SHF) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int c = 0; c < 8; ++c)
          asm volatile("shf.l.wrap.b32 %0, %0, %0, %1;" : "+r"(r[c]) : "r"(a));
    } else if (KIND == MOTIF_PROBE_IADD) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int c = 0; c < 8; ++c) asm volatile("add.u32 %0, %0, %1;" : "+r"(r[c]) : "r"(a));
    } else if (KIND == MOTIF_PROBE_IMAD) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int c = 0; c < 8; ++c)
          asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(r[c]) : "r"(a), "r"(b));
    } else if (KIND == MOTIF_PROBE_POPC_LOP3) {
      // 1 POPC and 3 LOP3 on independent chains: the rate shows whether POPC shares the LOP3 pipe.
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        asm volatile("popc.b32 %0, %0;" : "+r"(r[c]));
        asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(mn[c]) : "r"(a), "r"(b));
        asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(mn[c]) : "r"(b), "r"(a));
        asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(mn[c]) : "r"(a), "r"(a));
      }
    } else if (KIND == MOTIF_PROBE_CMP_SPLIT) {
      // Split-plane compare: two windows (even plane, odd plane) per 128-bit broadcast load.
      uint4 w = win[it & (kProbeSmemWords / 4 - 1)];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        uint32_t ce = r[c] & 0x15555555u, co = (r[c] >> 1) & 0x15555555u;
        uint32_t m0 = (ce ^ w.x) | (co ^ w.y);
        uint32_t m1 = (ce ^ w.z) | (co ^ w.w);
        mn[c] = min(mn[c], (uint32_t)__popc(m0));
        mn[c] = min(mn[c], (uint32_t)__popc(m1));
      }
    } else if (KIND == MOTIF_PROBE_CMP_FOLD) {
      // Folded compare: four packed windows per 128-bit broadcast load.
      uint4 w = win[it & (kProbeSmemWords / 4 - 1)];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        uint32_t x0 = r[c] ^ w.x, x1 = r[c] ^ w.y, x2 = r[c] ^ w.z, x3 = r[c] ^ w.w;
        mn[c] = min(mn[c], (uint32_t)__popc((x0 | (x0 >> 1)) & 0x55555555u));
        mn[c] = min(mn[c], (uint32_t)__popc((x1 | (x1 >> 1)) & 0x55555555u));
        mn[c] = min(mn[c], (uint32_t)__popc((x2 | (x2 >> 1)) & 0x55555555u));
        mn[c] = min(mn[c], (uint32_t)__popc((x3 | (x3 >> 1)) & 0x55555555u));
      }
    } else if (KIND == MOTIF_PROBE_ATOMS_OR) {
      // Shared-memory atomic ORs, result unused: word c * 1024 + tid (mod the array) puts every
      // lane of a warp on its own bank and no two threads on one word within a chain.
      uint32_t* wv = reinterpret_cast<uint32_t*>(win);
#pragma unroll
      for (int c = 0; c < 8; ++c)
        atomicOr(wv + (((c & 3) * 1024 + tid) & (kProbeSmemWords - 1)), r[c] + (uint32_t)it);
    } else if (KIND == MOTIF_PROBE_SHFL) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int c = 0; c < 8; ++c) r[c] = __shfl_xor_sync(0xffffffffu, r[c], 1 << (c & 3));
    } else if (KIND == MOTIF_PROBE_LDS64_DIV) {
      // Per-thread 64-bit shared loads at distinct, bank-conflict-free addresses.
      const uint2* w2 = reinterpret_cast<const uint2*>(win);
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        uint2 v = w2[((it * 8 + c) * 32 + (tid & 31)) & (kProbeSmemWords / 2 - 1)];
        r[c] |= v.x;
        mn[c] |= v.y;
      }
    }
  }
  long long t1 = clock64();
  __syncthreads();
  uint32_t acc = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) acc ^= r[c] ^ mn[c];
  sink[blockIdx.x * blockDim.x + tid] = acc;
  if (tid == 0) cycles[blockIdx.x] = t1 - t0;
}

template <int KIND>
cudaError_t launch_probe(int sms, uint32_t seed, int iters, long long* cyc, uint32_t* sink,
                         size_t smem_pad) {
  cudaError_t e = cudaFuncSetAttribute(probe_kernel<KIND>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_pad);
  if (e != cudaSuccess) return e;
  probe_kernel<KIND><<<sms, kProbeThreads, smem_pad>>>(seed, iters, cyc, sink);
  motif::note_launches(1);
  return cudaGetLastError();
}

// Operations counted per thread per loop iteration, by probe.
double ops_per_iter(int kind) {
  switch (kind) {
    case MOTIF_PROBE_POPC_LOP3: return 8.0 * 4.0;   // 8 POPC + 24 LOP3 instructions
    case MOTIF_PROBE_CMP_SPLIT: return 8.0 * 2.0;   // window compares
    case MOTIF_PROBE_CMP_FOLD: return 8.0 * 4.0;    // window compares
    case MOTIF_PROBE_LDS64_DIV: return 8.0;         // 64-bit shared loads
    case MOTIF_PROBE_ATOMS_OR: return 8.0;          // shared atomic ORs
    default: return 32.0;                           // 4 x 8 instructions of the probed kind
  }
}

}  // namespace

extern "C" int motif_probe_rate(int kind, int iters, double* ops_per_sm_clk, double* sm_cycles) {
  if (!ops_per_sm_clk || kind < 0 || kind >= MOTIF_PROBE_COUNT || iters <= 0) return MOTIF_ERR_ARG;
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
    return MOTIF_ERR_CUDA;
  const int sms = prop.multiProcessorCount;
  // Pad dynamic shared memory past half the SM's capacity so that one CTA owns each SM.
  size_t pad = prop.sharedMemPerMultiprocessor / 2 + 1024;
  if (pad + 16384 > prop.sharedMemPerBlockOptin) pad = prop.sharedMemPerBlockOptin - 16384;
  long long* cyc = nullptr;
  uint32_t* sink = nullptr;
  if (cudaMalloc(&cyc, sizeof(long long) * sms) != cudaSuccess) return MOTIF_ERR_OOM;
  if (cudaMalloc(&sink, sizeof(uint32_t) * (size_t)sms * kProbeThreads) != cudaSuccess) {
    cudaFree(cyc);
    return MOTIF_ERR_OOM;
  }
  cudaError_t e = cudaSuccess;
  switch (kind) {
#define PROBE_CASE(K) \
  case K: e = launch_probe<K>(sms, 12345u, iters, cyc, sink, pad); break;
    PROBE_CASE(MOTIF_PROBE_POPC)
    PROBE_CASE(MOTIF_PROBE_LOP3)
    PROBE_CASE(MOTIF_PROBE_IMNMX)
    PROBE_CASE(MOTIF_PROBE_SHF)
    PROBE_CASE(MOTIF_PROBE_IADD)
    PROBE_CASE(MOTIF_PROBE_IMAD)
    PROBE_CASE(MOTIF_PROBE_POPC_LOP3)
    PROBE_CASE(MOTIF_PROBE_CMP_SPLIT)
    PROBE_CASE(MOTIF_PROBE_CMP_FOLD)
    PROBE_CASE(MOTIF_PROBE_LDS64_DIV)
    PROBE_CASE(MOTIF_PROBE_ATOMS_OR)
    PROBE_CASE(MOTIF_PROBE_SHFL)
#undef PROBE_CASE
    default: e = cudaErrorInvalidValue;
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  std::vector<long long> h(sms);
  if (e == cudaSuccess) e = cudaMemcpy(h.data(), cyc, sizeof(long long) * sms, cudaMemcpyDeviceToHost);
  cudaFree(cyc);
  cudaFree(sink);
  if (e != cudaSuccess) return MOTIF_ERR_CUDA;
  std::sort(h.begin(), h.end());
  const double med = (double)h[sms / 2];
  const double ops = ops_per_iter(kind) * (double)iters * kProbeThreads;
  *ops_per_sm_clk = med > 0 ? ops / med : 0.0;
  if (sm_cycles) *sm_cycles = med;
  return MOTIF_OK;
}
