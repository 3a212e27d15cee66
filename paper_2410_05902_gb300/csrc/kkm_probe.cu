// Unit-rate probe: the per-SM issue rate of the two pipes the distance pass's
// epilogue leans on, measured on the device the library runs on.
//
//   op 0  ex2.approx.ftz.f32 (the MUFU exponential of the Gaussian and
//         Laplacian kernel values)
//   op 1  scalar FP32 fma.rn (the FMA pipe)
//   op 2  packed f32x2 fma.rn (two FP32 FMAs per lane and instruction)
//
// One block of 1024 threads per SM: the launch asks for more dynamic shared
// memory than half an SM holds, so no SM runs two blocks. Each thread keeps
// eight independent dependency chains (enough warps and chains in flight to
// cover the pipes' latency). Every block reads its SM's cycle counter around
// its loop, so the rate per clock needs no knowledge of the clock frequency.
// The loops are bounded by the caller's iteration count and contain no waits.
#include <algorithm>
#include <vector>

#include "kkm_internal.cuh"
#include "../../include/kkm.h"

#define KKM_API extern "C" __attribute__((visibility("default")))

namespace kkm {
namespace {

constexpr int PROBE_THREADS = 1024;
constexpr int PROBE_SMEM = 150 * 1024;   // above half of an SM's shared memory: one block per SM

__device__ __forceinline__ float probe_ex2(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__global__ void __launch_bounds__(PROBE_THREADS, 1)
    k_probe(int op, int64_t iters, unsigned long long* cycles, float* sink) {
  extern __shared__ float probe_smem[];
  float v[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) v[c] = 0.25f + 0.01f * (float)c + 1e-6f * (float)threadIdx.x;
  if (threadIdx.x == 0) probe_smem[0] = 0.0f;
  __syncthreads();
  const unsigned long long t0 = clock64();
  if (op == 0) {
    // y <- 2^(-y) stays in [0.5, 1] for y in [0, 1]
    for (int64_t i = 0; i < iters; ++i)
#pragma unroll
      for (int c = 0; c < 8; ++c) v[c] = probe_ex2(-v[c]);
  } else if (op == 1) {
    // y <- y * a + b with a < 1: a contraction toward b / (1 - a)
    const float a = 0.999f, b = 0.000999f;
    for (int64_t i = 0; i < iters; ++i)
#pragma unroll
      for (int c = 0; c < 8; ++c) v[c] = fmaf(v[c], a, b);
  } else {
    float2 p[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) p[c] = make_float2(v[2 * c], v[2 * c + 1]);
    const float2 a = make_float2(0.999f, 0.998f), b = make_float2(0.000999f, 0.000998f);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < 4; ++c) p[c] = __ffma2_rn(p[c], a, b);
#pragma unroll
      for (int c = 0; c < 4; ++c) p[c] = __ffma2_rn(p[c], a, b);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) { v[2 * c] = p[c].x; v[2 * c + 1] = p[c].y; }
  }
  __syncthreads();
  const unsigned long long t1 = clock64();
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += v[c];
  sink[(int64_t)blockIdx.x * PROBE_THREADS + threadIdx.x] = s + probe_smem[0];
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace
}  // namespace kkm

// Rates of op (0: ex2.approx, 1: FP32 fma, 2: f32x2 fma) on the current device:
// per SM and clock (median over the SMs' own cycle counts) and over the
// whole device per second (CUDA events). Allocates and frees its own small
// buffers and synchronises the stream.
KKM_API kkm_status kkm_probe_unit_rate(int32_t op, int64_t iters, double* per_clk_sm, double* per_second,
                                       void* stream) {
  if (op < 0 || op > 2 || iters < 1 || iters > (int64_t(1) << 24) || !per_clk_sm || !per_second)
    return KKM_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return KKM_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return KKM_ECUDA;
  unsigned long long* cyc = nullptr;
  float* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  static std::atomic<uint64_t> attr{0};
  cudaError_t e = kkm::smem_limit_once(kkm::k_probe, kkm::PROBE_SMEM, attr);
  if (e == cudaSuccess) e = cudaMalloc(&cyc, sizeof(unsigned long long) * sms);
  if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(float) * (size_t)sms * kkm::PROBE_THREADS);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float ms = 0.0f;
  std::vector<unsigned long long> h(sms > 0 ? sms : 1);
  if (e == cudaSuccess) {
    // one untimed launch (module load, clocks up), then the timed one
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
      if (rep == 1) e = cudaEventRecord(e0, st);
      if (e == cudaSuccess) {
        kkm::k_probe<<<sms, kkm::PROBE_THREADS, kkm::PROBE_SMEM, st>>>(op, iters, cyc, sink);
        e = cudaGetLastError();
      }
      if (rep == 1 && e == cudaSuccess) e = cudaEventRecord(e1, st);
    }
  }
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaMemcpy(h.data(), cyc, sizeof(unsigned long long) * sms, cudaMemcpyDeviceToHost);
  if (cyc) cudaFree(cyc);
  if (sink) cudaFree(sink);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return KKM_ECUDA;
  // eight instructions per thread and iteration; a packed one is two FP32 FMAs
  const double per_block = (double)kkm::PROBE_THREADS * (double)iters * 8.0 * (op == 2 ? 2.0 : 1.0);
  std::sort(h.begin(), h.end());
  const double med = (double)h[h.size() / 2];
  *per_clk_sm = med > 0.0 ? per_block / med : 0.0;
  *per_second = ms > 0.0f ? per_block * sms / (ms * 1e-3) : 0.0;
  return KKM_OK;
}

// The failure-detection path of the tcgen05 passes: one bounded mbarrier wait
// (the passes' own routine) that nothing satisfies when arrive == 0.
KKM_API kkm_status kkm_probe_bounded_wait(int64_t limit_ns, int32_t arrive, void* stream) {
  if (limit_ns < 1000 || limit_ns > 5000000000LL || (arrive != 0 && arrive != 1)) return KKM_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int* d_out = nullptr;
  int h_out = -1;
  cudaError_t e = cudaMalloc(&d_out, sizeof(int));
  if (e == cudaSuccess) e = kkm::launch_wait_probe((uint64_t)limit_ns, arrive, d_out, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_out, d_out, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (d_out) cudaFree(d_out);
  if (e != cudaSuccess) return KKM_ECUDA;
  return h_out == 1 ? KKM_ETIMEOUT : (h_out == 0 ? KKM_OK : KKM_ECUDA);
}
