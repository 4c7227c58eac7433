// Measured issue rates of the pipes the force kernels are bound by, on the
// GPU this library runs on: binary64 FMA (FP64 pipe), binary32 FMA scalar and
// packed (FMA pipes), and the SFU reciprocal square root.  Each rate comes from
// a kernel that runs only independent chains of that one instruction over a
// full wave of resident blocks, timed with CUDA events; the SM clock of the
// same run comes from the SMs' cycle counters (per SM, the span from the first
// block's start to the last block's end on it: warps are not scheduled fairly,
// so one block alone finishes early and would understate the span).  These
// are the denominators of the force kernels' rooflines: a kernel bound by a
// pipe can reach at most that pipe's rate divided by its instructions per
// interaction.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <vector>

#include "nbody_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;

__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ unsigned sm_id() {
  unsigned r;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
  return r;
}

// sink[0] keeps the results alive; rec[3 b .. 3 b + 2] = (SM id, start, end
// cycle counts) of block b.
__global__ void __launch_bounds__(kThreads) k_rate_dfma(double b, double c, int iters,
                                                        double *sink, unsigned long long *rec) {
  const unsigned long long t0 = clock64();
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; k++) a[k] = threadIdx.x * 1e-3 + k;
  for (int it = 0; it < iters; it++)
#pragma unroll
    for (int k = 0; k < kChains; k++) a[k] = fma(a[k], b, c);
  double s = 0;
#pragma unroll
  for (int k = 0; k < kChains; k++) s += a[k];
  if (s == 1234.5678) sink[0] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    rec[3 * blockIdx.x] = sm_id();
    rec[3 * blockIdx.x + 1] = t0;
    rec[3 * blockIdx.x + 2] = clock64();
  }
}

__global__ void __launch_bounds__(kThreads) k_rate_ffma(float b, float c, int iters, double *sink) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; k++) a[k] = threadIdx.x * 1e-3f + k;
  for (int it = 0; it < iters; it++)
#pragma unroll
    for (int k = 0; k < kChains; k++) a[k] = fmaf(a[k], b, c);
  float s = 0;
#pragma unroll
  for (int k = 0; k < kChains; k++) s += a[k];
  if (s == 1234.5678f) sink[0] = s;
}

__global__ void __launch_bounds__(kThreads) k_rate_ffma2(float b, float c, int iters,
                                                         double *sink) {
  float2 a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; k++) a[k] = make_float2(threadIdx.x * 1e-3f + k, k - 0.5f);
  const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
  for (int it = 0; it < iters; it++)
#pragma unroll
    for (int k = 0; k < kChains; k++) a[k] = __ffma2_rn(a[k], b2, c2);
  float s = 0;
#pragma unroll
  for (int k = 0; k < kChains; k++) s += a[k].x + a[k].y;
  if (s == 1234.5678f) sink[0] = s;
}

__global__ void __launch_bounds__(kThreads) k_rate_rsqrt(int iters, double *sink) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; k++) a[k] = 1.5f + threadIdx.x * 1e-3f + k;
  for (int it = 0; it < iters; it++)
#pragma unroll
    for (int k = 0; k < kChains; k++) a[k] = rsqrt_approx(a[k]);
  float s = 0;
#pragma unroll
  for (int k = 0; k < kChains; k++) s += a[k];
  if (s == 1234.5678f) sink[0] = s;
}

}  // namespace

extern "C" int nbody_measure_pipes(double *out, int nout) {
  if (!out || nout < NBODY_PIPE_FIELDS)
    return nb::record_error(NBODY_EINVAL, "out needs NBODY_PIPE_FIELDS doubles");
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rate_dfma, kThreads, 0);
  if (e != cudaSuccess) return nb::record_error(NBODY_ECUDA, "device query", e);
  if (per_sm < 1) per_sm = 1;
  const int blocks = sms * per_sm;  // one full wave
  const double threads = (double)blocks * kThreads;
  double *sink = nullptr;
  unsigned long long *rec = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaMalloc(&sink, sizeof(double)) != cudaSuccess ||
      cudaMalloc(&rec, sizeof(unsigned long long) * 3 * blocks) != cudaSuccess) {
    cudaFree(sink);
    return nb::record_error(NBODY_ENOMEM, "sink");
  }
  if ((e = cudaEventCreate(&a)) != cudaSuccess || (e = cudaEventCreate(&b)) != cudaSuccess) {
    cudaFree(sink);
    cudaFree(rec);
    return nb::record_error(NBODY_ECUDA, "events", e);
  }
  std::vector<unsigned long long> h((size_t)3 * blocks);
  // iteration counts for ~20-40 ms per kernel at nominal rates
  const int it_dfma = 8000, it_ffma = 160000, it_rsqrt = 40000;
  float ms[4] = {0, 0, 0, 0};
  double cycles = 0;
  int rc = NBODY_OK;
  for (int rep = 0; rep < 2 && rc == NBODY_OK; rep++) {  // the first pass warms up
    for (int k = 0; k < 4; k++) {
      cudaEventRecord(a, 0);
      if (k == 0) k_rate_dfma<<<blocks, kThreads>>>(1.0000001, -1e-9, it_dfma, sink, rec);
      if (k == 1) k_rate_ffma<<<blocks, kThreads>>>(1.0000001f, -1e-9f, it_ffma, sink);
      if (k == 2) k_rate_ffma2<<<blocks, kThreads>>>(1.0000001f, -1e-9f, it_ffma, sink);
      if (k == 3) k_rate_rsqrt<<<blocks, kThreads>>>(it_rsqrt, sink);
      cudaEventRecord(b, 0);
      if ((e = cudaEventSynchronize(b)) != cudaSuccess ||
          (e = cudaEventElapsedTime(&ms[k], a, b)) != cudaSuccess) {
        rc = nb::record_error(NBODY_ECUDA, "rate kernel", e);
        break;
      }
      if (k == 0) {
        if ((e = cudaMemcpy(h.data(), rec, sizeof(unsigned long long) * h.size(),
                            cudaMemcpyDeviceToHost)) != cudaSuccess) {
          rc = nb::record_error(NBODY_ECUDA, "cycle count", e);
          break;
        }
        // per SM: first start to last end; the median over SMs
        std::map<unsigned long long, std::pair<unsigned long long, unsigned long long>> span;
        for (int q = 0; q < blocks; q++) {
          auto it = span.find(h[3 * q]);
          if (it == span.end())
            span[h[3 * q]] = {h[3 * q + 1], h[3 * q + 2]};
          else {
            it->second.first = std::min(it->second.first, h[3 * q + 1]);
            it->second.second = std::max(it->second.second, h[3 * q + 2]);
          }
        }
        std::vector<double> cyc;
        for (auto &kv : span) cyc.push_back((double)(kv.second.second - kv.second.first));
        std::sort(cyc.begin(), cyc.end());
        cycles = cyc.empty() ? 0.0 : cyc[cyc.size() / 2];
      }
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(sink);
  cudaFree(rec);
  if (rc) return rc;
  if (!(cycles > 0)) return nb::record_error(NBODY_ECUDA, "no cycle count");
  const double clk = cycles / (ms[0] * 1e-3);  // SM cycles per second during the DFMA kernel
  const double dfma = threads * kChains * it_dfma / (ms[0] * 1e-3);
  const double ffma = threads * kChains * it_ffma / (ms[1] * 1e-3);
  const double ffma2 = threads * kChains * it_ffma * 2.0 / (ms[2] * 1e-3);  // lane-ops
  const double rsq = threads * kChains * it_rsqrt / (ms[3] * 1e-3);
  out[0] = sms;
  out[1] = clk / 1e6;
  out[2] = dfma / 1e9;
  out[3] = ffma / 1e9;
  out[4] = ffma2 / 1e9;
  out[5] = rsq / 1e9;
  out[6] = dfma / (clk * sms);
  out[7] = ffma2 / (clk * sms);
  out[8] = rsq / (clk * sms);
  return NBODY_OK;
}
