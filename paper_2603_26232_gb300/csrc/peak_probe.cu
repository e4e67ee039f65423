// Throughput probes of the GPU the library runs on: packed FP32 FMA
// (FFMA2, the butterfly instruction of the simulation kernels) and
// shared-memory load/store bandwidth (their transposes). The on-chip
// simulation of states of <= 14 qubits never touches HBM between layers;
// these two measured rates are its roofline. Plain HBM streams (write only,
// read only, copy) give the ceilings of the layer passes that only write
// (the first) or only read (the <C> pass).
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/paraqaoa.h"
#include "pq_internal.h"

namespace pq {

namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 16;  // independent FFMA2 chains per thread (hides the pipe latency)

// Every thread runs kChains independent chains x <- x * m + c of packed
// FP32 FMAs, `iters` times; the sum is written so that nothing is dead.
__global__ void __launch_bounds__(kProbeThreads) k_probe_ffma2(float2* out, int iters, float mval) {
  float2 x[kChains];
  const float t = (float)threadIdx.x * 1e-3f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = make_float2(t + k, t - k);
  const float2 m = make_float2(mval, mval), cst = make_float2(1e-7f, -1e-7f);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = __ffma2_rn(m, x[k], cst);
  }
  float2 s = make_float2(0.f, 0.f);
#pragma unroll
  for (int k = 0; k < kChains; ++k) s = make_float2(s.x + x[k].x, s.y + x[k].y);
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Every thread stores and reloads float2 words of a 32 KB shared buffer in
// conflict-free, consecutive order (a warp covers 256 contiguous bytes per
// access), `iters` rounds of 16 stores + 16 loads each.
__global__ void __launch_bounds__(kProbeThreads) k_probe_smem(float2* out, int iters) {
  __shared__ float2 buf[kProbeThreads * 16];
  const uint32_t tid = threadIdx.x;
  float2 v[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = make_float2((float)tid, (float)k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) buf[k * kProbeThreads + tid] = v[k];
    __syncwarp();
    // read another lane's words (same warp, so a warp barrier orders them)
    const uint32_t src = (tid & ~31u) | ((tid + 1 + i) & 31u);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const float2 w = buf[k * kProbeThreads + src];
      v[k] = make_float2(v[k].x + w.y, v[k].y + w.x);
    }
    __syncwarp();
  }
  float2 s = make_float2(0.f, 0.f);
#pragma unroll
  for (int k = 0; k < 16; ++k) s = make_float2(s.x + v[k].x, s.y + v[k].y);
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Grid-stride float4 streams over n4 elements.
__global__ void __launch_bounds__(kProbeThreads) k_stream_write(float4* p, size_t n4, float v) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x)
    p[i] = make_float4(v, v, v, v);
}
__global__ void __launch_bounds__(kProbeThreads) k_stream_read(const float4* p, size_t n4, float* out) {
  float s = 0.f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
    const float4 a = p[i];
    s += (a.x + a.y) + (a.z + a.w);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the loads live
}
__global__ void __launch_bounds__(kProbeThreads) k_stream_copy(const float4* a, float4* b, size_t n4) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x)
    b[i] = a[i];
}

}  // namespace

}  // namespace pq

extern "C" int paraqaoa_probe_streams(int device, int64_t bytes, double* write_gbs, double* read_gbs,
                                      double* copy_gbs) {
  using namespace pq;
  if (!write_gbs || !read_gbs || !copy_gbs || bytes < (int64_t(1) << 20) || bytes > (int64_t(1) << 34) ||
      bytes % 16 != 0)
    return PARAQAOA_E_INVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return PARAQAOA_E_INVAL;
  if (cudaSetDevice(device) != cudaSuccess) return PARAQAOA_E_CUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return PARAQAOA_E_CUDA;
  const int blocks = sms * 8;  // 8 resident CTAs of 256 threads per SM
  const size_t n4 = (size_t)bytes / 16;
  float4 *a = nullptr, *b = nullptr;
  float* out = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = PARAQAOA_OK;
  auto ck = [&](cudaError_t e) {
    if (e != cudaSuccess && rc == PARAQAOA_OK) rc = e == cudaErrorMemoryAllocation ? PARAQAOA_E_NOMEM : PARAQAOA_E_CUDA;
    return e == cudaSuccess;
  };
  ck(cudaMalloc(&a, (size_t)bytes));
  ck(cudaMalloc(&b, (size_t)bytes));
  ck(cudaMalloc(&out, sizeof(float) * (size_t)blocks * kProbeThreads));
  ck(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  ck(cudaEventCreate(&e0));
  ck(cudaEventCreate(&e1));
  if (rc == PARAQAOA_OK) {
    ck(cudaMemsetAsync(a, 0, (size_t)bytes, st));
    ck(cudaMemsetAsync(b, 0, (size_t)bytes, st));
  }
  float best[3] = {1e30f, 1e30f, 1e30f};
  for (int rep = 0; rep < 6 && rc == PARAQAOA_OK; ++rep) {  // the first round warms up
    for (int k = 0; k < 3 && rc == PARAQAOA_OK; ++k) {
      float ms = 0.f;
      ck(cudaEventRecord(e0, st));
      if (k == 0) k_stream_write<<<blocks, kProbeThreads, 0, st>>>(a, n4, 1.f);
      else if (k == 1) k_stream_read<<<blocks, kProbeThreads, 0, st>>>(b, n4, out);
      else k_stream_copy<<<blocks, kProbeThreads, 0, st>>>(a, b, n4);
      ck(cudaGetLastError());
      ck(cudaEventRecord(e1, st));
      ck(cudaEventSynchronize(e1));
      ck(cudaEventElapsedTime(&ms, e0, e1));
      if (rep > 0) best[k] = std::min(best[k], ms);
    }
  }
  if (rc == PARAQAOA_OK) {
    *write_gbs = (double)bytes / (best[0] * 1e-3) / 1e9;
    *read_gbs = (double)bytes / (best[1] * 1e-3) / 1e9;
    *copy_gbs = 2.0 * (double)bytes / (best[2] * 1e-3) / 1e9;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (out) cudaFree(out);
  if (b) cudaFree(b);
  if (a) cudaFree(a);
  return rc;
}

extern "C" int paraqaoa_probe_peaks(int device, double* fp32_tflops, double* smem_tbs) {
  using namespace pq;
  if (!fp32_tflops || !smem_tbs) return PARAQAOA_E_INVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return PARAQAOA_E_INVAL;
  if (cudaSetDevice(device) != cudaSuccess) return PARAQAOA_E_CUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return PARAQAOA_E_CUDA;
  const int blocks = sms * 8;  // 8 CTAs of 256 threads per SM: 64 warps, every scheduler busy
  float2* out = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = PARAQAOA_OK;
  auto ck = [&](cudaError_t e) {
    if (e != cudaSuccess && rc == PARAQAOA_OK) rc = e == cudaErrorMemoryAllocation ? PARAQAOA_E_NOMEM : PARAQAOA_E_CUDA;
    return e == cudaSuccess;
  };
  ck(cudaMalloc(&out, sizeof(float2) * (size_t)blocks * kProbeThreads));
  ck(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  ck(cudaEventCreate(&e0));
  ck(cudaEventCreate(&e1));
  const int fiters = 4096, siters = 2048;
  float best_f = 1e30f, best_s = 1e30f;
  for (int rep = 0; rep < 4 && rc == PARAQAOA_OK; ++rep) {  // the first round warms up
    float ms = 0.f;
    ck(cudaEventRecord(e0, st));
    k_probe_ffma2<<<blocks, kProbeThreads, 0, st>>>(out, fiters, 0.999999f);
    ck(cudaGetLastError());
    ck(cudaEventRecord(e1, st));
    ck(cudaEventSynchronize(e1));
    ck(cudaEventElapsedTime(&ms, e0, e1));
    if (rep > 0) best_f = std::min(best_f, ms);
    ck(cudaEventRecord(e0, st));
    k_probe_smem<<<blocks, kProbeThreads, 0, st>>>(out, siters);
    ck(cudaGetLastError());
    ck(cudaEventRecord(e1, st));
    ck(cudaEventSynchronize(e1));
    ck(cudaEventElapsedTime(&ms, e0, e1));
    if (rep > 0) best_s = std::min(best_s, ms);
  }
  if (rc == PARAQAOA_OK) {
    // an FFMA2 is two FMAs of two flops each
    const double flops = (double)blocks * kProbeThreads * fiters * kChains * 4.0;
    const double bytes = (double)blocks * kProbeThreads * siters * 16.0 * 2.0 * sizeof(float2);
    *fp32_tflops = flops / (best_f * 1e-3) / 1e12;
    *smem_tbs = bytes / (best_s * 1e-3) / 1e12;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (out) cudaFree(out);
  return rc;
}
