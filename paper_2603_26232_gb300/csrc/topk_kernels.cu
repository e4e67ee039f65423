// Selective Distribution Exploration (Sec. 3.3.2): the K most probable
// bitstrings of each final state, K <= 32.
//
// Each candidate is packed into one 64-bit key, (float bits of P(z)) << 32 |
// (~z), so that a larger key means a higher probability and, between equal
// probabilities, the smaller z. A warp keeps a running top-32 list, one key
// per lane, sorted descending; each batch of 32 new keys is sorted with a
// warp bitonic sort and merged in (elementwise max against the reversed list,
// then a bitonic merge). Stage 1 reduces chunks of 4096 entries to 32 keys;
// stage 2 merges the chunk lists of each instance.
#include <cuda_runtime.h>

#include <mutex>

#include "pq_internal.h"

namespace pq {

constexpr int kTopkChunk = 4096;

__device__ __forceinline__ uint64_t umax64(uint64_t a, uint64_t b) { return a > b ? a : b; }
__device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }

__device__ __forceinline__ uint64_t warp_sort_desc(uint64_t key, uint32_t lane) {
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      uint64_t o = __shfl_xor_sync(0xffffffffu, key, j);
      bool desc = (lane & k) == 0;
      bool lower = (lane & j) == 0;
      key = (lower == desc) ? umax64(key, o) : umin64(key, o);
    }
  }
  return key;
}

// Merge a descending list `b` (one key per lane) into descending `top`.
__device__ __forceinline__ uint64_t warp_merge_desc(uint64_t top, uint64_t b, uint32_t lane) {
  uint64_t rb = __shfl_sync(0xffffffffu, b, 31 - lane);
  uint64_t cnd = umax64(top, rb);  // bitonic, holds the 32 largest of both
#pragma unroll
  for (int j = 16; j > 0; j >>= 1) {
    uint64_t o = __shfl_xor_sync(0xffffffffu, cnd, j);
    cnd = ((lane & j) == 0) ? umax64(cnd, o) : umin64(cnd, o);
  }
  return cnd;
}

__device__ __forceinline__ uint64_t make_key(float2 a, uint32_t z) {
  float pz = fmaf(a.x, a.x, a.y * a.y);
  return ((uint64_t)__float_as_uint(pz) << 32) | (uint64_t)(~z);
}

// Stage 1: block b handles chunk (b - chunk_off[i]) of instance i.
__global__ void k_topk_chunks(const InstDev* __restrict__ inst, int32_t count,
                              const int64_t* __restrict__ chunk_off, int32_t raw,
                              const float2* __restrict__ states, uint64_t* __restrict__ scratch) {
  __shared__ uint64_t lists[8][32];
  const int64_t b = blockIdx.x;
  int lo = 0, hi = count - 1;
  while (lo < hi) {  // last i with chunk_off[i] <= b
    int mid = (lo + hi + 1) >> 1;
    if (chunk_off[mid] <= b) lo = mid; else hi = mid - 1;
  }
  const int i = lo;
  const InstDev I = inst[i];
  const uint64_t cnt = raw ? (1ull << I.n) : (I.n == 1 ? 1ull : (1ull << (I.n - 1)));
  const uint64_t base = (uint64_t)(b - chunk_off[i]) * kTopkChunk;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const float2* st = states + I.state_off;
  uint64_t top = 0;
  for (int it = 0; it < kTopkChunk / (8 * 32); ++it) {
    uint64_t z = base + (uint64_t)warp * (kTopkChunk / 8) + (uint64_t)it * 32 + lane;
    uint64_t key = (z < cnt) ? make_key(st[z], (uint32_t)z) : 0ull;
    key = warp_sort_desc(key, lane);
    top = warp_merge_desc(top, key, lane);
  }
  lists[warp][lane] = top;
  __syncthreads();
  if (warp == 0) {
    for (int w = 1; w < 8; ++w) top = warp_merge_desc(top, lists[w][lane], lane);
    scratch[(uint64_t)b * 32 + lane] = top;
  }
}

// Stage 2: merge the chunk lists of instance blockIdx.x; write the first K.
__global__ void k_topk_final(const int64_t* __restrict__ chunk_off, int32_t K,
                             const uint64_t* __restrict__ scratch, uint32_t* __restrict__ out_z,
                             float* __restrict__ out_p) {
  __shared__ uint64_t lists[8][32];
  const int i = blockIdx.x;
  const int64_t c0 = chunk_off[i], c1 = chunk_off[i + 1];
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  uint64_t top = 0;
  for (int64_t c = c0 + warp; c < c1; c += 8) top = warp_merge_desc(top, scratch[(uint64_t)c * 32 + lane], lane);
  lists[warp][lane] = top;
  __syncthreads();
  if (warp == 0) {
    for (int w = 1; w < 8; ++w) top = warp_merge_desc(top, lists[w][lane], lane);
    if ((int)lane < K) {
      out_z[(int64_t)i * K + lane] = ~(uint32_t)(top & 0xffffffffu);
      out_p[(int64_t)i * K + lane] = __uint_as_float((uint32_t)(top >> 32));
    }
  }
}

cudaError_t launch_topk_stages(const InstDev* inst, int32_t count, int32_t K, int32_t raw,
                               const int64_t* chunk_off_dev, int64_t total_chunks,
                               const float2* states, uint64_t* scratch, uint32_t* out_z,
                               float* out_p, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  if (total_chunks > 0x7fffffff) return cudaErrorInvalidValue;
  k_topk_chunks<<<(unsigned)total_chunks, 256, 0, st>>>(inst, count, chunk_off_dev, raw, states, scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_topk_final<<<count, 256, 0, st>>>(chunk_off_dev, K, scratch, out_z, out_p);
  return cudaGetLastError();
}

int64_t topk_chunks_of(int n, int raw) {
  uint64_t cnt = raw ? (1ull << n) : (n == 1 ? 1ull : (1ull << (n - 1)));
  return (int64_t)((cnt + kTopkChunk - 1) / kTopkChunk);
}

}  // namespace pq

// ---------------------------------------------------------------------------
// Allocation-free top-K for one state given by a device pointer.
//
// Some callers cannot let a library call cudaMalloc: a host process whose own
// caching allocator already holds nearly all device memory, or a
// latency-critical loop that cannot take cudaMalloc's implicit device
// synchronisation. For them the two top-K stages run here on a fixed
// file-scope scratch array instead of context-owned buffers.
//
// The array lives in every GPU that loads this library, for as long as the
// process runs. In host code its name is only a host-side stand-in, so its
// device address is fetched with cudaGetSymbolAddress once per device (on the
// first call made with that device current) and passed to the kernels.
// Every call shares the array: calls that overlap on the GPU race. Nothing in
// it needs clearing: stage 1 writes every entry stage 2 reads.

namespace {

constexpr int64_t kNoAllocMaxChunks = 8192;  // 2^25 ranked entries in chunks of 4096
static __device__ __align__(256) uint64_t g_topk_scratch[kNoAllocMaxChunks * 32];  // 2 MiB

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
uint64_t* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array for the current device (set-up once).
cudaError_t noalloc_scratch(uint64_t** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_topk_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = static_cast<uint64_t*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

__global__ void k_topk_chunks_one(const float2* __restrict__ st, uint64_t cnt,
                                  uint64_t* __restrict__ scratch) {
  __shared__ uint64_t lists[8][32];
  const uint64_t base = (uint64_t)blockIdx.x * pq::kTopkChunk;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  uint64_t top = 0;
  for (int it = 0; it < pq::kTopkChunk / (8 * 32); ++it) {
    const uint64_t z = base + (uint64_t)warp * (pq::kTopkChunk / 8) + (uint64_t)it * 32 + lane;
    uint64_t key = (z < cnt) ? pq::make_key(st[z], (uint32_t)z) : 0ull;
    key = pq::warp_sort_desc(key, lane);
    top = pq::warp_merge_desc(top, key, lane);
  }
  lists[warp][lane] = top;
  __syncthreads();
  if (warp == 0) {
    for (int w = 1; w < 8; ++w) top = pq::warp_merge_desc(top, lists[w][lane], lane);
    scratch[(uint64_t)blockIdx.x * 32 + lane] = top;
  }
}

__global__ void k_topk_final_one(int64_t chunks, int32_t K, const uint64_t* __restrict__ scratch,
                                 uint32_t* __restrict__ out_z, float* __restrict__ out_p) {
  __shared__ uint64_t lists[8][32];
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  uint64_t top = 0;
  for (int64_t c = warp; c < chunks; c += 8) top = pq::warp_merge_desc(top, scratch[(uint64_t)c * 32 + lane], lane);
  lists[warp][lane] = top;
  __syncthreads();
  if (warp == 0) {
    for (int w = 1; w < 8; ++w) top = pq::warp_merge_desc(top, lists[w][lane], lane);
    if ((int)lane < K) {
      out_z[lane] = ~(uint32_t)(top & 0xffffffffu);
      out_p[lane] = __uint_as_float((uint32_t)(top >> 32));
    }
  }
}

}  // namespace

extern "C" int paraqaoa_topk_noalloc(const float* state_dev, int32_t n, int32_t K, uint32_t flags,
                                     uint32_t* out_z_dev, float* out_p_dev, void* stream) {
  if (!state_dev || !out_z_dev || !out_p_dev || n < 1 || n > PARAQAOA_MAX_QUBITS || K < 1 ||
      K > PARAQAOA_MAX_TOPK)
    return PARAQAOA_E_INVAL;
  const int raw = (flags & PARAQAOA_TOPK_RAW) ? 1 : 0;
  const uint64_t cnt = raw ? (1ull << n) : (n == 1 ? 1ull : (1ull << (n - 1)));
  if ((uint64_t)K > cnt) return PARAQAOA_E_INVAL;
  const int64_t chunks = pq::topk_chunks_of(n, raw);
  if (chunks > kNoAllocMaxChunks) return PARAQAOA_E_SCRATCH_LIMIT;
  uint64_t* scratch = nullptr;
  cudaError_t e = noalloc_scratch(&scratch);
  if (e != cudaSuccess) return PARAQAOA_E_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_topk_chunks_one<<<(unsigned)chunks, 256, 0, st>>>(reinterpret_cast<const float2*>(state_dev), cnt, scratch);
  e = cudaGetLastError();
  if (e != cudaSuccess) return PARAQAOA_E_CUDA;
  k_topk_final_one<<<1, 256, 0, st>>>(chunks, K, scratch, out_z_dev, out_p_dev);
  return cudaGetLastError() == cudaSuccess ? PARAQAOA_OK : PARAQAOA_E_CUDA;
}
