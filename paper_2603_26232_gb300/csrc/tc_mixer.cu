// Split-precision tensor-core mixer (tcgen05, sm_103a).
//
// The mixer of QAOA (Sec. 2.2, U_M = exp(-i beta sum_j X_j)) restricted to k
// consecutive qubits [q0, q0 + k) is a dense 2^k x 2^k matrix. In the gauge
// the simulation kernels use (s_z = i^popcount(z) psi_z, see sim_kernels.cu)
// one qubit's factor is the real butterfly [[1, mu], [-mu, 1]] (the layer
// scalar is folded elsewhere), so the k-qubit block is the real Kronecker power
//   M[c', c] = mu^popcount(c' xor c) (-1)^popcount(c' and not c),
// and applying it is a real product D = A M^T with A[rows x 2^k] holding the
// real and imaginary parts of the amplitudes that share every other qubit.
//
// The product runs on the 5th-generation tensor cores with FP32 operands split
// into two 16-bit parts, x = x_hi + x_lo (BF16 or FP16), and three products
// A_hi M_hi^T + A_hi M_lo^T + A_lo M_hi^T accumulated in FP32 in tensor memory
// (the lo x lo term is below the split's own rounding). FP16 parts carry 11
// significant bits each but have a narrow exponent range, so A is scaled by a
// power of two (exact) before splitting and D scaled back. The gauge
// butterflies are unnormalised: each mixed qubit multiplies the state's norm
// by sqrt(1 + mu^2) (the layer scalar is folded into the next phase), so
// after the q0 qubits below the block the norm, and with it every amplitude,
// is at most (1 + mu^2)^(q0/2). The block's scale 2^(ceil(n/2) - e) with
// e = ceil((q0/2) log2(1 + mu^2)) keeps every scaled amplitude below
// 2^ceil(n/2) <= 2^15 (FP16 overflows at 65504) while a spread-out state's
// amplitudes, 2^(-n/2) of the norm, land near 1.
//
// One CTA of 256 threads owns a tile of 64 amplitude groups x 2^k amplitudes
// (128 rows: real parts, then imaginary parts). Per tile: coalesced FP32
// loads (all issued before the first use), split into shared memory in the
// canonical no-swizzle K-major layout,
// one thread issues 3 x 2^k/16 MMAs (M = 128, N = 2^k, K = 16) into 2^k TMEM
// columns, tcgen05.commit signals an mbarrier, and the accumulators come back
// with tcgen05.ld, are staged through shared memory and stored coalesced.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "pq_internal.h"

namespace pq {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor (tcgen05): no swizzle, K-major. Core
// matrices are 8 rows x 16 bytes; lbo = byte distance between core matrices
// adjacent along K, sbo = between core matrices adjacent along M (or N).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of sm_100-class tensor cores
  // base offset 0, absolute-offset mode 0, layout type 0 (no swizzle)
  return d;
}

// Instruction descriptor, kind::f16: D FP32, A and B both BF16 (or both FP16),
// K-major A and B, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t instr_desc(bool fp16, int M, int N) {
  return (1u << 4) | ((fp16 ? 0u : 1u) << 7) | ((fp16 ? 0u : 1u) << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

template <bool FP16>
struct Split;
template <>
struct Split<false> {
  __device__ static void run(float x, uint16_t& hi, uint16_t& lo) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(l);
  }
};
template <>
struct Split<true> {
  __device__ static void run(float x, uint16_t& hi, uint16_t& lo) {
    const __half h = __float2half_rn(x);
    const __half l = __float2half_rn(x - __half2float(h));
    hi = __half_as_ushort(h);
    lo = __half_as_ushort(l);
  }
};

// Byte offset of element (row, k) in the canonical layout of a [rows x K]
// 16-bit matrix: core matrix (row / 8, k / 8) at (row / 8) * sbo + (k / 8) * 128.
template <int K>
__device__ __forceinline__ uint32_t canon_off(uint32_t row, uint32_t k) {
  constexpr uint32_t sbo = K * 16;
  return (row >> 3) * sbo + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

constexpr int kRows = 128;      // MMA M: 64 amplitude groups x (re, im)
constexpr int kGroups = 64;
// Bounded waits are measured on the global nanosecond timer. After a wait
// gave up, the products still in flight get kDrainNs more before the TMEM
// columns are freed.
constexpr uint64_t kDrainNs = 1000000000ull;

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait until the mbarrier completes phase `phase`, for at most limit_ns
// (checked before each poll, so a limit of 0 gives up at once). True when the
// phase completed.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t phase, uint64_t limit_ns) {
  const uint64_t t0 = global_ns();
  for (;;) {
    if (global_ns() - t0 >= limit_ns) return false;
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(mbar), "r"(phase)
        : "memory");
    if (done) return true;
  }
}

}  // namespace

// Shared-memory bytes of one CTA for 2^KB columns.
__host__ __device__ constexpr size_t tc_smem_bytes(int KB) {
  // A_hi, A_lo (reused as the FP32 staging buffer), B_hi, B_lo, barrier + TMEM address
  return (size_t)2 * kRows * (1 << KB) * 2 + (size_t)2 * (1 << KB) * (1 << KB) * 2 + 64;
}

// Apply the mixer block [q0, q0 + KB) of layer `layer` to every instance in
// list (all with n qubits), in place on the interleaved complex64 states.
// Grid: nlist x ctas_per_inst CTAs; CTA (i, j) walks tiles j, j + ctas, ...
// of instance i. err (device int) is set to 1 if an mbarrier wait gave up
// (after wait_ns nanoseconds); the CTA then stops, lets the products in
// flight finish (bounded by kDrainNs), frees its TMEM columns and returns.
constexpr int kThreads = 256;  // 8 warps: TMEM lane quarter w % 4, column half w / 4

template <int KB, bool FP16>
__global__ void __launch_bounds__(kThreads, KB < 7 ? 2 : 1)
    k_mixer_tc(const InstDev* __restrict__ inst_all, const int32_t* __restrict__ list, int32_t n, int32_t q0,
               int32_t layer, int32_t ctas_per_inst, float2* __restrict__ states, uint64_t wait_ns,
               int* __restrict__ err) {
  constexpr int K = 1 << KB;       // MMA N and K extent
  constexpr int A_BYTES = kRows * K * 2;
  constexpr int B_BYTES = K * K * 2;
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* a_hi = smraw;
  unsigned char* a_lo = smraw + A_BYTES;
  unsigned char* b_hi = smraw + 2 * A_BYTES;
  unsigned char* b_lo = b_hi + B_BYTES;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(b_lo + B_BYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 1);
  // FP32 staging [kRows][K], column c of row r at c ^ (r & 31) (conflict-free
  // both ways); it aliases the A buffers, which the finished MMAs no longer read
  float* stage = reinterpret_cast<float*>(smraw);
  const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const InstDev I = inst_all[list[blockIdx.x / ctas_per_inst]];
  const int cta_j = blockIdx.x % ctas_per_inst;
  const float mu = I.mu[layer];
  float2* psi = states + I.state_off;
  const int64_t tiles = (int64_t)1 << (n - KB - 6);
  const uint32_t lomask = (1u << q0) - 1u;

  // ---- set-up: M_hi / M_lo, mbarrier, TMEM columns
  for (uint32_t e = tid; e < (uint32_t)(K * K); e += blockDim.x) {
    const uint32_t cp = e / K, c = e % K;  // B row (N index) c', column (K index) c
    const int d = __popc(cp ^ c), neg = __popc(cp & ~c) & 1;
    float v = 1.f;
    for (int t = 0; t < d; ++t) v *= mu;
    if (neg) v = -v;
    uint16_t hi, lo;
    Split<FP16>::run(v, hi, lo);
    *reinterpret_cast<uint16_t*>(b_hi + canon_off<K>(cp, c)) = hi;
    *reinterpret_cast<uint16_t*>(b_lo + canon_off<K>(cp, c)) = lo;
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"((uint32_t)(K < 32 ? 32 : K))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  // FP16 parts: the block's power-of-two scale (see the header comment)
  float scale = 1.f;
  if (FP16) {
    const int e = (int)ceilf(0.5f * (float)q0 * log2f(fmaf(mu, mu, 1.f)));
    scale = ldexpf(1.f, (n + 1) / 2 - e);
  }
  const float inv = 1.f / scale;
  uint32_t phase = 0;
  bool ok = true;

  for (int64_t t = cta_j; t < tiles && ok; t += ctas_per_inst) {
    // ---- load the tile (every load issued first), split into A_hi / A_lo:
    // thread (u, q) handles amplitude group u and column pairs c = 2q + 8i
    const uint32_t u = tid & (kGroups - 1), q = tid >> 6;
    const int64_t gi = t * kGroups + u;  // amplitude-group index (hi bits, lo bits)
    const int64_t base = ((gi >> q0) << (q0 + KB)) | (gi & lomask);
    constexpr int NP = K / 8;            // column pairs per thread
    constexpr int NB = NP < 8 ? NP : 8;  // pairs loaded per batch (caps the registers in flight)
#pragma unroll 1
    for (int i0 = 0; i0 < NP; i0 += NB) {
    float2 v[2 * NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const int c = 2 * (int)q + 8 * (i0 + i);
      v[2 * i] = psi[base + ((int64_t)c << q0)];
      v[2 * i + 1] = psi[base + ((int64_t)(c + 1) << q0)];
    }
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const int c = 2 * (int)q + 8 * (i0 + i);
      const float2 x0 = v[2 * i], x1 = v[2 * i + 1];
      uint16_t h0, l0, h1, l1;
      Split<FP16>::run(x0.x * scale, h0, l0);
      Split<FP16>::run(x1.x * scale, h1, l1);
      *reinterpret_cast<uint32_t*>(a_hi + canon_off<K>(u, c)) = (uint32_t)h0 | ((uint32_t)h1 << 16);
      *reinterpret_cast<uint32_t*>(a_lo + canon_off<K>(u, c)) = (uint32_t)l0 | ((uint32_t)l1 << 16);
      Split<FP16>::run(x0.y * scale, h0, l0);
      Split<FP16>::run(x1.y * scale, h1, l1);
      *reinterpret_cast<uint32_t*>(a_hi + canon_off<K>(u + kGroups, c)) = (uint32_t)h0 | ((uint32_t)h1 << 16);
      *reinterpret_cast<uint32_t*>(a_lo + canon_off<K>(u + kGroups, c)) = (uint32_t)l0 | ((uint32_t)l1 << 16);
    }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // ---- three split products, one issuing thread
    if (tid == 0) {
      constexpr uint32_t idesc = instr_desc(FP16, kRows, K);
      const uint32_t ah = smem_u32(a_hi), al = smem_u32(a_lo), bh = smem_u32(b_hi), bl = smem_u32(b_lo);
      constexpr uint32_t sboA = K * 16, sboB = K * 16;
#pragma unroll 1
      for (int prod = 0; prod < 3; ++prod) {
        const uint32_t a = prod == 2 ? al : ah, b = prod == 1 ? bl : bh;
#pragma unroll 1
        for (int s = 0; s < K / 16; ++s) {
          const uint64_t da = smem_desc(a + s * 256, 128, sboA);
          const uint64_t db = smem_desc(b + s * 256, 128, sboB);
          const uint32_t acc = (prod > 0 || s > 0) ? 1u : 0u;
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
              "l"(da), "l"(db), "r"(idesc), "r"(acc)
              : "memory");
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(mbar))
                   : "memory");
    }
    // ---- wait for the products (bounded)
    {
      const bool done = mbar_wait_bounded(smem_u32(mbar), phase, wait_ns);
      // every thread takes the same decision (the loads below are warp-collective)
      ok = !__syncthreads_or(!done);
      if (!ok && tid == 0) atomicExch(err, 1);
    }
    if (!ok) break;
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // ---- accumulators -> registers -> staging: warp w reads TMEM lanes
    // 32 (w % 4) .. + 31 (rows) and columns [(w / 4) K / 2, (w / 4 + 1) K / 2)
    const uint32_t row = (warp & 3) * 32 + lane;
    const uint32_t lane_base = tmem + (((warp & 3) * 32u) << 16);
    constexpr int CH = K / 2 < 32 ? K / 2 : 32;  // columns per tcgen05.ld
#pragma unroll 1
    for (int c0 = (int)(warp >> 2) * (K / 2); c0 < (int)(warp >> 2) * (K / 2) + K / 2; c0 += CH) {
      uint32_t r[32];
      if constexpr (CH == 32) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
              "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
              "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
              "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(lane_base + (uint32_t)c0));
      } else {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
              "=r"(r[15])
            : "r"(lane_base + (uint32_t)c0));
      }
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < CH; ++j) stage[row * K + ((c0 + j) ^ (row & 31))] = __uint_as_float(r[j]) * inv;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    // ---- coalesced stores of the tile
    for (int c = (int)q; c < K; c += 4)
      psi[base + ((int64_t)c << q0)] =
          make_float2(stage[u * K + (c ^ (u & 31))], stage[(u + kGroups) * K + (c ^ ((u + kGroups) & 31))]);
    __syncthreads();  // staging (aliasing A) is free for the next tile's split
  }
  if (!ok) mbar_wait_bounded(smem_u32(mbar), phase, kDrainNs);  // the products in flight, before the columns are freed
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)(K < 32 ? 32 : K))
                 : "memory");
  }
}

template <int KB, bool FP16>
static cudaError_t launch_tc_t(const InstDev* inst, const int32_t* list, int32_t nlist, int32_t n, int32_t q0,
                               int32_t layer, float2* states, uint64_t wait_ns, int* err, int num_sms, cudaStream_t st) {
  const size_t smem = tc_smem_bytes(KB);
  static_assert((size_t)2 * kRows * (1 << KB) * 2 == (size_t)kRows * (1 << KB) * 4, "staging fills the A buffers");
  cudaError_t e = cudaFuncSetAttribute(k_mixer_tc<KB, FP16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t tiles = (int64_t)1 << (n - KB - 6);
  const int per = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, ((int64_t)num_sms * 2 + nlist - 1) / nlist));
  const int64_t blocks = (int64_t)nlist * per;
  if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
  k_mixer_tc<KB, FP16><<<(unsigned)blocks, kThreads, smem, st>>>(inst, list, n, q0, layer, per, states, wait_ns, err);
  return cudaGetLastError();
}

cudaError_t launch_mixer_tc(int kb, bool fp16, const InstDev* inst, const int32_t* list, int32_t nlist, int32_t n,
                            int32_t q0, int32_t layer, float2* states, uint64_t wait_ns, int* err, int num_sms,
                            cudaStream_t st) {
  if (nlist <= 0) return cudaSuccess;
  if (n < kb + 6 || q0 < 0 || q0 + kb > n) return cudaErrorInvalidValue;
#define PQ_TC(KBV)                                                                                            \
  if (kb == KBV)                                                                                              \
    return fp16 ? launch_tc_t<KBV, true>(inst, list, nlist, n, q0, layer, states, wait_ns, err, num_sms, st)    \
                : launch_tc_t<KBV, false>(inst, list, nlist, n, q0, layer, states, wait_ns, err, num_sms, st);
  PQ_TC(5)
  PQ_TC(6)
  PQ_TC(7)
#undef PQ_TC
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Elementwise steps of the tensor-core variant, with the cut table C(z)
// (uint16, built by k_cut_table) read from HBM.
// Phase of layer l: s_z <- (init ? i^popcount(z) : s_z) * tab_l[C(z)].
__global__ void k_tc_phase(const InstDev* __restrict__ inst_all, const int32_t* __restrict__ list, int32_t n,
                           int32_t layer, int32_t init, const float2* __restrict__ tables,
                           const uint16_t* __restrict__ cuts, int64_t cut_stride, float2* __restrict__ states) {
  const InstDev I = inst_all[list[blockIdx.y]];
  const float2* tab = tables + I.table_off + (int64_t)layer * (I.W + 1);
  const uint16_t* C = cuts + (int64_t)blockIdx.y * cut_stride;
  float2* s = states + I.state_off;
  const int64_t dim = (int64_t)1 << n;
  for (int64_t z = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; z < dim; z += (int64_t)gridDim.x * blockDim.x) {
    float2 a;
    if (init) {
      const int r = __popcll((unsigned long long)z) & 3;
      const float sg = (r & 2) ? -1.f : 1.f;
      a = (r & 1) ? make_float2(0.f, sg) : make_float2(sg, 0.f);
    } else {
      a = s[z];
    }
    const float2 t = tab[min((int)C[z], I.W)];
    s[z] = make_float2(fmaf(a.x, t.x, -a.y * t.y), fmaf(a.x, t.y, a.y * t.x));
  }
}

// <C> partial sums (FP64 per block, fixed order) and the return from the gauge:
// psi_z = i^-popcount(z) lambda_p s_z.
__global__ void k_tc_finish(const InstDev* __restrict__ inst_all, const int32_t* __restrict__ list, int32_t n,
                            const uint16_t* __restrict__ cuts, int64_t cut_stride, float2* __restrict__ states,
                            double* __restrict__ partials, int32_t keep) {
  __shared__ double red[8];
  const InstDev I = inst_all[list[blockIdx.y]];
  const uint16_t* C = cuts + (int64_t)blockIdx.y * cut_stride;
  float2* s = states + I.state_off;
  const int64_t dim = (int64_t)1 << n;
  double acc = 0.0;
  for (int64_t z = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; z < dim; z += (int64_t)gridDim.x * blockDim.x) {
    const float2 a = s[z];
    acc += (double)fmaf(a.x, a.x, a.y * a.y) * (double)C[z];
    if (keep) {
      const int r = (-__popcll((unsigned long long)z)) & 3;
      const float2 f = I.final_scale;
      float2 b = make_float2(fmaf(a.x, f.x, -a.y * f.y), fmaf(a.x, f.y, a.y * f.x));
      if (r & 1) b = make_float2(-b.y, b.x);
      if (r & 2) b = make_float2(-b.x, -b.y);
      s[z] = b;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    partials[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
  }
}

__global__ void k_tc_expect(const InstDev* __restrict__ inst_all, const int32_t* __restrict__ list,
                            const double* __restrict__ partials, int32_t nb, int32_t nlist,
                            double* __restrict__ expect) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nlist) return;
  const int ii = list[i];
  double t = 0.0;
  for (int b = 0; b < nb; ++b) t += partials[(int64_t)i * nb + b];
  expect[ii] = t * (double)inst_all[ii].final_scale2;
}

cudaError_t launch_tc_phase(const InstDev* inst, const int32_t* list, int32_t nlist, int32_t n, int32_t layer,
                            int32_t init, const float2* tables, const uint16_t* cuts, int64_t cut_stride,
                            float2* states, cudaStream_t st) {
  if (nlist <= 0) return cudaSuccess;
  const int64_t dim = int64_t(1) << n;
  dim3 grid((unsigned)std::min<int64_t>((dim + 255) / 256, 1024), (unsigned)nlist);
  k_tc_phase<<<grid, 256, 0, st>>>(inst, list, n, layer, init, tables, cuts, cut_stride, states);
  return cudaGetLastError();
}

int tc_finish_blocks(int32_t n) { return (int)std::min<int64_t>(((int64_t(1) << n) + 255) / 256, 256); }

cudaError_t launch_tc_finish(const InstDev* inst, const int32_t* list, int32_t nlist, int32_t n, const uint16_t* cuts,
                             int64_t cut_stride, float2* states, double* partials, int32_t keep, double* expect,
                             cudaStream_t st) {
  if (nlist <= 0) return cudaSuccess;
  const int nb = tc_finish_blocks(n);
  k_tc_finish<<<dim3(nb, nlist), 256, 0, st>>>(inst, list, n, cuts, cut_stride, states, partials, keep);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_tc_expect<<<(nlist + 127) / 128, 128, 0, st>>>(inst, list, partials, nb, nlist, expect);
  return cudaGetLastError();
}

}  // namespace pq
