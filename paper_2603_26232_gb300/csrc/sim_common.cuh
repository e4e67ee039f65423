// Device helpers shared by the QAOA state-vector kernels for sm_103a: the
// on-chip simulation (sim_kernels.cu) and the HBM-streaming layer pass
// (layer_pass.cu).
//
// The state is complex64 (float2). A layer l applies exp(-i gamma_l C(z))
// (Sec. 2.2, the diagonal cost unitary of the Max-Cut objective of Sec. 2.1)
// and then exp(-i beta_l X_j) on every qubit j (the transverse-field mixer).
//
// Mixer arithmetic. exp(-i b X) = cos b I - i sin b X. Writing it as
//   cos b (I + i mu X),  mu = -tan b      when |cos b| >= |sin b|, or
//   (-i sin b) X (I + i mu X), mu = cot b otherwise,
// every qubit costs one butterfly (a, b) -> (a + i mu b, b + i mu a), two
// FMAs per amplitude, and the scalars cos^n b or (-i sin b)^n of a whole layer
// are folded into the next layer's phase table (or applied once at the end).
// The factor X^{(x)n} of the second form is dropped: |+>^n is invariant under
// the global flip and both unitaries commute with it (C(z) = C(not z)), so
// it acts as the identity on every state the circuit reaches.
//
// Gauge. The kernels hold s_z = i^popcount(z) psi_z instead of psi_z. The
// butterfly on qubit j then becomes real: with z' = z | 2^j,
//   (s_z, s_z') -> (s_z + mu s_z', s_z' - mu s_z),
// two packed FP32x2 FMAs with a broadcast mu and no re/im swaps. The phase is
// diagonal and |s_z| = |psi_z|, so phases, <C> and probabilities are
// unchanged; only the initial state and a stored final state carry the
// factor i^(+-popcount(z)).
//
// Cut values are integers computed on the fly from adjacency bit-planes, so
// the phase exp(-i gamma C) is a lookup into a table of W+1 entries built in
// FP64; nothing but the state itself moves through HBM.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "pq_internal.h"

namespace pq {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// Gauge butterfly (x, y) -> (x + mu y, y - mu x) on both components at once;
// in the untransformed state it is (a, b) -> (a + i mu b, b + i mu a).
__device__ __forceinline__ void bfly(float2& x, float2& y, float mu) {
  const float2 nx = __ffma2_rn(make_float2(mu, mu), y, x);
  const float2 ny = __ffma2_rn(make_float2(-mu, -mu), x, y);
  x = nx;
  y = ny;
}

// i^r * (x + i y) for a small integer r (any sign). Selects, not branches:
// with r known at compile time it folds to a register permutation.
__device__ __forceinline__ float2 rot_i(float2 a, int r) {
  const float2 t = (r & 1) ? make_float2(-a.y, a.x) : a;
  return (r & 2) ? make_float2(-t.x, -t.y) : t;
}

// Population count of a register index (< 64), written out so that it folds
// to a constant inside unrolled loops.
__host__ __device__ constexpr int popc_c(uint32_t x) {
  return (int)((x & 1u) + ((x >> 1) & 1u) + ((x >> 2) & 1u) + ((x >> 3) & 1u) + ((x >> 4) & 1u) + ((x >> 5) & 1u));
}

// C(z) = sum over u with z_u = 1 of the weight of u's neighbours with z_v = 0.
__device__ __forceinline__ int cut_eval(uint32_t z, const uint32_t* pl, int n, int P) {
  int c = 0;
  for (int u = 0; u < n; ++u) {
    uint32_t m = ((z >> u) & 1u) ? ~z : 0u;
    const uint32_t* q = pl + u * P;
    for (int b = 0; b < P; ++b) c += __popc(q[b] & m) << b;
  }
  return c;
}

// Change of C when qubit u (not in z0, u in kmask) is set, counting only
// neighbours outside kmask: weight to unset outsiders minus weight to set ones.
__device__ __forceinline__ int kappa(uint32_t z0, uint32_t kmask, int u, const uint32_t* pl, int P) {
  const uint32_t* q = pl + u * P;
  int c = 0;
  for (int b = 0; b < P; ++b) c += (__popc(q[b] & ~(z0 | kmask)) - __popc(q[b] & z0)) << b;
  return c;
}

// Phase-table index: a cut value is in [0, W] by construction; the clamp keeps
// the shared-memory read in bounds even if a caller's data broke that.
__device__ __forceinline__ uint32_t tix(int c, int W) { return min((uint32_t)c, (uint32_t)W); }

// Register layouts of a 2^TB tile held by 2^(TB-R) threads x 2^R registers.
// Layout RHO puts R local index bits in the register index k:
//   RHO 0: bits [TB-R, TB)   (load/store layout: lanes are consecutive)
//   RHO 1: bits [TB-2R, TB-R)
//   RHO 2: bits [0, R)       (overlaps RHO 1 when TB < 3R; only bits < TB-2R mix there)
// and the remaining bits, in increasing order, in the thread index.
//
// Shared-memory slot of local index li: one pad element after every 2^R,
// which makes every transpose between these layouts bank-conflict free
// (checked exhaustively for the tile shapes in use). It is additive over
// disjoint bits (pad(t | k) = pad(t) + pad(k)), so a thread's addresses are
// one base register plus compile-time offsets.
template <int R>
__host__ __device__ __forceinline__ constexpr uint32_t padr(uint32_t li) { return li + (li >> R); }
template <int TB, int R>
__host__ __device__ constexpr int padded_r() { return (1 << TB) + (1 << (TB - R)); }

template <int TB, int R, int RHO>
__device__ __forceinline__ uint32_t lir(uint32_t tid, uint32_t k) {
  if constexpr (RHO == 0) {
    return tid | (k << (TB - R));
  } else if constexpr (RHO == 1) {
    constexpr int lb = TB - 2 * R;
    return (tid & ((1u << lb) - 1u)) | (k << lb) | ((tid >> lb) << (TB - R));
  } else {
    return k | (tid << R);
  }
}

// The same layouts named by their register-bit offset O: registers hold local
// bits [O, O + R); thread bits fill [0, O) and [O + R, TB) in increasing order,
// so lanes stay on the lowest local bits (coalesced HBM access) whenever O >= 5.
// RHO 0, 1, 2 are O = TB - R, TB - 2R, 0.
template <int TB, int R, int O>
__device__ __forceinline__ uint32_t lir_o(uint32_t tid, uint32_t k) {
  return (tid & ((1u << O) - 1u)) | (k << O) | ((tid >> O) << (O + R));
}
// Local bit that thread-index bit b occupies in the layout of offset O.
template <int R, int O>
__host__ __device__ constexpr int thread_bit_local_o(int b) { return b < O ? b : b + R; }

// Layout offsets of the layer passes. Classic passes mix up to ceil(TB / R)
// rounds through layouts O = TB - R, TB - 2R, ..., and finally O = 0 (which
// overlaps the previous round's bits when R does not divide TB; only the
// bits below that round's offset mix there). Split passes (the low qubit
// group of 2R qubits) mix local bits [R, 2R) and [0, R) in two rounds with a
// single transpose, loading and storing in O = R.
__host__ __device__ constexpr int full_rounds(int TB, int R) { return (TB + R - 1) / R; }
__host__ __device__ constexpr int lay_off(int TB, int R, bool split, int rho) {
  return split ? (rho == 0 ? R : 0) : (rho + 1 < full_rounds(TB, R) ? TB - (rho + 1) * R : 0);
}
// Register slots round rho may mix: those whose local bit the rounds before
// it have not covered (every slot but in the last, overlapping round).
__host__ __device__ constexpr uint32_t round_slots(int TB, int R, bool split, int rho) {
  uint32_t m = 0;
  const int prev = rho == 0 ? TB : lay_off(TB, R, split, rho - 1);
  for (int j = 0; j < R; ++j)
    if (split || lay_off(TB, R, split, rho) + j < prev) m |= 1u << j;
  return m;
}

__host__ __device__ __forceinline__ int slot_lbr(int TB, int R, int rho, int j) {
  return rho == 0 ? TB - R + j : (rho == 1 ? TB - 2 * R + j : j);
}

// Transpose from layout FROM to TO through shared memory; TRAIL as for
// transposer_o below (the barrier after the reads, which a caller whose next
// buffer write is a transpose from TO does not need).
template <int TB, int R, int FROM, int TO, bool TRAIL = true>
__device__ __forceinline__ void transposer(float2 (&a)[1 << R], float2* sm, uint32_t tid) {
  float2* pf = sm + padr<R>(lir<TB, R, FROM>(tid, 0));
  float2* pt = sm + padr<R>(lir<TB, R, TO>(tid, 0));
#pragma unroll
  for (int k = 0; k < (1 << R); ++k) pf[padr<R>(lir<TB, R, FROM>(0, k))] = a[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < (1 << R); ++k) a[k] = pt[padr<R>(lir<TB, R, TO>(0, k))];
  if constexpr (TRAIL) __syncthreads();
}

// True when layouts OF and OT put the same local bits in the warp index
// (thread bits 5 and up): a transpose between them then only moves data
// among the lanes of one warp, through shared memory the warp alone
// touches, and a warp barrier is enough.
template <int TB, int R, int OF, int OT>
__host__ __device__ constexpr bool warp_local_transpose() {
  for (int b = 5; b < TB - R; ++b)
    if (thread_bit_local_o<R, OF>(b) != thread_bit_local_o<R, OT>(b)) return false;
  return true;
}

static_assert(warp_local_transpose<12, 4, 4, 0>() && warp_local_transpose<12, 5, 2, 0>() &&
                  warp_local_transpose<13, 5, 3, 0>() && warp_local_transpose<12, 5, 5, 0>(),
              "the second transpose of a three-round pass and the split pass's transpose stay in a warp");
static_assert(warp_local_transpose<13, 4, 5, 1>() && warp_local_transpose<13, 4, 1, 0>() &&
                  warp_local_transpose<14, 4, 2, 0>() && !warp_local_transpose<14, 4, 6, 2>(),
              "four-round passes: which transposes stay in a warp");
static_assert(!warp_local_transpose<12, 4, 8, 4>(), "load/store-layout transposes cross warps");
static_assert(lay_off(13, 4, false, 2) == 1 && lay_off(13, 4, false, 3) == 0 && round_slots(13, 4, false, 3) == 1u &&
                  round_slots(12, 5, false, 2) == 3u && round_slots(12, 4, false, 2) == 15u,
              "round offsets and slot masks");

// Transpose from layout OF to OT through shared memory. TRAIL = false leaves
// out the barrier after the reads. That is safe when the next write to the
// buffer is a transpose from OT: each thread then writes exactly the slots it
// has just read (padr is additive, so a thread's slots in a layout are
// padr(lir_o(tid, k)) whichever transpose addresses them), and the other
// threads read only their own slots. Any other next write needs a barrier
// of the caller's in between.
template <int TB, int R, int OF, int OT, bool TRAIL = true>
__device__ __forceinline__ void transposer_o(float2 (&a)[1 << R], float2* sm, uint32_t tid) {
  constexpr bool kWarp = warp_local_transpose<TB, R, OF, OT>();
  float2* pf = sm + padr<R>(lir_o<TB, R, OF>(tid, 0));
  float2* pt = sm + padr<R>(lir_o<TB, R, OT>(tid, 0));
#pragma unroll
  for (int k = 0; k < (1 << R); ++k) pf[padr<R>(lir_o<TB, R, OF>(0, k))] = a[k];
  if constexpr (kWarp) __syncwarp(); else __syncthreads();
#pragma unroll
  for (int k = 0; k < (1 << R); ++k) a[k] = pt[padr<R>(lir_o<TB, R, OT>(0, k))];
  if constexpr (TRAIL) {
    if constexpr (kWarp) __syncwarp(); else __syncthreads();
  }
}

template <int R>
__device__ __forceinline__ void mix_regs_r(float2 (&a)[1 << R], float mu, uint32_t mask) {
#pragma unroll
  for (int j = 0; j < R; ++j) {
    if ((mask >> j) & 1u) {
#pragma unroll
      for (int k = 0; k < (1 << R); ++k)
        if (!((k >> j) & 1)) bfly(a[k], a[k | (1 << j)], mu);
    }
  }
}

// Butterflies of one round without data-dependent branches: slots outside
// `mask` get mu = 0, an exact identity, so every register keeps one fixed
// home and no copies are needed where paths would join. Slots outside the
// compile-time set ALLOWED (never mixed in this round) are skipped.
template <int R, uint32_t ALLOWED>
__device__ __forceinline__ void mix_regs_sel(float2 (&a)[1 << R], float mu, uint32_t mask) {
#pragma unroll
  for (int j = 0; j < R; ++j) {
    if (!((ALLOWED >> j) & 1u)) continue;
    const float m = ((mask >> j) & 1u) ? mu : 0.f;
#pragma unroll
    for (int k = 0; k < (1 << R); ++k)
      if (!((k >> j) & 1)) bfly(a[k], a[k | (1 << j)], m);
  }
}

// One mixing round: with FULL every slot in ALLOWED mixes, so one broadcast
// multiplier serves them all; otherwise mix_regs_sel's per-slot selects.
template <int R, uint32_t ALLOWED>
__device__ __forceinline__ void mix_round(float2 (&a)[1 << R], float mu, uint32_t mask, bool full) {
  if (full) {
#pragma unroll
    for (int j = 0; j < R; ++j) {
      if (!((ALLOWED >> j) & 1u)) continue;
#pragma unroll
      for (int k = 0; k < (1 << R); ++k)
        if (!((k >> j) & 1)) bfly(a[k], a[k | (1 << j)], mu);
    }
  } else {
    mix_regs_sel<R, ALLOWED>(a, mu, mask);
  }
}

// Deterministic block sum of one double per thread (fixed reduction order).
__device__ __forceinline__ double block_sum(double v, double* red, uint32_t tid, uint32_t nt) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((tid & 31u) == 0) red[tid >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (tid == 0)
    for (uint32_t w = 0; w < (nt >> 5); ++w) s += red[w];
  __syncthreads();
  return s;
}

}  // namespace pq
