// QAOA state-vector kernels for sm_103a: cost phase, mixer, <C>, cut table.
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
#include <cuda_runtime.h>

#include <algorithm>

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

// Layout offsets of the layer passes. Classic passes mix up to three rounds
// through layouts O = TB - R, TB - 2R, 0. Split passes (the low qubit group of
// 2R qubits) mix local bits [R, 2R) and [0, R) in two rounds with a single
// transpose, loading and storing in O = R.
__host__ __device__ constexpr int lay_off(int TB, int R, bool split, int rho) {
  return split ? (rho == 0 ? R : 0) : (rho == 0 ? TB - R : (rho == 1 ? TB - 2 * R : 0));
}

__host__ __device__ __forceinline__ int slot_lbr(int TB, int R, int rho, int j) {
  return rho == 0 ? TB - R + j : (rho == 1 ? TB - 2 * R + j : j);
}

template <int TB, int R, int FROM, int TO>
__device__ __forceinline__ void transposer(float2 (&a)[1 << R], float2* sm, uint32_t tid) {
  float2* pf = sm + padr<R>(lir<TB, R, FROM>(tid, 0));
  float2* pt = sm + padr<R>(lir<TB, R, TO>(tid, 0));
#pragma unroll
  for (int k = 0; k < (1 << R); ++k) pf[padr<R>(lir<TB, R, FROM>(0, k))] = a[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < (1 << R); ++k) a[k] = pt[padr<R>(lir<TB, R, TO>(0, k))];
  __syncthreads();
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
static_assert(!warp_local_transpose<12, 4, 8, 4>(), "load/store-layout transposes cross warps");

template <int TB, int R, int OF, int OT>
__device__ __forceinline__ void transposer_o(float2 (&a)[1 << R], float2* sm, uint32_t tid) {
  constexpr bool kWarp = warp_local_transpose<TB, R, OF, OT>();
  float2* pf = sm + padr<R>(lir_o<TB, R, OF>(tid, 0));
  float2* pt = sm + padr<R>(lir_o<TB, R, OT>(tid, 0));
#pragma unroll
  for (int k = 0; k < (1 << R); ++k) pf[padr<R>(lir_o<TB, R, OF>(0, k))] = a[k];
  if constexpr (kWarp) __syncwarp(); else __syncthreads();
#pragma unroll
  for (int k = 0; k < (1 << R); ++k) a[k] = pt[padr<R>(lir_o<TB, R, OT>(0, k))];
  if constexpr (kWarp) __syncwarp(); else __syncthreads();
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

// The on-chip kernel uses the 32-register shape throughout.
__host__ __device__ __forceinline__ constexpr uint32_t pad(uint32_t li) { return padr<5>(li); }
template <int TB>
__host__ __device__ constexpr int padded_elems() { return padded_r<TB, 5>(); }
template <int TB, int RHO>
__device__ __forceinline__ uint32_t li_of(uint32_t tid, uint32_t k) { return lir<TB, 5, RHO>(tid, k); }
template <int TB>
__device__ __forceinline__ uint32_t li0_rt(int rho, uint32_t tid) {
  if (rho == 0) return li_of<TB, 0>(tid, 0);
  if (rho == 1) return li_of<TB, 1>(tid, 0);
  return li_of<TB, 2>(tid, 0);
}
__host__ __device__ __forceinline__ int slot_lb(int TB, int rho, int j) { return slot_lbr(TB, 5, rho, j); }
template <int TB, int FROM, int TO>
__device__ __forceinline__ void transpose(float2 (&a)[32], float2* sm, uint32_t tid) {
  transposer<TB, 5, FROM, TO>(a, sm, tid);
}

template <int TB>
__device__ __forceinline__ void goto_layout(float2 (&a)[32], float2* sm, uint32_t tid, int& cur, int to) {
  if (cur == to) return;
  const int code = cur * 3 + to;
  if (code == 1) transpose<TB, 0, 1>(a, sm, tid);
  else if (code == 2) transpose<TB, 0, 2>(a, sm, tid);
  else if (code == 3) transpose<TB, 1, 0>(a, sm, tid);
  else if (code == 5) transpose<TB, 1, 2>(a, sm, tid);
  else if (code == 6) transpose<TB, 2, 0>(a, sm, tid);
  else transpose<TB, 2, 1>(a, sm, tid);
  cur = to;
}

__device__ __forceinline__ void mix_regs(float2 (&a)[32], float mu, uint32_t mask) { mix_regs_r<5>(a, mu, mask); }

// Per-layout cut decomposition shared by the CTA: for the 5 register qubits
// Kq of layout rho, ckk[k] = C restricted to edges inside Kq at assignment k.
struct LayoutCut {
  int kq[3][5];
  uint32_t kmask[3];
  int ckk[3][32];
  int pad[2];  // 16-byte multiple: a double buffer follows it in shared memory
};
static_assert(sizeof(LayoutCut) % 16 == 0, "shared-memory carve-up needs 16-byte multiples");

// Fill LayoutCut for the layouts in use. qubit(lb) maps a local bit to a qubit.
template <int TB>
__device__ void build_layout_cut(LayoutCut& lc, int nrounds, int c, int s, const uint32_t* pl,
                                 int P, uint32_t tid) {
  if (tid < 3) {
    int rho = tid;
    uint32_t m = 0;
    for (int j = 0; j < 5; ++j) {
      int lb = slot_lb(TB, rho, j);
      int q = lb < c ? lb : s + (lb - c);
      lc.kq[rho][j] = q;
      m |= 1u << q;
    }
    lc.kmask[rho] = m;
  }
  __syncthreads();
  for (uint32_t q = tid; q < 32u * (uint32_t)nrounds; q += (1u << (TB - 5))) {
    int rho = q >> 5, k = q & 31;
    uint32_t zk = 0;
    for (int j = 0; j < 5; ++j)
      if ((k >> j) & 1) zk |= 1u << lc.kq[rho][j];
    int cc = 0;
    for (int j = 0; j < 5; ++j) {
      if (!((k >> j) & 1)) continue;
      const uint32_t* row = pl + lc.kq[rho][j] * P;
      for (int b = 0; b < P; ++b) cc += __popc(row[b] & lc.kmask[rho] & ~zk) << b;
    }
    lc.ckk[rho][k] = cc;
  }
  __syncthreads();
}

// Cut values of this thread's 32 amplitudes in layout rho: C = C0 + ckk[k] +
// sum of kap[j] over the set bits j of k.
struct ThreadCut {
  int C0;
  int kap[5];
};

__device__ __forceinline__ ThreadCut thread_cut(uint32_t z0, const LayoutCut& lc, int rho,
                                                const uint32_t* pl, int n, int P) {
  ThreadCut t;
  t.C0 = cut_eval(z0, pl, n, P);
#pragma unroll
  for (int j = 0; j < 5; ++j) t.kap[j] = kappa(z0, lc.kmask[rho], lc.kq[rho][j], pl, P);
  return t;
}

__device__ __forceinline__ int cut_of_reg(const ThreadCut& t, const int* ckk, int k) {
  int c = t.C0 + ckk[k];
#pragma unroll
  for (int j = 0; j < 5; ++j)
    if ((k >> j) & 1) c += t.kap[j];
  return c;
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

// ---------------------------------------------------------------------------
// Per-instance layer constants: phase tables tab_l[c] = exp(-i gamma_l c) S_l
// in FP64 rounded to complex64, with S_0 = 2^(-n/2) (the |+>^n amplitude)
// and S_l = lambda_{l-1}, the scalar left out of layer l-1's mixer.
// One warp per instance; the FP64 pipe is narrow, so the work is kept to
// one sincos per lane and layer plus one FP64 complex multiply per entry:
// lane t fills c = t, t + 32, ... by the recurrence z <- z exp(-i gamma 32)
// from z = S exp(-i gamma t). After k steps the relative error is about
// 4k 2^-53, below 1e-13 for every table that fits on chip, far under the
// FP32 rounding of the stored entry. The mixer scalars cos^n b and sin^n b
// are integer powers, taken by repeated squaring.
__device__ __forceinline__ double ipow(double x, int e) {
  double r = 1.0;
  for (; e > 0; e >>= 1) {
    if (e & 1) r *= x;
    x *= x;
  }
  return r;
}

__global__ void __launch_bounds__(32) k_prep_layers(const InstDev* __restrict__ inst_ro, int32_t p,
                                                    const double* __restrict__ gamma,
                                                    const double* __restrict__ beta, float2* __restrict__ tables,
                                                    InstDev* __restrict__ inst_rw) {
  const int i = blockIdx.x;
  const int lane = threadIdx.x;
  const InstDev I = inst_ro[i];
  const int n = I.n, W = I.W;
  // S_0 = 2^(-n/2), exactly
  double sre = (n & 1) ? ldexp(0.70710678118654752440, -(n >> 1)) : ldexp(1.0, -(n >> 1)), sim = 0.0;
  for (int l = 0; l < p; ++l) {
    const double g = gamma[(int64_t)i * p + l];
    float2* tab = tables + I.table_off + (int64_t)l * (W + 1);
    double sn, cs, sB, cB;
    sincos(g * (double)lane, &sn, &cs);  // exp(-i g t) = cs - i sn
    sincos(g * 32.0, &sB, &cB);          // the step exp(-i g 32) = cB - i sB
    double zr = cs * sre + sn * sim, zi = cs * sim - sn * sre;  // S exp(-i g t)
    for (int c = lane; c <= W; c += 32) {
      tab[c] = make_float2((float)zr, (float)zi);
      const double nr = fma(zr, cB, zi * sB), ni = fma(zi, cB, -(zr * sB));
      zr = nr;
      zi = ni;
    }
    const double b = beta[(int64_t)i * p + l];
    double sb, cb;
    sincos(b, &sb, &cb);
    double lre, lim, mu;
    if (fabs(cb) >= fabs(sb)) {
      mu = -sb / cb;
      lre = ipow(cb, n);
      lim = 0.0;
    } else {
      mu = cb / sb;
      const double mag = ipow(sb, n);  // (-i sb)^n = sb^n (-i)^n
      const int r = n & 3;
      lre = (r == 0) ? mag : (r == 2 ? -mag : 0.0);
      lim = (r == 1) ? -mag : (r == 3 ? mag : 0.0);
    }
    if (lane == 0) {
      inst_rw[i].mu[l] = (float)mu;
      if (l == p - 1) {
        inst_rw[i].final_scale = make_float2((float)lre, (float)lim);
        inst_rw[i].final_scale2 = (float)(lre * lre + lim * lim);
      }
    }
    sre = lre;
    sim = lim;
  }
}

cudaError_t launch_prep_layers(const InstDev* inst, int32_t count, int32_t p, const double* gamma,
                               const double* beta, float2* tables, InstDev* inst_rw,
                               cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  k_prep_layers<<<count, 32, 0, st>>>(inst, p, gamma, beta, tables, inst_rw);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// n <= 9: one 64-thread CTA per instance, state in shared memory, one qubit at
// a time. Used for tiny subgraphs and edge cases.
__global__ void k_tiny_sim(const InstDev* __restrict__ inst_all, const int32_t* __restrict__ list,
                           int32_t p, const SubDev* __restrict__ subs,
                           const uint32_t* __restrict__ planes_all, const float2* __restrict__ tables,
                           float2* __restrict__ states, double* __restrict__ expect, int32_t keep,
                           int32_t want_expect, int32_t tabcap) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* psi = reinterpret_cast<float2*>(smraw);    // 512
  float2* tab = psi + 512;                            // tabcap
  uint32_t* pl = reinterpret_cast<uint32_t*>(tab + tabcap);  // 9*16
  double* red = reinterpret_cast<double*>(pl + 9 * kMaxPlanes + 8);
  const int ii = list[blockIdx.x];
  const InstDev I = inst_all[ii];
  const SubDev S = subs[I.sub];
  const int n = I.n, P = I.P, W = I.W;
  const uint32_t dim = 1u << n, tid = threadIdx.x, nt = blockDim.x;
  for (uint32_t q = tid; q < (uint32_t)(n * P); q += nt) pl[q] = planes_all[S.plane_off + q];
  for (uint32_t z = tid; z < dim; z += nt) psi[z] = rot_i(make_float2(1.f, 0.f), __popc(z));
  for (int l = 0; l < p; ++l) {
    __syncthreads();
    const float2* tl = tables + I.table_off + (int64_t)l * (W + 1);
    for (int c = tid; c <= W; c += nt) tab[c] = tl[c];
    __syncthreads();
    for (uint32_t z = tid; z < dim; z += nt) psi[z] = cmul(psi[z], tab[tix(cut_eval(z, pl, n, P), W)]);
    const float mu = I.mu[l];
    for (int j = 0; j < n; ++j) {
      __syncthreads();
      for (uint32_t q = tid; q < (dim >> 1); q += nt) {
        uint32_t lo = q & ((1u << j) - 1u);
        uint32_t z0 = ((q >> j) << (j + 1)) | lo;
        float2 x = psi[z0], y = psi[z0 | (1u << j)];
        bfly(x, y, mu);
        psi[z0] = x;
        psi[z0 | (1u << j)] = y;
      }
    }
  }
  __syncthreads();
  if (want_expect) {
    double acc = 0.0;
    for (uint32_t z = tid; z < dim; z += nt) {
      float2 a = psi[z];
      acc += (double)(a.x * a.x + a.y * a.y) * (double)cut_eval(z, pl, n, P);
    }
    double s = block_sum(acc, red, tid, nt);
    if (tid == 0) expect[ii] = s * (double)I.final_scale2;
  }
  if (keep)
    for (uint32_t z = tid; z < dim; z += nt)
      states[I.state_off + z] = cmul(rot_i(psi[z], -__popc(z)), I.final_scale);
}

cudaError_t launch_tiny_sim(const InstDev* inst, const int32_t* list, int32_t nlist, int32_t p,
                            const SubDev* subs, const uint32_t* planes, const float2* tables,
                            float2* states, double* expect, int32_t keep, int32_t want_expect,
                            int32_t tabcap, cudaStream_t st) {
  if (nlist <= 0) return cudaSuccess;
  size_t smem = 512 * sizeof(float2) + tabcap * sizeof(float2) + (9 * kMaxPlanes + 8) * 4 + 8 * 8;
  cudaFuncSetAttribute(k_tiny_sim, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_tiny_sim<<<nlist, 64, smem, st>>>(inst, list, p, subs, planes, tables, states, expect, keep,
                                      want_expect, tabcap);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// 10 <= n <= 14: the whole state of one instance lives in one CTA (registers
// plus a shared-memory transpose buffer); all p layers, <C> and the optional
// state write happen without touching HBM in between.
template <int TB>
__global__ void __launch_bounds__(1 << (TB - 5))
    k_smem_sim(const InstDev* __restrict__ inst_all, const int32_t* __restrict__ list, int32_t p,
               const SubDev* __restrict__ subs, const uint32_t* __restrict__ planes_all,
               const float2* __restrict__ tables, float2* __restrict__ states,
               double* __restrict__ expect, int32_t keep, int32_t want_expect, int32_t tabcap) {
  constexpr uint32_t NT = 1u << (TB - 5);
  constexpr int NR = (TB > 10) ? 3 : 2;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* sm = reinterpret_cast<float2*>(smraw);               // padded 2^TB
  float2* tab = sm + padded_elems<TB>();                        // tabcap
  uint32_t* pl = reinterpret_cast<uint32_t*>(tab + tabcap);     // 14*16
  LayoutCut* lc = reinterpret_cast<LayoutCut*>(pl + kSmemMaxQubits * kMaxPlanes);
  double* red = reinterpret_cast<double*>(lc + 1);
  const uint32_t tid = threadIdx.x;
  const int ii = list[blockIdx.x];
  const InstDev I = inst_all[ii];
  const SubDev S = subs[I.sub];
  const int n = TB, P = I.P, W = I.W;
  for (uint32_t q = tid; q < (uint32_t)(n * P); q += NT) pl[q] = planes_all[S.plane_off + q];
  __syncthreads();
  build_layout_cut<TB>(*lc, NR, TB, TB, pl, P, tid);
  // mix masks: all slots, except that layout 2 only mixes local bits < TB-10
  const uint32_t mask2 = (1u << (TB - 10)) - 1u;
  float2 a[32];
  int cur = NR - 1;
  {
    const float2 b = rot_i(make_float2(1.f, 0.f), __popc(li0_rt<TB>(cur, tid)));
#pragma unroll
    for (int k = 0; k < 32; ++k) a[k] = rot_i(b, __popc(k));
  }
  for (int l = 0; l < p; ++l) {
    const float2* tl = tables + I.table_off + (int64_t)l * (W + 1);
    for (int c = tid; c <= W; c += NT) tab[c] = tl[c];
    __syncthreads();
    {
      ThreadCut t = thread_cut(li0_rt<TB>(cur, tid), *lc, cur, pl, n, P);
      const int* ckk = lc->ckk[cur];
#pragma unroll
      for (int k = 0; k < 32; ++k) a[k] = cmul(a[k], tab[tix(cut_of_reg(t, ckk, k), W)]);
    }
    const float mu = I.mu[l];
    if ((l & 1) == 0) {
      for (int r = NR - 1; r >= 0; --r) {
        goto_layout<TB>(a, sm, tid, cur, r);
        mix_regs(a, mu, r == 2 ? mask2 : 31u);
      }
    } else {
      for (int r = 0; r < NR; ++r) {
        goto_layout<TB>(a, sm, tid, cur, r);
        mix_regs(a, mu, r == 2 ? mask2 : 31u);
      }
    }
    __syncthreads();  // before the next table load overwrites tab
  }
  if (want_expect) {
    ThreadCut t = thread_cut(li0_rt<TB>(cur, tid), *lc, cur, pl, n, P);
    const int* ckk = lc->ckk[cur];
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < 32; ++k)
      acc = fmaf(fmaf(a[k].x, a[k].x, a[k].y * a[k].y), (float)cut_of_reg(t, ckk, k), acc);
    double s = block_sum((double)acc, red, tid, NT);
    if (tid == 0) expect[ii] = s * (double)I.final_scale2;
  }
  if (keep) {
    goto_layout<TB>(a, sm, tid, cur, 0);
    float2* out = states + I.state_off;
    const float2 fs = rot_i(I.final_scale, -__popc(tid));
#pragma unroll
    for (int k = 0; k < 32; ++k) out[li_of<TB, 0>(tid, k)] = cmul(a[k], rot_i(fs, -__popc(k)));
  }
}

template <int TB>
static cudaError_t launch_smem_t(const InstDev* inst, const int32_t* list, int32_t nlist, int32_t p,
                                 const SubDev* subs, const uint32_t* planes, const float2* tables,
                                 float2* states, double* expect, int32_t keep, int32_t want_expect,
                                 int32_t tabcap, cudaStream_t st) {
  size_t smem = (size_t)padded_elems<TB>() * sizeof(float2) + tabcap * sizeof(float2) +
                kSmemMaxQubits * kMaxPlanes * 4 + sizeof(LayoutCut) + 32 * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_smem_sim<TB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_smem_sim<TB><<<nlist, 1 << (TB - 5), smem, st>>>(inst, list, p, subs, planes, tables, states,
                                                      expect, keep, want_expect, tabcap);
  return cudaGetLastError();
}

cudaError_t launch_smem_sim(int n, const InstDev* inst, const int32_t* list, int32_t nlist,
                            int32_t p, const SubDev* subs, const uint32_t* planes,
                            const float2* tables, float2* states, double* expect, int32_t keep,
                            int32_t want_expect, int32_t tabcap, cudaStream_t st) {
  if (nlist <= 0) return cudaSuccess;
  switch (n) {
    case 10: return launch_smem_t<10>(inst, list, nlist, p, subs, planes, tables, states, expect, keep, want_expect, tabcap, st);
    case 11: return launch_smem_t<11>(inst, list, nlist, p, subs, planes, tables, states, expect, keep, want_expect, tabcap, st);
    case 12: return launch_smem_t<12>(inst, list, nlist, p, subs, planes, tables, states, expect, keep, want_expect, tabcap, st);
    case 13: return launch_smem_t<13>(inst, list, nlist, p, subs, planes, tables, states, expect, keep, want_expect, tabcap, st);
    case 14: return launch_smem_t<14>(inst, list, nlist, p, subs, planes, tables, states, expect, keep, want_expect, tabcap, st);
    default: return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------------------
// n >= 15: layer passes that stream the state through HBM. A tile is 2^TB
// amplitudes whose local bits [0, c) are qubits [0, c) (contiguous in HBM) and
// whose local bits [c, TB) are qubits [s, s + TB - c); the remaining qubits are
// fixed per tile. A pass may finish one layer's mixer on the tile's qubits,
// apply the next layer's phase and start its mixer, so p layers take p + 1
// passes when the qubits split into two groups (see make_schedule).
//
// One CTA per tile, tiles of an instance consecutive in blockIdx: the block
// scheduler then keeps the CTAs resident on the GPU on neighbouring tiles and
// refills an SM the moment a CTA retires, which measured faster than
// persistent CTAs walking their own tile ranges.
//
// Cut values. With T the tile's qubits, F the fixed ones, J the qubits of the
// thread index and K the 5 register qubits of the layout where the cut is
// needed, C(z) = sum_u d_u z_u - 2 sum_{u<v} w_uv z_u z_v splits into
//   C = C(z_F)                          per tile (z_T = 0)
//     + sum_{u in J} lam_u z_u          lam_u = d_u - 2 sum_{v in F} w_uv z_v, per tile
//     - 2 Q_J(z_J)                      per thread and instance (k_cut_consts)
//     + sum_{u in K} z_u (lam_u + B_u)  B_u = -2 sum_{v in J} w_uv z_v, per thread (k_cut_consts)
//     - 2 Q_K(z_K)                      32-entry table per instance (k_cut_consts)
// so a cut value costs a broadcast load and a few integer adds.
struct TileConst {
  int cf;        // C(z_F)
  int lam[16];   // lam_u per local bit
  int pad[3];    // keeps what follows in shared memory 16-byte aligned
};
static_assert(sizeof(TileConst) % 16 == 0, "shared-memory carve-up needs 16-byte multiples");

__host__ __device__ __forceinline__ uint32_t qubit_of(int lb, int c, int s) {
  return lb < c ? (uint32_t)lb : (uint32_t)(s + (lb - c));
}

// Visit the 32 registers in Gray-code order so that consecutive registers
// differ in one bit: per-register offsets then cost one add each.
__host__ __device__ constexpr int gray(int i) { return i ^ (i >> 1); }
__host__ __device__ constexpr int gray_bit(int i) { return i & 1 ? 0 : (i & 2 ? 1 : (i & 4 ? 2 : (i & 8 ? 3 : 4))); }

// Entries per instance of the k_cut_consts output: 2^R (Q_K table) + (1 + R) per thread.
__host__ __device__ constexpr int cut_consts_stride(int tb, int r) { return (1 << r) + (1 + r) * (1 << (tb - r)); }

// Cut constants of one pass for the part of each listed instance (one CTA
// per distinct part; the layer pass finds them by the instance's cc_slot),
// for the cut layout of offset OC, at out + blockIdx.x * stride:
// out[0..2^R) = -2 Q_K(k); out[2^R + t] = -2 Q_J(z_J(t)); out[2^R + (1+j) NT + t] =
// B_u(t) of register slot j.
template <int TB, int R, int OC>
__global__ void __launch_bounds__(1 << (TB - R))
    k_cut_consts(PassDesc pd, int32_t n, const InstDev* __restrict__ inst_all,
                 const int32_t* __restrict__ list, const SubDev* __restrict__ subs,
                 const uint32_t* __restrict__ planes_all, int32_t* __restrict__ out) {
  constexpr uint32_t NT = 1u << (TB - R);
  constexpr int KQ = 1 << R;
  __shared__ uint32_t pl[PARAQAOA_MAX_QUBITS * kMaxPlanes];
  const uint32_t tid = threadIdx.x;
  const InstDev* Ip = inst_all + list[blockIdx.x];
  const SubDev S = subs[Ip->sub];
  const int P = Ip->P, c = pd.c, s = pd.s;
  for (uint32_t q = tid; q < (uint32_t)(n * P); q += NT) pl[q] = planes_all[S.plane_off + q];
  __syncthreads();
  int32_t* o = out + (int64_t)blockIdx.x * cut_consts_stride(TB, R);
  if (tid < (uint32_t)KQ) {
    uint32_t zk = 0;
    for (int j = 0; j < R; ++j)
      if ((tid >> j) & 1u) zk |= 1u << qubit_of(OC + j, c, s);
    int acc = 0;
    for (int j = 0; j < R; ++j) {
      if (!((tid >> j) & 1u)) continue;
      const uint32_t* row = pl + qubit_of(OC + j, c, s) * P;
      for (int b = 0; b < P; ++b) acc += __popc(row[b] & zk) << b;
    }
    o[tid] = -acc;  // each pair of set K qubits counted from both ends
  }
  const uint32_t li0 = lir_o<TB, R, OC>(tid, 0);
  uint32_t zJ = 0;
  for (int lb = 0; lb < TB; ++lb)
    if ((li0 >> lb) & 1u) zJ |= 1u << qubit_of(lb, c, s);
  int acc = 0;
  for (int u = 0; u < n; ++u) {
    if (!((zJ >> u) & 1u)) continue;
    const uint32_t* row = pl + u * P;
    for (int b = 0; b < P; ++b) acc += __popc(row[b] & zJ) << b;
  }
  o[KQ + tid] = -acc;
  for (int j = 0; j < R; ++j) {
    const uint32_t* row = pl + qubit_of(OC + j, c, s) * P;
    int bj = 0;
    for (int b = 0; b < P; ++b) bj += __popc(row[b] & zJ) << b;
    o[KQ + (1 + j) * NT + tid] = -2 * bj;
  }
}

// Shapes whose CTAs may walk 2^tpc_log2 tiles of one instance (sharing the
// per-instance set-up loads).
__host__ __device__ constexpr bool layer_multi_tile(int tb, int r) { return r == 4; }

// Occupancy target of a tile shape: resident CTAs per SM. The 16-register
// shape fits 64 registers per thread (four CTAs of 256 threads); the 2^12 x 32
// shape is held to 96 registers for five CTAs of 128 threads (a few bytes of
// spills, measured 3% faster than four CTAs at 128 registers).
__host__ __device__ constexpr int layer_min_blocks(int tb, int r) { return r == 4 ? 4 : (tb >= 13 ? 2 : 5); }

template <int TB, int R, int NR, bool SPLIT>
__global__ void __launch_bounds__(1 << (TB - R), layer_min_blocks(TB, R))
    k_layer_pass(PassDesc pd, int32_t n, int32_t tiles_log2, const InstDev* __restrict__ inst_all,
                 const int32_t* __restrict__ list, const SubDev* __restrict__ subs,
                 const uint32_t* __restrict__ planes_all, const float2* __restrict__ tables,
                 float2* __restrict__ states, double* __restrict__ partials, int32_t tabcap,
                 const int32_t* __restrict__ consts, uint32_t mm0, uint32_t mm1, uint32_t mm2) {
  constexpr uint32_t NT = 1u << (TB - R);
  constexpr int KQ = 1 << R;  // registers per thread
  constexpr int O0 = lay_off(TB, R, SPLIT, 0), O1 = lay_off(TB, R, SPLIT, 1), O2 = lay_off(TB, R, SPLIT, 2);
  constexpr int OC = lay_off(TB, R, SPLIT, NR - 1);  // layout of the cut step (phase / <C>)
  static_assert(!SPLIT || NR == 2, "split passes mix two rounds");
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* tab = reinterpret_cast<float2*>(smraw);
  float2* sm = tab + tabcap;
  int* qk = reinterpret_cast<int*>(sm + padded_r<TB, R>());  // 2^R entries (<= 32)
  TileConst* tc = reinterpret_cast<TileConst*>(qk + 32);
  uint32_t* pls = reinterpret_cast<uint32_t*>(tc + 1);  // the instance's bit-planes
  double* red = reinterpret_cast<double*>(pls + PARAQAOA_MAX_QUBITS * kMaxPlanes);
  const uint32_t tid = threadIdx.x;
  const int c = pd.c, s = pd.s, g = TB - c;
  const uint32_t lowt = (uint32_t)(s - c);
  // this CTA's 2^tpc_log2 tiles, all of one instance, strided by the
  // instance's CTA count: CTAs that run side by side then cover consecutive
  // tiles, which keeps the DRAM pages of a pass with short contiguous runs
  // (a high qubit group) busy together
  const uint32_t per = (uint32_t)(tiles_log2 - pd.tpc_log2);
  const int li_idx = (int)(blockIdx.x >> per);
  const uint32_t tj = blockIdx.x & ((1u << per) - 1u);
  const InstDev* Ip = inst_all + list[li_idx];
  const int P = Ip->P, W = Ip->W;
  const uint32_t* pl = planes_all + subs[Ip->sub].plane_off;
  const bool need_cut = pd.layerP >= 0 || pd.expect;

  // ---- set-up. One round of global loads, all issued before the first
  // barrier (the state loads below too): the phase table, the instance's
  // adjacency bit-planes, the Q_K table and this thread's cut constants.
  // After the barrier warp 0 derives the tile constants from the planes in
  // shared memory.
  if (pd.layerP >= 0) {
    const float2* tl = tables + Ip->table_off + (int64_t)pd.layerP * (W + 1);
    for (int cc = tid; cc <= W; cc += NT) tab[cc] = tl[cc];
  }
  const int32_t* cc_inst = consts + (int64_t)Ip->cc_slot * cut_consts_stride(TB, R);
  int ccJ = 0, ccB[R];
#pragma unroll
  for (int j = 0; j < R; ++j) ccB[j] = 0;
  if (need_cut) {
    for (int q = tid; q < n * P; q += NT) pls[q] = pl[q];
    if (tid < (uint32_t)KQ) qk[tid] = cc_inst[tid];
    ccJ = cc_inst[KQ + tid];
#pragma unroll
    for (int j = 0; j < R; ++j) ccB[j] = cc_inst[KQ + (1 + j) * NT + tid];
  }
  // Local index -> qubit offset: local bits [0, c) are qubits [0, c), bits
  // [c, TB) move up by s - c (a monotone bit map, so it keeps popcounts).
  const uint32_t lowm = (1u << c) - 1u;
  const int sh = s - c;
  auto zmap = [&](uint32_t li) -> uint32_t { return (li & lowm) | ((li & ~lowm) << sh); };
  // load/store layout O0: this thread's amplitude offsets are zmap(lt | register bits)
  const uint32_t lt = lir_o<TB, R, O0>(tid, 0);
  // Tiles of one CTA share the set-up above. Across iterations the barriers
  // below order every reuse of shared memory: warp 0 rewrites the tile
  // constants only after the first barrier of the next tile, which every
  // thread reaches after its last read of them.
  // (Only the 16-register shape walks several tiles: the 32-register shapes
  // keep one tile per CTA, where the loop's live set would spill.)
  const uint32_t ntiles = layer_multi_tile(TB, R) ? (1u << pd.tpc_log2) : 1u;
  // this thread's <C> terms over the CTA's tiles, summed in FP32 in two
  // levels (2^R positive terms per tile, then at most 2^kMaxTpcLog2 tile
  // sums: relative error below 48 x 2^-24, about 3e-6), FP64 from the block
  // reduction on
  float acc_cta = 0.f;
  for (uint32_t tt = 0; tt < ntiles; ++tt) {
  const uint32_t tile = tj | (tt << per);
  const uint32_t zbase = ((tile & ((1u << lowt) - 1u)) << c) | ((tile >> lowt) << (s + g));
  float2* base = states + Ip->state_off + (zbase | zmap(lt));

  float2 a[KQ];
  const uint32_t li0 = lir_o<TB, R, OC>(tid, 0);
  if (pd.init) {  // s_z = i^popcount(z), z = tile base | thread qubits | register qubits
    const int r = __popc(zbase | zmap(li0));
    const float sg = (r & 2) ? -1.f : 1.f;
    const float2 b = (r & 1) ? make_float2(0.f, sg) : make_float2(sg, 0.f);
#pragma unroll
    for (int k = 0; k < KQ; ++k) a[k] = rot_i(b, popc_c(k));
  } else {
    uint32_t e[R];  // qubit offsets of the register slots
#pragma unroll
    for (int j = 0; j < R; ++j) e[j] = zmap(1u << (O0 + j));
    uint32_t off = 0;
    a[0] = base[0];
#pragma unroll
    for (int i = 1; i < KQ; ++i) {
      const int k = gray(i), b = gray_bit(i);
      off = ((k >> b) & 1) ? off + e[b] : off - e[b];
      a[k] = base[off];
    }
  }
  __syncthreads();  // phase table, planes and Q_K visible
  int A = 0, kap[R];
#pragma unroll
  for (int j = 0; j < R; ++j) kap[j] = 0;
  if (need_cut) {
    if (tid < 32) {
      // lane u < n: contribution of vertex u to C(z_F); lane u < TB: lam of local bit u
      int cfu = 0;
      if ((int)tid < n && ((zbase >> tid) & 1u)) {
        const uint32_t* row = pls + tid * P;
        for (int b = 0; b < P; ++b) cfu += __popc(row[b] & ~zbase) << b;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) cfu += __shfl_xor_sync(0xffffffffu, cfu, o);
      if (tid < (uint32_t)TB) {
        const uint32_t* row = pls + qubit_of(tid, c, s) * P;
        int d = 0, aa = 0;
        for (int b = 0; b < P; ++b) {
          d += __popc(row[b]) << b;
          aa += __popc(row[b] & zbase) << b;
        }
        tc->lam[tid] = d - 2 * aa;
      }
      if (tid == 0) tc->cf = cfu;
    }
    __syncthreads();  // tile constants visible
    A = tc->cf + ccJ;
#pragma unroll
    for (int b = 0; b < TB - R; ++b) A += ((tid >> b) & 1u) ? tc->lam[thread_bit_local_o<R, OC>(b)] : 0;
#pragma unroll
    for (int j = 0; j < R; ++j) kap[j] = tc->lam[OC + j] + ccB[j];
  }
  // round 2 (layout 2) only ever mixes slots below TB - 2R (the others repeat layout 1's)
  constexpr uint32_t kAll = (1u << R) - 1u;
  constexpr uint32_t kLow2 = SPLIT || (TB - 2 * R) >= R ? kAll : ((1u << (TB - 2 * R > 0 ? TB - 2 * R : 0)) - 1u);
  if (pd.layerA >= 0) {
    const float muA = Ip->mu[pd.layerA];
    mix_regs_sel<R, kAll>(a, muA, mm0);
    if constexpr (NR > 1) {
      transposer_o<TB, R, O0, O1>(a, sm, tid);
      mix_regs_sel<R, kAll>(a, muA, mm1);
    }
    if constexpr (NR > 2) {
      transposer_o<TB, R, O1, O2>(a, sm, tid);
      mix_regs_sel<R, kLow2>(a, muA, mm2);
    }
  }
  if (pd.layerP >= 0) {
    int S = A;
    a[0] = cmul(a[0], tab[tix(S + qk[0], W)]);
#pragma unroll
    for (int i = 1; i < KQ; ++i) {
      const int k = gray(i), b = gray_bit(i);
      S = ((k >> b) & 1) ? S + kap[b] : S - kap[b];
      a[k] = cmul(a[k], tab[tix(S + qk[k], W)]);
    }
  }
  if (pd.layerB >= 0) {
    const float muB = Ip->mu[pd.layerB];
    if constexpr (NR > 2) {
      mix_regs_sel<R, kLow2>(a, muB, mm2);
      transposer_o<TB, R, O2, O1>(a, sm, tid);
    }
    if constexpr (NR > 1) {
      mix_regs_sel<R, kAll>(a, muB, mm1);
      transposer_o<TB, R, O1, O0>(a, sm, tid);
    }
    mix_regs_sel<R, kAll>(a, muB, mm0);
  }
  if (pd.expect) {
    float acc = 0.f;
    int S = A;
#pragma unroll
    for (int i = 0; i < KQ; ++i) {
      const int k = gray(i);
      if (i > 0) {
        const int b = gray_bit(i);
        S = ((k >> b) & 1) ? S + kap[b] : S - kap[b];
      }
      acc = fmaf(fmaf(a[k].x, a[k].x, a[k].y * a[k].y), (float)(S + qk[k]), acc);
    }
    acc_cta += acc;
  }
  if (pd.store) {
    if (pd.layerB < 0) {  // a pass without a second mixer ends in the cut layout
      if constexpr (NR == 3) transposer_o<TB, R, O2, O0>(a, sm, tid);
      if constexpr (NR == 2) transposer_o<TB, R, O1, O0>(a, sm, tid);
    }
    if (pd.last) {  // back from the gauge, times lambda_p
      const float2 fs = rot_i(Ip->final_scale, -__popc(zbase | zmap(lt)));
#pragma unroll
      for (int k = 0; k < KQ; ++k) a[k] = cmul(a[k], rot_i(fs, -popc_c(k)));
    }
    uint32_t e[R];
#pragma unroll
    for (int j = 0; j < R; ++j) e[j] = zmap(1u << (O0 + j));
    uint32_t off = 0;
    base[0] = a[0];
#pragma unroll
    for (int i = 1; i < KQ; ++i) {
      const int k = gray(i), b = gray_bit(i);
      off = ((k >> b) & 1) ? off + e[b] : off - e[b];
      base[off] = a[k];
    }
  }
  }  // tiles of this CTA
  // One block reduction per CTA (the FP64 pipe is narrow and the reduction
  // serialises the CTA): the sum goes to the partial slot of the CTA's first
  // tile and its other tiles' slots get 0, so the per-instance reduction
  // over tile slots is unchanged.
  if (pd.expect) {
    const double sum = block_sum((double)acc_cta, red, tid, NT);
    if (tid == 0) {
      partials[Ip->part_off + tj] = sum;
      for (uint32_t tt = 1; tt < ntiles; ++tt) partials[Ip->part_off + (tj | (tt << per))] = 0.0;
    }
  }
}

size_t layer_pass_smem(int kind, int tabcap) {
  const int tb = kTileShapes[kind].tb, r = kTileShapes[kind].r;
  const size_t padded = (size_t(1) << tb) + (size_t(1) << (tb - r));
  return (size_t)tabcap * sizeof(float2) + padded * sizeof(float2) + 32 * 4 + sizeof(TileConst) +
         PARAQAOA_MAX_QUBITS * kMaxPlanes * 4 + 16 * sizeof(double);
}

bool layer_kind_multi_tile(int kind) { return layer_multi_tile(kTileShapes[kind].tb, kTileShapes[kind].r); }


int64_t cut_consts_elems(int kind, int32_t nlist) {
  return (int64_t)nlist * cut_consts_stride(kTileShapes[kind].tb, kTileShapes[kind].r);
}

static int pass_rounds(int tb, int r, const PassDesc& pd) {
  if (pd.split) return 2;
  return 1 + (pd.mix_lo < tb - r) + (pd.mix_lo < tb - 2 * r);
}

template <int TB, int R, int OC>
static cudaError_t launch_cc_t(int n, const PassDesc& pd, const InstDev* inst, const int32_t* list,
                               int32_t nlist, const SubDev* subs, const uint32_t* planes,
                               int32_t* consts, cudaStream_t st) {
  k_cut_consts<TB, R, OC><<<nlist, 1 << (TB - R), 0, st>>>(pd, n, inst, list, subs, planes, consts);
  return cudaGetLastError();
}

cudaError_t launch_cut_consts(int kind, int n, const PassDesc& pd, const InstDev* inst, const int32_t* list,
                              int32_t nlist, const SubDev* subs, const uint32_t* planes,
                              int32_t* consts, cudaStream_t st) {
  if (nlist <= 0 || !(pd.layerP >= 0 || pd.expect)) return cudaSuccess;
  const int tb = kTileShapes[kind].tb, r = kTileShapes[kind].r;
  const int rc = pass_rounds(tb, r, pd) - 1;
#define PQ_CC(TBV, RV) \
  do { \
    if (tb == TBV && r == RV) { \
      if (pd.split) return launch_cc_t<TBV, RV, lay_off(TBV, RV, true, 1)>(n, pd, inst, list, nlist, subs, planes, consts, st); \
      if (rc == 0) return launch_cc_t<TBV, RV, lay_off(TBV, RV, false, 0)>(n, pd, inst, list, nlist, subs, planes, consts, st); \
      if (rc == 1) return launch_cc_t<TBV, RV, lay_off(TBV, RV, false, 1)>(n, pd, inst, list, nlist, subs, planes, consts, st); \
      return launch_cc_t<TBV, RV, lay_off(TBV, RV, false, 2)>(n, pd, inst, list, nlist, subs, planes, consts, st); \
    } \
  } while (0)
  PQ_CC(12, 5);
  PQ_CC(12, 4);
  PQ_CC(13, 5);
#undef PQ_CC
  return cudaErrorInvalidValue;
}

template <int TB, int R, int NR, bool SPLIT>
static cudaError_t launch_layer_t(int kind, int n, const PassDesc& pd, const InstDev* inst,
                                  const int32_t* list, int32_t nlist, const SubDev* subs,
                                  const uint32_t* planes, const float2* tables, float2* states,
                                  double* partials, int32_t tabcap, int32_t* consts, cudaStream_t st) {
  const size_t smem = layer_pass_smem(kind, tabcap);
  cudaError_t e = cudaFuncSetAttribute(k_layer_pass<TB, R, NR, SPLIT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int tiles_log2 = n - TB;
  const int tpc = layer_multi_tile(TB, R) ? pd.tpc_log2 : 0;
  if (tpc < 0 || tpc > tiles_log2 || tpc > kMaxTpcLog2) return cudaErrorInvalidValue;
  const int64_t blocks = (int64_t)nlist << (tiles_log2 - tpc);
  if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
  // register slots each round mixes (mm0: layout 0, mm1: layout 1, mm2: layout 2)
  uint32_t mm0 = 0, mm1 = 0, mm2 = 0;
  for (int j = 0; j < R; ++j) {
    if (SPLIT || TB - R + j >= pd.mix_lo) mm0 |= 1u << j;
    if (SPLIT || TB - 2 * R + j >= pd.mix_lo) mm1 |= 1u << j;
    if (!SPLIT && j >= pd.mix_lo && j < TB - 2 * R) mm2 |= 1u << j;
  }
  k_layer_pass<TB, R, NR, SPLIT><<<(unsigned)blocks, 1 << (TB - R), smem, st>>>(
      pd, n, tiles_log2, inst, list, subs, planes, tables, states, partials, tabcap, consts, mm0, mm1, mm2);
  return cudaGetLastError();
}

cudaError_t launch_layer_pass(int kind, int n, const PassDesc& pd, const InstDev* inst,
                              const int32_t* list, int32_t nlist, const SubDev* subs,
                              const uint32_t* planes, const float2* tables, float2* states,
                              double* partials, int32_t tabcap, int32_t* consts, cudaStream_t st) {
  if (nlist <= 0) return cudaSuccess;
  if (kind < 0 || kind >= kTileKinds) return cudaErrorInvalidValue;
  const int tb = kTileShapes[kind].tb, r = kTileShapes[kind].r;
  if (n < tb) return cudaErrorInvalidValue;
  const int nr = pass_rounds(tb, r, pd);
#define PQ_LAUNCH(TBV, RV) \
  do { \
    if (tb == TBV && r == RV) { \
      if (pd.split) return launch_layer_t<TBV, RV, 2, true>(kind, n, pd, inst, list, nlist, subs, planes, tables, states, partials, tabcap, consts, st); \
      if (nr == 1) return launch_layer_t<TBV, RV, 1, false>(kind, n, pd, inst, list, nlist, subs, planes, tables, states, partials, tabcap, consts, st); \
      if (nr == 2) return launch_layer_t<TBV, RV, 2, false>(kind, n, pd, inst, list, nlist, subs, planes, tables, states, partials, tabcap, consts, st); \
      return launch_layer_t<TBV, RV, 3, false>(kind, n, pd, inst, list, nlist, subs, planes, tables, states, partials, tabcap, consts, st); \
    } \
  } while (0)
  PQ_LAUNCH(12, 5);
  PQ_LAUNCH(12, 4);
  PQ_LAUNCH(13, 5);
#undef PQ_LAUNCH
  return cudaErrorInvalidValue;
}

// Sum the per-tile partials of each instance in a fixed order, times |lambda_p|^2.
__global__ void k_expect_reduce(const InstDev* __restrict__ inst_all, const int32_t* __restrict__ list,
                                int32_t tiles, const double* __restrict__ partials,
                                double* __restrict__ expect) {
  __shared__ double red[8];
  const int ii = list[blockIdx.x];
  const InstDev I = inst_all[ii];
  double acc = 0.0;
  for (int t = threadIdx.x; t < tiles; t += blockDim.x) acc += partials[I.part_off + t];
  double s = block_sum(acc, red, threadIdx.x, blockDim.x);
  if (threadIdx.x == 0) expect[ii] = s * (double)I.final_scale2;
}

cudaError_t launch_expect_reduce(const InstDev* inst, const int32_t* list, int32_t nlist,
                                 int32_t tiles, const double* partials, double* expect,
                                 cudaStream_t st) {
  if (nlist <= 0) return cudaSuccess;
  k_expect_reduce<<<nlist, 256, 0, st>>>(inst, list, tiles, partials, expect);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Cut table (Sec. 2.1) of one subgraph: out[z] = C(z), one thread per z.
__global__ void k_cut_table(const SubDev* __restrict__ sub, const uint32_t* __restrict__ planes_all,
                            uint16_t* __restrict__ out) {
  __shared__ uint32_t pl[PARAQAOA_MAX_QUBITS * kMaxPlanes];
  const SubDev S = *sub;
  for (int q = threadIdx.x; q < S.n * S.P; q += blockDim.x) pl[q] = planes_all[S.plane_off + q];
  __syncthreads();
  const uint64_t dim = 1ull << S.n;
  for (uint64_t z = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; z < dim;
       z += (uint64_t)gridDim.x * blockDim.x)
    out[z] = (uint16_t)cut_eval((uint32_t)z, pl, S.n, S.P);
}

cudaError_t launch_cut_table(const SubDev* sub_dev_one, int n, const uint32_t* planes, uint16_t* out,
                             cudaStream_t st) {
  const uint64_t dim = 1ull << n;
  const unsigned blocks = (unsigned)std::min<uint64_t>((dim + 255) / 256, 152ull * 16);
  k_cut_table<<<blocks, 256, 0, st>>>(sub_dev_one, planes, out);
  return cudaGetLastError();
}

}  // namespace pq
