// QAOA state-vector kernels for sm_103a that are not the HBM-streaming
// layer pass (layer_pass.cu): layer constants, on-chip simulation of small
// states, the <C> reduction over tile partials and the cut table. The
// state representation (gauge, mixer arithmetic, cut values) is described
// in sim_common.cuh.
#include <cuda_runtime.h>

#include <algorithm>

#include "sim_common.cuh"

namespace pq {

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
// Every transpose of the on-chip kernel starts from the layout the one before
// it ended in (goto_layout tracks it), and the only other shared-memory
// writes (the next layer's phase table, the <C> reduction) sit behind
// barriers of their own, so the barrier after a transpose's reads is left out.
template <int TB, int FROM, int TO>
__device__ __forceinline__ void transpose(float2 (&a)[32], float2* sm, uint32_t tid) {
  transposer<TB, 5, FROM, TO, false>(a, sm, tid);
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
// Resident CTAs per SM the on-chip kernel is compiled for (registers capped
// at 65536 / (threads x CTAs)): two CTAs of 256 threads at 13 qubits and four
// of 128 at 12 (both at 128 registers, a few bytes of spills; uncapped they
// took 162 and 161 registers, one and three CTAs), four of 64 at 11 (a
// tighter cap spills 256 B), eight of 32 at 10; 14 qubits fill one SM's
// shared memory.
__host__ __device__ constexpr int smem_sim_min_blocks(int tb) {
  return tb >= 14 ? 1 : (tb == 13 ? 2 : (tb == 10 ? 8 : 4));
}

template <int TB>
__global__ void __launch_bounds__(1 << (TB - 5), smem_sim_min_blocks(TB))
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
    // The next layer's table load may overwrite tab now: every layer takes at
    // least one transpose after its phase, whose barrier all threads reach
    // only after their last read of the table.
    static_assert(NR >= 2, "a transpose per layer orders the table reads before the next load");
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
  // a halved state holds one of each pair z, not z of equal |psi|^2 and C
  if (threadIdx.x == 0) expect[ii] = s * (double)I.final_scale2 * (I.halved ? 2.0 : 1.0);
}

cudaError_t launch_expect_reduce(const InstDev* inst, const int32_t* list, int32_t nlist,
                                 int32_t tiles, const double* partials, double* expect,
                                 cudaStream_t st) {
  if (nlist <= 0) return cudaSuccess;
  k_expect_reduce<<<nlist, 256, 0, st>>>(inst, list, tiles, partials, expect);
  return cudaGetLastError();
}

// *dst |= *src (one thread): folds a launch's error word into a sticky one.
__global__ void k_flag_or(const uint64_t* __restrict__ src, uint64_t* __restrict__ dst) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && *src) *dst = 1;
}

cudaError_t launch_flag_or(const uint64_t* src, uint64_t* dst, cudaStream_t st) {
  k_flag_or<<<1, 32, 0, st>>>(src, dst);
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
