// The HBM-streaming layer pass (Sec. 2.2, Sec. 3.3): one pass over every
// tile of a batch of same-size QAOA states finishes one layer's mixer on a
// qubit group, applies the next cost phase and starts the next mixer, or
// reduces <C>. The state representation (gauge, mixer arithmetic, cut
// values) is described in sim_common.cuh.
#include <cuda_runtime.h>

#include <algorithm>

#include "sim_common.cuh"

namespace pq {

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

// Occupancy target of a tile shape: resident CTAs per SM. The 16-register
// shapes fit 64 registers per thread: four CTAs of 256 threads (2^12), two of
// 512 (2^13) or one of 1024 (2^14), 32 warps per SM each; the 2^12 x 32
// shape is held to 96 registers for five CTAs of 128 threads (a few bytes of
// spills, measured 3% faster than four CTAs at 128 registers); the 2^13 x 32
// shape runs two CTAs of 256 threads.
__host__ __device__ constexpr int layer_min_blocks(int tb, int r) {
  return r == 4 ? (1 << (14 - tb)) : (tb >= 13 ? 2 : 5);
}

// State loads of a layer pass. CG: through L2 only (the persistent kernel
// reads, in one launch, amplitudes that other SMs wrote earlier in the same
// launch, which a stale L1 line must not serve).
template <bool CG>
__device__ __forceinline__ float2 ld_state(const float2* p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}

// Tile constants (cf, lam) of each of a CTA's tiles tj + (u << per), one
// warp per tile: lane v < n adds vertex v's share of C(z_F), lane v < tb
// the lam of local bit v. Run once per CTA before its tile loop; kept out of
// line so that its registers do not weigh on the loop's.
__device__ __noinline__ void tile_consts(TileConst* tcs, const uint32_t* pls, uint32_t tid, uint32_t nt,
                                         uint32_t ntiles, uint32_t tj, uint32_t per, uint32_t lowt, int c, int s,
                                         int g, int n, int P, int tb) {
  const uint32_t lane = tid & 31u;
  for (uint32_t u = tid >> 5; u < ntiles; u += nt >> 5) {
    const uint32_t tu = tj | (u << per);
    const uint32_t zb = ((tu & ((1u << lowt) - 1u)) << c) | ((tu >> lowt) << (s + g));
    int cfu = 0;
    if ((int)lane < n && ((zb >> lane) & 1u)) {
      const uint32_t* row = pls + lane * P;
      for (int b = 0; b < P; ++b) cfu += __popc(row[b] & ~zb) << b;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cfu += __shfl_xor_sync(0xffffffffu, cfu, o);
    if (lane < (uint32_t)tb) {
      const uint32_t* row = pls + qubit_of(lane, c, s) * P;
      int d = 0, aa = 0;
      for (int b = 0; b < P; ++b) {
        d += __popc(row[b]) << b;
        aa += __popc(row[b] & zb) << b;
      }
      tcs[u].lam[lane] = d - 2 * aa;
    }
    if (lane == 0) tcs[u].cf = cfu;
  }
}

// One CTA's share of a layer pass, work unit `bid` of the pass: instance
// list[bid >> per] and its tiles tj, tj + 2^per, ... with tj = bid mod 2^per
// (per = tiles_log2 - tpc_log2, 2^tpc_log2 tiles).
// CONTIG: the pass's tile is 2^TB contiguous amplitudes (the low qubit
// group, c = s = TB), so every register slot's offset is a compile-time
// constant and loads and stores take immediate offsets from one base.
template <int TB, int R, int NR, bool SPLIT, bool CONTIG, bool CG>
__device__ __forceinline__ void layer_tiles(const PassDesc pd, int32_t n, int32_t tiles_log2, uint32_t bid,
                                            const InstDev* __restrict__ inst_all, const int32_t* __restrict__ list,
                                            const SubDev* __restrict__ subs, const uint32_t* __restrict__ planes_all,
                                            const float2* __restrict__ tables, float2* __restrict__ states,
                                            double* __restrict__ partials, int32_t tabcap,
                                            const int32_t* __restrict__ consts, uint32_t mm0, uint32_t mm1,
                                            uint32_t mm2, uint32_t mm3) {
  constexpr uint32_t NT = 1u << (TB - R);
  constexpr int KQ = 1 << R;  // registers per thread
  constexpr int O0 = lay_off(TB, R, SPLIT, 0), O1 = lay_off(TB, R, SPLIT, 1), O2 = lay_off(TB, R, SPLIT, 2),
                O3 = lay_off(TB, R, SPLIT, 3);
  constexpr int OC = lay_off(TB, R, SPLIT, NR - 1);  // layout of the cut step (phase / <C>)
  static_assert(!SPLIT || NR == 2, "split passes mix two rounds");
  static_assert(NR <= full_rounds(TB, R) || SPLIT, "no more rounds than the tile has register groups");
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* tab = reinterpret_cast<float2*>(smraw);
  float2* sm = tab + tabcap;
  int* qk = reinterpret_cast<int*>(sm + padded_r<TB, R>());  // 2^R entries (<= 32)
  int* qk8 = qk + 32;  // the same in bytes of the phase table (x sizeof(float2))
  TileConst* tcs = reinterpret_cast<TileConst*>(qk + 64);  // one per tile of the CTA
  uint32_t* pls = reinterpret_cast<uint32_t*>(tcs + (1 << kMaxTpcLog2));  // the instance's bit-planes
  double* red = reinterpret_cast<double*>(pls + PARAQAOA_MAX_QUBITS * kMaxPlanes);
  const uint32_t tid = threadIdx.x;
  const int c = CONTIG ? TB : pd.c, s = CONTIG ? TB : pd.s, g = TB - c;
  const uint32_t lowt = (uint32_t)(s - c);
  // this CTA's 2^tpc_log2 tiles, all of one instance, strided by the
  // instance's CTA count: CTAs that run side by side then cover consecutive
  // tiles, which keeps the DRAM pages of a pass with short contiguous runs
  // (a high qubit group) busy together
  const uint32_t per = (uint32_t)(tiles_log2 - pd.tpc_log2);
  const int li_idx = (int)(bid >> per);
  const uint32_t tj = bid & ((1u << per) - 1u);
  const InstDev* Ip = inst_all + list[li_idx];
  const int P = Ip->P, W = Ip->W;
  const uint32_t* pl = planes_all + subs[Ip->sub].plane_off;
  const bool need_cut = pd.layerP >= 0 || pd.expect;

  // ---- set-up. One round of global loads, all issued before the first
  // barrier (the first tile's state loads too): the phase table, the
  // instance's adjacency bit-planes, the Q_K table and this thread's cut
  // constants. After the barrier each warp derives the constants of one of
  // the CTA's tiles (more when the tiles outnumber the warps) from the planes
  // in shared memory, so the tile loop itself needs no barrier for them.
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
    if (tid < (uint32_t)KQ) {
      const int q = cc_inst[tid];
      qk[tid] = q;
      qk8[tid] = q * (int)sizeof(float2);
    }
    ccJ = cc_inst[KQ + tid];
#pragma unroll
    for (int j = 0; j < R; ++j) ccB[j] = cc_inst[KQ + (1 + j) * NT + tid];
  }
  // Local index -> qubit offset: local bits [0, c) are qubits [0, c), bits
  // [c, TB) move up by s - c (a monotone bit map, so it keeps popcounts).
  const uint32_t lowm = (1u << c) - 1u;
  const int sh = s - c;
  auto zmap = [&](uint32_t li) -> uint32_t { return CONTIG ? li : (li & lowm) | ((li & ~lowm) << sh); };
  // load/store layout O0: this thread's amplitude offsets are zmap(lt | register bits)
  const uint32_t lt = lir_o<TB, R, O0>(tid, 0);
  // Tiles of one CTA share the set-up above; inside the tile loop shared
  // memory is written only by the transposes. Those leave out the barrier
  // after their reads (each chains from the layout the one before it read).
  // Across tiles the chain holds when the pass starts in the layout it ends
  // in (O0 when it mixes first, else the cut layout OC); otherwise a barrier
  // follows the next tile's state loads (issued first, so that they are in
  // flight while warps wait).
  const uint32_t ntiles = 1u << pd.tpc_log2;
  const bool tr_a = pd.layerA >= 0, tr_b = pd.layerB >= 0, tr_s = pd.store && !tr_b;
  const bool trail_tile = NR > 1 && (tr_a || tr_b || tr_s) && (tr_a ? O0 : OC) != ((tr_b || tr_s) ? O0 : OC);
  // this thread's <C> terms over the CTA's tiles, summed in FP32 in two
  // levels (2^R positive terms per tile, then at most 2^kMaxTpcLog2 tile
  // sums: relative error below 48 x 2^-24, about 3e-6), FP64 from the block
  // reduction on
  float acc_cta = 0.f;
  // the last round of a classic pass overlaps the one before it when R does
  // not divide TB: only its slots below the previous offset ever mix
  constexpr uint32_t kS0 = round_slots(TB, R, SPLIT, 0), kS1 = round_slots(TB, R, SPLIT, 1),
                     kS2 = round_slots(TB, R, SPLIT, 2), kS3 = round_slots(TB, R, SPLIT, 3);
  // every slot a round may mix does (the pass's qubit group covers them all):
  // one broadcast multiplier per round instead of a select per slot
  const bool full_mix = (mm0 & kS0) == kS0 && (NR < 2 || (mm1 & kS1) == kS1) && (NR < 3 || (mm2 & kS2) == kS2) &&
                        (NR < 4 || (mm3 & kS3) == kS3);
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
    a[0] = ld_state<CG>(base);
#pragma unroll
    for (int i = 1; i < KQ; ++i) {
      const int k = gray(i), b = gray_bit(i);
      off = ((k >> b) & 1) ? off + e[b] : off - e[b];
      a[k] = ld_state<CG>(base + off);
    }
  }
  if (tt == 0) {
    __syncthreads();  // set-up loads visible
    if (need_cut) {
      tile_consts(tcs, pls, tid, NT, ntiles, tj, per, lowt, c, s, g, n, P, TB);
      __syncthreads();  // tile constants visible
    }
  } else if (trail_tile) {
    __syncthreads();  // the previous tile's last transpose reads, before this tile's first writes
  }
  int A = 0, kap[R];
#pragma unroll
  for (int j = 0; j < R; ++j) kap[j] = 0;
  if (need_cut) {
    const TileConst* tc = tcs + tt;
    A = tc->cf + ccJ;
#pragma unroll
    for (int b = 0; b < TB - R; ++b) A += ((tid >> b) & 1u) ? tc->lam[thread_bit_local_o<R, OC>(b)] : 0;
#pragma unroll
    for (int j = 0; j < R; ++j) kap[j] = tc->lam[OC + j] + ccB[j];
  }
  if (pd.layerA >= 0) {
    const float muA = Ip->mu[pd.layerA];
    mix_round<R, kS0>(a, muA, mm0, full_mix);
    if constexpr (NR > 1) {
      transposer_o<TB, R, O0, O1, false>(a, sm, tid);
      mix_round<R, kS1>(a, muA, mm1, full_mix);
    }
    if constexpr (NR > 2) {
      transposer_o<TB, R, O1, O2, false>(a, sm, tid);
      mix_round<R, kS2>(a, muA, mm2, full_mix);
    }
    if constexpr (NR > 3) {
      transposer_o<TB, R, O2, O3, false>(a, sm, tid);
      mix_round<R, kS3>(a, muA, mm3, full_mix);
    }
  }
  if (pd.layerP >= 0) {
    // cut values walked in bytes of the table: index, clamp, load
    const unsigned char* tb8 = reinterpret_cast<const unsigned char*>(tab);
    const uint32_t W8 = (uint32_t)W * (uint32_t)sizeof(float2);
    int S = A * (int)sizeof(float2);
    a[0] = cmul(a[0], *reinterpret_cast<const float2*>(tb8 + min((uint32_t)(S + qk8[0]), W8)));
#pragma unroll
    for (int i = 1; i < KQ; ++i) {
      const int k = gray(i), b = gray_bit(i);
      const int k8 = kap[b] * (int)sizeof(float2);
      S = ((k >> b) & 1) ? S + k8 : S - k8;
      a[k] = cmul(a[k], *reinterpret_cast<const float2*>(tb8 + min((uint32_t)(S + qk8[k]), W8)));
    }
  }
  if (pd.layerB >= 0) {
    const float muB = Ip->mu[pd.layerB];
    if constexpr (NR > 3) {
      mix_round<R, kS3>(a, muB, mm3, full_mix);
      transposer_o<TB, R, O3, O2, false>(a, sm, tid);
    }
    if constexpr (NR > 2) {
      mix_round<R, kS2>(a, muB, mm2, full_mix);
      transposer_o<TB, R, O2, O1, false>(a, sm, tid);
    }
    if constexpr (NR > 1) {
      mix_round<R, kS1>(a, muB, mm1, full_mix);
      transposer_o<TB, R, O1, O0, false>(a, sm, tid);
    }
    mix_round<R, kS0>(a, muB, mm0, full_mix);
  }
  if (pd.expect) {
    // sum_k |a_k|^2 C_k with C_k = A + sum_{j in k} kap_j + qk[k], and qk
    // (-2 Q_K) a sum over the pairs of set register bits, qk[{j, l}] each:
    // after superset sums nk[m] = sum over k containing m of |a_k|^2 it is
    // A nk[0] + sum_j kap_j nk[{j}] + sum_{j<l} qk[{j,l}] nk[{j,l}].
    float nk[KQ];
#pragma unroll
    for (int k = 0; k < KQ; ++k) nk[k] = fmaf(a[k].x, a[k].x, a[k].y * a[k].y);
#pragma unroll
    for (int j = 0; j < R; ++j)
#pragma unroll
      for (int k = 0; k < KQ; ++k)
        if (!((k >> j) & 1)) nk[k] += nk[k | (1 << j)];
    float acc = (float)A * nk[0];
#pragma unroll
    for (int j = 0; j < R; ++j) acc = fmaf((float)kap[j], nk[1 << j], acc);
#pragma unroll
    for (int j = 0; j < R; ++j)
#pragma unroll
      for (int l = j + 1; l < R; ++l) acc = fmaf((float)qk[(1 << j) | (1 << l)], nk[(1 << j) | (1 << l)], acc);
    acc_cta += acc;
  }
  if (pd.store) {
    if (pd.layerB < 0) {  // a pass without a second mixer ends in the cut layout
      if constexpr (NR > 1) transposer_o<TB, R, OC, O0, false>(a, sm, tid);
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

// One launch per pass: CTA b takes work unit b.
template <int TB, int R, int NR, bool SPLIT, bool CONTIG>
__global__ void __launch_bounds__(1 << (TB - R), layer_min_blocks(TB, R))
    k_layer_pass(PassDesc pd, int32_t n, int32_t tiles_log2, const InstDev* __restrict__ inst_all,
                 const int32_t* __restrict__ list, const SubDev* __restrict__ subs,
                 const uint32_t* __restrict__ planes_all, const float2* __restrict__ tables,
                 float2* __restrict__ states, double* __restrict__ partials, int32_t tabcap,
                 const int32_t* __restrict__ consts, uint32_t mm0, uint32_t mm1, uint32_t mm2, uint32_t mm3) {
  layer_tiles<TB, R, NR, SPLIT, CONTIG, false>(pd, n, tiles_log2, blockIdx.x, inst_all, list, subs, planes_all,
                                               tables, states, partials, tabcap, consts, mm0, mm1, mm2, mm3);
}

size_t layer_pass_smem(int kind, int tabcap) {
  const int tb = kTileShapes[kind].tb, r = kTileShapes[kind].r;
  const size_t padded = (size_t(1) << tb) + (size_t(1) << (tb - r));
  return (size_t)tabcap * sizeof(float2) + padded * sizeof(float2) + 64 * 4 + (sizeof(TileConst) << kMaxTpcLog2) +
         PARAQAOA_MAX_QUBITS * kMaxPlanes * 4 + 32 * sizeof(double);
}



int64_t cut_consts_elems(int kind, int32_t nlist) {
  return (int64_t)nlist * cut_consts_stride(kTileShapes[kind].tb, kTileShapes[kind].r);
}

// Rounds a pass needs: enough that the last one's offset is at or below the
// lowest local bit it mixes.
static int pass_rounds(int tb, int r, const PassDesc& pd) {
  if (pd.split) return 2;
  int k = 1;
  while (k < full_rounds(tb, r) && pd.mix_lo < lay_off(tb, r, false, k - 1)) ++k;
  return k;
}

int layer_pass_rounds(int kind, const PassDesc& pd) {
  return pass_rounds(kTileShapes[kind].tb, kTileShapes[kind].r, pd);
}

void layer_pass_masks(int kind, const PassDesc& pd, uint32_t mm[4]) {
  const int tb = kTileShapes[kind].tb, r = kTileShapes[kind].r;
  const int nr = pass_rounds(tb, r, pd);
  const bool split = pd.split != 0;
  for (int k = 0; k < 4; ++k) {
    mm[k] = 0;
    if (k >= nr) continue;
    for (int j = 0; j < r; ++j)
      if (((round_slots(tb, r, split, k) >> j) & 1u) && (split || lay_off(tb, r, split, k) + j >= pd.mix_lo))
        mm[k] |= 1u << j;
  }
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
#define PQ_CCA n, pd, inst, list, nlist, subs, planes, consts, st
#define PQ_CC(TBV, RV) \
  do { \
    if (tb == TBV && r == RV) { \
      if (pd.split) return launch_cc_t<TBV, RV, lay_off(TBV, RV, true, 1)>(PQ_CCA); \
      if (rc == 0) return launch_cc_t<TBV, RV, lay_off(TBV, RV, false, 0)>(PQ_CCA); \
      if (rc == 1) return launch_cc_t<TBV, RV, lay_off(TBV, RV, false, 1)>(PQ_CCA); \
      if (rc == 2) return launch_cc_t<TBV, RV, lay_off(TBV, RV, false, 2)>(PQ_CCA); \
      return launch_cc_t<TBV, RV, lay_off(TBV, RV, false, 3)>(PQ_CCA); \
    } \
  } while (0)
  PQ_CC(12, 5);
  PQ_CC(12, 4);
  PQ_CC(13, 5);
  PQ_CC(13, 4);
  PQ_CC(14, 4);
#undef PQ_CC
#undef PQ_CCA
  return cudaErrorInvalidValue;
}

template <int TB, int R, int NR, bool SPLIT, bool CONTIG>
static cudaError_t launch_layer_t(int kind, int n, int nq, const PassDesc& pd, const InstDev* inst,
                                  const int32_t* list, int32_t nlist, const SubDev* subs,
                                  const uint32_t* planes, const float2* tables, float2* states,
                                  double* partials, int32_t tabcap, int32_t* consts, cudaStream_t st) {
  const size_t smem = layer_pass_smem(kind, tabcap);
  if (CONTIG && (pd.c != TB || pd.s != TB)) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_layer_pass<TB, R, NR, SPLIT, CONTIG>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int tiles_log2 = nq - TB;
  const int tpc = pd.tpc_log2;
  if (tpc < 0 || tpc > tiles_log2 || tpc > kMaxTpcLog2) return cudaErrorInvalidValue;
  const int64_t blocks = (int64_t)nlist << (tiles_log2 - tpc);
  if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
  // register slots each round mixes: its slots at or above mix_lo that no
  // earlier round covered (split passes mix every slot of both rounds)
  uint32_t mm[4] = {0, 0, 0, 0};
  for (int k = 0; k < NR; ++k)
    for (int j = 0; j < R; ++j)
      if (((round_slots(TB, R, SPLIT, k) >> j) & 1u) && (SPLIT || lay_off(TB, R, SPLIT, k) + j >= pd.mix_lo))
        mm[k] |= 1u << j;
  k_layer_pass<TB, R, NR, SPLIT, CONTIG><<<(unsigned)blocks, 1 << (TB - R), smem, st>>>(
      pd, n, tiles_log2, inst, list, subs, planes, tables, states, partials, tabcap, consts, mm[0], mm[1], mm[2],
      mm[3]);
  return cudaGetLastError();
}

static cudaError_t launch_mirror(int kind, int n, int nq, const PassDesc& pd, const InstDev* inst, const int32_t* list,
                                 int32_t nlist, const SubDev* subs, const uint32_t* planes, const float2* tables,
                                 float2* states, double* partials, int32_t tabcap, int32_t* consts, cudaStream_t st);

cudaError_t launch_layer_pass(int kind, int n, int nq, const PassDesc& pd, const InstDev* inst,
                              const int32_t* list, int32_t nlist, const SubDev* subs,
                              const uint32_t* planes, const float2* tables, float2* states,
                              double* partials, int32_t tabcap, int32_t* consts, cudaStream_t st) {
  if (nlist <= 0) return cudaSuccess;
  if (kind < 0 || kind >= kTileKinds) return cudaErrorInvalidValue;
  const int tb = kTileShapes[kind].tb, r = kTileShapes[kind].r;
  if (nq < tb || nq > n) return cudaErrorInvalidValue;
  if (pd.mirrorA || pd.mirrorB)
    return launch_mirror(kind, n, nq, pd, inst, list, nlist, subs, planes, tables, states, partials, tabcap, consts,
                         st);
  const int nr = pass_rounds(tb, r, pd);
  // split passes always cover the contiguous low group; classic passes over
  // it mix all TB local bits in three rounds
  const bool contig = pd.c == tb && pd.s == tb;
  if (pd.split && !contig) return cudaErrorInvalidValue;
#define PQ_ARGS kind, n, nq, pd, inst, list, nlist, subs, planes, tables, states, partials, tabcap, consts, st
  // instantiated: split passes; the contiguous low group in all its rounds;
  // other groups in one to three rounds (every high group carries at least
  // two contiguous qubits, and the third round's offset is at most 2)
#define PQ_LAUNCH(TBV, RV) \
  do { \
    if (tb == TBV && r == RV) { \
      constexpr int kFull = full_rounds(TBV, RV); \
      if (pd.split) return launch_layer_t<TBV, RV, 2, true, true>(PQ_ARGS); \
      if (contig && nr == kFull) return launch_layer_t<TBV, RV, kFull, false, true>(PQ_ARGS); \
      if (contig) return cudaErrorInvalidValue; \
      if (nr == 1) return launch_layer_t<TBV, RV, 1, false, false>(PQ_ARGS); \
      if (nr == 2) return launch_layer_t<TBV, RV, 2, false, false>(PQ_ARGS); \
      if (nr == 3) return launch_layer_t<TBV, RV, 3, false, false>(PQ_ARGS); \
      return cudaErrorInvalidValue; \
    } \
  } while (0)
  PQ_LAUNCH(12, 5);
  PQ_LAUNCH(12, 4);
  PQ_LAUNCH(13, 5);
  PQ_LAUNCH(13, 4);
  PQ_LAUNCH(14, 4);
#undef PQ_LAUNCH
#undef PQ_ARGS
  return cudaErrorInvalidValue;
}

// ------------------------------------------------------------ halved states
// A QAOA state keeps psi_z = psi_(not z) (|+>^n and both unitaries commute
// with the global flip), so a halved state stores only y = z < 2^m, m = n - 1
// (vertex m on side 0). The mixer of qubits j < m acts on the half as usual;
// the mixer of qubit m pairs y with its complement y' = (2^m - 1) - y: in the
// untransformed state (a, b) = (psi_y, psi_y') -> (a + i mu b, b + i mu a), and
// with the gauge s_y = i^popc(y) psi_y that becomes
//   s_y  <- s_y  + mu sigma kappa s_y'
//   s_y' <- s_y' + mu sigma kappa (-1)^m s_y,   kappa = i^(1 - m), sigma = (-1)^popc(y).
// The cut of the complement is C(y') = C(y | 2^m) = C(y) + Delta(y), Delta(y) =
// d_m - 2 sum_u w_mu y_u: linear in y's bits, split like lam into a tile part,
// a thread part and register slots.
//
// k_layer_mirror is the low-group pass (contiguous 2^TB tiles, classic
// rounds) of a halved state: a CTA holds tile t (top tile bit 0) in a[] and
// its mirror tile t' = t xor (2^(tiles) - 1) in b[], b's slot k of thread tid
// being the complement of a's slot k in every layout, so the mirror butterfly
// is register-local; b's butterflies on the other qubits take -mu (the
// complemented pair swaps roles). Every step of the pass (phase, rounds,
// transposes, <C>, store) runs on both halves.
struct MirrorConst {
  int cf, dfv;   // C(z_F); d_m - 2 sum_{u in F} w_mu z_u
  int lam[16];   // lam_u per local bit
  int del[16];   // -2 w_mu per local bit
  int pad[2];
};
static_assert(sizeof(MirrorConst) % 16 == 0, "shared-memory carve-up needs 16-byte multiples");

__host__ __device__ constexpr int mirror_min_blocks(int tb) { return tb >= 13 ? 1 : 2; }

// mirror butterfly of one slot (f = mu sigma, the data a, b of the pair)
__device__ __forceinline__ void mirror_bfly(float2& a, float2& b, float f, int m) {
  const float2 kb = rot_i(b, 1 - m), ka = rot_i(a, 1 - m);
  const float g = (m & 1) ? -f : f;
  a = make_float2(fmaf(f, kb.x, a.x), fmaf(f, kb.y, a.y));
  b = make_float2(fmaf(g, ka.x, b.x), fmaf(g, ka.y, b.y));
}

template <int TB, int R, int X>
__device__ __forceinline__ void mirror_all(float2 (&a)[1 << R], float2 (&b)[1 << R], float mu, uint32_t zbase,
                                           uint32_t tid, int m) {
  const int par = __popc(zbase | lir_o<TB, R, X>(tid, 0)) & 1;
#pragma unroll
  for (int k = 0; k < (1 << R); ++k) {
    const float f = ((par + popc_c(k)) & 1) ? -mu : mu;
    mirror_bfly(a[k], b[k], f, m);
  }
}

template <int TB, int R, int NR>
__global__ void __launch_bounds__(1 << (TB - R), mirror_min_blocks(TB))
    k_layer_mirror(PassDesc pd, int32_t n, int32_t tiles_log2, const InstDev* __restrict__ inst_all,
                   const int32_t* __restrict__ list, const SubDev* __restrict__ subs,
                   const uint32_t* __restrict__ planes_all, const float2* __restrict__ tables,
                   float2* __restrict__ states, double* __restrict__ partials, int32_t tabcap,
                   const int32_t* __restrict__ consts, uint32_t mm0, uint32_t mm1, uint32_t mm2, uint32_t mm3) {
  constexpr uint32_t NT = 1u << (TB - R);
  constexpr int KQ = 1 << R;
  constexpr int O0 = lay_off(TB, R, false, 0), O1 = lay_off(TB, R, false, 1), O2 = lay_off(TB, R, false, 2),
                O3 = lay_off(TB, R, false, 3);
  constexpr int OC = lay_off(TB, R, false, NR - 1);
  static_assert(NR == full_rounds(TB, R), "the low-group pass mixes all its rounds");
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* tab = reinterpret_cast<float2*>(smraw);
  float2* sm = tab + tabcap;
  int* qk = reinterpret_cast<int*>(sm + padded_r<TB, R>());
  MirrorConst* tc = reinterpret_cast<MirrorConst*>(qk + 32);
  uint32_t* pls = reinterpret_cast<uint32_t*>(tc + 1);
  double* red = reinterpret_cast<double*>(pls + PARAQAOA_MAX_QUBITS * kMaxPlanes);
  const uint32_t tid = threadIdx.x;
  const int m = n - 1;  // stored qubits; vertex m is the one left on side 0
  // work unit: 2^tpc pairs of one instance, strided by the instance's CTA count
  const uint32_t per = (uint32_t)(tiles_log2 - 1 - pd.tpc_log2);
  const int li_idx = (int)(blockIdx.x >> per);
  const uint32_t tj = blockIdx.x & ((1u << per) - 1u);
  const uint32_t tmask = (1u << tiles_log2) - 1u, lmask = (1u << TB) - 1u;
  const InstDev* Ip = inst_all + list[li_idx];
  const int P = Ip->P, W = Ip->W;
  const uint32_t* pl = planes_all + subs[Ip->sub].plane_off;
  const bool need_cut = pd.layerP >= 0 || pd.expect;
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
  const uint32_t lt = lir_o<TB, R, O0>(tid, 0);
  const uint32_t ntiles = 1u << pd.tpc_log2;
  float acc_cta = 0.f;
  for (uint32_t tt = 0; tt < ntiles; ++tt) {
  const uint32_t tile = tj | (tt << per), mtile = tile ^ tmask;
  const uint32_t zbase = tile << TB;
  float2* base = states + Ip->state_off + (zbase | lt);
  float2* mbase = states + Ip->state_off + ((mtile << TB) | (lmask - lt));  // slot k at mbase - (k << O0)
  float2 a[KQ], b[KQ];
  if (pd.init) {  // layout OC: s_y = i^popc(y), s_y' = i^(m - popc(y))
    const int r = __popc(zbase | lir_o<TB, R, OC>(tid, 0));
    const float2 ba = rot_i(make_float2(1.f, 0.f), r), bb = rot_i(make_float2(1.f, 0.f), m - r);
#pragma unroll
    for (int k = 0; k < KQ; ++k) {
      a[k] = rot_i(ba, popc_c(k));
      b[k] = rot_i(bb, -popc_c(k));
    }
  } else {
#pragma unroll
    for (int k = 0; k < KQ; ++k) {
      a[k] = base[k << O0];
      b[k] = mbase[-(int32_t)(k << O0)];
    }
  }
  __syncthreads();  // set-up visible; the previous tile's constants read
  int A = 0, kap[R], D = 0, dk[R];
#pragma unroll
  for (int j = 0; j < R; ++j) kap[j] = dk[j] = 0;
  if (need_cut) {
    if (tid < 32) {
      int cfu = 0, dfu = 0;
      const uint32_t* rv = pls + m * P;  // vertex m's neighbourhood
      int wv = 0;                        // w_(m, lane)
      for (int bb = 0; bb < P; ++bb) wv += (int)((rv[bb] >> tid) & 1u) << bb;
      if ((int)tid < n && ((zbase >> tid) & 1u)) {
        const uint32_t* row = pls + tid * P;
        for (int bb = 0; bb < P; ++bb) cfu += __popc(row[bb] & ~zbase) << bb;
        dfu = wv;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        cfu += __shfl_xor_sync(0xffffffffu, cfu, o);
        dfu += __shfl_xor_sync(0xffffffffu, dfu, o);
      }
      if (tid < (uint32_t)TB) {
        const uint32_t* row = pls + tid * P;
        int d = 0, aa = 0;
        for (int bb = 0; bb < P; ++bb) {
          d += __popc(row[bb]) << bb;
          aa += __popc(row[bb] & zbase) << bb;
        }
        tc->lam[tid] = d - 2 * aa;
        tc->del[tid] = -2 * wv;
      }
      if (tid == 0) {
        int dm = 0;
        for (int bb = 0; bb < P; ++bb) dm += __popc(rv[bb]) << bb;
        tc->cf = cfu;
        tc->dfv = dm - 2 * dfu;
      }
    }
    __syncthreads();
    A = tc->cf + ccJ;
    D = tc->dfv;
#pragma unroll
    for (int bb = 0; bb < TB - R; ++bb)
      if ((tid >> bb) & 1u) {
        A += tc->lam[thread_bit_local_o<R, OC>(bb)];
        D += tc->del[thread_bit_local_o<R, OC>(bb)];
      }
#pragma unroll
    for (int j = 0; j < R; ++j) {
      kap[j] = tc->lam[OC + j] + ccB[j];
      dk[j] = tc->del[OC + j];
    }
  }
  constexpr uint32_t kS0 = round_slots(TB, R, false, 0), kS1 = round_slots(TB, R, false, 1),
                     kS2 = round_slots(TB, R, false, 2), kS3 = round_slots(TB, R, false, 3);
  if (pd.layerA >= 0) {
    const float muA = Ip->mu[pd.layerA];
    mix_regs_sel<R, kS0>(a, muA, mm0);
    mix_regs_sel<R, kS0>(b, -muA, mm0);
    if constexpr (NR > 1) {
      transposer_o<TB, R, O0, O1>(a, sm, tid);
      transposer_o<TB, R, O0, O1>(b, sm, tid);
      mix_regs_sel<R, kS1>(a, muA, mm1);
      mix_regs_sel<R, kS1>(b, -muA, mm1);
    }
    if constexpr (NR > 2) {
      transposer_o<TB, R, O1, O2>(a, sm, tid);
      transposer_o<TB, R, O1, O2>(b, sm, tid);
      mix_regs_sel<R, kS2>(a, muA, mm2);
      mix_regs_sel<R, kS2>(b, -muA, mm2);
    }
    if constexpr (NR > 3) {
      transposer_o<TB, R, O2, O3>(a, sm, tid);
      transposer_o<TB, R, O2, O3>(b, sm, tid);
      mix_regs_sel<R, kS3>(a, muA, mm3);
      mix_regs_sel<R, kS3>(b, -muA, mm3);
    }
    if (pd.mirrorA) mirror_all<TB, R, OC>(a, b, muA, zbase, tid, m);
  }
  if (pd.layerP >= 0) {
    int S = A, T = D;
    a[0] = cmul(a[0], tab[tix(S + qk[0], W)]);
    b[0] = cmul(b[0], tab[tix(S + qk[0] + T, W)]);
#pragma unroll
    for (int i = 1; i < KQ; ++i) {
      const int k = gray(i), bt = gray_bit(i);
      S = ((k >> bt) & 1) ? S + kap[bt] : S - kap[bt];
      T = ((k >> bt) & 1) ? T + dk[bt] : T - dk[bt];
      a[k] = cmul(a[k], tab[tix(S + qk[k], W)]);
      b[k] = cmul(b[k], tab[tix(S + qk[k] + T, W)]);
    }
  }
  if (pd.layerB >= 0) {
    const float muB = Ip->mu[pd.layerB];
    if constexpr (NR > 3) {
      mix_regs_sel<R, kS3>(a, muB, mm3);
      mix_regs_sel<R, kS3>(b, -muB, mm3);
      transposer_o<TB, R, O3, O2>(a, sm, tid);
      transposer_o<TB, R, O3, O2>(b, sm, tid);
    }
    if constexpr (NR > 2) {
      mix_regs_sel<R, kS2>(a, muB, mm2);
      mix_regs_sel<R, kS2>(b, -muB, mm2);
      transposer_o<TB, R, O2, O1>(a, sm, tid);
      transposer_o<TB, R, O2, O1>(b, sm, tid);
    }
    if constexpr (NR > 1) {
      mix_regs_sel<R, kS1>(a, muB, mm1);
      mix_regs_sel<R, kS1>(b, -muB, mm1);
      transposer_o<TB, R, O1, O0>(a, sm, tid);
      transposer_o<TB, R, O1, O0>(b, sm, tid);
    }
    mix_regs_sel<R, kS0>(a, muB, mm0);
    mix_regs_sel<R, kS0>(b, -muB, mm0);
    if (pd.mirrorB) mirror_all<TB, R, O0>(a, b, muB, zbase, tid, m);
  }
  if (pd.expect) {
    float acc = 0.f;
    int S = A, T = D;
#pragma unroll
    for (int i = 0; i < KQ; ++i) {
      const int k = gray(i);
      if (i > 0) {
        const int bt = gray_bit(i);
        S = ((k >> bt) & 1) ? S + kap[bt] : S - kap[bt];
        T = ((k >> bt) & 1) ? T + dk[bt] : T - dk[bt];
      }
      acc = fmaf(fmaf(a[k].x, a[k].x, a[k].y * a[k].y), (float)(S + qk[k]), acc);
      acc = fmaf(fmaf(b[k].x, b[k].x, b[k].y * b[k].y), (float)(S + qk[k] + T), acc);
    }
    acc_cta += acc;
  }
  if (pd.store) {
    if (pd.layerB < 0) {
      if constexpr (NR > 1) {
        transposer_o<TB, R, OC, O0>(a, sm, tid);
        transposer_o<TB, R, OC, O0>(b, sm, tid);
      }
    }
    if (pd.last) {  // back from the gauge, times lambda_p
      const int r = __popc(zbase | lt);
      const float2 fa = rot_i(Ip->final_scale, -r), fb = rot_i(Ip->final_scale, r - m);
#pragma unroll
      for (int k = 0; k < KQ; ++k) {
        a[k] = cmul(a[k], rot_i(fa, -popc_c(k)));
        b[k] = cmul(b[k], rot_i(fb, popc_c(k)));
      }
    }
#pragma unroll
    for (int k = 0; k < KQ; ++k) {
      base[k << O0] = a[k];
      mbase[-(int32_t)(k << O0)] = b[k];
    }
  }
  }  // pairs of this CTA
  if (pd.expect) {
    const double sum = block_sum((double)acc_cta, red, tid, NT);
    if (tid == 0) {  // the sum in the slot of the CTA's first tile, 0 in every other slot it covers
      for (uint32_t tt = 0; tt < ntiles; ++tt) {
        const uint32_t tile = tj | (tt << per);
        partials[Ip->part_off + tile] = tt == 0 ? sum : 0.0;
        partials[Ip->part_off + (tile ^ tmask)] = 0.0;
      }
    }
  }
}

bool layer_mirror_supported(int kind) {
  return kind >= 0 && kind < kTileKinds && kTileShapes[kind].r == 4 && kTileShapes[kind].tb <= 13;
}

template <int TB, int R>
static cudaError_t launch_mirror_t(int n, int nq, const PassDesc& pd, const InstDev* inst, const int32_t* list,
                                   int32_t nlist, const SubDev* subs, const uint32_t* planes, const float2* tables,
                                   float2* states, double* partials, int32_t tabcap, int32_t* consts, cudaStream_t st) {
  constexpr int kFull = full_rounds(TB, R);
  const size_t padded = (size_t(1) << TB) + (size_t(1) << (TB - R));
  const size_t smem = (size_t)tabcap * sizeof(float2) + padded * sizeof(float2) + 32 * 4 + sizeof(MirrorConst) +
                      PARAQAOA_MAX_QUBITS * kMaxPlanes * 4 + 32 * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_layer_mirror<TB, R, kFull>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int tiles_log2 = nq - TB;
  const int tpc = pd.tpc_log2;
  // the low group, contiguous, of a halved state of nq = n - 1 qubits, in pairs of tiles
  if (nq != n - 1 || pd.c != TB || pd.s != TB || pd.split || tiles_log2 < 1 || tpc < 0 || tpc > tiles_log2 - 1 ||
      tpc > kMaxTpcLog2)
    return cudaErrorInvalidValue;
  const int64_t blocks = (int64_t)nlist << (tiles_log2 - 1 - tpc);
  if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
  uint32_t mm[4] = {0, 0, 0, 0};
  for (int k = 0; k < kFull; ++k)
    for (int j = 0; j < R; ++j)
      if (((round_slots(TB, R, false, k) >> j) & 1u) && lay_off(TB, R, false, k) + j >= pd.mix_lo) mm[k] |= 1u << j;
  k_layer_mirror<TB, R, kFull><<<(unsigned)blocks, 1 << (TB - R), smem, st>>>(
      pd, n, tiles_log2, inst, list, subs, planes, tables, states, partials, tabcap, consts, mm[0], mm[1], mm[2],
      mm[3]);
  return cudaGetLastError();
}

static cudaError_t launch_mirror(int kind, int n, int nq, const PassDesc& pd, const InstDev* inst, const int32_t* list,
                                 int32_t nlist, const SubDev* subs, const uint32_t* planes, const float2* tables,
                                 float2* states, double* partials, int32_t tabcap, int32_t* consts, cudaStream_t st) {
  if (!layer_mirror_supported(kind)) return cudaErrorInvalidValue;
  if (kTileShapes[kind].tb == 12)
    return launch_mirror_t<12, 4>(n, nq, pd, inst, list, nlist, subs, planes, tables, states, partials, tabcap,
                                  consts, st);
  return launch_mirror_t<13, 4>(n, nq, pd, inst, list, nlist, subs, planes, tables, states, partials, tabcap, consts,
                                st);
}

// ------------------------------------------------------------ persistent form
// Every pass of every size class of one tile shape in one launch. Work items
// are ordered pass by pass (all classes' first passes, then their second
// passes, ...), instance by instance within a pass; a CTA takes the next item
// from a global counter, waits until every item of its instance's previous
// pass is done, runs the tile group and counts it done. An item only ever
// waits for items taken before it, and those belong to CTAs that are
// running, so the queue always progresses; every wait is bounded all the
// same (the global nanosecond timer), and one that gives up raises the
// error flag and lets the item through, so the launch ends.
__device__ __forceinline__ uint64_t pq_global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <int TB, int R>
__global__ void __launch_bounds__(1 << (TB - R), layer_min_blocks(TB, R))
    k_layer_persist(const PersistSeg* __restrict__ segs, int32_t nseg, int64_t items, uint64_t* ctrl,
                    uint32_t* done, const InstDev* __restrict__ inst_all, const int32_t* __restrict__ lists,
                    const SubDev* __restrict__ subs, const uint32_t* __restrict__ planes_all,
                    const float2* __restrict__ tables, float2* __restrict__ states, double* __restrict__ partials,
                    int32_t tabcap, const int32_t* __restrict__ consts, uint64_t wait_ns) {
  constexpr int kFull = full_rounds(TB, R);
  __shared__ int64_t s_item;
  __shared__ int32_t s_seg;
  const uint32_t tid = threadIdx.x;
  for (;;) {
    if (tid == 0) {
      const int64_t it = (int64_t)atomicAdd(reinterpret_cast<unsigned long long*>(ctrl), 1ull);
      int sg = 0;
      if (it < items) {
        while (sg + 1 < nseg && segs[sg + 1].item0 <= it) ++sg;
        const PersistSeg& S = segs[sg];
        if (S.prev >= 0 && S.prev < nseg) {  // this instance's previous pass, all of its tile groups
          const PersistSeg& Pv = segs[S.prev];
          const uint32_t* ctr = done + Pv.done_off + ((it - S.item0) >> S.per);
          const uint32_t need = 1u << Pv.per;
          const uint64_t t0 = pq_global_ns();
          while (ld_acquire_gpu(ctr) < need) {
            if (pq_global_ns() - t0 >= wait_ns) {
              atomicExch(reinterpret_cast<unsigned long long*>(ctrl) + 1, 1ull);
              break;
            }
            __nanosleep(128);
          }
        }
      }
      s_item = it;
      s_seg = sg;
    }
    __syncthreads();
    const int64_t it = s_item;
    if (it >= items) break;
    const PersistSeg& S = segs[s_seg];
    const PassDesc pd = S.pd;
    const uint32_t bid = (uint32_t)(it - S.item0);
    const int32_t* cc = consts + S.cc_off;
    const int32_t* lst = lists + S.list_off;
    const int tl = S.n - TB;
#define PQ_TILES(NRV, SPV, CTV)                                                                                  \
  layer_tiles<TB, R, NRV, SPV, CTV, true>(pd, S.n, tl, bid, inst_all, lst, subs, planes_all, tables, states, \
                                          partials, tabcap, cc, S.mm[0], S.mm[1], S.mm[2], S.mm[3])
    if (pd.split) PQ_TILES(2, true, true);
    else if (pd.c == TB && pd.s == TB) PQ_TILES(kFull, false, true);
    else if (S.nr == 1) PQ_TILES(1, false, false);
    else if (S.nr == 2) PQ_TILES(2, false, false);
    else PQ_TILES(3, false, false);
#undef PQ_TILES
    // the tile group's stores, then its completion count (release)
    __threadfence();
    __syncthreads();
    if (tid == 0) atomicAdd(done + S.done_off + (bid >> S.per), 1u);
  }
}

template <int TB, int R>
static cudaError_t launch_persist_t(int kind, const PersistSeg* segs, int32_t nseg, int64_t items, uint64_t* ctrl,
                                    uint32_t* done, const InstDev* inst, const int32_t* lists, const SubDev* subs,
                                    const uint32_t* planes, const float2* tables, float2* states, double* partials,
                                    int32_t tabcap, const int32_t* consts, uint64_t wait_ns, int num_sms,
                                    cudaStream_t st) {
  const size_t smem = layer_pass_smem(kind, tabcap);
  cudaError_t e = cudaFuncSetAttribute(k_layer_persist<TB, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_layer_persist<TB, R>, 1 << (TB - R), smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int64_t grid = std::min<int64_t>(items, (int64_t)per_sm * std::max(num_sms, 1));
  k_layer_persist<TB, R><<<(unsigned)grid, 1 << (TB - R), smem, st>>>(segs, nseg, items, ctrl, done, inst, lists, subs,
                                                                    planes, tables, states, partials, tabcap, consts,
                                                                    wait_ns);
  return cudaGetLastError();
}

cudaError_t launch_layer_persist(int kind, const PersistSeg* segs, int32_t nseg, int64_t items, uint64_t* ctrl,
                                 uint32_t* done, const InstDev* inst, const int32_t* lists, const SubDev* subs,
                                 const uint32_t* planes, const float2* tables, float2* states, double* partials,
                                 int32_t tabcap, const int32_t* consts, uint64_t wait_ns, int num_sms,
                                 cudaStream_t st) {
  if (items <= 0) return cudaSuccess;
  if (kind < 0 || kind >= kTileKinds || nseg < 1) return cudaErrorInvalidValue;
#define PQ_PERSIST(TBV, RV)                                                                                         \
  if (kTileShapes[kind].tb == TBV && kTileShapes[kind].r == RV)                                                     \
    return launch_persist_t<TBV, RV>(kind, segs, nseg, items, ctrl, done, inst, lists, subs, planes, tables, states, \
                                     partials, tabcap, consts, wait_ns, num_sms, st);
  PQ_PERSIST(12, 5)
  PQ_PERSIST(12, 4)
  PQ_PERSIST(13, 5)
  PQ_PERSIST(13, 4)
  PQ_PERSIST(14, 4)
#undef PQ_PERSIST
  return cudaErrorInvalidValue;
}

}  // namespace pq
