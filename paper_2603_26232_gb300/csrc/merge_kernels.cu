// Level-Aware Parallel Merge (Sec. 3.4, Alg. 2) on the GPU.
//
// Parts are index ranges [first_l, first_l + size_l) with one shared vertex
// between neighbours; a path picks candidate j_l for every level l. Level 0
// uses its candidate as is; level l > 0 uses the candidate or its complement
// so that the shared vertex first_l keeps the side level l-1 gave it.
// Vertices are assigned in index order, so the edges that become fully
// assigned at level l are (a) the induced edges E_l, whose cut is the
// candidate's own intra cut (orientation-independent), and (b) the
// inter-partition edges (u, v), u < v, whose larger end v is new at level l.
// A path's score after level l is the cut of all edges assigned so far; at the
// last level it is CutVal on the whole graph (Sec. 3.4.1).
#include <cuda_runtime.h>

#include "pq_internal.h"

namespace pq {

// Intra cut of every candidate: intra[l*K + j] = C_l(cand[l*K + j]).
__global__ void k_cand_intra(const SubDev* __restrict__ subs, const uint32_t* __restrict__ planes,
                             const uint32_t* __restrict__ cand, int32_t M, int32_t K,
                             int64_t* __restrict__ intra) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)M * K) return;
  const SubDev S = subs[t / K];
  const uint32_t z = cand[t];
  const uint32_t* pl = planes + S.plane_off;
  int64_t c = 0;
  for (int u = 0; u < S.n; ++u) {
    uint32_t m = ((z >> u) & 1u) ? ~z : 0u;
    for (int b = 0; b < S.P; ++b) c += (int64_t)__popc(pl[u * S.P + b] & m) << b;
  }
  intra[t] = c;
}



// ------------------------------------------------------------- exhaustive
// Side of vertex u on the path whose per-level choices are (jj, flips).
__device__ __forceinline__ int side_on_path(const MergeDev& md, int u, const uint8_t* jj, uint64_t flips) {
  const int lv = md.level_of[u];
  const uint32_t b = md.cand[lv * md.K + jj[lv]];
  return (int)(((b >> (u - md.first[lv])) & 1u) ^ (uint32_t)((flips >> lv) & 1ull));
}

// Score added at level l by choice j, given the choices of levels < l.
__device__ __forceinline__ int64_t level_gain(const MergeDev& md, int l, int j, const uint8_t* jj,
                                              uint64_t flips, int& flip_out) {
  uint32_t b = md.cand[l * md.K + j];
  int flip = 0;
  if (l > 0) flip = ((int)(b & 1u)) != side_on_path(md, md.first[l], jj, flips);
  flip_out = flip;
  int64_t g = md.intra[l * md.K + j];
  for (int64_t e = md.eoff[l]; e < md.eoff[l + 1]; ++e) {
    int su = side_on_path(md, md.eu[e], jj, flips);
    int sv = (int)(((b >> md.ev[e]) & 1u) ^ (uint32_t)flip);
    if (su != sv) g += md.ew[e];
  }
  return g;
}


// Alg. 2: thread t walks the subtree under starting path t (the digits of t
// in base K over the first L levels, level 0 most significant) depth-first
// in lexicographic order, keeping its first best leaf; the grid keeps the
// maximum of (score << 32 | ~t) so ties go to the smallest starting path.
// With want_path, only thread `winner` runs and writes its best path.
__global__ void k_merge_dfs(MergeDev md, int32_t L, int64_t nprefix, unsigned long long* best_key,
                            int64_t winner, int32_t* best_path) {
  const int64_t t = (best_path ? winner : (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
  if (best_path && (blockIdx.x != 0 || threadIdx.x != 0)) return;
  if (t >= nprefix) return;
  uint8_t jj[kMaxExhaustiveLevels];
  uint8_t bestj[kMaxExhaustiveLevels];
  int64_t sc[kMaxExhaustiveLevels + 1];
  uint64_t flips = 0;
  const int M = md.M, K = md.K;
  int64_t rest = t, div = nprefix / K;
  sc[0] = 0;
  for (int l = 0; l < L; ++l) {
    int j = (int)(rest / div);
    rest %= div;
    div = div > 1 ? div / K : 1;
    int f;
    sc[l + 1] = sc[l] + level_gain(md, l, j, jj, flips, f);
    jj[l] = (uint8_t)j;
    flips = (flips & ~(1ull << l)) | ((uint64_t)f << l);
  }
  int64_t best = -1;
  if (L == M) {
    best = sc[M];
    for (int l = 0; l < M; ++l) bestj[l] = jj[l];
  } else {
    // iterative DFS over levels L..M-1; jj[l] == K means "exhausted"
    int l = L;
    jj[l] = 0;
    while (l >= L) {
      if (jj[l] >= K) {
        --l;
        if (l >= L) jj[l]++;
        continue;
      }
      int f;
      sc[l + 1] = sc[l] + level_gain(md, l, jj[l], jj, flips, f);
      flips = (flips & ~(1ull << l)) | ((uint64_t)f << l);
      if (l == M - 1) {
        if (sc[M] > best) {
          best = sc[M];
          for (int q = 0; q < M; ++q) bestj[q] = jj[q];
        }
        jj[l]++;
      } else {
        ++l;
        jj[l] = 0;
      }
    }
  }
  if (best_path) {
    for (int q = 0; q < M; ++q) best_path[q] = bestj[q];
    return;
  }
  const unsigned long long key = ((unsigned long long)best << 32) | (unsigned long long)(0xffffffffu - (uint32_t)t);
  atomicMax(best_key, key);
}

// ------------------------------------------------------------- beam
// Keys of the extensions of level l: (score << 24) | (0xffffff - (rank*K + j))
// where rank is the parent's position in lexicographic tuple order, so a
// larger key is a higher score, then the lexicographically smaller tuple.
__global__ void k_beam_score(MergeDev md, int32_t l, int32_t nb, const uint32_t* __restrict__ sides,
                             const int64_t* __restrict__ score, const int32_t* __restrict__ rank,
                             uint64_t* __restrict__ keys) {
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gw >= (int64_t)nb * md.K) return;
  const int a = (int)(gw / md.K), j = (int)(gw % md.K);
  const uint32_t* sa = sides + (int64_t)a * md.words;
  const uint32_t b = md.cand[l * md.K + j];
  int flip = 0;
  if (l > 0) {
    const int f = md.first[l];
    flip = (int)(b & 1u) != (int)((sa[f >> 5] >> (f & 31)) & 1u);
  }
  int64_t g = 0;
  for (int64_t e = md.eoff[l] + lane; e < md.eoff[l + 1]; e += 32) {
    const int u = md.eu[e];
    int su = (int)((sa[u >> 5] >> (u & 31)) & 1u);
    int sv = (int)(((b >> md.ev[e]) & 1u) ^ (uint32_t)flip);
    if (su != sv) g += md.ew[e];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) g += __shfl_down_sync(0xffffffffu, g, o);
  if (lane == 0) {
    const int64_t tot = score[a] + md.intra[l * md.K + j] + g;
    const uint64_t code = (uint64_t)rank[a] * md.K + j;
    keys[gw] = ((uint64_t)tot << 24) | (0xffffffull - code);
  }
}

// Bitonic sort of n (power of two) keys in shared memory, descending.
// Thread t handles indices t, t + blockDim.x, ... (blockDim.x a multiple of
// 32), so a compare-exchange at a stride below 32 pairs two indices of one
// 32-element chunk, handled by lanes of one warp: a stage at such a stride
// that follows another one needs only a warp barrier.
__device__ void block_sort_desc(uint64_t* k, int n) {
  int prev = n;  // stride of the previous stage (n: the fill before the sort)
  for (int size = 2; size <= n; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      if (stride < 32 && prev < 32) __syncwarp();
      else __syncthreads();
      prev = stride;
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        int p = i ^ stride;
        if (p > i) {
          bool desc = (i & size) == 0;
          uint64_t x = k[i], y = k[p];
          if ((x < y) == desc) {
            k[i] = y;
            k[p] = x;
          }
        }
      }
    }
  }
  __syncthreads();
}


// Keep the best `beam` extensions, give them lexicographic ranks, and build
// their assignments (bit-packed sides) in the next buffer.
__global__ void k_beam_select(MergeDev md, int32_t l, int32_t nb, int64_t beam,
                              const uint64_t* __restrict__ keys, const uint32_t* __restrict__ sides,
                              const int64_t* __restrict__ score, const int32_t* __restrict__ rank2slot,
                              uint32_t* __restrict__ nsides, int64_t* __restrict__ nscore,
                              int32_t* __restrict__ nrank, int32_t* __restrict__ nrank2slot,
                              int32_t* __restrict__ nb_out) {
  extern __shared__ __align__(16) uint64_t sk[];  // kBeamSortCap
  uint64_t* sc2 = sk + kBeamSortCap;               // kBeamSortCap
  const int E = nb * md.K;
  int n2 = 1;
  while (n2 < E) n2 <<= 1;
  for (int i = threadIdx.x; i < n2; i += blockDim.x) sk[i] = i < E ? keys[i] : 0ull;
  block_sort_desc(sk, n2);
  const int keep = (int)((int64_t)E < beam ? E : beam);
  // lexicographic ranks of the kept ones: sort their codes ascending
  int m2 = 1;
  while (m2 < keep) m2 <<= 1;
  for (int i = threadIdx.x; i < m2; i += blockDim.x) {
    // descending sort of (~code << 32 | slot) gives ascending code order
    if (i < keep) {
      uint64_t code = 0xffffffull - (sk[i] & 0xffffffull);
      sc2[i] = ((uint64_t)(0xffffffull - code) << 32) | (uint64_t)i;
    } else {
      sc2[i] = 0ull;
    }
  }
  block_sort_desc(sc2, m2);
  for (int r = threadIdx.x; r < keep; r += blockDim.x) {
    const int slot = (int)(sc2[r] & 0xffffffffu);
    nrank[slot] = r;
    nrank2slot[r] = slot;
  }
  const int f = md.first[l], sz = md.size[l];
  for (int t = threadIdx.x >> 5; t < keep; t += blockDim.x >> 5) {
    const uint64_t key = sk[t];
    const uint64_t code = 0xffffffull - (key & 0xffffffull);
    const int prank = (int)(code / md.K), j = (int)(code % md.K);
    const int a = rank2slot[prank];
    const uint32_t* sa = sides + (int64_t)a * md.words;
    uint32_t* sn = nsides + (int64_t)t * md.words;
    for (int w = threadIdx.x & 31; w < md.words; w += 32) sn[w] = sa[w];
    __syncwarp();
    if ((threadIdx.x & 31) == 0) {
      uint32_t b = md.cand[l * md.K + j];
      if (l > 0 && (int)(b & 1u) != (int)((sa[f >> 5] >> (f & 31)) & 1u))
        b = ~b & (sz >= 32 ? 0xffffffffu : ((1u << sz) - 1u));
      for (int v = (l > 0 ? 1 : 0); v < sz; ++v) {
        const int gv = f + v;
        const uint32_t bit = 1u << (gv & 31);
        if ((b >> v) & 1u) sn[gv >> 5] |= bit;
        else sn[gv >> 5] &= ~bit;
      }
      nscore[t] = (int64_t)(key >> 24);
    }
  }
  if (threadIdx.x == 0) *nb_out = keep;
}

cudaError_t launch_cand_intra(const SubDev* subs, const uint32_t* planes, const uint32_t* cand,
                              int32_t M, int32_t K, int64_t* intra, cudaStream_t st) {
  const int64_t n = (int64_t)M * K;
  k_cand_intra<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(subs, planes, cand, M, K, intra);
  return cudaGetLastError();
}

cudaError_t launch_merge_dfs(const MergeDev& md, int32_t L, int64_t nprefix,
                             unsigned long long* best_key, cudaStream_t st) {
  const int64_t blocks = (nprefix + 127) / 128;
  if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
  k_merge_dfs<<<(unsigned)blocks, 128, 0, st>>>(md, L, nprefix, best_key, -1, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_merge_dfs_path(const MergeDev& md, int32_t L, int64_t nprefix, int64_t winner,
                                  int32_t* path, cudaStream_t st) {
  k_merge_dfs<<<1, 1, 0, st>>>(md, L, nprefix, nullptr, winner, path);
  return cudaGetLastError();
}

cudaError_t launch_beam_level(const MergeDev& md, int32_t l, int32_t nb, int64_t beam,
                              uint64_t* keys, const uint32_t* sides, const int64_t* score,
                              const int32_t* rank, const int32_t* rank2slot, uint32_t* nsides,
                              int64_t* nscore, int32_t* nrank, int32_t* nrank2slot,
                              int32_t* nb_out, cudaStream_t st) {
  const int64_t warps = (int64_t)nb * md.K;
  k_beam_score<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(md, l, nb, sides, score, rank, keys);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = 2 * kBeamSortCap * sizeof(uint64_t);
  e = cudaFuncSetAttribute(k_beam_select, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_beam_select<<<1, 1024, smem, st>>>(md, l, nb, beam, keys, sides, score, rank2slot, nsides,
                                       nscore, nrank, nrank2slot, nb_out);
  return cudaGetLastError();
}

}  // namespace pq
