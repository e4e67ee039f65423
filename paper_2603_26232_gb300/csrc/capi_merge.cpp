// C ABI: the merge of per-part candidates into a cut of the whole graph
// (Alg. 2, Sec. 3.4): exhaustive level-aware search or the beam reading.
#include "host_ctx.h"

using namespace pq;
using namespace pqh;

extern "C" {

int paraqaoa_merge(paraqaoa_ctx* c, const paraqaoa_csr* g, const paraqaoa_part* pt,
                   const uint32_t* cand, int32_t K, int32_t L, int64_t beam, uint8_t* out_side,
                   int64_t* out_cut) {
  if (!c || !pt || !cand || !out_side || !out_cut || K < 1 || K > PARAQAOA_MAX_TOPK || beam < 0)
    return PARAQAOA_E_INVAL;
  int rc = validate_csr(g);
  if (rc) return rc;
  if (g->n != pt->nv) return PARAQAOA_E_INVAL;
  const int32_t M = pt->M, nv = pt->nv;
  for (int32_t i = 0; i < M; ++i) {
    if (pt->size[i] > 32) return PARAQAOA_E_TOO_MANY_QUBITS;
    const uint32_t mask = pt->size[i] >= 32 ? 0xffffffffu : ((1u << pt->size[i]) - 1u);
    for (int32_t j = 0; j < K; ++j)
      if (cand[(int64_t)i * K + j] & ~mask) return PARAQAOA_E_INVAL;
  }
  int64_t total_w = 0;
  for (int64_t k = 0; k < g->nnz; ++k) total_w += g->w[k];
  total_w /= 2;
  PQ_CUDA(cudaSetDevice(c->device));
  rc = upload_part(c, pt, false);
  if (rc) return rc;
  // inter-partition edges bucketed by the level of their larger end
  std::vector<int32_t> lv = levels_of(pt);
  std::vector<int64_t> cnt(M + 1, 0);
  for (int32_t u = 0; u < nv; ++u)
    for (int64_t k = g->row_ptr[u]; k < g->row_ptr[u + 1]; ++k) {
      const int32_t v = g->col[k];
      if (u < v && u < pt->first[lv[v]]) cnt[lv[v] + 1]++;
    }
  for (int32_t i = 0; i < M; ++i) cnt[i + 1] += cnt[i];
  std::vector<int32_t> eu(cnt[M]), ev(cnt[M]), ew(cnt[M]);
  std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
  for (int32_t u = 0; u < nv; ++u)
    for (int64_t k = g->row_ptr[u]; k < g->row_ptr[u + 1]; ++k) {
      const int32_t v = g->col[k];
      if (u < v && u < pt->first[lv[v]]) {
        const int64_t at = fill[lv[v]]++;
        eu[at] = u;
        ev[at] = v - pt->first[lv[v]];
        ew[at] = g->w[k];
      }
    }
  const int64_t E = std::max<int64_t>(cnt[M], 1);
  PQ_CUDA(c->m_first.ensure(4 * M));
  PQ_CUDA(c->m_size.ensure(4 * M));
  PQ_CUDA(c->m_level.ensure(4 * (size_t)nv));
  PQ_CUDA(c->m_cand.ensure(4 * (size_t)M * K));
  PQ_CUDA(c->m_intra.ensure(8 * (size_t)M * K));
  PQ_CUDA(c->m_eoff.ensure(8 * (size_t)(M + 1)));
  PQ_CUDA(c->m_eu.ensure(4 * E));
  PQ_CUDA(c->m_ev.ensure(4 * E));
  PQ_CUDA(c->m_ew.ensure(4 * E));
  auto up = [&](DevBuf& b, const void* h, size_t n) {
    return n ? cudaMemcpyAsync(b.p, h, n, cudaMemcpyHostToDevice, c->stream) : cudaSuccess;
  };
  PQ_CUDA(up(c->m_first, pt->first.data(), 4 * M));
  PQ_CUDA(up(c->m_size, pt->size.data(), 4 * M));
  PQ_CUDA(up(c->m_level, lv.data(), 4 * (size_t)nv));
  PQ_CUDA(up(c->m_cand, cand, 4 * (size_t)M * K));
  PQ_CUDA(up(c->m_eoff, cnt.data(), 8 * (size_t)(M + 1)));
  PQ_CUDA(up(c->m_eu, eu.data(), 4 * cnt[M]));
  PQ_CUDA(up(c->m_ev, ev.data(), 4 * cnt[M]));
  PQ_CUDA(up(c->m_ew, ew.data(), 4 * cnt[M]));
  MergeDev md;
  md.M = M;
  md.K = K;
  md.nv = nv;
  md.words = (nv + 31) / 32;
  md.first = c->m_first.as<int32_t>();
  md.size = c->m_size.as<int32_t>();
  md.level_of = c->m_level.as<int32_t>();
  md.cand = c->m_cand.as<uint32_t>();
  md.intra = c->m_intra.as<int64_t>();
  md.eoff = c->m_eoff.as<int64_t>();
  md.eu = c->m_eu.as<int32_t>();
  md.ev = c->m_ev.as<int32_t>();
  md.ew = c->m_ew.as<int32_t>();
  std::vector<uint32_t> packed(md.words, 0u);
  {
    ProfScope ps(c, PARAQAOA_KCLASS_MERGE, 0);
    PQ_CUDA(launch_cand_intra(c->d_subs.as<SubDev>(), c->d_planes.as<uint32_t>(), md.cand, M, K,
                              c->m_intra.as<int64_t>(), c->stream));
  }
  if (beam == 0) {
    // exhaustive level-aware DFS (Alg. 2)
    const double space = std::pow((double)K, (double)M);
    if (space > 1099511627776.0 || M > kMaxExhaustiveLevels) return PARAQAOA_E_SEARCH_TOO_LARGE;
    if (total_w >= (int64_t(1) << 31)) return PARAQAOA_E_INVAL;
    if (L < 1) L = 1;
    if (L > M) L = M;
    int64_t nprefix = 1;
    for (int32_t i = 0; i < L; ++i) nprefix *= K;
    // The first best leaf in lexicographic order wins whatever the starting
    // level, so the walk may start deeper than L to give every SM work: at
    // least kMergeFillThreads starting paths when the tree has that many
    // (unless the context keeps exactly K^L, the paper's worker count).
    if (c->merge_fill)
      while (L < M && nprefix < kMergeFillThreads && nprefix * K <= (int64_t(1) << 30)) {
        ++L;
        nprefix *= K;
      }
    while (nprefix > (int64_t(1) << 30) && L > 1) {
      --L;
      nprefix /= K;
    }
    c->merge_levels_used = L;
    PQ_CUDA(c->m_key.ensure(8));
    PQ_CUDA(c->m_path.ensure(4 * (size_t)M));
    PQ_CUDA(cudaMemsetAsync(c->m_key.p, 0, 8, c->stream));
    unsigned long long key = 0;
    std::vector<int32_t> path(M);
    {
      ProfScope ps(c, PARAQAOA_KCLASS_MERGE, 0);
      PQ_CUDA(launch_merge_dfs(md, L, nprefix, c->m_key.as<unsigned long long>(), c->stream));
    }
    PQ_CUDA(cudaMemcpyAsync(&key, c->m_key.p, 8, cudaMemcpyDeviceToHost, c->stream));
    PQ_CUDA(cudaStreamSynchronize(c->stream));
    const int64_t winner = (int64_t)(0xffffffffu - (uint32_t)(key & 0xffffffffu));
    {
      ProfScope ps(c, PARAQAOA_KCLASS_MERGE, 0);
      PQ_CUDA(launch_merge_dfs_path(md, L, nprefix, winner, c->m_path.as<int32_t>(), c->stream));
    }
    PQ_CUDA(cudaMemcpyAsync(path.data(), c->m_path.p, 4 * (size_t)M, cudaMemcpyDeviceToHost, c->stream));
    PQ_CUDA(cudaStreamSynchronize(c->stream));
    // assignment of the winning path (orientation as in the kernels)
    std::vector<uint8_t> side(nv, 0);
    for (int32_t l = 0; l < M; ++l) {
      const int32_t f = pt->first[l], sz = pt->size[l];
      uint32_t b = cand[(int64_t)l * K + path[l]];
      if (l > 0 && (int)(b & 1u) != side[f]) b = ~b & (sz >= 32 ? 0xffffffffu : ((1u << sz) - 1u));
      for (int32_t v = 0; v < sz; ++v) side[f + v] = (uint8_t)((b >> v) & 1u);
    }
    const uint8_t flip = side[0];
    for (int32_t v = 0; v < nv; ++v) out_side[v] = side[v] ^ flip;
    *out_cut = (int64_t)(key >> 32);
    return PARAQAOA_OK;
  }
  // beam reading
  if ((int64_t)beam * K > kBeamSortCap) return PARAQAOA_E_INVAL;
  if (total_w >= (int64_t(1) << 38)) return PARAQAOA_E_INVAL;
  const int32_t B = (int32_t)beam;
  for (int q = 0; q < 2; ++q) {
    PQ_CUDA(c->m_sides[q].ensure(4 * (size_t)B * md.words));
    PQ_CUDA(c->m_score[q].ensure(8 * (size_t)B));
    PQ_CUDA(c->m_rank[q].ensure(4 * (size_t)B));
    PQ_CUDA(c->m_r2s[q].ensure(4 * (size_t)B));
  }
  PQ_CUDA(c->m_keys.ensure(8 * (size_t)B * K));
  PQ_CUDA(c->m_nb.ensure(4));
  PQ_CUDA(cudaMemsetAsync(c->m_sides[0].p, 0, 4 * (size_t)md.words, c->stream));
  PQ_CUDA(cudaMemsetAsync(c->m_score[0].p, 0, 8, c->stream));
  PQ_CUDA(cudaMemsetAsync(c->m_rank[0].p, 0, 4, c->stream));
  PQ_CUDA(cudaMemsetAsync(c->m_r2s[0].p, 0, 4, c->stream));
  int32_t nb = 1;
  int cur = 0;
  for (int32_t l = 0; l < M; ++l) {
    const int nx = cur ^ 1;
    {
      ProfScope ps(c, PARAQAOA_KCLASS_MERGE, 0, 2);
      PQ_CUDA(launch_beam_level(md, l, nb, B, c->m_keys.as<uint64_t>(), c->m_sides[cur].as<uint32_t>(),
                                c->m_score[cur].as<int64_t>(), c->m_rank[cur].as<int32_t>(),
                                c->m_r2s[cur].as<int32_t>(), c->m_sides[nx].as<uint32_t>(),
                                c->m_score[nx].as<int64_t>(), c->m_rank[nx].as<int32_t>(),
                                c->m_r2s[nx].as<int32_t>(), c->m_nb.as<int32_t>(), c->stream));
    }
    nb = (int32_t)std::min<int64_t>((int64_t)nb * K, B);
    cur = nx;
  }
  int64_t best = 0;
  PQ_CUDA(cudaMemcpyAsync(packed.data(), c->m_sides[cur].p, 4 * (size_t)md.words, cudaMemcpyDeviceToHost, c->stream));
  PQ_CUDA(cudaMemcpyAsync(&best, c->m_score[cur].p, 8, cudaMemcpyDeviceToHost, c->stream));
  PQ_CUDA(cudaStreamSynchronize(c->stream));
  const uint8_t flip = (uint8_t)(packed[0] & 1u);
  for (int32_t v = 0; v < nv; ++v) out_side[v] = (uint8_t)(((packed[v >> 5] >> (v & 31)) & 1u) ^ flip);
  *out_cut = best;
  return PARAQAOA_OK;
}

int paraqaoa_set_merge_fill(paraqaoa_ctx* c, int32_t enable, int32_t* levels_used) {
  if (!c) return PARAQAOA_E_INVAL;
  if (enable >= 0) c->merge_fill = enable != 0;
  if (levels_used) *levels_used = c->merge_levels_used;
  return PARAQAOA_OK;
}

}  // extern "C"
