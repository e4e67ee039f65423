// C ABI: the split-precision tensor-core mixer variant (paraqaoa_simulate_tc).
#include "host_ctx.h"

using namespace pq;
using namespace pqh;

extern "C" {

int paraqaoa_simulate_tc(paraqaoa_ctx* c, const paraqaoa_part* pt, const int32_t* ids, int32_t count, int32_t p,
                         const double* gamma, const double* beta, uint32_t flags, int32_t precision,
                         int32_t block_qubits) {
  if (!c || !pt || !ids || !gamma || !beta || count < 1 || p < 1 || p > PARAQAOA_MAX_P) return PARAQAOA_E_INVAL;
  if ((precision != PARAQAOA_TC_BF16 && precision != PARAQAOA_TC_FP16) || block_qubits < 5 || block_qubits > 7)
    return PARAQAOA_E_INVAL;
  for (int32_t i = 0; i < count; ++i) {
    if (ids[i] < 0 || ids[i] >= pt->M) return PARAQAOA_E_INVAL;
    if (pt->size[ids[i]] < 12) return PARAQAOA_E_INVAL;
  }
  PQ_CUDA(cudaSetDevice(c->device));
  int rc = upload_part(c, pt, false);
  if (rc) return rc;
  const uint32_t fl = (flags & (PARAQAOA_SIM_EXPECT | PARAQAOA_SIM_KEEP_STATE)) | PARAQAOA_SIM_KEEP_STATE;
  rc = plan_build(c, pt, ids, count, p, fl | kPlanFullStates);
  if (rc) return rc;
  SimPlan& pl = c->plan;
  pl.flags = flags | PARAQAOA_SIM_EXPECT;  // <C> is always reduced; states kept only on request
  // instances grouped by qubit count; cut tables (uint16, 2^n each) per instance
  std::map<int, std::vector<int32_t>> by_n;
  for (int32_t i = 0; i < count; ++i) by_n[pl.inst[i].n].push_back(i);
  std::vector<int32_t> lists;
  std::vector<std::pair<int, std::pair<int32_t, int32_t>>> groups;
  // each size group gets its own cut-table and partial-sum region, so that
  // the groups can run concurrently on side streams
  int64_t cut_elems = 0, part_elems = 0;
  std::vector<int64_t> cut_off, part_off;
  for (auto& kv : by_n) {
    groups.push_back({kv.first, {(int32_t)lists.size(), (int32_t)kv.second.size()}});
    lists.insert(lists.end(), kv.second.begin(), kv.second.end());
    cut_off.push_back(cut_elems);
    part_off.push_back(part_elems);
    cut_elems += (int64_t)kv.second.size() << kv.first;
    part_elems += (int64_t)kv.second.size() * tc_finish_blocks(kv.first);
  }
  const double extra = (double)cut_elems * 2 + (double)part_elems * 8;
  const double need = (double)pl.state_elems * 8 + (double)pl.table_elems * 8 + extra;
  if (need > (double)c->budget) return PARAQAOA_E_ADMISSION;
  PQ_CUDA(c->d_consts.ensure(std::max<size_t>(sizeof(int32_t) * lists.size(), 4)));
  PQ_CUDA(c->d_topk_scratch.ensure((size_t)cut_elems * 2 + 256));
  PQ_CUDA(c->d_partials.ensure(sizeof(double) * std::max<int64_t>(part_elems, 1)));
  PQ_CUDA(c->d_tc_err.ensure(sizeof(int)));
  int32_t* dl = c->d_consts.as<int32_t>();
  uint16_t* cuts = reinterpret_cast<uint16_t*>(c->d_topk_scratch.p);
  int* err = c->d_tc_err.as<int>();
  PQ_CUDA(cudaMemcpyAsync(dl, lists.data(), sizeof(int32_t) * lists.size(), cudaMemcpyHostToDevice, c->stream));
  PQ_CUDA(cudaMemsetAsync(err, 0, sizeof(int), c->stream));
  PQ_CUDA(cudaMemcpyAsync(c->d_gamma.p, gamma, sizeof(double) * count * p, cudaMemcpyHostToDevice, c->stream));
  PQ_CUDA(cudaMemcpyAsync(c->d_beta.p, beta, sizeof(double) * count * p, cudaMemcpyHostToDevice, c->stream));
  InstDev* inst = c->d_inst.as<InstDev>();
  {
    ProfScope ps(c, PARAQAOA_KCLASS_OTHER, 0);
    PQ_CUDA(launch_prep_layers(inst, count, p, c->d_gamma.as<double>(), c->d_beta.as<double>(),
                               c->d_tables.as<float2>(), inst, c->stream));
  }
  const bool fp16 = precision == PARAQAOA_TC_FP16;
  float2* states = c->d_states.as<float2>();
  // size groups on side streams (as in plan_run) unless per-kernel profiling is on
  const bool fork = !c->prof && groups.size() > 1;
  if (fork) {
    PQ_CUDA(ensure_side_streams(c));
    PQ_CUDA(cudaEventRecord(c->fork_ev, c->stream));
    for (int k = 0; k < kSideStreams; ++k) PQ_CUDA(cudaStreamWaitEvent(c->side[k], c->fork_ev, 0));
  }
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    const auto& gr = groups[gi];
    cudaStream_t st = fork ? c->side[gi % kSideStreams] : c->stream;
    const int n = gr.first;
    const int32_t off = gr.second.first, cnt = gr.second.second;
    const int64_t stride = int64_t(1) << n;
    uint16_t* gcuts = cuts + cut_off[gi];
    double* gparts = c->d_partials.as<double>() + part_off[gi];
    for (int32_t j = 0; j < cnt; ++j) {
      ProfScope ps(c, PARAQAOA_KCLASS_OTHER, (double)stride * 2);
      PQ_CUDA(launch_cut_table(c->d_subs.as<SubDev>() + pl.inst[lists[off + j]].sub, n, c->d_planes.as<uint32_t>(),
                               gcuts + (int64_t)j * stride, st));
    }
    // ceil(n / block_qubits) blocks of as even sizes as possible; fewer blocks
    // (sizes up to 7) when that would leave blocks under 5 qubits. Every block
    // has 5..7 qubits and at most n - 6, so that a tile holds 64 groups.
    int nb = (n + block_qubits - 1) / block_qubits;
    if (n / nb < 5) nb = n / 5;
    std::vector<int> bs(nb, n / nb);
    for (int b = 0; b < n % nb; ++b) ++bs[b];
    for (int b : bs)
      if (b < 5 || b > n - 6) return PARAQAOA_E_INVAL;
    for (int l = 0; l < p; ++l) {
      {
        ProfScope ps(c, PARAQAOA_KCLASS_OTHER, (double)cnt * stride * (l == 0 ? 10.0 : 18.0));
        PQ_CUDA(launch_tc_phase(inst, dl + off, cnt, n, l, l == 0, c->d_tables.as<float2>(), gcuts, stride, states,
                                st));
      }
      int q0 = 0;
      for (int b : bs) {
        ProfScope ps(c, PARAQAOA_KCLASS_TC_MIXER, (double)cnt * stride * 16.0);
        PQ_CUDA(launch_mixer_tc(b, fp16, inst, dl + off, cnt, n, q0, l, states, c->wait_ns, err, c->num_sms, st));
        q0 += b;
      }
    }
    ProfScope ps(c, PARAQAOA_KCLASS_OTHER, (double)cnt * stride * (flags & PARAQAOA_SIM_KEEP_STATE ? 18.0 : 10.0));
    PQ_CUDA(launch_tc_finish(inst, dl + off, cnt, n, gcuts, stride, states, gparts,
                             (flags & PARAQAOA_SIM_KEEP_STATE) ? 1 : 0, c->d_expect.as<double>(), st));
  }
  if (fork)
    for (int k = 0; k < kSideStreams; ++k) {
      PQ_CUDA(cudaEventRecord(c->join_ev[k], c->side[k]));
      PQ_CUDA(cudaStreamWaitEvent(c->stream, c->join_ev[k], 0));
    }
  int herr = 0;
  PQ_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  PQ_CUDA(cudaStreamSynchronize(c->stream));
  if (herr) {
    pl.valid = false;
    return PARAQAOA_E_TIMEOUT;
  }
  if (!(flags & PARAQAOA_SIM_KEEP_STATE)) pl.flags &= ~PARAQAOA_SIM_KEEP_STATE;
  return PARAQAOA_OK;
}

int paraqaoa_set_wait_limit(paraqaoa_ctx* c, int64_t ns) {
  if (!c || ns < 0 || ns > 10000000000ll) return PARAQAOA_E_INVAL;
  c->wait_ns = (uint64_t)ns;
  return PARAQAOA_OK;
}

}  // extern "C"
