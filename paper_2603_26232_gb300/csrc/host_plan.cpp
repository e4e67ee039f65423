// The batch plan behind every simulate, search and autotune entry point:
// admission and instance layout (plan_build), the launches of one run
// (plan_run: phase tables, cut constants, layer passes, <C> reductions, size
// classes on side streams), partition upload, the profiler's event
// bookkeeping, and the pass schedule of a state (make_schedule).
#include "host_ctx.h"

using namespace pq;
using namespace pqh;

namespace pqh {

std::atomic<uint64_t> g_part_serial{1};

cudaEvent_t get_event(paraqaoa_ctx* c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void prof_flush(paraqaoa_ctx* c) {
  if (c->pending.empty()) return;
  cudaStreamSynchronize(c->stream);
  for (auto& r : c->pending) {
    float t = 0.f;
    cudaEventElapsedTime(&t, r.a, r.b);
    c->ms[r.cls] += t;
    c->pool.push_back(r.a);
    c->pool.push_back(r.b);
  }
  c->pending.clear();
}

int validate_csr(const paraqaoa_csr* g) {
  if (!g || g->n < 1 || g->nnz < 0 || !g->row_ptr || (g->nnz > 0 && (!g->col || !g->w)))
    return PARAQAOA_E_INVAL;
  if (g->row_ptr[0] != 0 || g->row_ptr[g->n] != g->nnz) return PARAQAOA_E_INVAL;
  int64_t up = 0, down = 0, wbal = 0;
  for (int32_t u = 0; u < g->n; ++u) {
    if (g->row_ptr[u + 1] < g->row_ptr[u]) return PARAQAOA_E_INVAL;
    for (int64_t k = g->row_ptr[u]; k < g->row_ptr[u + 1]; ++k) {
      const int32_t v = g->col[k];
      if (v < 0 || v >= g->n || v == u || g->w[k] <= 0) return PARAQAOA_E_INVAL;
      if (u < v) {
        ++up;
        wbal += g->w[k];
      } else {
        ++down;
        wbal -= g->w[k];
      }
    }
  }
  if (up != down || wbal != 0) return PARAQAOA_E_INVAL;  // not symmetric
  return PARAQAOA_OK;
}

// Level (part index) at which each vertex is first assigned.
std::vector<int32_t> levels_of(const paraqaoa_part* pt) {
  std::vector<int32_t> lv(pt->nv, 0);
  for (int32_t i = 0; i < pt->M; ++i)
    for (int32_t v = (i == 0 ? 0 : 1); v < pt->size[i]; ++v) lv[pt->first[i] + v] = i;
  return lv;
}

int upload_part(paraqaoa_ctx* c, const paraqaoa_part* pt, bool force) {
  if (!force && c->part_serial == pt->serial) return PARAQAOA_OK;
  std::vector<SubDev> subs(pt->M);
  for (int32_t i = 0; i < pt->M; ++i) {
    subs[i].n = pt->size[i];
    subs[i].P = pt->P[i];
    subs[i].W = (int32_t)std::min<int64_t>(pt->weight[i], 0x7fffffff);
    subs[i].first = pt->first[i];
    subs[i].plane_off = pt->plane_off[i];
  }
  PQ_CUDA(c->d_subs.ensure(sizeof(SubDev) * std::max<size_t>(subs.size(), 1)));
  PQ_CUDA(c->d_planes.ensure(sizeof(uint32_t) * std::max<size_t>(pt->planes.size(), 1)));
  PQ_CUDA(cudaMemcpyAsync(c->d_subs.p, subs.data(), sizeof(SubDev) * subs.size(),
                          cudaMemcpyHostToDevice, c->stream));
  if (!pt->planes.empty())
    PQ_CUDA(cudaMemcpyAsync(c->d_planes.p, pt->planes.data(), sizeof(uint32_t) * pt->planes.size(),
                            cudaMemcpyHostToDevice, c->stream));
  PQ_CUDA(cudaStreamSynchronize(c->stream));  // host vectors are temporaries
  c->part_serial = pt->serial;
  return PARAQAOA_OK;
}

cudaError_t ensure_side_streams(paraqaoa_ctx* c) {
  if (c->fork_ev) return cudaSuccess;
  for (int k = 0; k < kSideStreams; ++k) {
    cudaError_t e = cudaStreamCreateWithFlags(&c->side[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->join_ev[k], cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
  }
  return cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming);
}

// Tile shape of size class n: the context's choice, except that a halved
// class uses the choice for its n - 1 stored qubits when that shape has a
// halved low-group pass and leaves at least two tiles, else 2^12 x 16.
// Tiles per CTA of a size class's passes (both launch forms, so that their
// <C> sums group alike): the context's choice for the stored qubit count,
// capped by the tiles a pass has (a halved class's low-group passes walk
// tile pairs: one tile bit fewer), and lowered while a launch of `ninst`
// instances would fill fewer than four waves of the shape's resident CTAs on
// every SM: the idle slots of a short grid's last wave cost more than the
// set-up the extra CTAs repeat (an 84-instance Adam batch of 2^20 states on
// the 2^13 tile walking 16 tiles is 672 CTAs, 2.2 waves of 304).
static int class_tpc(const paraqaoa_ctx* c, int kind, int tb, int nq, bool halved, int64_t ninst) {
  const int tiles_log2 = halved ? nq - tb - 1 : nq - tb;
  int tpc = std::min<int>(c->tpc_log2[nq], tiles_log2);
  const int64_t slots = (int64_t)c->num_sms * kTileResidentCtas[kind];
  while (tpc > 0 && (ninst << (tiles_log2 - tpc)) < 4 * slots) --tpc;
  return tpc;
}

int class_kind(const paraqaoa_ctx* c, int n, bool halved) {
  if (!halved) return c->tile_kind[n];
  const int k = c->tile_kind[n - 1];
  if (layer_mirror_supported(k) && n - 1 - kTileShapes[k].tb >= 1) return k;
  return 1;
}

// Build the plan of a batch (validation, admission, memory layout).
int plan_build(paraqaoa_ctx* c, const paraqaoa_part* pt, const int32_t* ids, int32_t count,
               int32_t p, uint32_t flags) {
  SimPlan& pl = c->plan;
  pl = SimPlan();
  if (count < 1 || p < 1 || p > PARAQAOA_MAX_P || !ids) return PARAQAOA_E_INVAL;
  pl.count = count;
  pl.p = p;
  pl.flags = flags;
  pl.inst.resize(count);
  const bool keep = flags & PARAQAOA_SIM_KEEP_STATE;
  const bool halve = (flags & PARAQAOA_SIM_HALVED) || (c->halved && !(flags & kPlanFullStates));
  std::vector<int32_t> tiny;
  std::map<int, std::vector<int32_t>> smem, hbm;
  for (int32_t i = 0; i < count; ++i) {
    const int32_t s = ids[i];
    if (s < 0 || s >= pt->M) return PARAQAOA_E_INVAL;
    const int n = pt->size[s];
    if (n > PARAQAOA_MAX_QUBITS) return PARAQAOA_E_TOO_MANY_QUBITS;
    if (pt->weight[s] > PARAQAOA_MAX_SUBGRAPH_WEIGHT) return PARAQAOA_E_INVAL;
    InstDev& I = pl.inst[i];
    std::memset(&I, 0, sizeof(I));
    I.sub = s;
    I.n = n;
    I.P = pt->P[s];
    I.W = (int32_t)pt->weight[s];
    I.table_off = pl.table_elems;
    pl.tabcap = std::max(pl.tabcap, I.W + 1);
    pl.table_elems += (int64_t)p * (I.W + 1);
    I.state_off = -1;
    I.part_off = -1;
    const bool big = n > kSmemMaxQubits;
    // halved: streaming parts of >= 16 qubits keep z < 2^(n-1) only
    I.halved = (halve && n > kSmemMaxQubits + 1) ? 1 : 0;
    const int nq = n - I.halved;
    if (big || keep) {
      I.state_off = pl.state_elems;
      pl.state_elems += int64_t(1) << nq;
    }
    if (big) {
      I.part_off = pl.partial_elems;
      pl.partial_elems += int64_t(1) << (nq - kTileShapes[class_kind(c, n, I.halved)].tb);
      hbm[n].push_back(i);
    } else if (n >= 10) {
      smem[n].push_back(i);
    } else {
      tiny.push_back(i);
    }
  }
  pl.tabcap = (pl.tabcap + 15) & ~15;
  auto add = [&](std::vector<int32_t>& v) {
    std::pair<int32_t, int32_t> r((int32_t)pl.lists.size(), (int32_t)v.size());
    pl.lists.insert(pl.lists.end(), v.begin(), v.end());
    return r;
  };
  auto t = add(tiny);
  pl.tiny = t;
  for (auto& kv : smem) pl.smem[kv.first] = add(kv.second);
  for (auto& kv : hbm) pl.hbm[kv.first] = add(kv.second);
  for (auto& kv : hbm) {
    std::map<int32_t, int32_t> slot;  // part -> slot, in order of first appearance
    std::vector<int32_t> reps;
    for (int32_t i : kv.second) {
      auto it = slot.find(pl.inst[i].sub);
      if (it == slot.end()) {
        it = slot.emplace(pl.inst[i].sub, (int32_t)reps.size()).first;
        reps.push_back(i);
      }
      pl.inst[i].cc_slot = it->second;
    }
    pl.hbm_reps[kv.first] = add(reps);
  }
  // admission: every byte this batch puts on the device
  const double need = (double)pl.state_elems * 8 + (double)pl.table_elems * 8 +
                      (double)pl.partial_elems * 8 + (double)count * (sizeof(InstDev) + 8 + 16 * p) +
                      (double)pl.lists.size() * 4;
  if (need > (double)c->budget) return PARAQAOA_E_ADMISSION;
  PQ_CUDA(c->d_inst.ensure(sizeof(InstDev) * count));
  PQ_CUDA(c->d_lists.ensure(sizeof(int32_t) * std::max<size_t>(pl.lists.size(), 1)));
  PQ_CUDA(c->d_gamma.ensure(sizeof(double) * count * p));
  PQ_CUDA(c->d_beta.ensure(sizeof(double) * count * p));
  PQ_CUDA(c->d_tables.ensure(sizeof(float2) * std::max<int64_t>(pl.table_elems, 1)));
  PQ_CUDA(c->d_states.ensure(sizeof(float2) * std::max<int64_t>(pl.state_elems, 1)));
  PQ_CUDA(c->d_partials.ensure(sizeof(double) * std::max<int64_t>(pl.partial_elems, 1)));
  PQ_CUDA(c->d_expect.ensure(sizeof(double) * count));
  PQ_CUDA(cudaMemcpyAsync(c->d_inst.p, pl.inst.data(), sizeof(InstDev) * count,
                          cudaMemcpyHostToDevice, c->stream));
  PQ_CUDA(cudaMemcpyAsync(c->d_lists.p, pl.lists.data(), sizeof(int32_t) * pl.lists.size(),
                          cudaMemcpyHostToDevice, c->stream));
  PQ_CUDA(cudaStreamSynchronize(c->stream));  // pl vectors may change before the copy ran
  pl.valid = true;
  return PARAQAOA_OK;
}

// Enqueue the whole simulation of the current plan; angles in c->d_gamma/d_beta.
int plan_run(paraqaoa_ctx* c) {
  SimPlan& pl = c->plan;
  const int32_t p = pl.p;
  const bool keep = pl.flags & PARAQAOA_SIM_KEEP_STATE;
  const bool want = pl.flags & PARAQAOA_SIM_EXPECT;
  InstDev* inst = c->d_inst.as<InstDev>();
  const int32_t* lists = c->d_lists.as<int32_t>();
  const SubDev* subs = c->d_subs.as<SubDev>();
  const uint32_t* planes = c->d_planes.as<uint32_t>();
  float2* tables = c->d_tables.as<float2>();
  float2* states = c->d_states.as<float2>();
  double* partials = c->d_partials.as<double>();
  double* expect = c->d_expect.as<double>();
  {
    ProfScope ps(c, PARAQAOA_KCLASS_OTHER, 0);
    PQ_CUDA(launch_prep_layers(inst, pl.count, p, c->d_gamma.as<double>(), c->d_beta.as<double>(),
                               tables, inst, c->stream));
  }
  // Size classes are independent (disjoint instances, states, partials and
  // cut-constant regions): without per-kernel profiling they run on side
  // streams forked from and joined back to the context stream, so that small
  // classes fill the GPU next to large ones. Stream capture follows the fork.
  const int ncls = (pl.tiny.second > 0 ? 1 : 0) + (int)pl.smem.size() + (int)pl.hbm.size();
  const bool fork = !c->prof && ncls > 1;
  int used = 0;
  if (fork) {
    PQ_CUDA(ensure_side_streams(c));
    PQ_CUDA(cudaEventRecord(c->fork_ev, c->stream));
    for (int k = 0; k < kSideStreams; ++k) PQ_CUDA(cudaStreamWaitEvent(c->side[k], c->fork_ev, 0));
  }
  auto cls_stream = [&]() -> cudaStream_t {
    if (!fork) return c->stream;
    const int k = used++ % kSideStreams;
    return c->side[k];
  };
  // Cut constants: one array per size class and distinct cut layout of its
  // schedule (a layout is fixed by the pass's qubit group and round count),
  // computed by the first run of the plan and reused by the later ones (Adam
  // steps, replayed graphs, the autotuner's timed runs).
  struct ClassSched {
    int kind, tb, nq;  // nq: stored qubits (n - 1 for a halved class)
    bool halved;
    std::vector<PassDesc> sched;
    std::vector<int> set;  // per pass: index of its cut layout (-1: no cut)
    int nsets = 0;
    int64_t off = 0, elems = 0;
  };
  std::map<int, ClassSched> cs;
  int64_t cc_total = 0;
  for (auto& kv : pl.hbm) {
    const int n = kv.first;
    ClassSched& q = cs[n];
    q.halved = pl.inst[pl.lists[kv.second.first]].halved != 0;  // a class is halved or not as a whole
    q.nq = n - (q.halved ? 1 : 0);
    q.kind = class_kind(c, n, q.halved);
    q.tb = kTileShapes[q.kind].tb;
    if (q.halved) {
      // classic schedule of the n - 1 stored qubits; every pass over the
      // contiguous low group also applies the top qubit's mixer of each
      // layer it mixes (each layer mixes the low group exactly once)
      q.sched = make_schedule(q.nq, p, q.tb, c->c_min[q.nq], keep, want, 0);
      for (PassDesc& pd : q.sched)
        if (pd.c == q.tb && pd.s == q.tb) {
          pd.mirrorA = pd.layerA >= 0;
          pd.mirrorB = pd.layerB >= 0;
        }
    } else {
      q.sched = make_schedule(n, p, q.tb, c->c_min[n], keep, want, (c->split[n] & 1) ? kTileShapes[q.kind].r : 0,
                              (c->split[n] & 2) != 0);
    }
    std::vector<std::array<int, 4>> keys;
    for (const PassDesc& pd : q.sched) {
      int k = -1;
      if (pd.layerP >= 0 || pd.expect) {
        const std::array<int, 4> key{pd.c, pd.s, pd.split, pd.mix_lo};
        k = (int)(std::find(keys.begin(), keys.end(), key) - keys.begin());
        if (k == (int)keys.size()) keys.push_back(key);
      }
      q.set.push_back(k);
    }
    q.nsets = (int)keys.size();
    q.elems = cut_consts_elems(q.kind, pl.hbm_reps[n].second);
    q.off = cc_total;
    cc_total += q.nsets * q.elems;
  }
  if (!pl.cc_ready) PQ_CUDA(c->d_consts.ensure(sizeof(int32_t) * std::max<int64_t>(cc_total, 1)));
  // Persistent form: the size classes of one tile shape share one launch
  // over a work queue of (pass, instance, tile group) items, ordered pass by
  // pass across the classes. The queue (segment table) is built and uploaded
  // by the plan's first run, outside any stream capture; later runs (Adam
  // steps, replayed graphs) only zero the control blocks and launch.
  bool any_halved = false;
  for (auto& kv : cs) any_halved = any_halved || kv.second.halved;
  if (c->persistent && !any_halved && !pl.hbm.empty() && !pl.cc_ready) {
    pl.persist.clear();
    std::vector<PersistSeg> segs;
    std::map<int, std::vector<int>> by_kind;
    for (auto& kv : pl.hbm) by_kind[cs[kv.first].kind].push_back(kv.first);
    int64_t ctl = 0;
    for (auto& kk : by_kind) {
      SimPlan::PersistGroup grp;
      grp.kind = kk.first;
      grp.classes = kk.second;
      grp.seg0 = (int32_t)segs.size();
      grp.ctl_off = (int32_t)ctl;
      grp.bytes = 0.0;
      int64_t item = 0, done = 0;
      size_t maxp = 0;
      for (int n : kk.second) maxp = std::max(maxp, cs[n].sched.size());
      std::map<int, int32_t> last;  // class -> its previous pass's segment
      for (size_t j = 0; j < maxp; ++j)
        for (int n : kk.second) {
          const ClassSched& q = cs[n];
          if (j >= q.sched.size()) continue;
          const auto& lst = pl.hbm[n];
          PersistSeg sg;
          std::memset(&sg, 0, sizeof(sg));
          sg.pd = q.sched[j];
          sg.pd.tpc_log2 = class_tpc(c, q.kind, q.tb, q.nq, q.halved, lst.second);
          sg.n = n;
          sg.nr = layer_pass_rounds(q.kind, sg.pd);
          sg.list_off = lst.first;
          sg.nlist = lst.second;
          sg.per = (n - q.tb) - sg.pd.tpc_log2;
          sg.prev = j == 0 ? -1 : last[n] - grp.seg0;  // the kernel indexes its group's segments
          sg.done_off = (int32_t)done;
          sg.item0 = item;
          sg.cc_off = q.off + (int64_t)std::max(q.set[j], 0) * q.elems;
          layer_pass_masks(q.kind, sg.pd, sg.mm);
          last[n] = (int32_t)segs.size();
          segs.push_back(sg);
          item += (int64_t)lst.second << sg.per;
          done += lst.second;
          grp.bytes += (double)lst.second * (double)(int64_t(1) << n) *
                       ((sg.pd.init ? 0.0 : 8.0) + (sg.pd.store ? 8.0 : 0.0));
        }
      grp.nseg = (int32_t)segs.size() - grp.seg0;
      grp.items = item;
      ctl += 2 + (done + 1) / 2;  // head and error words, then 32-bit counters packed two per word
      pl.persist.push_back(grp);
    }
    pl.persist_ctl_words = ctl;
    if (!c->d_perr.p) {
      PQ_CUDA(c->d_perr.ensure(sizeof(uint64_t)));
      PQ_CUDA(cudaMemsetAsync(c->d_perr.p, 0, sizeof(uint64_t), c->stream));
    }
    PQ_CUDA(c->d_pseg.ensure(sizeof(PersistSeg) * segs.size()));
    PQ_CUDA(c->d_pctl.ensure(sizeof(uint64_t) * std::max<int64_t>(ctl, 1)));
    PQ_CUDA(cudaMemcpyAsync(c->d_pseg.p, segs.data(), sizeof(PersistSeg) * segs.size(), cudaMemcpyHostToDevice,
                            c->stream));
    PQ_CUDA(cudaStreamSynchronize(c->stream));  // segs is a temporary
    pl.persist_used = true;
  }
  if (pl.tiny.second > 0) {
    cudaStream_t st = cls_stream();
    ProfScope ps(c, PARAQAOA_KCLASS_SMEM_SIM, 0);
    PQ_CUDA(launch_tiny_sim(inst, lists + pl.tiny.first, pl.tiny.second, p, subs, planes, tables,
                            states, expect, keep, want, pl.tabcap, st));
  }
  for (auto& kv : pl.smem) {
    cudaStream_t st = cls_stream();
    ProfScope ps(c, PARAQAOA_KCLASS_SMEM_SIM, keep ? (double)kv.second.second * 8.0 * (1 << kv.first) : 0.0);
    PQ_CUDA(launch_smem_sim(kv.first, inst, lists + kv.second.first, kv.second.second, p, subs,
                            planes, tables, states, expect, keep, want, pl.tabcap, st));
  }
  if (pl.persist_used) {
    for (const auto& grp : pl.persist) {
      cudaStream_t st = cls_stream();
      uint64_t* ctl = c->d_pctl.as<uint64_t>() + grp.ctl_off;
      uint32_t* done = reinterpret_cast<uint32_t*>(ctl + 2);
      const size_t ctl_bytes = sizeof(uint64_t) * (size_t)(
          (&grp == &pl.persist.back() ? pl.persist_ctl_words : (&grp + 1)->ctl_off) - grp.ctl_off);
      PQ_CUDA(cudaMemsetAsync(ctl, 0, ctl_bytes, st));
      for (int n : grp.classes) {
        const ClassSched& q = cs[n];
        std::vector<char> done_cc(q.nsets, pl.cc_ready ? 1 : 0);
        const auto reps = pl.hbm_reps[n];
        for (size_t ip = 0; ip < q.sched.size(); ++ip) {
          const int k = q.set[ip];
          if (k < 0 || done_cc[k]) continue;
          PassDesc pd = q.sched[ip];
          int32_t* consts = c->d_consts.as<int32_t>() + q.off + (int64_t)k * q.elems;
          ProfScope ps(c, PARAQAOA_KCLASS_OTHER, 0);
          PQ_CUDA(launch_cut_consts(q.kind, n, pd, inst, lists + reps.first, reps.second, subs, planes, consts, st));
          done_cc[k] = 1;
        }
      }
      {
        ProfScope ps(c, PARAQAOA_KCLASS_LAYER_PASS, grp.bytes);
        PQ_CUDA(launch_layer_persist(grp.kind, c->d_pseg.as<PersistSeg>() + grp.seg0, grp.nseg, grp.items, ctl, done,
                                     inst, lists, subs, planes, tables, states, partials, pl.tabcap,
                                     c->d_consts.as<int32_t>(), c->wait_ns, c->num_sms, st));
      }
      {  // a wait that gave up in this run stays reported until the next clear
        ProfScope ps(c, PARAQAOA_KCLASS_OTHER, 0);
        PQ_CUDA(launch_flag_or(ctl + 1, c->d_perr.as<uint64_t>(), st));
      }
      if (want)
        for (int n : grp.classes) {
          ProfScope ps(c, PARAQAOA_KCLASS_OTHER, 0);
          const auto& lst = pl.hbm[n];
          PQ_CUDA(launch_expect_reduce(inst, lists + lst.first, lst.second, 1 << (n - cs[n].tb), partials, expect, st));
        }
    }
  }
  for (auto& kv : pl.hbm) {
    if (pl.persist_used) break;
    cudaStream_t st = cls_stream();
    const int n = kv.first;
    const ClassSched& q = cs[n];
    const int kind = q.kind, tb = q.tb;
    const double amps = (double)kv.second.second * (double)(int64_t(1) << q.nq);
    const auto reps = pl.hbm_reps[n];
    std::vector<char> done(q.nsets, pl.cc_ready ? 1 : 0);
    for (size_t ip = 0; ip < q.sched.size(); ++ip) {
      PassDesc pd = q.sched[ip];
      pd.tpc_log2 = class_tpc(c, kind, tb, q.nq, q.halved, kv.second.second);
      const int k = q.set[ip];
      int32_t* consts = c->d_consts.as<int32_t>() + q.off + (int64_t)std::max(k, 0) * q.elems;
      if (k >= 0 && !done[k]) {
        ProfScope ps(c, PARAQAOA_KCLASS_OTHER, 0);
        PQ_CUDA(launch_cut_consts(kind, n, pd, inst, lists + reps.first, reps.second, subs, planes, consts, st));
        done[k] = 1;
      }
      const double bytes = amps * ((pd.init ? 0.0 : 8.0) + (pd.store ? 8.0 : 0.0));
      ProfScope ps(c, PARAQAOA_KCLASS_LAYER_PASS, bytes);
      PQ_CUDA(launch_layer_pass(kind, n, q.nq, pd, inst, lists + kv.second.first, kv.second.second, subs,
                                planes, tables, states, partials, pl.tabcap, consts, st));
    }
    if (want) {
      ProfScope ps(c, PARAQAOA_KCLASS_OTHER, 0);
      PQ_CUDA(launch_expect_reduce(inst, lists + kv.second.first, kv.second.second,
                                   1 << (q.nq - tb), partials, expect, st));
    }
  }
  if (fork)
    for (int k = 0; k < kSideStreams; ++k) {
      PQ_CUDA(cudaEventRecord(c->join_ev[k], c->side[k]));
      PQ_CUDA(cudaStreamWaitEvent(c->stream, c->join_ev[k], 0));
    }
  pl.cc_ready = true;
  return PARAQAOA_OK;
}

int persist_clear(paraqaoa_ctx* c) {
  PQ_CUDA(c->d_perr.ensure(sizeof(uint64_t)));
  PQ_CUDA(cudaMemsetAsync(c->d_perr.p, 0, sizeof(uint64_t), c->stream));
  return PARAQAOA_OK;
}

int persist_status(paraqaoa_ctx* c) {
  if (!c->d_perr.p) return PARAQAOA_OK;
  uint64_t e = 0;
  PQ_CUDA(cudaMemcpyAsync(&e, c->d_perr.p, sizeof(e), cudaMemcpyDeviceToHost, c->stream));
  PQ_CUDA(cudaStreamSynchronize(c->stream));
  return e ? PARAQAOA_E_TIMEOUT : PARAQAOA_OK;
}

}  // namespace pqh

namespace pq {

cudaStream_t ctx_stream(paraqaoa_ctx* c) { return c->stream; }
int ctx_device(paraqaoa_ctx* c) { return c->device; }
int ctx_part_device(paraqaoa_ctx* c, const paraqaoa_part* pt, const SubDev** subs, const uint32_t** planes) {
  int rc = upload_part(c, pt, false);
  if (rc) return rc;
  *subs = c->d_subs.as<SubDev>();
  *planes = c->d_planes.as<uint32_t>();
  return PARAQAOA_OK;
}

// p layers over G qubit groups: group 0 = qubits [0, tb) (a tile is 2^tb
// consecutive amplitudes), groups 1.. split qubits [tb, n) evenly, each tile
// carrying the lowest tb - g qubits (>= c_min) so that HBM accesses stay in
// runs of 2^(tb-g) amplitudes. Layer l visits the groups in increasing order
// for even l and decreasing for odd l, so the last group of layer l is the
// first of layer l+1 and one pass can finish layer l, apply the phase of
// l+1 and start its mixer: 1 + p (G - 1) passes in all. high_first reverses
// every layer's visiting order (layer 0 runs from the highest group down to
// group 0): the same number of passes, but the first pass (which only
// writes) mixes the highest group, and at even p so does the last (which
// only reads); a high group mixes fewer qubits, in fewer register rounds,
// than the tile-wide low group.
// Split schedules (split_r = R > 0) give group 0 only the 2R lowest qubits,
// which a pass mixes in two register rounds with a single transpose; the
// tile still loads 2^tb contiguous amplitudes, and qubits [2R, n) form the
// higher groups.
int schedule_groups(int n, int tb, int c_min, int split_r) {
  const int gmax = tb - std::max(0, std::min(c_min, tb - 1));
  const int low = split_r > 0 ? 2 * split_r : tb;
  return 1 + (n - low + gmax - 1) / gmax;
}

std::vector<PassDesc> make_schedule(int n, int p, int tb, int c_min, bool keep, bool expect, int split_r,
                                   bool high_first) {
  const int TB = tb;
  struct Grp {
    int c, s, mix_lo, split;
  };
  std::vector<Grp> grp;
  const int low = split_r > 0 ? 2 * split_r : TB;
  grp.push_back({TB, TB, 0, split_r > 0 ? 1 : 0});
  const int rest = n - low;
  const int H = schedule_groups(n, tb, c_min, split_r) - 1;
  int s = low;
  for (int h = 0; h < H; ++h) {
    const int g = rest / H + (h < rest % H ? 1 : 0);
    grp.push_back({TB - g, s, TB - g, 0});
    s += g;
  }
  const int G = (int)grp.size();
  auto mk = [&](int gi) {
    PassDesc d;
    std::memset(&d, 0, sizeof(d));
    d.c = grp[gi].c;
    d.s = grp[gi].s;
    d.mix_lo = grp[gi].mix_lo;
    d.split = grp[gi].split;
    d.layerA = d.layerP = d.layerB = -1;
    return d;
  };
  std::vector<PassDesc> out;
  // layer l visits the groups upward when l + high_first is even
  auto order = [&](int l, int i) { return ((l + (high_first ? 1 : 0)) % 2 == 0) ? i : G - 1 - i; };
  PassDesc first = mk(order(0, 0));
  first.init = 1;
  first.layerP = 0;
  first.layerB = 0;
  first.store = 1;
  out.push_back(first);
  for (int l = 0; l < p; ++l) {
    std::vector<int> ord(G);
    for (int i = 0; i < G; ++i) ord[i] = order(l, i);
    for (int idx = 1; idx < G; ++idx) {
      PassDesc d = mk(ord[idx]);
      d.layerA = l;
      if (idx < G - 1) {
        d.store = 1;
      } else if (l < p - 1) {
        d.layerP = l + 1;
        d.layerB = l + 1;
        d.store = 1;
      } else {
        d.store = keep ? 1 : 0;
        d.expect = expect ? 1 : 0;
        d.last = 1;
      }
      out.push_back(d);
    }
  }
  return out;
}

}  // namespace pq
