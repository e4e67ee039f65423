// C ABI of the ParaQAOA hot path: context, partition, admission, pass
// scheduling and the host side of every entry point in include/paraqaoa.h.
// Every numerical step runs in the CUDA kernels of this directory; this file
// validates arguments, lays out device memory and enqueues launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "pq_internal.h"

using namespace pq;

namespace {

std::atomic<uint64_t> g_part_serial{1};

// Grow-only device buffer.
struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t bytes) {
    if (bytes <= cap) return cudaSuccess;
    if (p) cudaFree(p);  // synchronous: no queued kernel still uses it
    p = nullptr;
    cap = 0;
    const size_t want = (bytes + 255) & ~size_t(255);
    cudaError_t e = cudaMalloc(&p, want);
    if (e == cudaSuccess) cap = want;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
  template <class T>
  T* as() const { return reinterpret_cast<T*>(p); }
};

int cuda_rc(cudaError_t e) {
  if (e == cudaSuccess) return PARAQAOA_OK;
  if (e == cudaErrorMemoryAllocation) return PARAQAOA_E_NOMEM;
  return PARAQAOA_E_CUDA;
}

#define PQ_CUDA(call)                       \
  do {                                      \
    cudaError_t e_ = (call);                \
    if (e_ != cudaSuccess) return cuda_rc(e_); \
  } while (0)

int bitlen(int64_t x) {
  int b = 0;
  while (x > 0) {
    ++b;
    x >>= 1;
  }
  return b;
}

struct ProfRec {
  int cls;
  cudaEvent_t a, b;
};

}  // namespace

struct paraqaoa_part {
  uint64_t serial;
  int32_t nv = 0, M = 0;
  std::vector<int32_t> first, size;
  std::vector<int64_t> eoff;  // M+1 into eu/ev/ew
  std::vector<int32_t> eu, ev, ew;
  std::vector<int64_t> weight;
  std::vector<int32_t> P;
  std::vector<int32_t> plane_off;
  std::vector<uint32_t> planes;
};

// A simulate plan: the instances of one batch and where their data lives.
struct SimPlan {
  int32_t count = 0, p = 0;
  uint32_t flags = 0;
  std::vector<InstDev> inst;
  std::vector<int32_t> lists;                   // concatenated instance lists
  std::pair<int32_t, int32_t> tiny{0, 0};       // offset, length into lists
  std::map<int, std::pair<int32_t, int32_t>> smem, hbm;  // n -> (offset, length)
  // n -> (offset, length) into lists: one instance per distinct part of the
  // class (the instances of a part share their cut constants)
  std::map<int, std::pair<int32_t, int32_t>> hbm_reps;
  int64_t table_elems = 0, state_elems = 0, partial_elems = 0;
  int32_t tabcap = 1;  // largest W + 1 of the batch (phase-table entries on chip)
  bool valid = false;
  // the layer passes' cut constants (functions of the parts and the pass
  // layouts only) are on the device from an earlier run of this plan
  bool cc_ready = false;
};

constexpr int kSideStreams = 4;

struct paraqaoa_ctx {
  int device = 0;
  size_t budget = 0;
  cudaStream_t own = nullptr, stream = nullptr;
  // per qubit count n: tile bits of the layer passes and the fewest contiguous
  // low qubits a high-group tile carries (heuristic, or measured by autotune)
  int8_t tile_kind[PARAQAOA_MAX_QUBITS + 1] = {};  // index into kTileShapes
  int8_t c_min[PARAQAOA_MAX_QUBITS + 1] = {};
  // split schedule (the low group is 2R qubits, one transpose per pass) per n
  int8_t split[PARAQAOA_MAX_QUBITS + 1] = {};
  // tiles per CTA of the layer passes (log2) per n
  int8_t tpc_log2[PARAQAOA_MAX_QUBITS + 1] = {};
  int num_sms = 0;
  // partition on the device
  uint64_t part_serial = 0;
  DevBuf d_subs, d_planes;
  // simulate
  SimPlan plan;
  DevBuf d_inst, d_lists, d_gamma, d_beta, d_tables, d_states, d_partials, d_expect;
  DevBuf d_consts;  // cut constants of the current plan's layer passes (the tensor-core variant: its lists)
  // top-K
  DevBuf d_chunk_off, d_topk_scratch, d_topk_z, d_topk_p;
  // merge
  DevBuf m_first, m_size, m_level, m_cand, m_intra, m_eoff, m_eu, m_ev, m_ew, m_key, m_path;
  DevBuf m_sides[2], m_score[2], m_rank[2], m_r2s[2], m_keys, m_nb;
  // angle loop
  DevBuf o_vals, o_best, o_theta, o_m, o_v, o_w, o_g2, o_b2;
  // tensor-core variant: device error flag of its bounded waits
  DevBuf d_tc_err;
  // Adam step counter on the device (read by the update kernel)
  DevBuf o_step;
  // side streams for concurrent size classes, with their fork / join events
  cudaStream_t side[kSideStreams] = {};
  cudaEvent_t fork_ev = nullptr, join_ev[kSideStreams] = {};
  // profiling
  bool prof = false;
  uint32_t prof_mask = ~0u;  // classes bracketed by events while profiling
  std::vector<ProfRec> pending;
  std::vector<cudaEvent_t> pool;
  int64_t launches[PARAQAOA_KCLASS_COUNT] = {};
  double ms[PARAQAOA_KCLASS_COUNT] = {}, bytes[PARAQAOA_KCLASS_COUNT] = {};
};

namespace {

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

void prof_flush(paraqaoa_ctx* c);

// Records kept unread before a flush; the event pool is filled to cover them
// when profiling is switched on, so a profiled run neither synchronises nor
// creates events in the middle of a call.
constexpr size_t kProfPendingMax = 16384;

struct ProfScope {
  paraqaoa_ctx* c;
  int cls;
  double bytes;
  int kernels;
  cudaEvent_t a = nullptr;
  ProfScope(paraqaoa_ctx* c_, int cls_, double bytes_, int kernels_ = 1)
      : c(c_), cls(cls_), bytes(bytes_), kernels(kernels_) {
    if (c->prof) {
      c->launches[cls] += kernels;
      c->bytes[cls] += bytes;
      if ((c->prof_mask >> cls) & 1u) {
        a = get_event(c);
        cudaEventRecord(a, c->stream);
      }
    }
  }
  ~ProfScope() {
    if (c->prof && a) {
      cudaEvent_t b = get_event(c);
      cudaEventRecord(b, c->stream);
      c->pending.push_back({cls, a, b});
      if (c->pending.size() >= kProfPendingMax) prof_flush(c);
    }
  }
};

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
    if (big || keep) {
      I.state_off = pl.state_elems;
      pl.state_elems += int64_t(1) << n;
    }
    if (big) {
      I.part_off = pl.partial_elems;
      pl.partial_elems += int64_t(1) << (n - kTileShapes[c->tile_kind[n]].tb);
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
    int kind, tb;
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
    q.kind = c->tile_kind[n];
    q.tb = kTileShapes[q.kind].tb;
    q.sched = make_schedule(n, p, q.tb, c->c_min[n], keep, want, c->split[n] ? kTileShapes[q.kind].r : 0);
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
  for (auto& kv : pl.hbm) {
    cudaStream_t st = cls_stream();
    const int n = kv.first;
    const ClassSched& q = cs[n];
    const int kind = q.kind, tb = q.tb;
    const double amps = (double)kv.second.second * (double)(int64_t(1) << n);
    const auto reps = pl.hbm_reps[n];
    std::vector<char> done(q.nsets, pl.cc_ready ? 1 : 0);
    for (size_t ip = 0; ip < q.sched.size(); ++ip) {
      PassDesc pd = q.sched[ip];
      pd.tpc_log2 = std::min<int>(c->tpc_log2[n], n - tb);
      const int k = q.set[ip];
      int32_t* consts = c->d_consts.as<int32_t>() + q.off + (int64_t)std::max(k, 0) * q.elems;
      if (k >= 0 && !done[k]) {
        ProfScope ps(c, PARAQAOA_KCLASS_OTHER, 0);
        PQ_CUDA(launch_cut_consts(kind, n, pd, inst, lists + reps.first, reps.second, subs, planes, consts, st));
        done[k] = 1;
      }
      const double bytes = amps * ((pd.init ? 0.0 : 8.0) + (pd.store ? 8.0 : 0.0));
      ProfScope ps(c, PARAQAOA_KCLASS_LAYER_PASS, bytes);
      PQ_CUDA(launch_layer_pass(kind, n, pd, inst, lists + kv.second.first, kv.second.second, subs,
                                planes, tables, states, partials, pl.tabcap, consts, st));
    }
    if (want) {
      ProfScope ps(c, PARAQAOA_KCLASS_OTHER, 0);
      PQ_CUDA(launch_expect_reduce(inst, lists + kv.second.first, kv.second.second,
                                   1 << (n - tb), partials, expect, st));
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

}  // namespace

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
// l+1 and start its mixer: 1 + p (G - 1) passes in all.
// Split schedules (split_r = R > 0) give group 0 only the 2R lowest qubits,
// which a pass mixes in two register rounds with a single transpose; the
// tile still loads 2^tb contiguous amplitudes, and qubits [2R, n) form the
// higher groups.
int schedule_groups(int n, int tb, int c_min, int split_r) {
  const int gmax = tb - std::max(0, std::min(c_min, tb - 1));
  const int low = split_r > 0 ? 2 * split_r : tb;
  return 1 + (n - low + gmax - 1) / gmax;
}

std::vector<PassDesc> make_schedule(int n, int p, int tb, int c_min, bool keep, bool expect, int split_r) {
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
  PassDesc first = mk(0);
  first.init = 1;
  first.layerP = 0;
  first.layerB = 0;
  first.store = 1;
  out.push_back(first);
  for (int l = 0; l < p; ++l) {
    std::vector<int> ord(G);
    for (int i = 0; i < G; ++i) ord[i] = (l % 2 == 0) ? i : G - 1 - i;
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

extern "C" {

const char* paraqaoa_strerror(int code) {
  switch (code) {
    case PARAQAOA_OK: return "ok";
    case PARAQAOA_E_INVAL: return "invalid argument";
    case PARAQAOA_E_TOO_MANY_QUBITS: return "subgraph has too many vertices to simulate";
    case PARAQAOA_E_ADMISSION: return "batch exceeds the context's device-memory budget";
    case PARAQAOA_E_NOMEM: return "out of memory";
    case PARAQAOA_E_SEARCH_TOO_LARGE: return "exhaustive merge space too large";
    case PARAQAOA_E_CUDA: return "CUDA runtime error";
    case PARAQAOA_E_TIMEOUT: return "device-side wait timed out";
    case PARAQAOA_E_NO_RESULT: return "no matching simulate results";
    case PARAQAOA_E_SCRATCH_LIMIT: return "input larger than the fixed no-allocation scratch";
    default: return "unknown error";
  }
}

int paraqaoa_create(paraqaoa_ctx** out, int device, size_t hbm_budget) {
  if (!out) return PARAQAOA_E_INVAL;
  *out = nullptr;
  int ndev = 0;
  PQ_CUDA(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return PARAQAOA_E_INVAL;
  PQ_CUDA(cudaSetDevice(device));
  paraqaoa_ctx* c = new (std::nothrow) paraqaoa_ctx();
  if (!c) return PARAQAOA_E_NOMEM;
  c->device = device;
  cudaError_t e = cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete c;
    return cuda_rc(e);
  }
  c->stream = c->own;
  if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) c->num_sms = 1;
  if (hbm_budget == 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    hbm_budget = (size_t)(0.8 * (double)fr);
  }
  c->budget = hbm_budget;
  for (int n = 0; n <= PARAQAOA_MAX_QUBITS; ++n) {
    // Default schedules: the autotuner's choices on the p = 2 amplitude-layer
    // sweep (parts of G(*, 0.3), weights 1..10): 2^12 x 32-register split
    // schedules up to 18 qubits, 2^12 x 16 classic walking 8 tiles per CTA for
    // 19-20, 2^13 x 32 classic walking 4 tiles for 21-24, and the split
    // schedule walking 4 tiles from 25 qubits (three qubit groups). Parts of
    // other graphs may prefer another; paraqaoa_autotune measures.
    c->c_min[n] = 2;
    if (n <= 18) {
      c->tile_kind[n] = 0;
      c->split[n] = 1;
      c->tpc_log2[n] = 1;
    } else if (n <= 20) {
      c->tile_kind[n] = 1;
      c->split[n] = 0;
      c->tpc_log2[n] = 3;
    } else if (n <= 24) {
      c->tile_kind[n] = 2;
      c->split[n] = 0;
      c->tpc_log2[n] = 2;
    } else {
      c->tile_kind[n] = 0;
      c->split[n] = 1;
      c->tpc_log2[n] = 2;
    }
  }
  *out = c;
  return PARAQAOA_OK;
}

void paraqaoa_destroy(paraqaoa_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  for (auto& r : c->pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : c->pool) cudaEventDestroy(e);
  DevBuf* bufs[] = {&c->d_subs, &c->d_planes, &c->d_inst, &c->d_lists, &c->d_gamma, &c->d_beta,
                    &c->d_tables, &c->d_states, &c->d_partials, &c->d_expect, &c->d_chunk_off,
                    &c->d_topk_scratch, &c->d_topk_z, &c->d_topk_p, &c->m_first, &c->m_size,
                    &c->m_level, &c->m_cand, &c->m_intra, &c->m_eoff, &c->m_eu, &c->m_ev, &c->m_ew,
                    &c->m_key, &c->m_path, &c->m_sides[0], &c->m_sides[1], &c->m_score[0],
                    &c->m_score[1], &c->m_rank[0], &c->m_rank[1], &c->m_r2s[0], &c->m_r2s[1],
                    &c->m_keys, &c->m_nb, &c->o_vals, &c->o_best, &c->o_theta, &c->o_m, &c->o_v,
                    &c->o_w, &c->o_g2, &c->o_b2, &c->d_consts, &c->d_tc_err, &c->o_step};
  for (DevBuf* b : bufs) b->release();
  for (int k = 0; k < kSideStreams; ++k) {
    if (c->side[k]) cudaStreamDestroy(c->side[k]);
    if (c->join_ev[k]) cudaEventDestroy(c->join_ev[k]);
  }
  if (c->fork_ev) cudaEventDestroy(c->fork_ev);
  if (c->own) cudaStreamDestroy(c->own);
  delete c;
}

int paraqaoa_set_stream(paraqaoa_ctx* c, void* stream) {
  if (!c) return PARAQAOA_E_INVAL;
  PQ_CUDA(cudaSetDevice(c->device));
  PQ_CUDA(cudaStreamSynchronize(c->stream));
  c->stream = stream ? (cudaStream_t)stream : c->own;
  return PARAQAOA_OK;
}

int paraqaoa_partition(const paraqaoa_csr* g, int32_t M, int32_t mode, const int32_t* sizes,
                       paraqaoa_part** out) {
  if (!out) return PARAQAOA_E_INVAL;
  *out = nullptr;
  int rc = validate_csr(g);
  if (rc != PARAQAOA_OK) return rc;
  const int32_t nv = g->n;
  if (M < 1 || M > nv) return PARAQAOA_E_INVAL;
  std::vector<int32_t> first(M), size(M);
  if (mode == PARAQAOA_PART_BALANCED) {
    if (M > 1 && nv - 1 < M) return PARAQAOA_E_INVAL;
    if (M == 1) {
      first[0] = 0;
      size[0] = nv;
    } else {
      const int32_t q = (nv - 1) / M, r = (nv - 1) % M;
      int32_t o = 0;
      for (int32_t i = 0; i < M; ++i) {
        const int32_t t = q + (i < r ? 1 : 0);
        first[i] = o;
        size[i] = t + 1;
        o += t;
      }
    }
  } else if (mode == PARAQAOA_PART_ALG1_LITERAL) {
    const int32_t s = nv / M - 1;
    if (M > 1 && s < 1) return PARAQAOA_E_INVAL;
    for (int32_t i = 0; i < M; ++i) {
      first[i] = i * s;
      size[i] = (i == M - 1) ? nv - i * s : s + 1;
    }
  } else if (mode == PARAQAOA_PART_SIZES) {
    if (!sizes) return PARAQAOA_E_INVAL;
    int64_t tot = 0;
    for (int32_t i = 0; i < M; ++i) {
      if (sizes[i] < (M > 1 ? 2 : 1)) return PARAQAOA_E_INVAL;
      tot += sizes[i];
    }
    if (tot - (M - 1) != nv) return PARAQAOA_E_INVAL;
    int32_t o = 0;
    for (int32_t i = 0; i < M; ++i) {
      first[i] = o;
      size[i] = sizes[i];
      o += sizes[i] - 1;
    }
  } else {
    return PARAQAOA_E_INVAL;
  }
  paraqaoa_part* pt = new (std::nothrow) paraqaoa_part();
  if (!pt) return PARAQAOA_E_NOMEM;
  pt->serial = g_part_serial.fetch_add(1);
  pt->nv = nv;
  pt->M = M;
  pt->first = first;
  pt->size = size;
  // GetSubgraph for all parts in one pass: an edge (u, v), u < v, lies in a
  // part iff u is in the part where v is first assigned.
  std::vector<int32_t> lv = levels_of(pt);
  std::vector<int64_t> cnt(M, 0);
  for (int32_t u = 0; u < nv; ++u)
    for (int64_t k = g->row_ptr[u]; k < g->row_ptr[u + 1]; ++k) {
      const int32_t v = g->col[k];
      if (u < v && u >= first[lv[v]]) cnt[lv[v]]++;
    }
  pt->eoff.assign(M + 1, 0);
  for (int32_t i = 0; i < M; ++i) pt->eoff[i + 1] = pt->eoff[i] + cnt[i];
  pt->eu.resize(pt->eoff[M]);
  pt->ev.resize(pt->eoff[M]);
  pt->ew.resize(pt->eoff[M]);
  std::vector<int64_t> fill(pt->eoff.begin(), pt->eoff.end() - 1);
  for (int32_t u = 0; u < nv; ++u)
    for (int64_t k = g->row_ptr[u]; k < g->row_ptr[u + 1]; ++k) {
      const int32_t v = g->col[k];
      if (u < v && u >= first[lv[v]]) {
        const int32_t i = lv[v];
        const int64_t at = fill[i]++;
        pt->eu[at] = u - first[i];
        pt->ev[at] = v - first[i];
        pt->ew[at] = g->w[k];
      }
    }
  // edges within a part are visited by increasing u, then v: sorted already
  pt->weight.assign(M, 0);
  pt->P.assign(M, 1);
  pt->plane_off.assign(M, 0);
  size_t planes = 0;
  for (int32_t i = 0; i < M; ++i) {
    int32_t wmax = 1;
    for (int64_t e = pt->eoff[i]; e < pt->eoff[i + 1]; ++e) {
      pt->weight[i] += pt->ew[e];
      wmax = std::max(wmax, pt->ew[e]);
    }
    pt->P[i] = std::min(bitlen(wmax), kMaxPlanes);
    pt->plane_off[i] = (int32_t)planes;
    planes += (size_t)std::min(size[i], 32) * pt->P[i];
  }
  pt->planes.assign(planes, 0u);
  for (int32_t i = 0; i < M; ++i) {
    if (size[i] > 32) continue;  // bit-planes need n <= 32; such parts cannot be simulated
    const int P = pt->P[i];
    uint32_t* pl = pt->planes.data() + pt->plane_off[i];
    for (int64_t e = pt->eoff[i]; e < pt->eoff[i + 1]; ++e) {
      const int a = pt->eu[e], b = pt->ev[e], w = pt->ew[e];
      for (int bit = 0; bit < P; ++bit)
        if ((w >> bit) & 1) {
          pl[a * P + bit] |= 1u << b;
          pl[b * P + bit] |= 1u << a;
        }
    }
  }
  *out = pt;
  return PARAQAOA_OK;
}

void paraqaoa_part_free(paraqaoa_part* pt) { delete pt; }

int paraqaoa_part_info(const paraqaoa_part* pt, int32_t* M, int32_t* first, int32_t* size,
                       int64_t* edges, int64_t* weight) {
  if (!pt) return PARAQAOA_E_INVAL;
  if (M) *M = pt->M;
  for (int32_t i = 0; i < pt->M; ++i) {
    if (first) first[i] = pt->first[i];
    if (size) size[i] = pt->size[i];
    if (edges) edges[i] = pt->eoff[i + 1] - pt->eoff[i];
    if (weight) weight[i] = pt->weight[i];
  }
  return PARAQAOA_OK;
}

int paraqaoa_part_edges(const paraqaoa_part* pt, int32_t id, int32_t* u, int32_t* v, int32_t* w) {
  if (!pt || id < 0 || id >= pt->M) return PARAQAOA_E_INVAL;
  for (int64_t e = pt->eoff[id], k = 0; e < pt->eoff[id + 1]; ++e, ++k) {
    if (u) u[k] = pt->eu[e];
    if (v) v[k] = pt->ev[e];
    if (w) w[k] = pt->ew[e];
  }
  return PARAQAOA_OK;
}

int paraqaoa_part_upload(paraqaoa_ctx* c, const paraqaoa_part* pt, int32_t force) {
  if (!c || !pt) return PARAQAOA_E_INVAL;
  PQ_CUDA(cudaSetDevice(c->device));
  return upload_part(c, pt, force != 0);
}

int paraqaoa_cut_table(paraqaoa_ctx* c, const paraqaoa_part* pt, int32_t id, uint16_t* out_host) {
  if (!c || !pt || !out_host || id < 0 || id >= pt->M) return PARAQAOA_E_INVAL;
  if (pt->size[id] > PARAQAOA_MAX_QUBITS) return PARAQAOA_E_TOO_MANY_QUBITS;
  if (pt->weight[id] > 65535) return PARAQAOA_E_INVAL;
  PQ_CUDA(cudaSetDevice(c->device));
  int rc = upload_part(c, pt, false);
  if (rc) return rc;
  const size_t bytes = sizeof(uint16_t) << pt->size[id];
  PQ_CUDA(c->d_states.ensure(bytes));  // scratch: the cut table replaces any kept states
  c->plan.valid = false;
  {
    ProfScope ps(c, PARAQAOA_KCLASS_OTHER, (double)bytes);
    PQ_CUDA(launch_cut_table(c->d_subs.as<SubDev>() + id, pt->size[id], c->d_planes.as<uint32_t>(),
                             c->d_states.as<uint16_t>(), c->stream));
  }
  PQ_CUDA(cudaMemcpyAsync(out_host, c->d_states.p, bytes, cudaMemcpyDeviceToHost, c->stream));
  PQ_CUDA(cudaStreamSynchronize(c->stream));
  return PARAQAOA_OK;
}

int paraqaoa_simulate_batch(paraqaoa_ctx* c, const paraqaoa_part* pt, const int32_t* ids,
                            int32_t count, int32_t p, const double* gamma, const double* beta,
                            uint32_t flags) {
  if (!c || !pt || !gamma || !beta) return PARAQAOA_E_INVAL;
  PQ_CUDA(cudaSetDevice(c->device));
  int rc = upload_part(c, pt, false);
  if (rc) return rc;
  rc = plan_build(c, pt, ids, count, p, flags);
  if (rc) return rc;
  PQ_CUDA(cudaMemcpyAsync(c->d_gamma.p, gamma, sizeof(double) * count * p, cudaMemcpyHostToDevice, c->stream));
  PQ_CUDA(cudaMemcpyAsync(c->d_beta.p, beta, sizeof(double) * count * p, cudaMemcpyHostToDevice, c->stream));
  return plan_run(c);
}

int paraqaoa_expect(paraqaoa_ctx* c, int32_t count, double* out_host) {
  if (!c || !out_host) return PARAQAOA_E_INVAL;
  if (!c->plan.valid || c->plan.count != count || !(c->plan.flags & PARAQAOA_SIM_EXPECT))
    return PARAQAOA_E_NO_RESULT;
  PQ_CUDA(cudaSetDevice(c->device));
  PQ_CUDA(cudaMemcpyAsync(out_host, c->d_expect.p, sizeof(double) * count, cudaMemcpyDeviceToHost, c->stream));
  PQ_CUDA(cudaStreamSynchronize(c->stream));
  return PARAQAOA_OK;
}

int paraqaoa_topk(paraqaoa_ctx* c, int32_t count, int32_t K, uint32_t* out_z, float* out_p,
                  uint32_t flags) {
  if (!c || !out_z || !out_p || K < 1 || K > PARAQAOA_MAX_TOPK) return PARAQAOA_E_INVAL;
  if (!c->plan.valid || c->plan.count != count || !(c->plan.flags & PARAQAOA_SIM_KEEP_STATE))
    return PARAQAOA_E_NO_RESULT;
  PQ_CUDA(cudaSetDevice(c->device));
  const int raw = (flags & PARAQAOA_TOPK_RAW) ? 1 : 0;
  std::vector<int64_t> off(count + 1, 0);
  for (int32_t i = 0; i < count; ++i) {
    const int n = c->plan.inst[i].n;
    const int64_t cnt = raw ? (int64_t(1) << n) : (n == 1 ? 1 : (int64_t(1) << (n - 1)));
    if (K > cnt) return PARAQAOA_E_INVAL;
    off[i + 1] = off[i] + topk_chunks_of(n, raw);
  }
  PQ_CUDA(c->d_chunk_off.ensure(sizeof(int64_t) * (count + 1)));
  PQ_CUDA(c->d_topk_scratch.ensure(sizeof(uint64_t) * 32 * std::max<int64_t>(off[count], 1)));
  PQ_CUDA(c->d_topk_z.ensure(sizeof(uint32_t) * count * K));
  PQ_CUDA(c->d_topk_p.ensure(sizeof(float) * count * K));
  PQ_CUDA(cudaMemcpyAsync(c->d_chunk_off.p, off.data(), sizeof(int64_t) * (count + 1),
                          cudaMemcpyHostToDevice, c->stream));
  {
    ProfScope ps(c, PARAQAOA_KCLASS_TOPK, 0, 2);
    PQ_CUDA(launch_topk_stages(c->d_inst.as<InstDev>(), count, K, raw, c->d_chunk_off.as<int64_t>(),
                               off[count], c->d_states.as<float2>(), c->d_topk_scratch.as<uint64_t>(),
                               c->d_topk_z.as<uint32_t>(), c->d_topk_p.as<float>(), c->stream));
  }
  PQ_CUDA(cudaMemcpyAsync(out_z, c->d_topk_z.p, sizeof(uint32_t) * count * K, cudaMemcpyDeviceToHost, c->stream));
  PQ_CUDA(cudaMemcpyAsync(out_p, c->d_topk_p.p, sizeof(float) * count * K, cudaMemcpyDeviceToHost, c->stream));
  PQ_CUDA(cudaStreamSynchronize(c->stream));
  return PARAQAOA_OK;
}

int paraqaoa_state(paraqaoa_ctx* c, int32_t i, float* out_host) {
  if (!c || !out_host) return PARAQAOA_E_INVAL;
  if (!c->plan.valid || !(c->plan.flags & PARAQAOA_SIM_KEEP_STATE)) return PARAQAOA_E_NO_RESULT;
  if (i < 0 || i >= c->plan.count) return PARAQAOA_E_INVAL;
  PQ_CUDA(cudaSetDevice(c->device));
  const InstDev& I = c->plan.inst[i];
  PQ_CUDA(cudaMemcpyAsync(out_host, c->d_states.as<float2>() + I.state_off, sizeof(float2) << I.n,
                          cudaMemcpyDeviceToHost, c->stream));
  PQ_CUDA(cudaStreamSynchronize(c->stream));
  return PARAQAOA_OK;
}

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
    while (nprefix > (int64_t(1) << 30) && L > 1) {
      --L;
      nprefix /= K;
    }
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

int paraqaoa_grid_search(paraqaoa_ctx* c, const paraqaoa_part* pt, const int32_t* ids,
                         int32_t count, int32_t points, double* out_gamma, double* out_beta,
                         double* out_best, double* out_values) {
  if (!c || !pt || !ids || count < 1 || points < 1 || points > 1024 || !out_gamma || !out_beta || !out_best)
    return PARAQAOA_E_INVAL;
  PQ_CUDA(cudaSetDevice(c->device));
  int rc = upload_part(c, pt, false);
  if (rc) return rc;
  const int32_t G = points * points;
  const int64_t total = (int64_t)count * G;
  if (total > 0x7fffffff) return PARAQAOA_E_INVAL;
  std::vector<int32_t> inst_ids(total);
  std::vector<double> gam(total), bet(total);
  const double pi = 3.14159265358979323846;
  for (int32_t s = 0; s < count; ++s)
    for (int32_t k = 0; k < G; ++k) {
      inst_ids[(int64_t)s * G + k] = ids[s];
      gam[(int64_t)s * G + k] = pi * (double)(k / points) / (double)points;
      bet[(int64_t)s * G + k] = 0.5 * pi * (double)(k % points) / (double)points;
    }
  PQ_CUDA(c->o_vals.ensure(sizeof(double) * total));
  PQ_CUDA(c->o_best.ensure(sizeof(double) * 3 * count));
  // chunk subgraphs so that each batch passes admission
  int32_t s0 = 0;
  while (s0 < count) {
    int32_t ns = count - s0;
    for (;;) {
      rc = plan_build(c, pt, inst_ids.data() + (int64_t)s0 * G, ns * G, 1, PARAQAOA_SIM_EXPECT);
      if (rc != PARAQAOA_E_ADMISSION || ns == 1) break;
      ns = (ns + 1) / 2;
    }
    if (rc) return rc;
    PQ_CUDA(cudaMemcpyAsync(c->d_gamma.p, gam.data() + (int64_t)s0 * G, sizeof(double) * ns * G, cudaMemcpyHostToDevice, c->stream));
    PQ_CUDA(cudaMemcpyAsync(c->d_beta.p, bet.data() + (int64_t)s0 * G, sizeof(double) * ns * G, cudaMemcpyHostToDevice, c->stream));
    rc = plan_run(c);
    if (rc) return rc;
    PQ_CUDA(cudaMemcpyAsync(c->o_vals.as<double>() + (int64_t)s0 * G, c->d_expect.p, sizeof(double) * ns * G,
                            cudaMemcpyDeviceToDevice, c->stream));
    PQ_CUDA(cudaStreamSynchronize(c->stream));  // host angle arrays are reused by the next chunk
    s0 += ns;
  }
  double* ob = c->o_best.as<double>();
  {
    ProfScope ps(c, PARAQAOA_KCLASS_OTHER, 0);
    PQ_CUDA(launch_grid_argmax(c->o_vals.as<double>(), count, points, ob, ob + count, ob + 2 * count, c->stream));
  }
  PQ_CUDA(cudaMemcpyAsync(out_gamma, ob, sizeof(double) * count, cudaMemcpyDeviceToHost, c->stream));
  PQ_CUDA(cudaMemcpyAsync(out_beta, ob + count, sizeof(double) * count, cudaMemcpyDeviceToHost, c->stream));
  PQ_CUDA(cudaMemcpyAsync(out_best, ob + 2 * count, sizeof(double) * count, cudaMemcpyDeviceToHost, c->stream));
  if (out_values)
    PQ_CUDA(cudaMemcpyAsync(out_values, c->o_vals.p, sizeof(double) * total, cudaMemcpyDeviceToHost, c->stream));
  PQ_CUDA(cudaStreamSynchronize(c->stream));
  c->plan.valid = false;
  return PARAQAOA_OK;
}

int paraqaoa_optimize(paraqaoa_ctx* c, const paraqaoa_part* pt, const int32_t* ids, int32_t count,
                      int32_t p, int32_t steps, double lr, double h, double* gamma_io,
                      double* beta_io, double* out_value) {
  if (!c || !pt || !ids || count < 1 || p < 1 || p > PARAQAOA_MAX_P || steps < 0 || !(h > 0) ||
      !gamma_io || !beta_io || !out_value)
    return PARAQAOA_E_INVAL;
  PQ_CUDA(cudaSetDevice(c->device));
  int rc = upload_part(c, pt, false);
  if (rc) return rc;
  const int32_t D = 2 * p, E = 4 * p;
  std::vector<double> theta((size_t)count * D), wsum(count);
  for (int32_t s = 0; s < count; ++s) {
    if (ids[s] < 0 || ids[s] >= pt->M) return PARAQAOA_E_INVAL;
    for (int32_t l = 0; l < p; ++l) {
      theta[(size_t)s * D + l] = gamma_io[(size_t)s * p + l];
      theta[(size_t)s * D + p + l] = beta_io[(size_t)s * p + l];
    }
    wsum[s] = (double)std::max<int64_t>(pt->weight[ids[s]], 1);
  }
  PQ_CUDA(c->o_theta.ensure(sizeof(double) * count * D));
  PQ_CUDA(c->o_m.ensure(sizeof(double) * count * D));
  PQ_CUDA(c->o_v.ensure(sizeof(double) * count * D));
  PQ_CUDA(c->o_w.ensure(sizeof(double) * count));
  PQ_CUDA(c->o_step.ensure(sizeof(int32_t)));
  PQ_CUDA(cudaMemcpyAsync(c->o_theta.p, theta.data(), sizeof(double) * count * D, cudaMemcpyHostToDevice, c->stream));
  PQ_CUDA(cudaMemcpyAsync(c->o_w.p, wsum.data(), sizeof(double) * count, cudaMemcpyHostToDevice, c->stream));
  PQ_CUDA(cudaMemsetAsync(c->o_m.p, 0, sizeof(double) * count * D, c->stream));
  PQ_CUDA(cudaMemsetAsync(c->o_v.p, 0, sizeof(double) * count * D, c->stream));
  // Subgraphs are independent: chunk them so that each batch of 4p shifted
  // evaluations per subgraph passes admission (halving until it does).
  std::vector<int32_t> ev_ids((size_t)count * E);
  for (int32_t s = 0; s < count; ++s)
    for (int32_t e = 0; e < E; ++e) ev_ids[(size_t)s * E + e] = ids[s];
  int32_t s0 = 0;
  while (steps > 0 && s0 < count) {
    int32_t ns = count - s0;
    for (;;) {
      rc = plan_build(c, pt, ev_ids.data() + (size_t)s0 * E, ns * E, p, PARAQAOA_SIM_EXPECT);
      if (rc != PARAQAOA_E_ADMISSION || ns == 1) break;
      ns = (ns + 1) / 2;
    }
    if (rc) return rc;
    double* th = c->o_theta.as<double>() + (size_t)s0 * D;
    double* mm = c->o_m.as<double>() + (size_t)s0 * D;
    double* vv = c->o_v.as<double>() + (size_t)s0 * D;
    const double* ww = c->o_w.as<double>() + s0;
    int32_t* step = c->o_step.as<int32_t>();
    PQ_CUDA(cudaMemsetAsync(step, 0, sizeof(int32_t), c->stream));
    // one Adam step: shifted angles (and the step counter), the batch, the update
    auto one_step = [&]() -> int {
      {
        ProfScope ps(c, PARAQAOA_KCLASS_OTHER, 0);
        PQ_CUDA(launch_adam_shifts(th, ns, p, h, c->d_gamma.as<double>(), c->d_beta.as<double>(), step, c->stream));
      }
      int r = plan_run(c);
      if (r) return r;
      ProfScope ps(c, PARAQAOA_KCLASS_OTHER, 0);
      PQ_CUDA(launch_adam_update(c->d_expect.as<double>(), ww, ns, p, h, lr, step, th, mm, vv, c->stream));
      return PARAQAOA_OK;
    };
    if ((rc = one_step())) return rc;  // the first step also sizes every buffer
    if (steps > 1 && !c->prof) {
      // the remaining steps replay one captured step as a CUDA graph (the
      // launches depend only on device data: angles, counter, moments)
      cudaGraph_t graph = nullptr;
      cudaGraphExec_t exec = nullptr;
      PQ_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed));
      rc = one_step();
      cudaError_t ce = cudaStreamEndCapture(c->stream, &graph);
      if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
      }
      PQ_CUDA(ce);
      ce = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      PQ_CUDA(ce);
      for (int32_t t = 2; t <= steps && ce == cudaSuccess; ++t) ce = cudaGraphLaunch(exec, c->stream);
      cudaGraphExecDestroy(exec);
      PQ_CUDA(ce);
    } else {
      for (int32_t t = 2; t <= steps; ++t)
        if ((rc = one_step())) return rc;
    }
    s0 += ns;
  }
  // final <C> at the optimised angles, chunked the same way
  PQ_CUDA(c->o_vals.ensure(sizeof(double) * count));
  s0 = 0;
  while (s0 < count) {
    int32_t ns = count - s0;
    for (;;) {
      rc = plan_build(c, pt, ids + s0, ns, p, PARAQAOA_SIM_EXPECT);
      if (rc != PARAQAOA_E_ADMISSION || ns == 1) break;
      ns = (ns + 1) / 2;
    }
    if (rc) return rc;
    {
      ProfScope ps(c, PARAQAOA_KCLASS_OTHER, 0);
      PQ_CUDA(launch_theta_split(c->o_theta.as<double>() + (size_t)s0 * D, ns, p, c->d_gamma.as<double>(),
                                 c->d_beta.as<double>(), c->stream));
    }
    rc = plan_run(c);
    if (rc) return rc;
    PQ_CUDA(cudaMemcpyAsync(gamma_io + (size_t)s0 * p, c->d_gamma.p, sizeof(double) * ns * p, cudaMemcpyDeviceToHost,
                            c->stream));
    PQ_CUDA(cudaMemcpyAsync(beta_io + (size_t)s0 * p, c->d_beta.p, sizeof(double) * ns * p, cudaMemcpyDeviceToHost,
                            c->stream));
    PQ_CUDA(cudaMemcpyAsync(out_value + s0, c->d_expect.p, sizeof(double) * ns, cudaMemcpyDeviceToHost, c->stream));
    PQ_CUDA(cudaStreamSynchronize(c->stream));
    s0 += ns;
  }
  return PARAQAOA_OK;
}

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
  rc = plan_build(c, pt, ids, count, p, fl);
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
    const float scale = fp16 ? std::ldexp(1.f, (n + 1) / 2) : 1.f;
    for (int l = 0; l < p; ++l) {
      {
        ProfScope ps(c, PARAQAOA_KCLASS_OTHER, (double)cnt * stride * (l == 0 ? 10.0 : 18.0));
        PQ_CUDA(launch_tc_phase(inst, dl + off, cnt, n, l, l == 0, c->d_tables.as<float2>(), gcuts, stride, states,
                                st));
      }
      int q0 = 0;
      for (int b : bs) {
        ProfScope ps(c, PARAQAOA_KCLASS_TC_MIXER, (double)cnt * stride * 16.0);
        PQ_CUDA(launch_mixer_tc(b, fp16, inst, dl + off, cnt, n, q0, l, states, scale, err, c->num_sms, st));
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

int paraqaoa_schedule(int32_t n, int32_t p, int32_t tile_bits, int32_t reg_bits, int32_t c_min, int32_t split,
                      int32_t keep, int32_t expect, int32_t max_passes, int32_t* out, int32_t* out_count) {
  if (!out_count || max_passes < 0 || (max_passes > 0 && !out)) return PARAQAOA_E_INVAL;
  if (n > PARAQAOA_MAX_QUBITS || p < 1 || p > PARAQAOA_MAX_P || c_min < 0 || c_min > 8 || (split != 0 && split != 1))
    return PARAQAOA_E_INVAL;
  int kind = -1;
  for (int k = 0; k < kTileKinds; ++k)
    if (kTileShapes[k].tb == tile_bits && kTileShapes[k].r == reg_bits) kind = k;
  if (kind < 0 || n < tile_bits || (split && n <= 2 * reg_bits)) return PARAQAOA_E_INVAL;
  const auto sched = make_schedule(n, p, tile_bits, c_min, keep != 0, expect != 0, split ? reg_bits : 0);
  *out_count = (int32_t)sched.size();
  for (int32_t i = 0; i < (int32_t)sched.size() && i < max_passes; ++i) {
    const PassDesc& d = sched[i];
    const int32_t rec[PARAQAOA_PASS_FIELDS] = {d.c,    d.s,     d.mix_lo, d.layerA, d.layerP, d.layerB,
                                               d.init, d.store, d.expect, d.last,   d.split};
    std::memcpy(out + (int64_t)i * PARAQAOA_PASS_FIELDS, rec, sizeof(rec));
  }
  return PARAQAOA_OK;
}

int paraqaoa_set_schedule(paraqaoa_ctx* c, int32_t n, int32_t tile_bits, int32_t reg_bits, int32_t c_min,
                          int32_t split, int32_t tiles_per_cta_log2) {
  if (!c || n < kSmemMaxQubits + 1 || n > PARAQAOA_MAX_QUBITS || c_min < 0 || c_min > 8 || (split != 0 && split != 1) ||
      tiles_per_cta_log2 < 0 || tiles_per_cta_log2 > kMaxTpcLog2)
    return PARAQAOA_E_INVAL;
  for (int kind = 0; kind < kTileKinds; ++kind)
    if (kTileShapes[kind].tb == tile_bits && kTileShapes[kind].r == reg_bits) {
      if (n < tile_bits || (split && n <= 2 * reg_bits)) return PARAQAOA_E_INVAL;
      c->tile_kind[n] = (int8_t)kind;
      c->c_min[n] = (int8_t)c_min;
      c->split[n] = (int8_t)split;
      c->tpc_log2[n] = (int8_t)tiles_per_cta_log2;
      c->plan.valid = false;
      return PARAQAOA_OK;
    }
  return PARAQAOA_E_INVAL;
}

int paraqaoa_autotune(paraqaoa_ctx* c, const paraqaoa_part* pt, int32_t p, int32_t* out_tile_bits,
                      int32_t* out_reg_bits, int32_t* out_c_min, int32_t* out_split, int32_t* out_tiles_per_cta_log2) {
  if (!c || !pt || p < 1 || p > PARAQAOA_MAX_P) return PARAQAOA_E_INVAL;
  PQ_CUDA(cudaSetDevice(c->device));
  int rc = upload_part(c, pt, false);
  if (rc) return rc;
  cudaEvent_t e0 = get_event(c), e1 = get_event(c);
  const bool prof = c->prof;
  c->prof = false;
  for (int n = kSmemMaxQubits + 1; n <= PARAQAOA_MAX_QUBITS; ++n) {
    std::vector<int32_t> reps;  // every part of this size (their phase tables and cut structure differ)
    for (int32_t i = 0; i < pt->M; ++i)
      if (pt->size[i] == n && pt->weight[i] <= PARAQAOA_MAX_SUBGRAPH_WEIGHT) reps.push_back(i);
    if (reps.empty()) continue;
    // the parts cycled until the batch streams >= 1 GB (well past L2)
    const int64_t copies = std::max<int64_t>(1, std::min<int64_t>(256, (int64_t(1) << 30) / (int64_t(8) << n)));
    std::vector<int32_t> ids(copies);
    for (int64_t k = 0; k < copies; ++k) ids[k] = reps[k % reps.size()];
    std::vector<double> ang(copies * p, 0.5);
    struct Cand {
      int kind, cm, sp, tpc;
      float ms;
    };
    std::vector<Cand> cands;
    std::vector<std::pair<int, int>> seen;  // (kind, groups, split; carried bits): one timing per schedule
    for (int kind = 0; kind < kTileKinds; ++kind) {
      const int tb = kTileShapes[kind].tb, r = kTileShapes[kind].r;
      if (n < tb) continue;
      for (int sp = 0; sp <= 1; ++sp)
        for (int cm = 2; cm <= 4; ++cm) {
          const int G = schedule_groups(n, tb, cm, sp ? r : 0);
          const auto sched = make_schedule(n, p, tb, cm, false, true, sp ? r : 0);
          const std::pair<int, int> key(G * 1000 + kind * 10 + sp, sched.size() > 1 ? sched[1].c : 0);
          if (std::find(seen.begin(), seen.end(), key) != seen.end()) continue;
          seen.push_back(key);
          for (int tpc = 0; tpc <= kMaxTpcLog2 && tpc <= n - tb; ++tpc)
            cands.push_back({kind, cm, sp, tpc, 1e30f});
        }
    }
    // three rounds over all candidates, each keeping its fastest round: the
    // rounds interleave the candidates so that clock and thermal drift
    // cannot favour the ones timed first
    for (int round = 0; round < 3 && !rc; ++round)
      for (Cand& cd : cands) {
        c->tile_kind[n] = (int8_t)cd.kind;
        c->c_min[n] = (int8_t)cd.cm;
        c->split[n] = (int8_t)cd.sp;
        c->tpc_log2[n] = (int8_t)cd.tpc;
        rc = plan_build(c, pt, ids.data(), (int32_t)copies, p, PARAQAOA_SIM_EXPECT);
        if (rc == PARAQAOA_E_ADMISSION) {
          rc = PARAQAOA_OK;
          continue;
        }
        if (rc) break;
        PQ_CUDA(cudaMemcpyAsync(c->d_gamma.p, ang.data(), sizeof(double) * ang.size(), cudaMemcpyHostToDevice, c->stream));
        PQ_CUDA(cudaMemcpyAsync(c->d_beta.p, ang.data(), sizeof(double) * ang.size(), cudaMemcpyHostToDevice, c->stream));
        if ((rc = plan_run(c))) break;  // warm-up
        PQ_CUDA(cudaEventRecord(e0, c->stream));
        for (int r = 0; r < 2 && !rc; ++r) rc = plan_run(c);
        PQ_CUDA(cudaEventRecord(e1, c->stream));
        PQ_CUDA(cudaEventSynchronize(e1));
        if (rc) break;
        float ms = 0.f;
        PQ_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        cd.ms = std::min(cd.ms, ms);
      }
    if (rc) break;
    Cand best{c->tile_kind[n], c->c_min[n], c->split[n], c->tpc_log2[n], 1e30f};
    for (const Cand& cd : cands)
      if (cd.ms < best.ms) best = cd;
    c->tile_kind[n] = (int8_t)best.kind;
    c->c_min[n] = (int8_t)best.cm;
    c->split[n] = (int8_t)best.sp;
    c->tpc_log2[n] = (int8_t)best.tpc;
  }
  c->pool.push_back(e0);
  c->pool.push_back(e1);
  c->prof = prof;
  c->plan.valid = false;
  if (rc) return rc;
  for (int n = 0; n <= PARAQAOA_MAX_QUBITS; ++n) {
    if (out_tile_bits) out_tile_bits[n] = kTileShapes[c->tile_kind[n]].tb;
    if (out_reg_bits) out_reg_bits[n] = kTileShapes[c->tile_kind[n]].r;
    if (out_c_min) out_c_min[n] = c->c_min[n];
    if (out_split) out_split[n] = c->split[n];
    if (out_tiles_per_cta_log2) out_tiles_per_cta_log2[n] = c->tpc_log2[n];
  }
  return PARAQAOA_OK;
}

int paraqaoa_profile_enable(paraqaoa_ctx* c, int32_t enable) {
  if (!c) return PARAQAOA_E_INVAL;
  prof_flush(c);
  c->prof = enable != 0;
  // Event records are read back only by paraqaoa_profile_read (or when
  // kProfPendingMax records are waiting), so that API calls return without
  // a pass over their events while the GPU idles.
  while (c->prof && c->pool.size() < 2 * kProfPendingMax) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) break;
    c->pool.push_back(e);
  }
  for (int k = 0; k < PARAQAOA_KCLASS_COUNT; ++k) {
    c->launches[k] = 0;
    c->ms[k] = 0;
    c->bytes[k] = 0;
  }
  return PARAQAOA_OK;
}

int paraqaoa_profile_classes(paraqaoa_ctx* c, uint32_t mask) {
  if (!c) return PARAQAOA_E_INVAL;
  c->prof_mask = mask;
  return PARAQAOA_OK;
}

int paraqaoa_profile_read(paraqaoa_ctx* c, int32_t which, int64_t* launches, double* ms,
                          double* bytes) {
  if (!c || which < 0 || which >= PARAQAOA_KCLASS_COUNT) return PARAQAOA_E_INVAL;
  prof_flush(c);
  if (launches) *launches = c->launches[which];
  if (ms) *ms = c->ms[which];
  if (bytes) *bytes = c->bytes[which];
  return PARAQAOA_OK;
}

}  // extern "C"
