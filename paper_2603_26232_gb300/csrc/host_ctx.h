// Host-side state shared by the C ABI's translation units: device buffers,
// the context and partition objects, the per-kernel profiler, and the
// batch plan (admission, instance layout, pass scheduling) that every
// simulate, search and autotune entry point builds and runs. Internal to the
// library; include/paraqaoa.h is the public interface.
#pragma once

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

namespace pqh {
using namespace pq;
extern std::atomic<uint64_t> g_part_serial;  // serial numbers of partitions

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

inline int cuda_rc(cudaError_t e) {
  if (e == cudaSuccess) return PARAQAOA_OK;
  if (e == cudaErrorMemoryAllocation) return PARAQAOA_E_NOMEM;
  return PARAQAOA_E_CUDA;
}

#define PQ_CUDA(call)                       \
  do {                                      \
    cudaError_t e_ = (call);                \
    if (e_ != cudaSuccess) return cuda_rc(e_); \
  } while (0)

inline int bitlen(int64_t x) {
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
}  // namespace pqh

namespace pqh {
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
  // persistent form: per tile shape used, its segments' range in the
  // segment array, its work items and its control block (uploaded by the
  // plan's first run)
  struct PersistGroup {
    int kind;
    int32_t seg0, nseg;
    int64_t items;
    int32_t ctl_off;          // uint64 offset of its control block (2 words + counters)
    std::vector<int> classes;  // qubit counts of its size classes
    double bytes;
  };
  std::vector<PersistGroup> persist;
  bool persist_used = false;
  int64_t persist_ctl_words = 0;
};

constexpr int kSideStreams = 4;
}  // namespace pqh

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
  pqh::DevBuf d_subs, d_planes;
  // simulate
  pqh::SimPlan plan;
  pqh::DevBuf d_inst, d_lists, d_gamma, d_beta, d_tables, d_states, d_partials, d_expect;
  pqh::DevBuf d_consts;  // cut constants of the current plan's layer passes (the tensor-core variant: its lists)
  // top-K
  pqh::DevBuf d_chunk_off, d_topk_scratch, d_topk_z, d_topk_p;
  // merge
  pqh::DevBuf m_first, m_size, m_level, m_cand, m_intra, m_eoff, m_eu, m_ev, m_ew, m_key, m_path;
  pqh::DevBuf m_sides[2], m_score[2], m_rank[2], m_r2s[2], m_keys, m_nb;
  // angle loop
  pqh::DevBuf o_vals, o_best, o_theta, o_m, o_v, o_w, o_g2, o_b2;
  // tensor-core variant: device error flag of its bounded waits, and their
  // limit in nanoseconds (paraqaoa_set_wait_limit)
  pqh::DevBuf d_tc_err;
  uint64_t wait_ns = 200000000ull;
  // persistent layer passes (paraqaoa_set_persistent): segment table,
  // control blocks and the sticky error word of their bounded waits
  bool persistent = false;
  pqh::DevBuf d_pseg, d_pctl, d_perr;
  // exhaustive merge: start the walk deeper than the caller's L when that
  // gives the GPU more starting paths (paraqaoa_set_merge_fill), and the
  // starting level the last exhaustive merge used
  bool merge_fill = true;
  int32_t merge_levels_used = 0;
  // every simulate call of the context (the angle search's included) halves
  // the states it can (paraqaoa_set_halved)
  bool halved = false;
  // Adam step counter on the device (read by the update kernel)
  pqh::DevBuf o_step;
  // side streams for concurrent size classes, with their fork / join events
  cudaStream_t side[pqh::kSideStreams] = {};
  cudaEvent_t fork_ev = nullptr, join_ev[pqh::kSideStreams] = {};
  // profiling
  bool prof = false;
  uint32_t prof_mask = ~0u;  // classes bracketed by events while profiling
  std::vector<pqh::ProfRec> pending;
  std::vector<cudaEvent_t> pool;
  int64_t launches[PARAQAOA_KCLASS_COUNT] = {};
  double ms[PARAQAOA_KCLASS_COUNT] = {}, bytes[PARAQAOA_KCLASS_COUNT] = {};
};

namespace pqh {

cudaEvent_t get_event(paraqaoa_ctx* c);
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

// Defined in host_plan.cpp.
int validate_csr(const paraqaoa_csr* g);
std::vector<int32_t> levels_of(const paraqaoa_part* pt);
int upload_part(paraqaoa_ctx* c, const paraqaoa_part* pt, bool force);
cudaError_t ensure_side_streams(paraqaoa_ctx* c);
// flags: PARAQAOA_SIM_*, or kPlanFullStates to ignore the context's halved
// setting (the tensor-core variant and the autotuner simulate full states)
constexpr uint32_t kPlanFullStates = 0x80000000u;
int plan_build(paraqaoa_ctx* c, const paraqaoa_part* pt, const int32_t* ids, int32_t count, int32_t p, uint32_t flags);
int plan_run(paraqaoa_ctx* c);
// Clear / read the sticky error word of the persistent layer passes' bounded
// waits (PARAQAOA_E_TIMEOUT when one gave up since the last clear).
int persist_clear(paraqaoa_ctx* c);
int class_kind(const paraqaoa_ctx* c, int n, bool halved);
int grid_search_impl(paraqaoa_ctx* c, const paraqaoa_part* pt, const int32_t* ids, int32_t count, int32_t points,
                     bool weight_scaled, double* out_gamma, double* out_beta, double* out_best, double* out_values);
int persist_status(paraqaoa_ctx* c);

}  // namespace pqh
