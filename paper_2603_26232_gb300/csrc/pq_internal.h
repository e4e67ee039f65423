// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/paraqaoa.h"

namespace pq {

// Tile shapes of the HBM-streaming layer passes: 2^tb amplitudes per CTA held
// as 2^r registers per thread (2^(tb-r) threads). The shape per qubit count is
// a context setting (heuristic default, or measured by paraqaoa_autotune).
struct TileShape {
  int tb, r;
};
constexpr int kTileKinds = 5;
constexpr TileShape kTileShapes[kTileKinds] = {{12, 5}, {12, 4}, {13, 5}, {13, 4}, {14, 4}};
// Resident CTAs per SM of each shape's layer pass: the occupancy its launch
// bounds are compiled for (layer_min_blocks in layer_pass.cu: five CTAs of
// 128 threads, four of 256, two of 256, two of 512, one of 1024). Used only
// to size grids in whole waves, so a mismatch costs speed, not results.
constexpr int kTileResidentCtas[kTileKinds] = {5, 4, 2, 2, 1};
constexpr int kSmemMaxQubits = 14;  // states of <= 14 qubits stay on chip
constexpr int kTinyMaxQubits = 9;   // n <= 9: one small CTA, plain loops
constexpr int kMaxPlanes = 16;      // weight bit-planes (weights < 2^16)
constexpr int kMaxTpcLog2 = 4;      // a layer-pass CTA walks at most 2^4 tiles

// One subgraph on the device. Adjacency is stored as bit-planes: bit v of
// planes[u*P + b] is bit b of w_uv (0 when u, v are not adjacent), so the
// weighted neighbourhood of u restricted to a vertex mask m has weight
// sum_b 2^b popc(planes[u*P+b] & m).
struct SubDev {
  int32_t n, P, W, first;
  int32_t plane_off;  // into the planes array
  int32_t pad[3];
};

// One simulated instance (a subgraph at one set of angles).
struct InstDev {
  int32_t sub;
  int32_t n, P, W;
  int64_t state_off;  // float2 offset of its state buffer (-1: none)
  int64_t table_off;  // float2 offset of its p phase tables of W+1 entries
  int64_t part_off;   // offset of its per-tile expectation partials
  float mu[PARAQAOA_MAX_P];  // mixer butterfly coefficient per layer
  float2 final_scale;        // lambda_p: scalar the last mixer left out
  float final_scale2;        // |lambda_p|^2
  int32_t cc_slot;           // its part's slot in the layer passes' cut-constant arrays
  int32_t halved;            // the state holds only z < 2^(n-1) (psi_z = psi_(not z)); <C> counts both halves
};

// One layer pass over every tile of a group of same-size instances.
struct PassDesc {
  int32_t c;        // local bits [0, c) are qubits [0, c) (contiguous in HBM)
  int32_t s;        // local bits [c, tb) are qubits [s, s + tb - c)
  int32_t mix_lo;   // local bits >= mix_lo are mixed by this pass
  int32_t layerA;   // finish the mixer of this layer (-1: none)
  int32_t layerP;   // apply this layer's cost phase (-1: none)
  int32_t layerB;   // start the mixer of this layer (-1: none)
  int32_t init;     // start from |+>^n instead of loading
  int32_t store;    // write the tile back
  int32_t expect;   // reduce sum |psi|^2 C into the tile partial
  int32_t last;     // the final pass (stores apply lambda_p)
  int32_t split;    // low-group pass of a split schedule: mix local bits [0, 2R) in two rounds
  int32_t tpc_log2; // each CTA processes 2^tpc_log2 tiles of one instance (strided by the CTAs per instance)
  // halved states (PARAQAOA_SIM_HALVED): this low-group pass also applies the
  // mixer of the unstored top qubit, after the layerA mixing and/or after the
  // layerB mixing (k_layer_mirror)
  int32_t mirrorA, mirrorB;
};

// One segment of the persistent layer-pass kernel's work queue: one pass of
// one size class, its instances' tile groups as consecutive work items.
struct PersistSeg {
  PassDesc pd;
  int32_t n, nr;       // qubits; register rounds of the pass
  int32_t list_off;    // instances: lists[list_off .. list_off + nlist)
  int32_t nlist;
  int32_t per;         // log2 of the tile groups per instance (work items per instance)
  int32_t prev;        // segment of the same class's previous pass (-1: none)
  int32_t done_off;    // this segment's per-instance completion counters
  int32_t pad;
  int64_t item0;       // first work item of the segment
  int64_t cc_off;      // cut constants of the pass (int32 offset into the consts array)
  uint32_t mm[4];      // register slots each round mixes
};

// Kernel launchers (sim_kernels.cu). All enqueue on `st` and return the
// launch error (cudaSuccess when queued).
cudaError_t launch_prep_layers(const InstDev* inst, int32_t count, int32_t p, const double* gamma,
                               const double* beta, float2* tables, InstDev* inst_rw,
                               cudaStream_t st);
cudaError_t launch_tiny_sim(const InstDev* inst, const int32_t* list, int32_t nlist, int32_t p,
                            const SubDev* subs, const uint32_t* planes, const float2* tables,
                            float2* states, double* expect, int32_t keep, int32_t want_expect,
                            int32_t tabcap, cudaStream_t st);
cudaError_t launch_smem_sim(int n, const InstDev* inst, const int32_t* list, int32_t nlist,
                            int32_t p, const SubDev* subs, const uint32_t* planes,
                            const float2* tables, float2* states, double* expect, int32_t keep,
                            int32_t want_expect, int32_t tabcap, cudaStream_t st);
// n: the parts' vertices; nq: the stored qubits (n, or n - 1 for halved states)
cudaError_t launch_layer_pass(int kind, int n, int nq, const PassDesc& pd, const InstDev* inst,
                              const int32_t* list, int32_t nlist, const SubDev* subs,
                              const uint32_t* planes, const float2* tables, float2* states,
                              double* partials, int32_t tabcap, int32_t* consts, cudaStream_t st);
// Whether the tile shape has a halved-state (mirror) low-group pass.
bool layer_mirror_supported(int kind);
int64_t cut_consts_elems(int kind, int32_t nlist);
// Register rounds of a pass and the slots each mixes (as launch_layer_pass uses them).
int layer_pass_rounds(int kind, const PassDesc& pd);
void layer_pass_masks(int kind, const PassDesc& pd, uint32_t mm[4]);
// The persistent form: every pass of every size class of one tile shape in a
// single launch over a work queue (ctrl[0]: next item, ctrl[1]: error flag;
// done: per-segment, per-instance completion counters; both zeroed by the
// caller). A work item waits for its instance's previous pass, at most
// wait_ns per wait; a wait that gives up sets ctrl[1] and lets the item
// through. Returns the launch error.
cudaError_t launch_layer_persist(int kind, const PersistSeg* segs, int32_t nseg, int64_t items, uint64_t* ctrl,
                                 uint32_t* done, const InstDev* inst, const int32_t* lists, const SubDev* subs,
                                 const uint32_t* planes, const float2* tables, float2* states, double* partials,
                                 int32_t tabcap, const int32_t* consts, uint64_t wait_ns, int num_sms,
                                 cudaStream_t st);
// `list`: one instance per distinct part, in cc_slot order
cudaError_t launch_cut_consts(int kind, int n, const PassDesc& pd, const InstDev* inst, const int32_t* list,
                              int32_t nlist, const SubDev* subs, const uint32_t* planes,
                              int32_t* consts, cudaStream_t st);
cudaError_t launch_expect_reduce(const InstDev* inst, const int32_t* list, int32_t nlist,
                                 int32_t tiles, const double* partials, double* expect,
                                 cudaStream_t st);
cudaError_t launch_cut_table(const SubDev* sub_dev_one, int n, const uint32_t* planes,
                             uint16_t* out, cudaStream_t st);
cudaError_t launch_flag_or(const uint64_t* src, uint64_t* dst, cudaStream_t st);
cudaError_t launch_topk_stages(const InstDev* inst, int32_t count, int32_t K, int32_t raw,
                               const int64_t* chunk_off_dev, int64_t total_chunks,
                               const float2* states, uint64_t* scratch, uint32_t* out_z,
                               float* out_p, cudaStream_t st);
int64_t topk_chunks_of(int n, int raw);

// Merge (merge_kernels.cu).
struct MergeDev {
  int32_t M, K, nv, words;
  const int32_t* first;     // M
  const int32_t* size;      // M
  const int32_t* level_of;  // nv: level at which the vertex is first assigned
  const uint32_t* cand;     // M*K
  const int64_t* intra;     // M*K
  const int64_t* eoff;      // M+1: inter edges bucketed by the level of their larger end
  const int32_t* eu;        // global smaller end
  const int32_t* ev;        // local index of the larger end in its level's part
  const int32_t* ew;
};
constexpr int kMaxExhaustiveLevels = 64;
constexpr int64_t kMergeFillThreads = int64_t(1) << 17;  // starting paths that fill the GPU
constexpr int kBeamSortCap = 8192;
cudaError_t launch_cand_intra(const SubDev* subs, const uint32_t* planes, const uint32_t* cand,
                              int32_t M, int32_t K, int64_t* intra, cudaStream_t st);
cudaError_t launch_merge_dfs(const MergeDev& md, int32_t L, int64_t nprefix,
                             unsigned long long* best_key, cudaStream_t st);
cudaError_t launch_merge_dfs_path(const MergeDev& md, int32_t L, int64_t nprefix, int64_t winner,
                                  int32_t* path, cudaStream_t st);
cudaError_t launch_beam_level(const MergeDev& md, int32_t l, int32_t nb, int64_t beam,
                              uint64_t* keys, const uint32_t* sides, const int64_t* score,
                              const int32_t* rank, const int32_t* rank2slot, uint32_t* nsides,
                              int64_t* nscore, int32_t* nrank, int32_t* nrank2slot,
                              int32_t* nb_out, cudaStream_t st);

// Angle loop (opt_kernels.cu).
// gscale (device, S entries, or NULL for 1): part s's grid runs gamma_a = pi a / (points gscale[s])
cudaError_t launch_grid_argmax(const double* vals, int32_t S, int32_t points, const double* gscale, double* gamma,
                               double* beta, double* best, cudaStream_t st);
cudaError_t launch_adam_shifts(const double* theta, int32_t S, int32_t p, double h,
                               double* gamma, double* beta, int32_t* step, cudaStream_t st);
cudaError_t launch_adam_update(const double* expect, const double* wsum, int32_t S, int32_t p,
                               double h, double lr, const int32_t* step, double* theta, double* m, double* v,
                               cudaStream_t st);
cudaError_t launch_theta_split(const double* theta, int32_t S, int32_t p, double* gamma,
                               double* beta, cudaStream_t st);

// Learned angles (mlp_kernels.cu). Operands __nv_bfloat16 are passed as
// uint16_t storage so that host translation units need no CUDA BF16 header.
constexpr int kFeatures = 64;
constexpr int kHidden = 256;
typedef uint16_t bf16_t;
cudaError_t launch_features(const SubDev* subs, const uint32_t* planes, const int32_t* ids, int32_t count,
                            float* out, cudaStream_t st);
cudaError_t launch_gemm_bf16_raw(bool ta, bool tb, int M, int N, int K, const bf16_t* A, int lda, const bf16_t* B,
                                 int ldb, float* C, int ldc, const float* bias, int relu, bf16_t* Cb, cudaStream_t st);
cudaError_t launch_to_bf16_raw(const float* x, bf16_t* y, int64_t n, cudaStream_t st);
cudaError_t launch_gather_rows_raw(const float* X, int cols, const float* T, int tcols, const int32_t* idx, int rows,
                                   bf16_t* Xb, float* Tb, cudaStream_t st);
cudaError_t launch_mse_grad_raw(const float* Y, const float* T, int64_t n, float* dY, bf16_t* dYb, double* loss,
                                cudaStream_t st);
cudaError_t launch_relu_back_raw(float* dH, const float* Z, int64_t n, bf16_t* dZb, cudaStream_t st);
cudaError_t launch_colsum(const float* dZ, int rows, int cols, float* db, cudaStream_t st);
cudaError_t launch_adam_raw(float* w, const float* g, float* m, float* v, int64_t n, float lr, int t, bf16_t* wb,
                            cudaStream_t st);

// Split-precision tensor-core mixer variant (tc_mixer.cu).
cudaError_t launch_mixer_tc(int kb, bool fp16, const InstDev* inst, const int32_t* list, int32_t nlist, int32_t n,
                            int32_t q0, int32_t layer, float2* states, uint64_t wait_ns, int* err, int num_sms,
                            cudaStream_t st);
cudaError_t launch_tc_phase(const InstDev* inst, const int32_t* list, int32_t nlist, int32_t n, int32_t layer,
                            int32_t init, const float2* tables, const uint16_t* cuts, int64_t cut_stride,
                            float2* states, cudaStream_t st);
int tc_finish_blocks(int32_t n);
cudaError_t launch_tc_finish(const InstDev* inst, const int32_t* list, int32_t nlist, int32_t n, const uint16_t* cuts,
                             int64_t cut_stride, float2* states, double* partials, int32_t keep, double* expect,
                             cudaStream_t st);

// The plain angle search's p = 1 grid with each part's gamma axis divided by
// its mean edge weight (capi_search.cpp).
int grid_search_weight_scaled(paraqaoa_ctx* c, const paraqaoa_part* pt, const int32_t* ids, int32_t count,
                              int32_t points, double* out_gamma, double* out_beta, double* out_best);

// Context internals the learned-angle entry points share (capi.cpp).
cudaStream_t ctx_stream(paraqaoa_ctx* c);
int ctx_device(paraqaoa_ctx* c);
int ctx_part_device(paraqaoa_ctx* c, const paraqaoa_part* pt, const SubDev** subs, const uint32_t** planes);

// Pass schedule for an n-qubit instance group (layer_pass.cu host helper).
std::vector<PassDesc> make_schedule(int n, int p, int tb, int c_min, bool keep, bool expect, int split_r,
                                   bool high_first = false);
int schedule_groups(int n, int tb, int c_min, int split_r);

}  // namespace pq
