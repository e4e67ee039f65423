/*
 * paraqaoa.h -- C ABI of the GB300 (sm_103a) ParaQAOA hot path.
 *
 * The library runs the data-parallel part of ParaQAOA (arXiv 2603.26232):
 * partition a Max-Cut graph into a chain of subgraphs (Sec. 3.2, Alg. 1),
 * simulate one QAOA circuit per subgraph on the GPU (Sec. 2.2, Sec. 3.3),
 * reduce <C> and pick the top-K bitstrings (Sec. 3.3.2), and merge the
 * candidates into a cut of the whole graph (Sec. 3.4, Alg. 2).
 *
 * Conventions shared by every entry point
 *  - Return value: PARAQAOA_OK (0) or a negative PARAQAOA_E_* code;
 *    paraqaoa_strerror() names it. A failed call leaves its outputs
 *    unspecified and the context usable, except after PARAQAOA_E_CUDA
 *    (a CUDA runtime error), after which the context should be destroyed.
 *  - Pointers named *_host (and every pointer not said otherwise) are host
 *    memory owned by the caller; the library copies what it needs before the
 *    call returns and never keeps them. Pointers named *_dev are device
 *    memory of the context's GPU, also owned by the caller.
 *  - The library owns paraqaoa_ctx, paraqaoa_part and all device state they
 *    create; free them with paraqaoa_destroy / paraqaoa_part_free.
 *  - Bit order: bit j of a bitstring z is local vertex j of its subgraph, i.e.
 *    global vertex first_i + j. z_j = 1 puts the vertex in S. (The paper
 *    prints bitstrings vertex by vertex, so its "110" is z = 0b011.)
 *  - Angles: U_C(gamma) = exp(-i gamma C), U_M(beta) = exp(-i beta sum_j X_j),
 *    layer l = 0..p-1 applies U_C(gamma[l]) then U_M(beta[l]) (Sec. 2.2).
 *  - Threading: one context per host thread. Work is queued on the context's
 *    stream; calls that return results to the host synchronise it.
 *  - Weights are positive int32; a subgraph's total weight must be
 *    <= PARAQAOA_MAX_SUBGRAPH_WEIGHT for simulation (its cut values index an
 *    on-chip phase table).
 */
#ifndef PARAQAOA_H
#define PARAQAOA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PARAQAOA_OK 0
#define PARAQAOA_E_INVAL (-1)            /* bad argument, size or ordering of calls */
#define PARAQAOA_E_TOO_MANY_QUBITS (-2)  /* a subgraph has more than PARAQAOA_MAX_QUBITS vertices */
#define PARAQAOA_E_ADMISSION (-3)        /* the batch's device memory exceeds the context budget */
#define PARAQAOA_E_NOMEM (-4)            /* host or device allocation failed */
#define PARAQAOA_E_SEARCH_TOO_LARGE (-5) /* exhaustive merge requested over too many leaves */
#define PARAQAOA_E_CUDA (-6)             /* CUDA runtime error */
#define PARAQAOA_E_TIMEOUT (-7)          /* a bounded device-side wait gave up */
#define PARAQAOA_E_NO_RESULT (-8)        /* results requested before a matching simulate call */
#define PARAQAOA_E_SCRATCH_LIMIT (-9)    /* larger than the fixed scratch of paraqaoa_topk_noalloc */

#define PARAQAOA_MAX_QUBITS 30
#define PARAQAOA_MAX_SUBGRAPH_WEIGHT 4095
#define PARAQAOA_MAX_TOPK 32
#define PARAQAOA_MAX_P 16

/* Partition modes (Sec. 3.2, Alg. 1). */
#define PARAQAOA_PART_BALANCED 0     /* |V|-1 steps split evenly, larger first; |V_i cap V_i+1| = 1 */
#define PARAQAOA_PART_ALG1_LITERAL 1 /* s = floor(|V|/M) - 1 as printed in Alg. 1; last part takes the rest */
#define PARAQAOA_PART_SIZES 2        /* explicit sizes[M], sum(sizes) - (M-1) = |V| */

/* simulate_batch flags */
#define PARAQAOA_SIM_EXPECT 0x1u     /* reduce <C> for every instance (paraqaoa_expect) */
#define PARAQAOA_SIM_KEEP_STATE 0x2u /* keep the final states (paraqaoa_topk, paraqaoa_state) */
#define PARAQAOA_SIM_HALVED 0x4u     /* parts of >= 16 qubits keep z < 2^(n-1) only (psi_z = psi_(not z)) */

/* topk flags */
#define PARAQAOA_TOPK_CANONICAL 0x0u /* rank only z with bit n-1 = 0 (P(z) = P(not z)) */
#define PARAQAOA_TOPK_RAW 0x1u       /* rank every z */

/* Symmetric CSR: both directions of every edge stored, no self-loops, w > 0,
 * row_ptr[n] = nnz. All arrays are host memory owned by the caller. */
typedef struct {
  int32_t n;
  int64_t nnz;
  const int64_t *row_ptr;
  const int32_t *col;
  const int32_t *w;
} paraqaoa_csr;

typedef struct paraqaoa_ctx paraqaoa_ctx;
typedef struct paraqaoa_part paraqaoa_part;

/* Create a context on CUDA device `device`. hbm_budget (bytes) caps the
 * device memory one simulate batch may use; 0 means 80% of the device's free
 * memory at creation. */
int paraqaoa_create(paraqaoa_ctx **out, int device, size_t hbm_budget);
void paraqaoa_destroy(paraqaoa_ctx *ctx);

/* Run subsequent work of ctx on `stream` (a cudaStream_t of ctx's device, or
 * NULL for the context's own stream). The caller keeps ownership. */
int paraqaoa_set_stream(paraqaoa_ctx *ctx, void *stream);

/* Sec. 3.2, Alg. 1 (Connectivity-Preserving Partitioning + GetSubgraph):
 * split vertices 0..n-1 into M index ranges, neighbours sharing one vertex,
 * and keep for each part the induced edges E_i; the remaining edges are
 * E_inter (Sec. 3.4.1). `sizes` is read only in PARAQAOA_PART_SIZES mode.
 * Host-only; O(|V| + |E|). */
int paraqaoa_partition(const paraqaoa_csr *g, int32_t M, int32_t mode, const int32_t *sizes,
                       paraqaoa_part **out);
void paraqaoa_part_free(paraqaoa_part *part);

/* Describe a partition: M, and per part its first global vertex, size,
 * edge count and total weight (each array M entries, any may be NULL). */
int paraqaoa_part_info(const paraqaoa_part *part, int32_t *M, int32_t *first, int32_t *size,
                       int64_t *edges, int64_t *weight);

/* Sec. 3.3.1 (the solver pool balances subgraphs across GPUs by size): an
 * assignment of the partition's parts to `world` ranks by longest processing
 * time first. Part i costs 2^n_i * p * evals[i] (evals NULL: 1 each); parts
 * are taken by cost descending, ties by index, and each goes to the rank
 * with the least load so far, ties to the lowest rank, so every rank computes
 * the same plan. Graham's bound holds: the largest load is at most
 * (4/3 - 1/(3 world)) of the best possible. out_rank (M entries) receives
 * each part's rank, out_load (optional, world entries) each rank's load.
 * Host-only. */
int paraqaoa_shard_plan(const paraqaoa_part *part, int32_t world, int32_t p, const double *evals,
                        int32_t *out_rank, double *out_load);

/* Sec. 3.5, Performance Efficiency Index: EF = 1 / (1 + exp(alpha (t_alg -
 * t_base))) (the efficiency factor; 0.5 at t_alg = t_base, towards 1 when
 * the evaluated run is much faster than the baseline) and PEI = AR x EF x
 * 100 with AR = CutVal_ALG / CutVal_OPT. Times in the unit alpha is given
 * per (the paper takes alpha = 0.001); ar, times and alpha must be >= 0.
 * ef_out / pei_out optional. Host-only. */
int paraqaoa_pei(double ar, double t_alg, double t_base, double alpha, double *ef_out, double *pei_out);

/* Local edge list (u < v, sorted) of part `id`; arrays sized by part_info. */
int paraqaoa_part_edges(const paraqaoa_part *part, int32_t id, int32_t *u, int32_t *v, int32_t *w);

/* Copy the partition's subgraph data (adjacency bit-planes, degrees) to the
 * device. Simulation uploads on first use; calling this first keeps the copy
 * out of a timed region. Re-uploads if `force` is non-zero. */
int paraqaoa_part_upload(paraqaoa_ctx *ctx, const paraqaoa_part *part, int32_t force);

/* Sec. 2.1 cut table of part `id`: out_host[z] = C(z) = sum of w_uv over
 * edges (u, v) of E_id with z_u != z_v, for z in [0, 2^n). 2^n entries. */
int paraqaoa_cut_table(paraqaoa_ctx *ctx, const paraqaoa_part *part, int32_t id, uint16_t *out_host);

/* Sec. 2.2 / Sec. 3.3: simulate `count` QAOA instances. Instance i runs on
 * part ids[i] with angles gamma[i*p + l], beta[i*p + l] (FP64, host), starting
 * from |+>^n; the state is complex64. With PARAQAOA_SIM_EXPECT the
 * expectation <C> is reduced (per-thread FP32 sums of a few hundred
 * terms at most, FP64 across threads and tiles); with
 * PARAQAOA_SIM_KEEP_STATE the final states stay on the device for
 * paraqaoa_topk / paraqaoa_state. With PARAQAOA_SIM_HALVED, instances of
 * parts of at least 16 vertices store only the amplitudes of z < 2^(n-1)
 * (the circuit keeps psi_z = psi_(not z), since |+>^n and both unitaries
 * commute with the global flip): half the memory and half the HBM traffic
 * per layer; the mixer of qubit n-1 then pairs each stored z with its
 * complement over the other n-1 bits and is applied in the passes over the
 * lowest qubit group (classic schedules; the persistent form is not used).
 * <C> counts both halves; paraqaoa_topk ranks the canonical half (RAW is
 * refused) and paraqaoa_state returns the whole state. Results replace those
 * of the previous call. Returns PARAQAOA_E_ADMISSION if the states would
 * exceed the budget. */
int paraqaoa_simulate_batch(paraqaoa_ctx *ctx, const paraqaoa_part *part, const int32_t *ids,
                            int32_t count, int32_t p, const double *gamma, const double *beta,
                            uint32_t flags);

/* <C> of the last simulate call's instances (count must match). Synchronises. */
int paraqaoa_expect(paraqaoa_ctx *ctx, int32_t count, double *out_host);

/* Sec. 3.3.2: the K most probable bitstrings of each instance of the last
 * simulate call (made with PARAQAOA_SIM_KEEP_STATE), ranked by probability
 * (FP32) descending, then z ascending. out_z and out_p hold count*K entries.
 * 1 <= K <= PARAQAOA_MAX_TOPK. Synchronises. */
int paraqaoa_topk(paraqaoa_ctx *ctx, int32_t count, int32_t K, uint32_t *out_z, float *out_p,
                  uint32_t flags);

/* Final complex64 state of instance i of the last KEEP_STATE simulate call,
 * written interleaved (re, im): 2 * 2^n floats. Synchronises. */
int paraqaoa_state(paraqaoa_ctx *ctx, int32_t i, float *out_host);

/* Sec. 3.4, Alg. 2: merge candidates cand[i*K + j] (bitstring j of part i,
 * local bit order) into a cut of the whole graph g. Level i > 0 takes the
 * candidate or its complement so that the shared vertex keeps its side.
 *  - beam == 0: exhaustive level-aware depth-first merge (Alg. 2): K^L
 *    starting paths walked in parallel, each to the last level; the best
 *    leaf (ties: first in lexicographic candidate order) wins.
 *    PARAQAOA_E_SEARCH_TOO_LARGE when K^M > 2^40.
 *  - beam  > 0: beam reading for large M: keep the best `beam` partial
 *    paths per level, ranked by the cut of the edges whose ends are both
 *    assigned, ties by lexicographic candidate order. Exact when
 *    beam >= K^(M-1).
 * out_side[v] in {0,1} for every vertex (vertex 0 on side 0); *out_cut is
 * CutVal of that assignment. */
int paraqaoa_merge(paraqaoa_ctx *ctx, const paraqaoa_csr *g, const paraqaoa_part *part,
                   const uint32_t *cand, int32_t K, int32_t L, int64_t beam, uint8_t *out_side,
                   int64_t *out_cut);

/* Exhaustive merge parallelism. Sec. 3.4.2 walks K^L starting paths in
 * parallel processes (2K^L workers with both orientations); the answer, the
 * first best leaf in lexicographic order, does not depend on L. With fill on
 * (the default) paraqaoa_merge starts its GPU walk at the first level L' >= L
 * with K^L' >= 2^17 starting paths (at most M levels and 2^30 paths), so
 * that every SM has work; off, it walks exactly K^L paths, one GPU thread
 * each, as the paper's L prescribes (for comparing against its worker
 * counts). enable < 0 leaves the setting; levels_used (optional) receives the
 * starting level the last exhaustive merge of ctx used. */
int paraqaoa_set_merge_fill(paraqaoa_ctx *ctx, int32_t enable, int32_t *levels_used);

/* p = 1 grid search (angle loop, first stage): gamma_a = pi a / points,
 * beta_b = (pi/2) b / points for a, b in [0, points); every part in ids is
 * simulated at every grid point; per part the first maximum of <C> in
 * row-major (a, b) order is returned. out_values (optional, count*points^2)
 * receives every <C>. */
int paraqaoa_grid_search(paraqaoa_ctx *ctx, const paraqaoa_part *part, const int32_t *ids,
                         int32_t count, int32_t points, double *out_gamma, double *out_beta,
                         double *out_best, double *out_values);

/* Fixed-iteration Adam (angle loop, second stage) on f = -<C>/W with
 * central-difference gradients of step h; all scalar updates in FP64 on the
 * device. gamma_io / beta_io (count*p, host) hold the start angles and
 * receive the final ones; out_value (count) receives <C> there. */
int paraqaoa_optimize(paraqaoa_ctx *ctx, const paraqaoa_part *part, const int32_t *ids,
                      int32_t count, int32_t p, int32_t steps, double lr, double h,
                      double *gamma_io, double *beta_io, double *out_value);

/* The plain angle search with its grid size, learning rate and difference
 * step as arguments: the p = 1 grid of points x points (as
 * paraqaoa_grid_search, except that part i's gamma axis is divided by
 * s_i = max(1, W_i / |E_i|), its mean edge weight: gamma_a = pi a /
 * (points s_i); the first maximum of <C> in gamma for integer weights lies
 * near 0.5 / s_i, inside one unscaled grid step), `steps` Adam steps of learning
 * rate lr and central-difference step h (paraqaoa_optimize), then for
 * d = 2..p INTERP (Zhou et al., PRX 10, 021067, 2020) from depth d-1 and
 * `steps` Adam steps at depth d; angles folded as in paraqaoa_solve_plain
 * (which is this call with points 16, lr 0.02, h 1e-3). Sec. 2.2 leaves the
 * optimiser open; the INTERP start and the folding change no <C>.
 * gamma_out / beta_out: count x p (host), value_out (optional): <C> there.
 * steps = 0: grid only at p = 1, INTERP and evaluation above. */
int paraqaoa_angle_search(paraqaoa_ctx *ctx, const paraqaoa_part *part, const int32_t *ids, int32_t count,
                          int32_t p, int32_t points, int32_t steps, double lr, double h, double *gamma_out,
                          double *beta_out, double *value_out);

/* Final simulation and top-K of a solve (Sec. 3.3.2): simulate the parts in
 * ids at the given angles (count x p each, host) with their states kept, in
 * chunks that pass the context's admission (halving until a chunk fits), and
 * rank each state's bitstrings as paraqaoa_topk does (flags CANONICAL or
 * RAW). out_z / out_p: count x K (host); out_expect (optional): count <C>.
 * Synchronises. */
int paraqaoa_final_topk(paraqaoa_ctx *ctx, const paraqaoa_part *part, const int32_t *ids, int32_t count,
                        int32_t p, const double *gamma, const double *beta, int32_t K, uint32_t flags,
                        double *out_expect, uint32_t *out_z, float *out_p);

/* Limit, in nanoseconds, of the context's bounded device-side waits (the
 * split-precision mixer waits for its tensor-core products on an mbarrier,
 * timed by the GPU's global nanosecond timer). A wait that runs longer gives
 * up: the kernel sets an error flag, gives the products already issued up to
 * one more second to finish, frees its tensor memory and returns, and the
 * call returns PARAQAOA_E_TIMEOUT with the context still usable. Default
 * 200 ms; 0 makes every such wait give up before its first poll (the error
 * path without a fault); at most 10 s. No counterpart in the paper. */
int paraqaoa_set_wait_limit(paraqaoa_ctx *ctx, int64_t ns);

/* Top-K of one state without any device allocation (the paper has no
 * counterpart; this is a deployment variant of paraqaoa_topk).
 * For callers that must not let a library allocate device memory: a host
 * whose own caching allocator already holds nearly all device memory, or a
 * latency-critical loop that cannot take cudaMalloc's implicit device
 * synchronisation. The call uses a fixed 2 MiB scratch array compiled into
 * the library, which every GPU that loads the library holds until the
 * process exits; it calls no cudaMalloc or cudaFree.
 *  - state_dev: device pointer to 2^n complex64 amplitudes, interleaved
 *    (re, im), on the calling thread's current device; caller-owned.
 *  - out_z_dev / out_p_dev: device pointers to K entries each; caller-owned.
 *    Ranking and flags as paraqaoa_topk (PARAQAOA_TOPK_CANONICAL / RAW).
 *  - stream: cudaStream_t to run on (NULL: the legacy default stream). The
 *    call only enqueues work; synchronise the stream before reading outputs.
 *  - Limits: at most 2^25 ranked entries (canonical n <= 26, raw n <= 25);
 *    larger inputs return PARAQAOA_E_SCRATCH_LIMIT.
 *  - The first call on a device looks up the scratch array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.
 *  - Every call shares the one scratch array: calls whose work overlaps on
 *    the GPU (other streams, other host threads) race and must be ordered by
 *    the caller. */
int paraqaoa_topk_noalloc(const float *state_dev, int32_t n, int32_t K, uint32_t flags,
                          uint32_t *out_z_dev, float *out_p_dev, void *stream);

/* ---------------------------------------------------------------------------
 * Learned angles. The paper leaves the classical optimiser's starting angles
 * open and notes that initialisation matters (Sec. 2.2). The plain form
 * below is the optimiser this library uses (p = 1 grid, fixed-iteration
 * Adam, INTERP to deeper circuits); the learned form predicts its angles
 * with a 64 -> 256 -> 256 -> 2p network from subgraph features, judges each
 * prediction by <C> and sends the rejected subgraphs to the plain form.
 * Network arithmetic: matrix products take BF16 operands (round to nearest
 * even) and accumulate in FP32; biases, ReLU masks, the loss and Adam are
 * FP32 on FP32 master weights.
 * ------------------------------------------------------------------------- */

#define PARAQAOA_FEATURES 64

/* The 64 features of each part in ids (count x 64 floats, row-major),
 * computed over the m vertices that have at least one edge (an isolated
 * vertex changes neither <C> nor the best angles; all features are 0 when
 * m = 0): [0] m/32, [1] edge density |E| / C(m,2), [2]/[3] mean/std edge
 * weight over 16, [4..8) mean/std/max/min degree over m, [8..24) degree
 * histogram (bin min(deg, 15)) over m, [24..40) weight histogram (bin
 * min(w, 16) - 1) over |E|, [40..56) weighted-degree histogram (bin
 * min(15, floor(16 D / (max D + 1)))) over m, [56] triangles / C(m,3),
 * [57] total weight / (10 C(m,2)), [58..64) zero. Parts must have at most
 * 32 vertices. Synchronises. */
int paraqaoa_features(paraqaoa_ctx *ctx, const paraqaoa_part *part, const int32_t *ids, int32_t count,
                      float *out_host);

/* Plain form of the angle search for depth p: the p = 1 grid search
 * (16 x 16 points, gamma axis divided by the part's mean edge weight as in
 * paraqaoa_angle_search), `steps` Adam steps (lr 0.02, central differences h =
 * 1e-3), then for d = 2..p INTERP (Zhou et al., PRX 10, 021067, 2020) from
 * depth d-1 and `steps` Adam steps at depth d. gamma_out / beta_out receive
 * count x p angles folded into the fundamental domain (gamma_0 in [0, pi],
 * other gammas in (-pi, pi], betas in (-pi/4, pi/4]; (gamma, beta) ->
 * (-gamma, -beta), gamma period 2 pi and beta period pi/2 leave <C>
 * unchanged), value_out (optional) <C> there. steps = 0 skips Adam. */
int paraqaoa_solve_plain(paraqaoa_ctx *ctx, const paraqaoa_part *part, const int32_t *ids, int32_t count,
                         int32_t p, int32_t steps, double *gamma_out, double *beta_out, double *value_out);

typedef struct paraqaoa_mlp paraqaoa_mlp;

/* Number of FP32 parameters of the depth-p network: W1[64 x 256], b1[256],
 * W2[256 x 256], b2[256], W3[256 x 2p], b3[2p] in this order (W stored in x
 * out, row-major). 0 for an invalid p. */
int64_t paraqaoa_mlp_param_count(int32_t p);

/* Create a depth-p angle network on ctx's device from init_params
 * (paraqaoa_mlp_param_count(p) floats, host, copied). The network's outputs
 * are [gamma_0..gamma_{p-1} | beta_0..beta_{p-1}]. Free with paraqaoa_mlp_free. */
int paraqaoa_mlp_create(paraqaoa_ctx *ctx, int32_t p, const float *init_params, paraqaoa_mlp **out);
void paraqaoa_mlp_free(paraqaoa_mlp *mlp);

/* Current FP32 master parameters (param_count floats). Synchronises. */
int paraqaoa_mlp_get_params(paraqaoa_mlp *mlp, float *out_host);

/* Loss L = sum (Y - T)^2 / (rows * 2p) over the rows of X (rows x 64) and
 * targets T (rows x 2p), and its gradient (param_count floats) at the
 * current parameters, without updating them. Synchronises. */
int paraqaoa_mlp_grad(paraqaoa_mlp *mlp, const float *X, const float *T, int32_t rows, float *grad_out,
                      double *loss_out);

/* Minibatch Adam (Kingma and Ba, 2015; beta1 0.9, beta2 0.999, eps 1e-8,
 * learning rate lr) on the MSE loss. Epoch e visits rows order[e*rows ..
 * (e+1)*rows) (each a permutation of 0..rows-1) in consecutive slices of
 * `batch` rows; epoch_loss (optional, `epochs` entries) receives the mean
 * minibatch loss of each epoch. Afterwards the judge's reference angles are
 * the column means of T (the best constant predictor). Synchronises. */
int paraqaoa_mlp_train(paraqaoa_mlp *mlp, const float *X, const float *T, int32_t rows, int32_t epochs,
                       int32_t batch, double lr, const int32_t *order, double *epoch_loss);

/* Predicted angles for the rows of X (rows x 64): gamma / beta rows x p. */
int paraqaoa_mlp_predict(paraqaoa_mlp *mlp, const float *X, int32_t rows, double *gamma, double *beta);

/* The judge's reference angles (p entries each). */
int paraqaoa_mlp_reference(paraqaoa_mlp *mlp, double *gamma_out, double *beta_out);

/* Learned form of the angle search at the network's depth p: features,
 * prediction, then batches that evaluate <C> at the prediction and at the
 * reference angles (the judge). Per part, with W its total weight:
 *  - <C>(prediction) >= <C>(reference): the prediction is kept (verdict 0);
 *  - otherwise, if <C>(prediction) >= <C>(reference) - tol W: the reference
 *    angles are taken (verdict 2);
 *  - otherwise the part goes to paraqaoa_solve_plain(fallback_steps) (verdict 1).
 * tol >= 0 (tol = 0: any loss against the reference means fallback).
 * gamma_out / beta_out receive count x p angles, value_out (optional) <C>
 * there, fallback_out (optional) the verdicts. The network must belong to ctx. */
int paraqaoa_solve_learned(paraqaoa_ctx *ctx, const paraqaoa_part *part, const int32_t *ids, int32_t count,
                           paraqaoa_mlp *mlp, int32_t fallback_steps, double tol, double *gamma_out,
                           double *beta_out, double *value_out, int32_t *fallback_out);

/* Split-precision tensor-core variant of paraqaoa_simulate_batch.
 * The mixer of each layer is applied as dense 2^k x 2^k products on blocks
 * of consecutive qubits, ceil(n / block_qubits) blocks of even sizes
 * (block_qubits in 5..7; fewer, larger blocks of up to 7 qubits where that
 * would leave blocks of under 5), on the tcgen05 tensor
 * cores: every FP32 amplitude component and matrix entry is split into two
 * 16-bit parts (precision PARAQAOA_TC_BF16 or PARAQAOA_TC_FP16; FP16 parts
 * are taken of the amplitudes scaled by 2^ceil(n/2)) and the three products
 * hi*hi + hi*lo + lo*hi accumulate in FP32. Phases use an integer cut table
 * per instance. Every part must have at least 12 vertices. <C> is always
 * reduced (paraqaoa_expect); with PARAQAOA_SIM_KEEP_STATE in flags the final
 * states stay for paraqaoa_state / paraqaoa_topk. The paper has no such
 * variant: it exists to measure what 16-bit tensor-core arithmetic costs in
 * accuracy against the FP32 butterflies of paraqaoa_simulate_batch.
 * Synchronises; PARAQAOA_E_TIMEOUT if a bounded device wait gave up. */
#define PARAQAOA_TC_BF16 0
#define PARAQAOA_TC_FP16 1
int paraqaoa_simulate_tc(paraqaoa_ctx *ctx, const paraqaoa_part *part, const int32_t *ids, int32_t count, int32_t p,
                         const double *gamma, const double *beta, uint32_t flags, int32_t precision,
                         int32_t block_qubits);

/* Autotuner for the HBM-streaming layer passes (no counterpart in the paper,
 * which runs a fixed solver per subgraph). For every qubit count n >= 15
 * present in `part`, times the candidate schedules at depth p on the batch
 * one Adam step of the parts of that size runs (4p evaluations per part),
 * repeated to >= 1 GB (>= 1 GB of the parts cycled when one step holds more
 * than 4 GB), and keeps the fastest
 * for ctx: tile shapes (2^12
 * amplitudes per CTA as 32 or 16 registers per thread, or 2^13 as 32),
 * minimum contiguous-qubit runs of the higher groups (2..4), the schedule
 * form (PARAQAOA_SCHED_*: classic or split, low or high group first) and 1,
 * 2, 4, 8 or 16 tiles per CTA (sharing the per-instance set-up loads and
 * the <C> reduction). Choices that give the same pass schedule are timed
 * once. Optional outputs (31 entries each, indexed by n): chosen tile bits,
 * register bits per thread, minimum run, form bits, log2 tiles per CTA.
 * Without a call the context uses the choices measured on a p = 2 sweep of
 * G(*, 0.3) parts: (13/5, run 2, split + high first, 8 tiles per CTA),
 * except (12/4, 2, split + high first, 16) at 16 qubits and (13/5, 2,
 * classic + high first, 8) for 21-24. */
int paraqaoa_autotune(paraqaoa_ctx *ctx, const paraqaoa_part *part, int32_t p, int32_t *out_tile_bits,
                      int32_t *out_reg_bits, int32_t *out_c_min, int32_t *out_split,
                      int32_t *out_tiles_per_cta_log2);

/* Halved states for every simulate call of ctx (on/off; off by default):
 * as if each call passed PARAQAOA_SIM_HALVED, including the calls the angle
 * search (paraqaoa_grid_search, paraqaoa_optimize, paraqaoa_angle_search,
 * paraqaoa_solve_plain), the learned form and paraqaoa_final_topk make.
 * The paper stores full states; this is a deployment setting (half the
 * state memory and HBM traffic of parts of >= 16 vertices). */
int paraqaoa_set_halved(paraqaoa_ctx *ctx, int32_t enable);

/* Persistent layer passes (on/off; off by default). On: every pass of every
 * size class of n >= 15 qubits that shares a tile shape runs in ONE launch
 * of a persistent kernel (grid: the resident CTAs of the shape on every SM)
 * over a work queue of (pass, instance, tile group) items, ordered pass by
 * pass across the size classes; a CTA takes the next item from a global
 * counter and waits for its instance's previous pass to finish (every item
 * waits only for items taken before it, so the queue always progresses).
 * Each wait is bounded (paraqaoa_set_wait_limit); one that gives up lets its
 * item run on, and the call that returns the results (paraqaoa_expect,
 * paraqaoa_topk, paraqaoa_grid_search, paraqaoa_optimize) returns
 * PARAQAOA_E_TIMEOUT. The phase tables and cut constants are built by
 * separate launches before it, <C> is reduced by one launch per size class
 * after it, and the on-chip classes (n <= 14) run beside it; Adam steps
 * replay all of it from one CUDA graph. Results equal the per-pass
 * launches' bit for bit. No counterpart in the paper, which runs one solver
 * per subgraph (Sec. 3.3). */
int paraqaoa_set_persistent(paraqaoa_ctx *ctx, int32_t enable);

/* Schedule form bits (the `split` argument of the schedule calls).
 * SPLIT: the low group is the 2R lowest qubits, mixed in two register rounds
 * with one transpose (otherwise classic: the low group is the tile's 2^tb
 * contiguous qubits, mixed in up to four rounds). HIGH_FIRST: every layer
 * visits the qubit groups in the reverse order, so layer 0 starts on the
 * highest group; the first pass (write only) and, at even p, the last (read
 * only) then mix a high group, fewer qubits than the low group. Either order
 * is the circuit of Sec. 2.2: one layer's mixers commute qubit by qubit. */
#define PARAQAOA_SCHED_SPLIT 0x1
#define PARAQAOA_SCHED_HIGH_FIRST 0x2

/* Set the layer-pass schedule of n-qubit parts by hand (the choice the
 * autotuner makes): tile bits and register bits per thread (one of the
 * shapes 12/5, 12/4, 13/5, 13/4, 14/4), minimum contiguous run c_min of the
 * higher groups, split = PARAQAOA_SCHED_* form bits (0..3) and log2 of the
 * tiles each CTA walks (0..4). Affects later simulate calls of ctx. States
 * kept halved (PARAQAOA_SIM_HALVED) use the classic low-group-first form. */
int paraqaoa_set_schedule(paraqaoa_ctx *ctx, int32_t n, int32_t tile_bits, int32_t reg_bits, int32_t c_min,
                          int32_t split, int32_t tiles_per_cta_log2);

/* The layer-pass schedule of one n-qubit state at depth p for a tile shape
 * (tile_bits/reg_bits one of 12/5, 12/4, 13/5, 13/4, 14/4), minimum
 * contiguous run c_min of the higher groups and PARAQAOA_SCHED_* form bits
 * `split` (0..3), without a context or a GPU
 * (Sec. 2.2: the p layers' mixers commute qubit by qubit, so a layer can be
 * applied in qubit groups that fit a tile, and one pass ends layer l on a
 * group, applies phase l + 1 and starts layer l + 1 on the same group).
 * keep: the last pass stores the state; expect: the last pass reduces <C>.
 * Writes up to max_passes records of PARAQAOA_PASS_FIELDS int32 each into
 * out (caller-owned) and the pass count into *out_count; a record is
 * {c, s, mix_lo, layerA, layerP, layerB, init, store, expect, last, split}:
 * the tile holds qubits [0, c) and [s, s + tile_bits - c) as its local bits
 * 0..tile_bits-1, the pass mixes local bits >= mix_lo (split passes: bits
 * [0, 2 reg_bits)), finishes mixer layerA, applies phase layerP and starts
 * mixer layerB (-1: none). Returns PARAQAOA_E_INVAL for an unknown shape, n
 * below the tile or above PARAQAOA_MAX_QUBITS, p outside 1..PARAQAOA_MAX_P,
 * or a split schedule that does not fit; *out_count holds the full count
 * even when max_passes is smaller (then only max_passes records are
 * written). */
#define PARAQAOA_PASS_FIELDS 11
int paraqaoa_schedule(int32_t n, int32_t p, int32_t tile_bits, int32_t reg_bits, int32_t c_min, int32_t split,
                      int32_t keep, int32_t expect, int32_t max_passes, int32_t *out, int32_t *out_count);

/* Measured throughput of device `device` for the roofline of the on-chip
 * simulation (states of <= 14 qubits, which stay in registers and shared
 * memory between layers): packed FP32 FMA (FFMA2; two FMAs, four flops,
 * per instruction) in TFLOP/s, and shared-memory store + load bandwidth in
 * TB/s, each the best of three timed launches of a probe kernel that keeps
 * every SM busy. Allocates and frees its own small buffers; synchronises.
 * No counterpart in the paper. */
int paraqaoa_probe_peaks(int device, double *fp32_tflops, double *smem_tbs);

/* Measured HBM stream bandwidth of device `device`, the ceilings of the
 * layer passes that only write (a batch's first pass) or only read (its
 * <C> pass): grid-stride float4 writes, reads and copies over buffers of
 * `bytes` each (1 MiB .. 16 GiB, a multiple of 16; use >> L2), 8 resident
 * CTAs of 256 threads per SM, best of five timed launches after one
 * warm-up, in GB/s (copy counts read + written bytes). Allocates and frees
 * two buffers of `bytes`; synchronises. Returns PARAQAOA_E_INVAL for bad
 * arguments, PARAQAOA_E_NOMEM when the buffers do not fit. No counterpart
 * in the paper. */
int paraqaoa_probe_streams(int device, int64_t bytes, double *write_gbs, double *read_gbs, double *copy_gbs);

/* Per-kernel device time recorded with CUDA events on the context stream.
 * enable != 0 starts recording (and clears the counters). While it is on,
 * size classes run in order on the context stream and Adam steps are
 * launched one by one (no side streams, no graph replay), so that every
 * launch can be bracketed. */
int paraqaoa_profile_enable(paraqaoa_ctx *ctx, int32_t enable);
/* Restrict the event brackets to the kernel classes whose bit is set in
 * mask (bit k = PARAQAOA_KCLASS k; the default is every class). Launches
 * and algorithmic bytes are still counted for every class; the device
 * milliseconds of an unbracketed class read as 0. Fewer brackets leave
 * fewer gaps between launches. */
int paraqaoa_profile_classes(paraqaoa_ctx *ctx, uint32_t mask);
/* Read one counter set: kernel class `which` (see PARAQAOA_KCLASS_*):
 * launches, summed device milliseconds and algorithmic bytes moved. */
int paraqaoa_profile_read(paraqaoa_ctx *ctx, int32_t which, int64_t *launches, double *ms,
                          double *bytes);

#define PARAQAOA_KCLASS_LAYER_PASS 0 /* HBM-streaming layer passes (n >= 15) */
#define PARAQAOA_KCLASS_SMEM_SIM 1   /* whole-state-on-chip simulation (n <= 14) */
#define PARAQAOA_KCLASS_TOPK 2
#define PARAQAOA_KCLASS_MERGE 3
#define PARAQAOA_KCLASS_OTHER 4
#define PARAQAOA_KCLASS_TC_MIXER 5 /* split-precision tensor-core mixer passes */
#define PARAQAOA_KCLASS_COUNT 6

const char *paraqaoa_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* PARAQAOA_H */
