// C ABI: the plain angle search (Sec. 2.2): the p = 1 grid and Adam with
// central differences, batched over parts and replayed as a CUDA graph.
#include "host_ctx.h"

using namespace pq;
using namespace pqh;

extern "C" {

}  // extern "C"

namespace pqh {

// The p = 1 grid of paraqaoa_grid_search; with weight_scaled, part s's gamma
// axis is divided by s_i = max(1, W_i / |E_i|), its mean edge weight.
int grid_search_impl(paraqaoa_ctx* c, const paraqaoa_part* pt, const int32_t* ids, int32_t count, int32_t points,
                     bool weight_scaled, double* out_gamma, double* out_beta, double* out_best, double* out_values) {
  if (!c || !pt || !ids || count < 1 || points < 1 || points > 1024 || !out_gamma || !out_beta || !out_best)
    return PARAQAOA_E_INVAL;
  for (int32_t s = 0; s < count; ++s)
    if (ids[s] < 0 || ids[s] >= pt->M) return PARAQAOA_E_INVAL;
  PQ_CUDA(cudaSetDevice(c->device));
  int rc = upload_part(c, pt, false);
  if (rc) return rc;
  if (c->persistent && (rc = persist_clear(c))) return rc;
  const int32_t G = points * points;
  const int64_t total = (int64_t)count * G;
  if (total > 0x7fffffff) return PARAQAOA_E_INVAL;
  std::vector<int32_t> inst_ids(total);
  std::vector<double> gam(total), bet(total), gsc(count, 1.0);
  const double pi = 3.14159265358979323846;
  for (int32_t s = 0; s < count; ++s) {
    const int32_t id = ids[s];
    const int64_t ne = pt->eoff[id + 1] - pt->eoff[id];
    if (weight_scaled && ne > 0) gsc[s] = std::max(1.0, (double)pt->weight[id] / (double)ne);
    for (int32_t k = 0; k < G; ++k) {
      inst_ids[(int64_t)s * G + k] = id;
      gam[(int64_t)s * G + k] = pi * (double)(k / points) / ((double)points * gsc[s]);
      bet[(int64_t)s * G + k] = 0.5 * pi * (double)(k % points) / (double)points;
    }
  }
  PQ_CUDA(c->o_vals.ensure(sizeof(double) * total));
  PQ_CUDA(c->o_best.ensure(sizeof(double) * 4 * count));
  PQ_CUDA(cudaMemcpyAsync(c->o_best.as<double>() + 3 * count, gsc.data(), sizeof(double) * count,
                          cudaMemcpyHostToDevice, c->stream));
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
    PQ_CUDA(launch_grid_argmax(c->o_vals.as<double>(), count, points, ob + 3 * count, ob, ob + count, ob + 2 * count,
                               c->stream));
  }
  PQ_CUDA(cudaMemcpyAsync(out_gamma, ob, sizeof(double) * count, cudaMemcpyDeviceToHost, c->stream));
  PQ_CUDA(cudaMemcpyAsync(out_beta, ob + count, sizeof(double) * count, cudaMemcpyDeviceToHost, c->stream));
  PQ_CUDA(cudaMemcpyAsync(out_best, ob + 2 * count, sizeof(double) * count, cudaMemcpyDeviceToHost, c->stream));
  if (out_values)
    PQ_CUDA(cudaMemcpyAsync(out_values, c->o_vals.p, sizeof(double) * total, cudaMemcpyDeviceToHost, c->stream));
  PQ_CUDA(cudaStreamSynchronize(c->stream));
  c->plan.valid = false;
  return c->persistent ? persist_status(c) : PARAQAOA_OK;
}

}  // namespace pqh

namespace pq {
int grid_search_weight_scaled(paraqaoa_ctx* c, const paraqaoa_part* pt, const int32_t* ids, int32_t count,
                              int32_t points, double* out_gamma, double* out_beta, double* out_best) {
  return grid_search_impl(c, pt, ids, count, points, true, out_gamma, out_beta, out_best, nullptr);
}
}  // namespace pq

extern "C" {

int paraqaoa_grid_search(paraqaoa_ctx* c, const paraqaoa_part* pt, const int32_t* ids, int32_t count, int32_t points,
                         double* out_gamma, double* out_beta, double* out_best, double* out_values) {
  return grid_search_impl(c, pt, ids, count, points, false, out_gamma, out_beta, out_best, out_values);
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
  if (c->persistent && (rc = persist_clear(c))) return rc;
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
  return c->persistent ? persist_status(c) : PARAQAOA_OK;
}

}  // extern "C"
