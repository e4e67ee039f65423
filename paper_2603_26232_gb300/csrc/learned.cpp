// Learned QAOA angles: the angle network object and the plain / learned
// solve drivers. The paper names the classical optimiser only loosely and
// notes that initialisation matters (Sec. 2.2); the plain form here is the
// 16 x 16 p = 1 grid, fixed-iteration Adam and INTERP to deeper circuits, and
// the learned form predicts those angles from subgraph features, judges each
// prediction by <C> and sends the rejected subgraphs to the plain form.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "pq_internal.h"

using namespace pq;

namespace {

int rc_of(cudaError_t e) {
  if (e == cudaSuccess) return PARAQAOA_OK;
  if (e == cudaErrorMemoryAllocation) return PARAQAOA_E_NOMEM;
  return PARAQAOA_E_CUDA;
}

#define LQ_CUDA(call)                          \
  do {                                         \
    cudaError_t e_ = (call);                   \
    if (e_ != cudaSuccess) return rc_of(e_);   \
  } while (0)
#define LQ_RC(call)            \
  do {                         \
    int r_ = (call);           \
    if (r_) return r_;         \
  } while (0)

struct Buf {
  void* p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t bytes) {
    if (bytes <= cap) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    const size_t want = (bytes + 255) & ~size_t(255);
    cudaError_t e = cudaMalloc(&p, want);
    if (e == cudaSuccess) cap = want;
    return e;
  }
  ~Buf() {
    if (p) cudaFree(p);
  }
  template <class T>
  T* as() const { return reinterpret_cast<T*>(p); }
};

int64_t param_count(int p) {
  return (int64_t)kFeatures * kHidden + kHidden + (int64_t)kHidden * kHidden + kHidden +
         (int64_t)kHidden * 2 * p + 2 * p;
}

}  // namespace

struct paraqaoa_mlp {
  paraqaoa_ctx* ctx = nullptr;
  int p = 0;
  int64_t np = 0;
  int t = 0;  // Adam steps taken
  // parameters: FP32 master, BF16 copy, gradient, Adam moments
  Buf w, wb, g, m, v;
  // activations for up to `cap` rows
  int cap = 0;
  Buf xb, tt, z1, h1b, z2, h2b, y, dy, dyb, dz2b, dz1b, loss, idx;
  // training data on the device
  Buf X, T, order, epoch_losses;
  // reference angles of the judge (mean training label), gamma then beta
  std::vector<double> ref;
  // offsets of the parameter tensors in the flat arrays
  int64_t oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0;
};

namespace {

int ensure_rows(paraqaoa_mlp* q, int rows) {
  if (rows <= q->cap) return PARAQAOA_OK;
  const size_t r = (size_t)rows, o = 2 * (size_t)q->p;
  LQ_CUDA(q->xb.ensure(r * kFeatures * 2));
  LQ_CUDA(q->tt.ensure(r * o * 4));
  LQ_CUDA(q->z1.ensure(r * kHidden * 4));
  LQ_CUDA(q->h1b.ensure(r * kHidden * 2));
  LQ_CUDA(q->z2.ensure(r * kHidden * 4));
  LQ_CUDA(q->h2b.ensure(r * kHidden * 2));
  LQ_CUDA(q->y.ensure(r * o * 4));
  LQ_CUDA(q->dy.ensure(r * std::max<size_t>(o, kHidden) * 4));
  LQ_CUDA(q->dyb.ensure(r * o * 2));
  LQ_CUDA(q->dz2b.ensure(r * kHidden * 2));
  LQ_CUDA(q->dz1b.ensure(r * kHidden * 2));
  LQ_CUDA(q->idx.ensure(r * 4));
  q->cap = rows;
  return PARAQAOA_OK;
}

// Forward pass over `rows` rows already in q->xb (BF16). Y in q->y (FP32).
int forward(paraqaoa_mlp* q, int rows, cudaStream_t st) {
  const float* w = q->w.as<float>();
  const bf16_t* wb = q->wb.as<bf16_t>();
  const int o = 2 * q->p;
  LQ_CUDA(launch_gemm_bf16_raw(false, false, rows, kHidden, kFeatures, q->xb.as<bf16_t>(), kFeatures, wb + q->oW1,
                               kHidden, q->z1.as<float>(), kHidden, w + q->ob1, 1, q->h1b.as<bf16_t>(), st));
  LQ_CUDA(launch_gemm_bf16_raw(false, false, rows, kHidden, kHidden, q->h1b.as<bf16_t>(), kHidden, wb + q->oW2,
                               kHidden, q->z2.as<float>(), kHidden, w + q->ob2, 1, q->h2b.as<bf16_t>(), st));
  LQ_CUDA(launch_gemm_bf16_raw(false, false, rows, o, kHidden, q->h2b.as<bf16_t>(), kHidden, wb + q->oW3, o,
                               q->y.as<float>(), o, w + q->ob3, 0, nullptr, st));
  return PARAQAOA_OK;
}

// Loss and gradient of the rows in q->xb against targets q->tt; gradient in
// q->g, loss (FP64) in *loss_dev. The forward kernels keep relu(Z) in z1/z2,
// whose positive entries are exactly the ReLU mask Z > 0.
int backward(paraqaoa_mlp* q, int rows, double* loss_dev, cudaStream_t st) {
  const int o = 2 * q->p;
  const bf16_t* wb = q->wb.as<bf16_t>();
  float* g = q->g.as<float>();
  float* dy = q->dy.as<float>();
  LQ_CUDA(launch_mse_grad_raw(q->y.as<float>(), q->tt.as<float>(), (int64_t)rows * o, dy, q->dyb.as<bf16_t>(),
                              loss_dev, st));
  // layer 3: dW3 = H2b^T dYb, db3 = colsum dY, dH2 = dYb W3b^T
  LQ_CUDA(launch_gemm_bf16_raw(true, false, kHidden, o, rows, q->h2b.as<bf16_t>(), kHidden, q->dyb.as<bf16_t>(), o,
                               g + q->oW3, o, nullptr, 0, nullptr, st));
  LQ_CUDA(launch_colsum(dy, rows, o, g + q->ob3, st));
  float* dh = q->dy.as<float>();  // reuse: rows x 256 FP32 (dY is consumed above)
  LQ_CUDA(launch_gemm_bf16_raw(false, true, rows, kHidden, o, q->dyb.as<bf16_t>(), o, wb + q->oW3, o, dh, kHidden,
                               nullptr, 0, nullptr, st));
  LQ_CUDA(launch_relu_back_raw(dh, q->z2.as<float>(), (int64_t)rows * kHidden, q->dz2b.as<bf16_t>(), st));
  // layer 2
  LQ_CUDA(launch_gemm_bf16_raw(true, false, kHidden, kHidden, rows, q->h1b.as<bf16_t>(), kHidden,
                               q->dz2b.as<bf16_t>(), kHidden, g + q->oW2, kHidden, nullptr, 0, nullptr, st));
  LQ_CUDA(launch_colsum(dh, rows, kHidden, g + q->ob2, st));
  LQ_CUDA(launch_gemm_bf16_raw(false, true, rows, kHidden, kHidden, q->dz2b.as<bf16_t>(), kHidden, wb + q->oW2,
                               kHidden, dh, kHidden, nullptr, 0, nullptr, st));
  LQ_CUDA(launch_relu_back_raw(dh, q->z1.as<float>(), (int64_t)rows * kHidden, q->dz1b.as<bf16_t>(), st));
  // layer 1
  LQ_CUDA(launch_gemm_bf16_raw(true, false, kFeatures, kHidden, rows, q->xb.as<bf16_t>(), kFeatures,
                               q->dz1b.as<bf16_t>(), kHidden, g + q->oW1, kHidden, nullptr, 0, nullptr, st));
  LQ_CUDA(launch_colsum(dh, rows, kHidden, g + q->ob1, st));
  return PARAQAOA_OK;
}

int upload_rows(paraqaoa_mlp* q, const float* X, const float* T, int rows, cudaStream_t st) {
  LQ_RC(ensure_rows(q, rows));
  LQ_CUDA(q->X.ensure((size_t)rows * kFeatures * 4));
  LQ_CUDA(cudaMemcpyAsync(q->X.p, X, (size_t)rows * kFeatures * 4, cudaMemcpyHostToDevice, st));
  if (T) {
    LQ_CUDA(q->T.ensure((size_t)rows * 2 * q->p * 4));
    LQ_CUDA(cudaMemcpyAsync(q->T.p, T, (size_t)rows * 2 * q->p * 4, cudaMemcpyHostToDevice, st));
  }
  std::vector<int32_t> id(rows);
  for (int i = 0; i < rows; ++i) id[i] = i;
  LQ_CUDA(cudaMemcpyAsync(q->idx.p, id.data(), sizeof(int32_t) * rows, cudaMemcpyHostToDevice, st));
  LQ_CUDA(launch_gather_rows_raw(q->X.as<float>(), kFeatures, T ? q->T.as<float>() : nullptr, 2 * q->p,
                                 q->idx.as<int32_t>(), rows, q->xb.as<bf16_t>(), q->tt.as<float>(), st));
  LQ_CUDA(cudaStreamSynchronize(st));  // id is a temporary
  return PARAQAOA_OK;
}

void interp(const std::vector<double>& x, int p, std::vector<double>& out) {
  // INTERP (Zhou et al., PRX 10, 021067, 2020): depth-p angles -> depth p+1
  out.assign(p + 1, 0.0);
  for (int i = 1; i <= p + 1; ++i) {
    const double lo = (i - 2 >= 0) ? x[i - 2] : 0.0;
    const double hi = (i - 1 < p) ? x[i - 1] : 0.0;
    out[i - 1] = ((double)(i - 1) / p) * lo + ((double)(p - i + 1) / p) * hi;
  }
}

// Fold depth-p angles into one fundamental domain: (gamma, beta) -> (-gamma,
// -beta) keeps every probability (complex conjugation), gamma has period 2 pi
// for integer cut values and beta period pi / 2 (X^n commutes with both
// unitaries). Result: gamma_0 in [0, pi], other gammas in (-pi, pi], betas in
// (-pi/4, pi/4].
void canonicalize(double* g, double* b, int p) {
  const double pi = 3.14159265358979323846;
  auto wrap = [](double x, double period) {  // into (-period/2, period/2]
    double y = x - period * std::floor(x / period + 0.5);
    if (y <= -0.5 * period) y += period;
    if (y > 0.5 * period) y -= period;
    return y;
  };
  for (int l = 0; l < p; ++l) g[l] = wrap(g[l], 2.0 * pi);
  if (g[0] < 0.0)
    for (int l = 0; l < p; ++l) {
      g[l] = -g[l];
      b[l] = -b[l];
    }
  for (int l = 0; l < p; ++l) {
    g[l] = wrap(g[l], 2.0 * pi);
    b[l] = wrap(b[l], 0.5 * pi);
  }
}

// <C> of count instances through simulate/expect, in chunks that pass the
// context's admission (halving the chunk until it does).
int expect_chunked(paraqaoa_ctx* ctx, const paraqaoa_part* part, const int32_t* ids, int32_t count, int p,
                   const double* g, const double* b, double* out) {
  int32_t s0 = 0;
  while (s0 < count) {
    int32_t ns = count - s0;
    int rc;
    for (;;) {
      rc = paraqaoa_simulate_batch(ctx, part, ids + s0, ns, p, g + (size_t)s0 * p, b + (size_t)s0 * p,
                                   PARAQAOA_SIM_EXPECT);
      if (rc != PARAQAOA_E_ADMISSION || ns == 1) break;
      ns = (ns + 1) / 2;
    }
    if (rc) return rc;
    LQ_RC(paraqaoa_expect(ctx, ns, out + s0));
    s0 += ns;
  }
  return PARAQAOA_OK;
}

}  // namespace

extern "C" {

int64_t paraqaoa_mlp_param_count(int32_t p) {
  if (p < 1 || p > PARAQAOA_MAX_P) return 0;
  return param_count(p);
}

int paraqaoa_mlp_create(paraqaoa_ctx* ctx, int32_t p, const float* init_params, paraqaoa_mlp** out) {
  if (!ctx || !out || p < 1 || p > PARAQAOA_MAX_P || !init_params) return PARAQAOA_E_INVAL;
  *out = nullptr;
  LQ_CUDA(cudaSetDevice(ctx_device(ctx)));
  paraqaoa_mlp* q = new (std::nothrow) paraqaoa_mlp();
  if (!q) return PARAQAOA_E_NOMEM;
  q->ctx = ctx;
  q->p = p;
  q->np = param_count(p);
  q->oW1 = 0;
  q->ob1 = q->oW1 + (int64_t)kFeatures * kHidden;
  q->oW2 = q->ob1 + kHidden;
  q->ob2 = q->oW2 + (int64_t)kHidden * kHidden;
  q->oW3 = q->ob2 + kHidden;
  q->ob3 = q->oW3 + (int64_t)kHidden * 2 * p;
  q->ref.assign(2 * p, 0.0);
  const size_t n = (size_t)q->np;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = q->w.ensure(n * 4);
  if (e == cudaSuccess) e = q->wb.ensure(n * 2);
  if (e == cudaSuccess) e = q->g.ensure(n * 4);
  if (e == cudaSuccess) e = q->m.ensure(n * 4);
  if (e == cudaSuccess) e = q->v.ensure(n * 4);
  if (e == cudaSuccess) e = q->loss.ensure(8 * 2);
  cudaStream_t st = ctx_stream(ctx);
  if (e == cudaSuccess) e = cudaMemcpyAsync(q->w.p, init_params, n * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(q->m.p, 0, n * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(q->v.p, 0, n * 4, st);
  if (e == cudaSuccess) e = launch_to_bf16_raw(q->w.as<float>(), q->wb.as<bf16_t>(), q->np, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    delete q;
    return rc_of(e);
  }
  *out = q;
  return PARAQAOA_OK;
}

void paraqaoa_mlp_free(paraqaoa_mlp* q) {
  if (!q) return;
  cudaSetDevice(ctx_device(q->ctx));
  cudaStreamSynchronize(ctx_stream(q->ctx));
  delete q;
}

int paraqaoa_mlp_get_params(paraqaoa_mlp* q, float* out_host) {
  if (!q || !out_host) return PARAQAOA_E_INVAL;
  LQ_CUDA(cudaSetDevice(ctx_device(q->ctx)));
  cudaStream_t st = ctx_stream(q->ctx);
  LQ_CUDA(cudaMemcpyAsync(out_host, q->w.p, (size_t)q->np * 4, cudaMemcpyDeviceToHost, st));
  LQ_CUDA(cudaStreamSynchronize(st));
  return PARAQAOA_OK;
}

int paraqaoa_mlp_reference(paraqaoa_mlp* q, double* gamma_out, double* beta_out) {
  if (!q || !gamma_out || !beta_out) return PARAQAOA_E_INVAL;
  for (int l = 0; l < q->p; ++l) {
    gamma_out[l] = q->ref[l];
    beta_out[l] = q->ref[q->p + l];
  }
  return PARAQAOA_OK;
}

int paraqaoa_mlp_grad(paraqaoa_mlp* q, const float* X, const float* T, int32_t rows, float* grad_out,
                      double* loss_out) {
  if (!q || !X || !T || rows < 1 || !grad_out) return PARAQAOA_E_INVAL;
  LQ_CUDA(cudaSetDevice(ctx_device(q->ctx)));
  cudaStream_t st = ctx_stream(q->ctx);
  LQ_RC(upload_rows(q, X, T, rows, st));
  LQ_RC(forward(q, rows, st));
  LQ_RC(backward(q, rows, q->loss.as<double>(), st));
  LQ_CUDA(cudaMemcpyAsync(grad_out, q->g.p, (size_t)q->np * 4, cudaMemcpyDeviceToHost, st));
  double loss = 0.0;
  LQ_CUDA(cudaMemcpyAsync(&loss, q->loss.p, 8, cudaMemcpyDeviceToHost, st));
  LQ_CUDA(cudaStreamSynchronize(st));
  if (loss_out) *loss_out = loss;
  return PARAQAOA_OK;
}

int paraqaoa_mlp_train(paraqaoa_mlp* q, const float* X, const float* T, int32_t rows, int32_t epochs,
                       int32_t batch, double lr, const int32_t* order, double* epoch_loss) {
  if (!q || !X || !T || rows < 1 || epochs < 1 || batch < 1 || !order || !(lr > 0.0)) return PARAQAOA_E_INVAL;
  for (int64_t i = 0; i < (int64_t)rows * epochs; ++i)
    if (order[i] < 0 || order[i] >= rows) return PARAQAOA_E_INVAL;
  LQ_CUDA(cudaSetDevice(ctx_device(q->ctx)));
  cudaStream_t st = ctx_stream(q->ctx);
  const int o = 2 * q->p;
  const int bmax = std::min(batch, rows);
  LQ_RC(ensure_rows(q, bmax));
  LQ_CUDA(q->X.ensure((size_t)rows * kFeatures * 4));
  LQ_CUDA(q->T.ensure((size_t)rows * o * 4));
  LQ_CUDA(q->order.ensure((size_t)rows * epochs * 4));
  const int nb = (rows + batch - 1) / batch;
  LQ_CUDA(q->epoch_losses.ensure(sizeof(double) * (size_t)epochs * nb));
  LQ_CUDA(cudaMemcpyAsync(q->X.p, X, (size_t)rows * kFeatures * 4, cudaMemcpyHostToDevice, st));
  LQ_CUDA(cudaMemcpyAsync(q->T.p, T, (size_t)rows * o * 4, cudaMemcpyHostToDevice, st));
  LQ_CUDA(cudaMemcpyAsync(q->order.p, order, (size_t)rows * epochs * 4, cudaMemcpyHostToDevice, st));
  double* losses = q->epoch_losses.as<double>();
  for (int e = 0; e < epochs; ++e) {
    for (int b = 0; b < nb; ++b) {
      const int s0 = b * batch, r = std::min(batch, rows - s0);
      LQ_CUDA(launch_gather_rows_raw(q->X.as<float>(), kFeatures, q->T.as<float>(), o,
                                     q->order.as<int32_t>() + (int64_t)e * rows + s0, r, q->xb.as<bf16_t>(),
                                     q->tt.as<float>(), st));
      LQ_RC(forward(q, r, st));
      LQ_RC(backward(q, r, losses + (int64_t)e * nb + b, st));
      ++q->t;
      LQ_CUDA(launch_adam_raw(q->w.as<float>(), q->g.as<float>(), q->m.as<float>(), q->v.as<float>(), q->np,
                              (float)lr, q->t, q->wb.as<bf16_t>(), st));
    }
  }
  std::vector<double> all((size_t)epochs * nb);
  LQ_CUDA(cudaMemcpyAsync(all.data(), losses, sizeof(double) * all.size(), cudaMemcpyDeviceToHost, st));
  LQ_CUDA(cudaStreamSynchronize(st));
  if (epoch_loss)
    for (int e = 0; e < epochs; ++e) {
      double s = 0.0;
      for (int b = 0; b < nb; ++b) s += all[(size_t)e * nb + b];
      epoch_loss[e] = s / nb;
    }
  // judge reference: the mean training label (the best constant predictor)
  for (int c = 0; c < o; ++c) {
    double s = 0.0;
    for (int i = 0; i < rows; ++i) s += (double)T[(int64_t)i * o + c];
    q->ref[c] = s / rows;
  }
  return PARAQAOA_OK;
}

int paraqaoa_mlp_predict(paraqaoa_mlp* q, const float* X, int32_t rows, double* gamma, double* beta) {
  if (!q || !X || rows < 1 || !gamma || !beta) return PARAQAOA_E_INVAL;
  LQ_CUDA(cudaSetDevice(ctx_device(q->ctx)));
  cudaStream_t st = ctx_stream(q->ctx);
  LQ_RC(upload_rows(q, X, nullptr, rows, st));
  LQ_RC(forward(q, rows, st));
  std::vector<float> y((size_t)rows * 2 * q->p);
  LQ_CUDA(cudaMemcpyAsync(y.data(), q->y.p, y.size() * 4, cudaMemcpyDeviceToHost, st));
  LQ_CUDA(cudaStreamSynchronize(st));
  for (int r = 0; r < rows; ++r)
    for (int l = 0; l < q->p; ++l) {
      gamma[(int64_t)r * q->p + l] = y[(size_t)r * 2 * q->p + l];
      beta[(int64_t)r * q->p + l] = y[(size_t)r * 2 * q->p + q->p + l];
    }
  return PARAQAOA_OK;
}

int paraqaoa_solve_plain(paraqaoa_ctx* ctx, const paraqaoa_part* part, const int32_t* ids, int32_t count, int32_t p,
                         int32_t steps, double* gamma_out, double* beta_out, double* value_out) {
  return paraqaoa_angle_search(ctx, part, ids, count, p, 16, steps, 0.02, 1e-3, gamma_out, beta_out, value_out);
}

int paraqaoa_angle_search(paraqaoa_ctx* ctx, const paraqaoa_part* part, const int32_t* ids, int32_t count, int32_t p,
                          int32_t points, int32_t steps, double lr, double h, double* gamma_out, double* beta_out,
                          double* value_out) {
  if (!ctx || !part || !ids || count < 1 || p < 1 || p > PARAQAOA_MAX_P || steps < 0 || !gamma_out || !beta_out ||
      points < 1 || points > 1024 || !(h > 0.0) || !(lr > 0.0))
    return PARAQAOA_E_INVAL;
  std::vector<double> g(count), b(count), best(count), val(count);
  LQ_RC(grid_search_weight_scaled(ctx, part, ids, count, points, g.data(), b.data(), best.data()));
  if (steps > 0) LQ_RC(paraqaoa_optimize(ctx, part, ids, count, 1, steps, lr, h, g.data(), b.data(), val.data()));
  else val = best;
  std::vector<double> x, y;
  for (int d = 2; d <= p; ++d) {
    std::vector<double> g2((size_t)count * d), b2((size_t)count * d);
    for (int i = 0; i < count; ++i) {
      interp(std::vector<double>(g.begin() + (size_t)i * (d - 1), g.begin() + (size_t)(i + 1) * (d - 1)), d - 1, x);
      interp(std::vector<double>(b.begin() + (size_t)i * (d - 1), b.begin() + (size_t)(i + 1) * (d - 1)), d - 1, y);
      std::copy(x.begin(), x.end(), g2.begin() + (size_t)i * d);
      std::copy(y.begin(), y.end(), b2.begin() + (size_t)i * d);
    }
    g.swap(g2);
    b.swap(b2);
    if (steps > 0) {
      LQ_RC(paraqaoa_optimize(ctx, part, ids, count, d, steps, lr, h, g.data(), b.data(), val.data()));
    } else {
      LQ_RC(expect_chunked(ctx, part, ids, count, d, g.data(), b.data(), val.data()));
    }
  }
  for (int i = 0; i < count; ++i) canonicalize(g.data() + (size_t)i * p, b.data() + (size_t)i * p, p);
  std::copy(g.begin(), g.end(), gamma_out);
  std::copy(b.begin(), b.end(), beta_out);
  if (value_out) std::copy(val.begin(), val.end(), value_out);
  return PARAQAOA_OK;
}

int paraqaoa_final_topk(paraqaoa_ctx* ctx, const paraqaoa_part* part, const int32_t* ids, int32_t count, int32_t p,
                        const double* gamma, const double* beta, int32_t K, uint32_t flags, double* out_expect,
                        uint32_t* out_z, float* out_p) {
  if (!ctx || !part || !ids || count < 1 || p < 1 || p > PARAQAOA_MAX_P || !gamma || !beta || K < 1 ||
      K > PARAQAOA_MAX_TOPK || !out_z || !out_p)
    return PARAQAOA_E_INVAL;
  int32_t s0 = 0;
  while (s0 < count) {
    int32_t ns = count - s0;
    int rc;
    for (;;) {  // halve the chunk until its states pass the context's admission
      rc = paraqaoa_simulate_batch(ctx, part, ids + s0, ns, p, gamma + (size_t)s0 * p, beta + (size_t)s0 * p,
                                   PARAQAOA_SIM_EXPECT | PARAQAOA_SIM_KEEP_STATE);
      if (rc != PARAQAOA_E_ADMISSION || ns == 1) break;
      ns = (ns + 1) / 2;
    }
    LQ_RC(rc);
    if (out_expect) LQ_RC(paraqaoa_expect(ctx, ns, out_expect + s0));
    LQ_RC(paraqaoa_topk(ctx, ns, K, out_z + (size_t)s0 * K, out_p + (size_t)s0 * K, flags));
    s0 += ns;
  }
  return PARAQAOA_OK;
}

int paraqaoa_features(paraqaoa_ctx* ctx, const paraqaoa_part* part, const int32_t* ids, int32_t count,
                      float* out_host) {
  if (!ctx || !part || !ids || count < 1 || !out_host) return PARAQAOA_E_INVAL;
  int32_t M = 0;
  LQ_RC(paraqaoa_part_info(part, &M, nullptr, nullptr, nullptr, nullptr));
  std::vector<int32_t> size(M);
  LQ_RC(paraqaoa_part_info(part, &M, nullptr, size.data(), nullptr, nullptr));
  for (int i = 0; i < count; ++i)
    if (ids[i] < 0 || ids[i] >= M || size[ids[i]] > 32) return PARAQAOA_E_INVAL;
  LQ_CUDA(cudaSetDevice(ctx_device(ctx)));
  const SubDev* subs = nullptr;
  const uint32_t* planes = nullptr;
  LQ_RC(ctx_part_device(ctx, part, &subs, &planes));
  cudaStream_t st = ctx_stream(ctx);
  Buf d_ids, d_out;
  LQ_CUDA(d_ids.ensure(sizeof(int32_t) * count));
  LQ_CUDA(d_out.ensure(sizeof(float) * kFeatures * count));
  LQ_CUDA(cudaMemcpyAsync(d_ids.p, ids, sizeof(int32_t) * count, cudaMemcpyHostToDevice, st));
  LQ_CUDA(launch_features(subs, planes, d_ids.as<int32_t>(), count, d_out.as<float>(), st));
  LQ_CUDA(cudaMemcpyAsync(out_host, d_out.p, sizeof(float) * kFeatures * count, cudaMemcpyDeviceToHost, st));
  LQ_CUDA(cudaStreamSynchronize(st));
  return PARAQAOA_OK;
}

int paraqaoa_solve_learned(paraqaoa_ctx* ctx, const paraqaoa_part* part, const int32_t* ids, int32_t count,
                           paraqaoa_mlp* q, int32_t fallback_steps, double tol, double* gamma_out, double* beta_out,
                           double* value_out, int32_t* fallback_out) {
  if (!ctx || !part || !ids || count < 1 || !q || q->ctx != ctx || fallback_steps < 0 || !gamma_out || !beta_out ||
      !(tol >= 0.0))
    return PARAQAOA_E_INVAL;
  int32_t M = 0;
  LQ_RC(paraqaoa_part_info(part, &M, nullptr, nullptr, nullptr, nullptr));
  std::vector<int64_t> weight(M);
  LQ_RC(paraqaoa_part_info(part, &M, nullptr, nullptr, nullptr, weight.data()));
  for (int i = 0; i < count; ++i)
    if (ids[i] < 0 || ids[i] >= M) return PARAQAOA_E_INVAL;
  const int p = q->p;
  std::vector<float> X((size_t)count * kFeatures);
  LQ_RC(paraqaoa_features(ctx, part, ids, count, X.data()));
  std::vector<double> g((size_t)count * p), b((size_t)count * p);
  LQ_RC(paraqaoa_mlp_predict(q, X.data(), count, g.data(), b.data()));
  // judge: <C> at the prediction and at the reference angles, one batch
  std::vector<int32_t> ids2(2 * (size_t)count);
  std::vector<double> g2(2 * (size_t)count * p), b2(2 * (size_t)count * p), ex(2 * (size_t)count);
  for (int i = 0; i < count; ++i) {
    ids2[i] = ids[i];
    ids2[count + i] = ids[i];
    for (int l = 0; l < p; ++l) {
      g2[(size_t)i * p + l] = g[(size_t)i * p + l];
      b2[(size_t)i * p + l] = b[(size_t)i * p + l];
      g2[(size_t)(count + i) * p + l] = q->ref[l];
      b2[(size_t)(count + i) * p + l] = q->ref[p + l];
    }
  }
  LQ_RC(expect_chunked(ctx, part, ids2.data(), 2 * count, p, g2.data(), b2.data(), ex.data()));
  std::vector<int32_t> rej;
  std::vector<double> val(count);
  for (int i = 0; i < count; ++i) {
    val[i] = ex[i];
    int verdict = 0;                                  // keep the prediction
    if (ex[i] < ex[count + i]) {
      if (ex[i] >= ex[count + i] - tol * (double)std::max<int64_t>(weight[ids[i]], 1)) {
        verdict = 2;                                  // the reference is better by less than tol W: take it
        val[i] = ex[count + i];
        for (int l = 0; l < p; ++l) {
          g[(size_t)i * p + l] = q->ref[l];
          b[(size_t)i * p + l] = q->ref[p + l];
        }
      } else {
        verdict = 1;                                  // the network missed: plain form
        rej.push_back(i);
      }
    }
    if (fallback_out) fallback_out[i] = verdict;
  }
  if (!rej.empty()) {
    std::vector<int32_t> rid(rej.size());
    for (size_t k = 0; k < rej.size(); ++k) rid[k] = ids[rej[k]];
    std::vector<double> fg(rej.size() * p), fb(rej.size() * p), fv(rej.size());
    LQ_RC(paraqaoa_solve_plain(ctx, part, rid.data(), (int32_t)rid.size(), p, fallback_steps, fg.data(), fb.data(),
                               fv.data()));
    for (size_t k = 0; k < rej.size(); ++k) {
      const int i = rej[k];
      for (int l = 0; l < p; ++l) {
        g[(size_t)i * p + l] = fg[k * p + l];
        b[(size_t)i * p + l] = fb[k * p + l];
      }
      val[i] = fv[k];
    }
  }
  std::copy(g.begin(), g.end(), gamma_out);
  std::copy(b.begin(), b.end(), beta_out);
  if (value_out) std::copy(val.begin(), val.end(), value_out);
  return PARAQAOA_OK;
}

}  // extern "C"
