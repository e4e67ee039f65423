// Angle loop on the device: grid argmax and fixed-iteration Adam with
// central-difference gradients, FP64 scalars throughout.
//
// The paper fixes neither the optimiser nor its initialisation (Sec. 2.2
// names gradient descent or evolutionary strategies and notes that the
// initialisation matters); the reading implemented here is a p = 1 grid,
// INTERP initialisation for deeper circuits and Adam on f = -<C>/W.
#include <cuda_runtime.h>

#include "pq_internal.h"

namespace pq {

// vals[s*G + a*points + b] -> first maximum per subgraph (row-major order).
__global__ void k_grid_argmax(const double* __restrict__ vals, int32_t S, int32_t points,
                              const double* __restrict__ gscale, double* __restrict__ gamma,
                              double* __restrict__ beta, double* __restrict__ best) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const int G = points * points;
  const double* v = vals + (int64_t)s * G;
  int arg = 0;
  double bv = v[0];
  for (int k = 1; k < G; ++k)
    if (v[k] > bv) {
      bv = v[k];
      arg = k;
    }
  const double pi = 3.14159265358979323846;
  gamma[s] = pi * (double)(arg / points) / ((double)points * (gscale ? gscale[s] : 1.0));
  beta[s] = 0.5 * pi * (double)(arg % points) / (double)points;
  best[s] = bv;
}

// Angles of the 4p shifted evaluations per subgraph: theta +- h e_k, in the
// order (k = 0, +), (k = 0, -), (k = 1, +), ... ; theta = (gamma_0..p-1, beta_0..p-1).
// Also advances the Adam step counter *step (read by k_adam_update), so that
// one captured step can be replayed as a CUDA graph.
__global__ void k_adam_shifts(const double* __restrict__ theta, int32_t S, int32_t p, double h,
                              double* __restrict__ gamma, double* __restrict__ beta, int32_t* __restrict__ step) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) *step += 1;
  const int E = 4 * p;
  if (t >= (int64_t)S * E) return;
  const int s = (int)(t / E), e = (int)(t % E);
  const int k = e >> 1;
  const double d = (e & 1) ? -h : h;
  const double* th = theta + (int64_t)s * 2 * p;
  for (int l = 0; l < p; ++l) {
    gamma[t * p + l] = th[l] + (k == l ? d : 0.0);
    beta[t * p + l] = th[p + l] + (k == p + l ? d : 0.0);
  }
}

__global__ void k_adam_update(const double* __restrict__ expect, const double* __restrict__ wsum,
                              int32_t S, int32_t p, double h, double lr, const int32_t* __restrict__ step,
                              double* __restrict__ theta, double* __restrict__ m,
                              double* __restrict__ v) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int t = *step;
  const int D = 2 * p;
  if (q >= (int64_t)S * D) return;
  const int s = (int)(q / D), k = (int)(q % D);
  const double W = wsum[s];
  const double fp = -expect[(int64_t)s * 4 * p + 2 * k] / W;
  const double fm = -expect[(int64_t)s * 4 * p + 2 * k + 1] / W;
  const double g = (fp - fm) / (2.0 * h);
  const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
  const double mm = b1 * m[q] + (1.0 - b1) * g;
  const double vv = b2 * v[q] + (1.0 - b2) * g * g;
  m[q] = mm;
  v[q] = vv;
  // bias corrections b^t by binary powering: t is the step count, and a
  // chain of a few FP64 multiplies is far shorter than pow() on the narrow
  // FP64 pipe (relative difference ~1e-15)
  double p1 = 1.0, p2 = 1.0, q1 = b1, q2 = b2;
  for (int e = t; e > 0; e >>= 1) {
    if (e & 1) {
      p1 *= q1;
      p2 *= q2;
    }
    q1 *= q1;
    q2 *= q2;
  }
  const double mh = mm / (1.0 - p1);
  const double vh = vv / (1.0 - p2);
  theta[q] -= lr * mh / (sqrt(vh) + eps);
}

__global__ void k_theta_split(const double* __restrict__ theta, int32_t S, int32_t p,
                              double* __restrict__ gamma, double* __restrict__ beta) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)S * p) return;
  const int64_t s = q / p;
  const int l = (int)(q % p);
  gamma[q] = theta[s * 2 * p + l];
  beta[q] = theta[s * 2 * p + p + l];
}

static unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t launch_grid_argmax(const double* vals, int32_t S, int32_t points, const double* gscale, double* gamma,
                               double* beta, double* best, cudaStream_t st) {
  k_grid_argmax<<<nblk(S, 128), 128, 0, st>>>(vals, S, points, gscale, gamma, beta, best);
  return cudaGetLastError();
}

cudaError_t launch_adam_shifts(const double* theta, int32_t S, int32_t p, double h, double* gamma,
                               double* beta, int32_t* step, cudaStream_t st) {
  k_adam_shifts<<<nblk((int64_t)S * 4 * p, 128), 128, 0, st>>>(theta, S, p, h, gamma, beta, step);
  return cudaGetLastError();
}

cudaError_t launch_adam_update(const double* expect, const double* wsum, int32_t S, int32_t p,
                               double h, double lr, const int32_t* step, double* theta, double* m, double* v,
                               cudaStream_t st) {
  k_adam_update<<<nblk((int64_t)S * 2 * p, 128), 128, 0, st>>>(expect, wsum, S, p, h, lr, step, theta, m, v);
  return cudaGetLastError();
}

cudaError_t launch_theta_split(const double* theta, int32_t S, int32_t p, double* gamma,
                               double* beta, cudaStream_t st) {
  k_theta_split<<<nblk((int64_t)S * p, 128), 128, 0, st>>>(theta, S, p, gamma, beta);
  return cudaGetLastError();
}

}  // namespace pq
