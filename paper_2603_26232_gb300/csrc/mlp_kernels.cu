// Learned QAOA angles: subgraph features and the 64 -> 256 -> 256 -> 2p MLP,
// trained and evaluated by hand-written kernels with BF16 operands and FP32
// accumulation. The paper leaves angle initialisation open and notes that it
// matters (Sec. 2.2); the network predicts the angles the plain optimiser
// would find, and the solver judges every prediction by <C> and falls back to
// that optimiser.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "pq_internal.h"

namespace pq {

// ---------------------------------------------------------------------------
// Features of one subgraph (kFeatures floats), from its adjacency bit-planes.
// Isolated vertices are left out (they change neither C(z)'s dependence on the
// other qubits nor <C>, so neither the best angles); m = number of vertices
// with at least one edge, all features 0 when m = 0:
//   [0] m / 32           [1] |E| / C(m,2)        [2] mean w / 16    [3] std w / 16
//   [4] mean degree / m  [5] std degree / m      [6] max degree / m [7] min degree / m
//   [8..24)  degree histogram, bin min(deg, 15), counts / m
//   [24..40) weight histogram, bin min(w, 16) - 1, counts / |E|
//   [40..56) weighted-degree histogram, bin min(15, floor(16 D_u / (max D + 1))), counts / m
//   [56] triangles / C(m,3)   [57] total weight / (10 C(m,2))   [58..64) 0
// (degrees over the m non-isolated vertices). One warp per subgraph, lane u
// owns vertex u; histogram bins are integer counts from warp ballots, so every
// entry is one FP32 division.
__global__ void k_features(const SubDev* __restrict__ subs, const uint32_t* __restrict__ planes,
                           const int32_t* __restrict__ ids, int32_t count, float* __restrict__ out) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= count) return;
  const SubDev S = subs[ids[w]];
  const uint32_t* pl = planes + S.plane_off;
  const int n = S.n, P = S.P;
  int deg = 0, wdeg = 0, esum = 0, esq = 0, ecnt = 0, tri = 0;
  int whist_lane[16];
#pragma unroll
  for (int b = 0; b < 16; ++b) whist_lane[b] = 0;
  if (lane < n) {
    uint32_t any = 0;
    for (int b = 0; b < P; ++b) any |= pl[lane * P + b];
    deg = __popc(any);
    for (int b = 0; b < P; ++b) wdeg += __popc(pl[lane * P + b]) << b;
    uint32_t hi = any & ~((2u << lane) - 1u);  // neighbours v > u
    while (hi) {
      const int v = __ffs(hi) - 1;
      hi &= hi - 1;
      int wv = 0;
      for (int b = 0; b < P; ++b) wv |= (int)((pl[lane * P + b] >> v) & 1u) << b;
      esum += wv;
      esq += wv * wv;
      ++ecnt;
      const int bin = min(wv, 16) - 1;
#pragma unroll
      for (int b = 0; b < 16; ++b) whist_lane[b] += (b == bin);
      uint32_t anyv = 0;
      for (int b = 0; b < P; ++b) anyv |= pl[v * P + b];
      tri += __popc(any & anyv & ~((2u << v) - 1u));  // triangles u < v < x
    }
  }
  const bool own = lane < n && deg > 0;  // a non-isolated vertex
  const int m = __popc(__ballot_sync(0xffffffffu, own));
  auto wsum = [](int x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
  };
  const int E = wsum(ecnt), Wt = wsum(esum), Wsq = wsum(esq), T = wsum(tri);
  const int dsum = wsum(deg), dsq = wsum(deg * deg);
  int dmax = own ? deg : -1, dmin = own ? deg : (1 << 30), wdmax = own ? wdeg : 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dmax = max(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    dmin = min(dmin, __shfl_xor_sync(0xffffffffu, dmin, o));
    wdmax = max(wdmax, __shfl_xor_sync(0xffffffffu, wdmax, o));
  }
  const int dbin = min(deg, 15);
  const int wdbin = min(15, (16 * wdeg) / (wdmax + 1));
  float* f = out + (int64_t)w * kFeatures;
  if (m == 0) {  // edgeless: every feature 0
    f[lane] = 0.f;
    f[32 + lane] = 0.f;
    return;
  }
  const float fm = (float)m, pairs = 0.5f * fm * (fm - 1.f);
  const float triples = fm * (fm - 1.f) * (fm - 2.f) / 6.f;
  // lane b < 16 writes the three histograms' bin b; the others the scalars and zeros
  int hd = 0, hw = 0, hwd = 0;
#pragma unroll
  for (int b = 0; b < 16; ++b) {
    const int cd = __popc(__ballot_sync(0xffffffffu, own && dbin == b));
    const int cwd = __popc(__ballot_sync(0xffffffffu, own && wdbin == b));
    const int cw = wsum(whist_lane[b]);
    if (lane == b) {
      hd = cd;
      hwd = cwd;
      hw = cw;
    }
  }
  if (lane < 16) {
    f[8 + lane] = (float)hd / fm;
    f[24 + lane] = (float)hw / (float)E;
    f[40 + lane] = (float)hwd / fm;
  } else if (lane == 16) {
    f[0] = fm / 32.f;
    f[1] = (float)E / pairs;
    const float mw = (float)Wt / (float)E;
    f[2] = mw / 16.f;
    f[3] = sqrtf(fmaxf((float)Wsq / (float)E - mw * mw, 0.f)) / 16.f;
    const float md = (float)dsum / fm;
    f[4] = md / fm;
    f[5] = sqrtf(fmaxf((float)dsq / fm - md * md, 0.f)) / fm;
    f[6] = (float)dmax / fm;
    f[7] = (float)dmin / fm;
  } else if (lane == 17) {
    f[56] = triples > 0.f ? (float)T / triples : 0.f;
    f[57] = (float)Wt / (10.f * pairs);
  } else if (lane < 24) {
    f[58 + (lane - 18)] = 0.f;
  }
}

cudaError_t launch_features(const SubDev* subs, const uint32_t* planes, const int32_t* ids, int32_t count,
                            float* out, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  k_features<<<(count * 32 + 127) / 128, 128, 0, st>>>(subs, planes, ids, count, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// C[M x N] (FP32) = op(A) op(B), op(A) M x K, op(B) K x N, BF16 operands,
// FP32 accumulation in a fixed order (k ascending). TA: A is stored K x M;
// TB: B is stored N x K. Epilogue: + bias[N] (optional), ReLU (optional),
// BF16 copy Cb (optional). 64 x 64 tiles, 256 threads, 4 x 4 outputs per
// thread, K-steps of 16 through shared memory.
template <bool TA, bool TB>
__global__ void __launch_bounds__(256)
    k_gemm_bf16(int M, int N, int K, const __nv_bfloat16* __restrict__ A, int lda,
                const __nv_bfloat16* __restrict__ B, int ldb, float* __restrict__ C, int ldc,
                const float* __restrict__ bias, int relu, __nv_bfloat16* __restrict__ Cb) {
  __shared__ float As[16][64 + 1];
  __shared__ float Bs[16][64 + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int e = threadIdx.x; e < 16 * 64; e += 256) {
      // element (kk, mm) of the A tile and (kk, nn) of the B tile; the index
      // order follows each operand's storage so that loads are coalesced
      int kk, mm;
      if (TA) { kk = e / 64; mm = e % 64; } else { mm = e / 16; kk = e % 16; }
      const int gm = m0 + mm, gk = k0 + kk;
      float va = 0.f;
      if (gm < M && gk < K) va = __bfloat162float(TA ? A[(int64_t)gk * lda + gm] : A[(int64_t)gm * lda + gk]);
      As[kk][mm] = va;
      int kb, nn;
      if (TB) { nn = e / 16; kb = e % 16; } else { kb = e / 64; nn = e % 64; }
      const int gn = n0 + nn, gkb = k0 + kb;
      float vb = 0.f;
      if (gn < N && gkb < K) vb = __bfloat162float(TB ? B[(int64_t)gn * ldb + gkb] : B[(int64_t)gkb * ldb + gn]);
      Bs[kb][nn] = vb;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty * 4 + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx * 4 + j;
      if (gn >= N) continue;
      float v = acc[i][j] + (bias ? bias[gn] : 0.f);
      if (relu) v = fmaxf(v, 0.f);
      C[(int64_t)gm * ldc + gn] = v;
      if (Cb) Cb[(int64_t)gm * ldc + gn] = __float2bfloat16(v);
    }
  }
}

cudaError_t launch_gemm_bf16(bool ta, bool tb, int M, int N, int K, const __nv_bfloat16* A, int lda,
                             const __nv_bfloat16* B, int ldb, float* C, int ldc, const float* bias,
                             int relu, __nv_bfloat16* Cb, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  dim3 grid((N + 63) / 64, (M + 63) / 64);
  if (!ta && !tb) k_gemm_bf16<false, false><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, relu, Cb);
  else if (ta && !tb) k_gemm_bf16<true, false><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, relu, Cb);
  else if (!ta && tb) k_gemm_bf16<false, true><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, relu, Cb);
  else k_gemm_bf16<true, true><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, relu, Cb);
  return cudaGetLastError();
}

static unsigned nblk(int64_t n) { return (unsigned)std::min<int64_t>(std::max<int64_t>((n + 255) / 256, 1), 152 * 8); }

// FP32 -> BF16 (round to nearest even).
__global__ void k_to_bf16(const float* __restrict__ x, __nv_bfloat16* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16(x[i]);
}

// Minibatch gather: rows idx[0..rows) of X (FP32, cols wide) -> BF16 Xb, and
// of T (FP32, tcols wide) -> Tb (FP32).
__global__ void k_gather_rows(const float* __restrict__ X, int cols, const float* __restrict__ T, int tcols,
                              const int32_t* __restrict__ idx, int rows, __nv_bfloat16* __restrict__ Xb,
                              float* __restrict__ Tb) {
  const int64_t nx = (int64_t)rows * cols, nt = (int64_t)rows * tcols;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nx + nt; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < nx) {
      const int r = (int)(i / cols), cc = (int)(i % cols);
      Xb[i] = __float2bfloat16(X[(int64_t)idx[r] * cols + cc]);
    } else if (T) {
      const int64_t j = i - nx;
      const int r = (int)(j / tcols), cc = (int)(j % tcols);
      Tb[j] = T[(int64_t)idx[r] * tcols + cc];
    }
  }
}

// MSE head: dY = 2 (Y - T) / n (FP32, plus BF16 copy); loss[slot] = sum (Y - T)^2 / n
// summed in FP64 in a fixed order (one CTA).
__global__ void __launch_bounds__(256) k_mse_grad(const float* __restrict__ Y, const float* __restrict__ T, int64_t n,
                                                  float* __restrict__ dY, __nv_bfloat16* __restrict__ dYb,
                                                  double* __restrict__ loss) {
  __shared__ double red[8];
  double acc = 0.0;
  const float s = 2.f / (float)n;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const float d = Y[i] - T[i];
    acc += (double)d * (double)d;
    const float g = s * d;
    dY[i] = g;
    dYb[i] = __float2bfloat16(g);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    *loss = t / (double)n;
  }
}

// dZ = dH [Z > 0] in place, with a BF16 copy.
__global__ void k_relu_back(float* __restrict__ dH, const float* __restrict__ Z, int64_t n,
                            __nv_bfloat16* __restrict__ dZb) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float v = Z[i] > 0.f ? dH[i] : 0.f;
    dH[i] = v;
    dZb[i] = __float2bfloat16(v);
  }
}

// db[j] = sum_i dZ[i, j], rows ascending (FP32).
__global__ void k_colsum(const float* __restrict__ dZ, int rows, int cols, float* __restrict__ db) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cols) return;
  float s = 0.f;
  for (int i = 0; i < rows; ++i) s += dZ[(int64_t)i * cols + j];
  db[j] = s;
}

// Adam (Kingma and Ba, 2015) on FP32 master weights; refreshes the BF16 copy.
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float bc1,
                       float bc2, __nv_bfloat16* __restrict__ wb) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    w[i] = wi;
    wb[i] = __float2bfloat16(wi);
  }
}

cudaError_t launch_to_bf16(const float* x, __nv_bfloat16* y, int64_t n, cudaStream_t st) {
  k_to_bf16<<<nblk(n), 256, 0, st>>>(x, y, n);
  return cudaGetLastError();
}
cudaError_t launch_gather_rows(const float* X, int cols, const float* T, int tcols, const int32_t* idx, int rows,
                               __nv_bfloat16* Xb, float* Tb, cudaStream_t st) {
  k_gather_rows<<<nblk((int64_t)rows * (cols + tcols)), 256, 0, st>>>(X, cols, T, tcols, idx, rows, Xb, Tb);
  return cudaGetLastError();
}
cudaError_t launch_mse_grad(const float* Y, const float* T, int64_t n, float* dY, __nv_bfloat16* dYb,
                            double* loss, cudaStream_t st) {
  k_mse_grad<<<1, 256, 0, st>>>(Y, T, n, dY, dYb, loss);
  return cudaGetLastError();
}
cudaError_t launch_relu_back(float* dH, const float* Z, int64_t n, __nv_bfloat16* dZb, cudaStream_t st) {
  k_relu_back<<<nblk(n), 256, 0, st>>>(dH, Z, n, dZb);
  return cudaGetLastError();
}
cudaError_t launch_colsum(const float* dZ, int rows, int cols, float* db, cudaStream_t st) {
  k_colsum<<<(cols + 127) / 128, 128, 0, st>>>(dZ, rows, cols, db);
  return cudaGetLastError();
}
cudaError_t launch_adam(float* w, const float* g, float* m, float* v, int64_t n, float lr, int t,
                        __nv_bfloat16* wb, cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f;
  k_adam<<<nblk(n), 256, 0, st>>>(w, g, m, v, n, lr, b1, b2, 1e-8f, 1.f - powf(b1, (float)t),
                                  1.f - powf(b2, (float)t), wb);
  return cudaGetLastError();
}

static_assert(sizeof(__nv_bfloat16) == sizeof(bf16_t), "BF16 storage is 16 bits");
static const __nv_bfloat16* bfc(const bf16_t* p) { return reinterpret_cast<const __nv_bfloat16*>(p); }
static __nv_bfloat16* bfm(bf16_t* p) { return reinterpret_cast<__nv_bfloat16*>(p); }

cudaError_t launch_gemm_bf16_raw(bool ta, bool tb, int M, int N, int K, const bf16_t* A, int lda, const bf16_t* B,
                                 int ldb, float* C, int ldc, const float* bias, int relu, bf16_t* Cb, cudaStream_t st) {
  return launch_gemm_bf16(ta, tb, M, N, K, bfc(A), lda, bfc(B), ldb, C, ldc, bias, relu, bfm(Cb), st);
}
cudaError_t launch_to_bf16_raw(const float* x, bf16_t* y, int64_t n, cudaStream_t st) {
  return launch_to_bf16(x, bfm(y), n, st);
}
cudaError_t launch_gather_rows_raw(const float* X, int cols, const float* T, int tcols, const int32_t* idx, int rows,
                                   bf16_t* Xb, float* Tb, cudaStream_t st) {
  return launch_gather_rows(X, cols, T, tcols, idx, rows, bfm(Xb), Tb, st);
}
cudaError_t launch_mse_grad_raw(const float* Y, const float* T, int64_t n, float* dY, bf16_t* dYb, double* loss,
                                cudaStream_t st) {
  return launch_mse_grad(Y, T, n, dY, bfm(dYb), loss, st);
}
cudaError_t launch_relu_back_raw(float* dH, const float* Z, int64_t n, bf16_t* dZb, cudaStream_t st) {
  return launch_relu_back(dH, Z, n, bfm(dZb), st);
}
cudaError_t launch_adam_raw(float* w, const float* g, float* m, float* v, int64_t n, float lr, int t, bf16_t* wb,
                            cudaStream_t st) {
  return launch_adam(w, g, m, v, n, lr, t, bfm(wb), st);
}

}  // namespace pq
