// Learned initial guess for the pseudo-time Newton solve (not part of the
// paper, whose Newton iteration starts from zero interior velocity with the
// Dirichlet data in place, section 2.4):
//   y0 = ybar + Phi diag(sigma) f(x),
// Phi a POD basis of solution snapshots (method of snapshots: Gram matrix of
// the centred snapshots, its eigenpairs on the host, Phi = X^T U Sigma^-1),
// f a fully connected tanh network from inflow coefficients, Re and Wo to the
// normalised POD coefficients, trained with Adam (Kingma & Ba 2015) on
// solves of the method itself.  The solver then iterates to the same
// tolerance as from the plain guess: the converged field is the plain method's.
//
// Every product is one FP32 tiled GEMM kernel with a fused epilogue (bias,
// tanh, or the tanh derivative of the backward pass); the problem sizes
// (batch <= a few thousand, width 512, POD rank <= 128) are far below the
// point where tensor cores would pay for the reduced precision.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <random>
#include <vector>

#include "abi_util.h"
#include "kernels.h"

namespace ts {
namespace {

constexpr int GT_M = 64, GT_N = 64, GT_K = 16;
enum { EPI_NONE = 0, EPI_TANH = 1, EPI_DTANH = 2, EPI_ATOMIC = 3 };

// C[M][N] = op(A) op(B) (+ bias[N]) with an epilogue; row-major storage,
// op(A)[i][k] = TA ? A[k lda + i] : A[i lda + k], op(B)[k][j] = TB ? B[j ldb + k] : B[k ldb + j].
// EPI_DTANH multiplies by (1 - aux^2); EPI_ATOMIC adds into C (split-K over blockIdx.z).
template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, const float* __restrict__ A,
                                                   int64_t lda, const float* __restrict__ B, int64_t ldb,
                                                   float* __restrict__ C, int64_t ldc,
                                                   const float* __restrict__ bias,
                                                   const float* __restrict__ aux, int64_t ldaux,
                                                   int k_chunk) {
  __shared__ float As[GT_K][GT_M + 4];
  __shared__ float Bs[GT_K][GT_N + 4];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i0 = blockIdx.y * GT_M, j0 = blockIdx.x * GT_N;
  const int kb = blockIdx.z * k_chunk;
  const int ke = K < kb + k_chunk ? K : kb + k_chunk;
  float acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
  for (int k0 = kb; k0 < ke; k0 += GT_K) {
    for (int t = threadIdx.x; t < GT_M * GT_K; t += 256) {
      const int ii = TA ? t % GT_M : t / GT_K;
      const int kk = TA ? t / GT_M : t % GT_K;
      const int gi = i0 + ii, gk = k0 + kk;
      float v = 0.f;
      if (gi < M && gk < ke) v = TA ? A[(int64_t)gk * lda + gi] : A[(int64_t)gi * lda + gk];
      As[kk][ii] = v;
    }
    for (int t = threadIdx.x; t < GT_N * GT_K; t += 256) {
      const int jj = TB ? t / GT_K : t % GT_N;
      const int kk = TB ? t % GT_K : t / GT_N;
      const int gj = j0 + jj, gk = k0 + kk;
      float v = 0.f;
      if (gj < N && gk < ke) v = TB ? B[(int64_t)gj * ldb + gk] : B[(int64_t)gk * ldb + gj];
      Bs[kk][jj] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GT_K; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int gi = i0 + ty + 16 * r;
    if (gi >= M) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int gj = j0 + tx + 16 * c;
      if (gj >= N) continue;
      float v = acc[r][c];
      if (EPI == EPI_ATOMIC) {
        atomicAdd(&C[(int64_t)gi * ldc + gj], v);
        continue;
      }
      if (bias) v += bias[gj];
      if (EPI == EPI_TANH) v = tanhf(v);
      if (EPI == EPI_DTANH) {
        const float h = aux[(int64_t)gi * ldaux + gj];
        v *= 1.f - h * h;
      }
      C[(int64_t)gi * ldc + gj] = v;
    }
  }
}

template <bool TA, bool TB, int EPI>
int gemm(int M, int N, int K, const float* A, int64_t lda, const float* B, int64_t ldb, float* C,
         int64_t ldc, const float* bias, const float* aux, int64_t ldaux, cudaStream_t st) {
  if (M <= 0 || N <= 0) return 0;
  const int gx = (N + GT_N - 1) / GT_N, gy = (M + GT_M - 1) / GT_M;
  int splits = 1, k_chunk = K;
  if (EPI == EPI_ATOMIC) {
    // enough blocks to fill the GPU; chunks a multiple of the k tile
    const int64_t tiles = (int64_t)gx * gy;
    int64_t want = (4 * 152 + tiles - 1) / tiles;
    int64_t max_split = (K + 4 * GT_K - 1) / (4 * GT_K);
    splits = (int)(want < max_split ? want : max_split);
    if (splits < 1) splits = 1;
    k_chunk = (int)(((K + splits - 1) / splits + GT_K - 1) / GT_K * GT_K);
    splits = (K + k_chunk - 1) / k_chunk;
  }
  if (splits > 65535 || gy > 65535) return -1;
  count_launches(1);
  gemm_kernel<TA, TB, EPI><<<dim3(gx, gy, splits), 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, bias,
                                                                 aux, ldaux, k_chunk);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

// delta = (out - T) / B, partial sums of (out - T)^2 per block
__global__ void loss_kernel(const float* __restrict__ out, const float* __restrict__ T, int64_t n, float invB,
                            float* __restrict__ delta, double* __restrict__ loss) {
  __shared__ double red[8];
  double acc = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float d = out[i] - T[i];
    delta[i] = d * invB;
    acc += (double)d * d;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    loss[blockIdx.x] = s;
  }
}

// db[j] = sum_b delta[b][j]
__global__ void colsum_kernel(const float* __restrict__ delta, int B, int N, float* __restrict__ db) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += delta[(int64_t)b * N + j];
  db[j] = s;
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t n, float lr, float b1, float b2, float c1,
                            float c2, float eps) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// mean over snapshots (FP64), one column per thread
__global__ void mean_kernel(const double* __restrict__ Y, int S, int64_t n, double* __restrict__ mean) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0;
    for (int k = 0; k < S; ++k) s += Y[(int64_t)k * n + i];
    mean[i] = s / S;
  }
}

// X[s][i] = Y[s][i] - mean[i] in FP32
__global__ void center_kernel(const double* __restrict__ Y, const double* __restrict__ mean, int S, int64_t n,
                              float* __restrict__ X) {
  const int64_t total = (int64_t)S * n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x)
    X[t] = (float)(Y[t] - mean[t % n]);
}

// rows idx[b] of src[.][w] into dst[b][w]
__global__ void gather_rows_kernel(const float* __restrict__ src, const int* __restrict__ idx, int B, int w,
                                   float* __restrict__ dst) {
  const int64_t total = (int64_t)B * w;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = t / w, c = t - b * w;
    dst[t] = src[(int64_t)idx[b] * w + c];
  }
}

// y[i] = mean[i] + sum_j Phi[i][j] sigma_j a_j on free entries; fixed entries keep y
__global__ void reconstruct_kernel(const double* __restrict__ mean, const float* __restrict__ phi, int k,
                                   const float* __restrict__ coef, const uint8_t* __restrict__ dmask, int C,
                                   int64_t n, double* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t node = i / (4 * C);
    const int f = (int)((i / C) % 4), c = (int)(i % C);
    if (c == 1) continue;                          // Im of mode 0 stays zero
    if (dmask && f < 3 && dmask[node]) continue;   // Dirichlet velocity keeps its data
    double s = mean[i];
    const float* row = phi + i * k;
    for (int j = 0; j < k; ++j) s += (double)row[j] * coef[j];
    y[i] = s;
  }
}

int grid1(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 8) b = 152 * 8;
  return (int)(b < 1 ? 1 : b);
}

// cyclic Jacobi eigenpairs of a symmetric n x n matrix (host, FP64), descending
void host_sym_eig(std::vector<double>& A, int n, std::vector<double>& w, std::vector<double>& V) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0, dia = 0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) (i == j ? dia : off) += A[(size_t)i * n + j] * A[(size_t)i * n + j];
    if (off <= 1e-30 * dia) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[(size_t)p * n + q];
        if (apq == 0.0) continue;
        const double zeta = (A[(size_t)q * n + q] - A[(size_t)p * n + p]) / (2 * apq);
        double t = 1.0 / (std::fabs(zeta) + std::sqrt(1 + zeta * zeta));
        if (zeta < 0) t = -t;
        const double c = 1 / std::sqrt(1 + t * t), s = t * c;
        for (int k = 0; k < n; ++k) {
          const double ap = A[(size_t)k * n + p], aq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = c * ap - s * aq;
          A[(size_t)k * n + q] = s * ap + c * aq;
        }
        for (int k = 0; k < n; ++k) {
          const double ap = A[(size_t)p * n + k], aq = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = c * ap - s * aq;
          A[(size_t)q * n + k] = s * ap + c * aq;
        }
        for (int k = 0; k < n; ++k) {
          const double vp = V[(size_t)k * n + p], vq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = c * vp - s * vq;
          V[(size_t)k * n + q] = s * vp + c * vq;
        }
      }
  }
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::sort(order.begin(), order.end(),
            [&](int a, int b) { return A[(size_t)a * n + a] > A[(size_t)b * n + b]; });
  std::vector<double> Vs((size_t)n * n);
  w.resize(n);
  for (int j = 0; j < n; ++j) {
    w[j] = A[(size_t)order[j] * n + order[j]];
    for (int i = 0; i < n; ++i) Vs[(size_t)i * n + j] = V[(size_t)i * n + order[j]];
  }
  V.swap(Vs);
}

}  // namespace
}  // namespace ts

using namespace ts;

struct ts_surrogate {
  std::vector<int> sizes;            // n_in, hidden..., n_out
  std::vector<int64_t> w_off, b_off; // offsets into the flat parameter vector
  int64_t n_params = 0;
  int64_t n_dof = 0;
  float *d_p = nullptr, *d_m = nullptr, *d_v = nullptr, *d_g = nullptr;
  int adam_t = 0;
  // activations for a batch of up to bmax rows
  int bmax = 0;
  std::vector<float*> d_h;           // h_0 .. h_L (h_L = output)
  float *d_delta0 = nullptr, *d_delta1 = nullptr, *d_T = nullptr;
  double* d_loss = nullptr;
  int* d_idx = nullptr;
  // POD
  int k = 0;                         // fitted rank
  double* d_mean = nullptr;
  float* d_phi = nullptr;            // [n_dof][n_out]
  std::vector<double> sigma;
  float* d_coef = nullptr;
};

namespace {

int ensure_batch(ts_surrogate* s, int B) {
  if (B <= s->bmax) return 0;
  for (float*& p : s->d_h) dfree(p);
  dfree(s->d_delta0);
  dfree(s->d_delta1);
  dfree(s->d_T);
  dfree(s->d_idx);
  const int L = (int)s->sizes.size() - 1;
  s->d_h.assign(L + 1, nullptr);
  int wmax = 0;
  for (int l = 0; l <= L; ++l) {
    TS_TRY(dalloc(&s->d_h[l], (size_t)B * s->sizes[l]));
    wmax = std::max(wmax, s->sizes[l]);
  }
  TS_TRY(dalloc(&s->d_delta0, (size_t)B * wmax));
  TS_TRY(dalloc(&s->d_delta1, (size_t)B * wmax));
  TS_TRY(dalloc(&s->d_T, (size_t)B * s->sizes[L]));
  TS_TRY(dalloc(&s->d_idx, (size_t)B));
  s->bmax = B;
  return 0;
}

// forward pass of the batch already in d_h[0]
int forward(ts_surrogate* s, int B, cudaStream_t st) {
  const int L = (int)s->sizes.size() - 1;
  for (int l = 0; l < L; ++l) {
    const int nin = s->sizes[l], nout = s->sizes[l + 1];
    const float* W = s->d_p + s->w_off[l];
    const float* b = s->d_p + s->b_off[l];
    int rc = (l < L - 1)
                 ? gemm<false, true, EPI_TANH>(B, nout, nin, s->d_h[l], nin, W, nin, s->d_h[l + 1], nout, b,
                                               nullptr, 0, st)
                 : gemm<false, true, EPI_NONE>(B, nout, nin, s->d_h[l], nin, W, nin, s->d_h[l + 1], nout, b,
                                               nullptr, 0, st);
    if (rc) return fail(TS_ERR_CUDA, "surrogate forward gemm");
  }
  return 0;
}

// gradient of (1 / 2B) sum ||f(x) - t||^2 for the batch in d_h[0] / d_T, into d_g
int backward(ts_surrogate* s, int B, double* loss_out, cudaStream_t st) {
  const int L = (int)s->sizes.size() - 1;
  const int nout = s->sizes[L];
  const int lb = grid1((int64_t)B * nout);
  count_launches(1);
  loss_kernel<<<lb, 256, 0, st>>>(s->d_h[L], s->d_T, (int64_t)B * nout, 1.f / B, s->d_delta0, s->d_loss);
  float* delta = s->d_delta0;
  float* other = s->d_delta1;
  for (int l = L - 1; l >= 0; --l) {
    const int nin = s->sizes[l], no = s->sizes[l + 1];
    // dW_l = delta^T h_l ; db_l = column sums of delta
    if (gemm<true, false, EPI_NONE>(no, nin, B, delta, no, s->d_h[l], nin, s->d_g + s->w_off[l], nin, nullptr,
                                    nullptr, 0, st))
      return fail(TS_ERR_CUDA, "surrogate dW gemm");
    count_launches(1);
    colsum_kernel<<<(no + 127) / 128, 128, 0, st>>>(delta, B, no, s->d_g + s->b_off[l]);
    if (l > 0) {
      // delta_{l-1} = (delta W_l) * (1 - h_l^2)
      if (gemm<false, false, EPI_DTANH>(B, nin, no, delta, no, s->d_p + s->w_off[l], nin, other, nin, nullptr,
                                        s->d_h[l], nin, st))
        return fail(TS_ERR_CUDA, "surrogate delta gemm");
      std::swap(delta, other);
    }
  }
  if (loss_out) {
    std::vector<double> part(lb);
    TS_CUDA(cudaMemcpyAsync(part.data(), s->d_loss, lb * sizeof(double), cudaMemcpyDeviceToHost, st));
    TS_CUDA(cudaStreamSynchronize(st));
    double sum = 0;
    for (double x : part) sum += x;
    *loss_out = 0.5 * sum / B;
  }
  return 0;
}

int adam(ts_surrogate* s, double lr, cudaStream_t st) {
  ++s->adam_t;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)s->adam_t), c2 = 1.f - std::pow(b2, (float)s->adam_t);
  count_launches(1);
  adam_kernel<<<grid1(s->n_params), 256, 0, st>>>(s->d_p, s->d_g, s->d_m, s->d_v, s->n_params, (float)lr, b1,
                                                  b2, c1, c2, 1e-8f);
  return cudaGetLastError() == cudaSuccess ? 0 : fail(TS_ERR_CUDA, "adam kernel");
}

}  // namespace

extern "C" {

int ts_surrogate_create(int n_in, int hidden, int n_hidden_layers, int n_out, int64_t n_dof, uint64_t seed,
                        ts_surrogate** out) {
  if (!out) return fail(TS_ERR_ARG, "NULL output handle");
  *out = nullptr;
  if (n_in <= 0 || hidden <= 0 || n_hidden_layers < 0 || n_out <= 0 || n_dof < 0 || n_out > 1024)
    return fail(TS_ERR_ARG, "surrogate sizes out of range");
  ts_surrogate* s = new ts_surrogate();
  s->sizes.push_back(n_in);
  for (int l = 0; l < n_hidden_layers; ++l) s->sizes.push_back(hidden);
  s->sizes.push_back(n_out);
  s->n_dof = n_dof;
  const int L = (int)s->sizes.size() - 1;
  int64_t off = 0;
  for (int l = 0; l < L; ++l) {
    s->w_off.push_back(off);
    off += (int64_t)s->sizes[l] * s->sizes[l + 1];
    s->b_off.push_back(off);
    off += s->sizes[l + 1];
  }
  s->n_params = off;
  // weights ~ U(-1/sqrt(n_in), 1/sqrt(n_in)), biases zero (53-bit uniforms from a 64-bit Mersenne twister)
  std::vector<float> host(off, 0.f);
  std::mt19937_64 rng(seed);
  for (int l = 0; l < L; ++l) {
    const double lim = 1.0 / std::sqrt((double)s->sizes[l]);
    for (int64_t i = 0; i < (int64_t)s->sizes[l] * s->sizes[l + 1]; ++i) {
      const double u = (double)(rng() >> 11) * (1.0 / 9007199254740992.0);
      host[s->w_off[l] + i] = (float)((2 * u - 1) * lim);
    }
  }
  int rc = 0;
  if ((rc = dalloc(&s->d_p, off)) || (rc = dalloc(&s->d_m, off)) || (rc = dalloc(&s->d_v, off)) ||
      (rc = dalloc(&s->d_g, off)) || (rc = dalloc(&s->d_loss, 152 * 8)) || (rc = dalloc(&s->d_coef, n_out))) {
    ts_surrogate_free(s);
    return rc;
  }
  if (cudaMemcpy(s->d_p, host.data(), off * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(s->d_m, 0, off * sizeof(float)) != cudaSuccess ||
      cudaMemset(s->d_v, 0, off * sizeof(float)) != cudaSuccess) {
    ts_surrogate_free(s);
    return fail(TS_ERR_CUDA, "surrogate initialisation copy");
  }
  *out = s;
  return 0;
}

void ts_surrogate_free(ts_surrogate* s) {
  if (!s) return;
  cudaDeviceSynchronize();
  for (float*& p : s->d_h) dfree(p);
  dfree(s->d_p);
  dfree(s->d_m);
  dfree(s->d_v);
  dfree(s->d_g);
  dfree(s->d_delta0);
  dfree(s->d_delta1);
  dfree(s->d_T);
  dfree(s->d_loss);
  dfree(s->d_idx);
  dfree(s->d_mean);
  dfree(s->d_phi);
  dfree(s->d_coef);
  delete s;
}

int64_t ts_surrogate_num_params(const ts_surrogate* s) { return s ? s->n_params : -1; }

int ts_surrogate_get_params(const ts_surrogate* s, float* host, int64_t n) {
  if (!s || !host || n != s->n_params) return fail(TS_ERR_ARG, "parameter buffer size mismatch");
  TS_CUDA(cudaMemcpy(host, s->d_p, n * sizeof(float), cudaMemcpyDeviceToHost));
  return 0;
}

int ts_surrogate_set_params(ts_surrogate* s, const float* host, int64_t n) {
  if (!s || !host || n != s->n_params) return fail(TS_ERR_ARG, "parameter buffer size mismatch");
  TS_CUDA(cudaMemcpy(s->d_p, host, n * sizeof(float), cudaMemcpyHostToDevice));
  TS_CUDA(cudaMemset(s->d_m, 0, n * sizeof(float)));
  TS_CUDA(cudaMemset(s->d_v, 0, n * sizeof(float)));
  s->adam_t = 0;
  return 0;
}

int ts_surrogate_forward(ts_surrogate* s, const float* X, int B, float* out, void* stream) {
  if (!s || !X || !out || B <= 0) return fail(TS_ERR_ARG, "ts_surrogate_forward: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  TS_TRY(ensure_batch(s, B));
  const int L = (int)s->sizes.size() - 1;
  TS_CUDA(cudaMemcpyAsync(s->d_h[0], X, (size_t)B * s->sizes[0] * sizeof(float), cudaMemcpyDeviceToDevice, st));
  TS_TRY(forward(s, B, st));
  TS_CUDA(cudaMemcpyAsync(out, s->d_h[L], (size_t)B * s->sizes[L] * sizeof(float), cudaMemcpyDeviceToDevice, st));
  return 0;
}

int ts_surrogate_gradient(ts_surrogate* s, const float* X, const float* T, int B, float* grad, double* loss,
                          void* stream) {
  if (!s || !X || !T || B <= 0) return fail(TS_ERR_ARG, "ts_surrogate_gradient: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  TS_TRY(ensure_batch(s, B));
  const int L = (int)s->sizes.size() - 1;
  TS_CUDA(cudaMemcpyAsync(s->d_h[0], X, (size_t)B * s->sizes[0] * sizeof(float), cudaMemcpyDeviceToDevice, st));
  TS_CUDA(cudaMemcpyAsync(s->d_T, T, (size_t)B * s->sizes[L] * sizeof(float), cudaMemcpyDeviceToDevice, st));
  TS_TRY(forward(s, B, st));
  TS_TRY(backward(s, B, loss, st));
  if (grad) TS_CUDA(cudaMemcpyAsync(grad, s->d_g, s->n_params * sizeof(float), cudaMemcpyDeviceToDevice, st));
  return 0;
}

int ts_surrogate_adam(ts_surrogate* s, const float* grad, double lr, void* stream) {
  if (!s || !grad || !(lr > 0)) return fail(TS_ERR_ARG, "ts_surrogate_adam: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  if (grad != s->d_g)
    TS_CUDA(cudaMemcpyAsync(s->d_g, grad, s->n_params * sizeof(float), cudaMemcpyDeviceToDevice, st));
  return adam(s, lr, st);
}

int ts_surrogate_fit_basis(ts_surrogate* s, const double* Y, int S, void* stream) {
  if (!s || !Y || S < 2) return fail(TS_ERR_ARG, "ts_surrogate_fit_basis: need >= 2 snapshots");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = s->n_dof;
  const int kmax = s->sizes.back();
  dfree(s->d_mean);
  dfree(s->d_phi);
  TS_TRY(dalloc(&s->d_mean, n));
  TS_TRY(dalloc(&s->d_phi, (size_t)n * kmax));
  float *X = nullptr, *G = nullptr, *U = nullptr;
  TS_TRY(dalloc(&X, (size_t)S * n));
  int rc = 0;
  do {
    if ((rc = dalloc(&G, (size_t)S * S)) || (rc = dalloc(&U, (size_t)S * kmax))) break;
    count_launches(2);
    mean_kernel<<<grid1(n), 256, 0, st>>>(Y, S, n, s->d_mean);
    center_kernel<<<grid1((int64_t)S * n), 256, 0, st>>>(Y, s->d_mean, S, n, X);
    if (cudaMemsetAsync(G, 0, (size_t)S * S * sizeof(float), st) != cudaSuccess) { rc = fail(TS_ERR_CUDA, "memset"); break; }
    // Gram matrix X X^T (split over the long dimension)
    if (gemm<false, true, EPI_ATOMIC>(S, S, (int)std::min<int64_t>(n, INT32_MAX), X, n, X, n, G, S, nullptr,
                                      nullptr, 0, st)) { rc = fail(TS_ERR_CUDA, "gram gemm"); break; }
    std::vector<float> g32((size_t)S * S);
    if (cudaMemcpyAsync(g32.data(), G, g32.size() * sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) { rc = fail(TS_ERR_CUDA, "gram copy"); break; }
    std::vector<double> A((size_t)S * S), w, V;
    for (int i = 0; i < S; ++i)
      for (int j = 0; j < S; ++j) A[(size_t)i * S + j] = 0.5 * ((double)g32[(size_t)i * S + j] + g32[(size_t)j * S + i]);
    host_sym_eig(A, S, w, V);
    const double wmax = w.empty() ? 0 : w[0];
    int k = 0;
    while (k < kmax && k < S && w[k] > 1e-10 * wmax && w[k] > 0) ++k;
    if (k == 0) { rc = fail(TS_ERR_ARG, "snapshots have no variation"); break; }
    s->k = k;
    s->sigma.assign(k, 0.0);
    // U'[s][j] = V[s][j] / sigma_j, zero beyond the fitted rank
    std::vector<float> up((size_t)S * kmax, 0.f);
    for (int j = 0; j < k; ++j) {
      s->sigma[j] = std::sqrt(w[j]);
      for (int i = 0; i < S; ++i) up[(size_t)i * kmax + j] = (float)(V[(size_t)i * S + j] / s->sigma[j]);
    }
    if (cudaMemcpyAsync(U, up.data(), up.size() * sizeof(float), cudaMemcpyHostToDevice, st) != cudaSuccess) {
      rc = fail(TS_ERR_CUDA, "basis copy");
      break;
    }
    // Phi = X^T U'  ([n][S] x [S][kmax])
    if (gemm<true, false, EPI_NONE>((int)std::min<int64_t>(n, INT32_MAX), kmax, S, X, n, U, kmax, s->d_phi, kmax,
                                    nullptr, nullptr, 0, st)) { rc = fail(TS_ERR_CUDA, "basis gemm"); break; }
    if (cudaStreamSynchronize(st) != cudaSuccess) { rc = fail(TS_ERR_CUDA, "basis sync"); break; }
  } while (0);
  dfree(X);
  dfree(G);
  dfree(U);
  return rc;
}

int ts_surrogate_basis_rank(const ts_surrogate* s, double* sigma_host) {
  if (!s) return fail(TS_ERR_ARG, "NULL surrogate");
  if (sigma_host)
    for (int j = 0; j < s->k; ++j) sigma_host[j] = s->sigma[j];
  return s->k;
}

int ts_surrogate_coefficients(ts_surrogate* s, const double* Y, int S, float* A, void* stream) {
  if (!s || !Y || !A || S <= 0 || s->k == 0) return fail(TS_ERR_ARG, "ts_surrogate_coefficients: fit a basis first");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = s->n_dof;
  const int kmax = s->sizes.back();
  float* X = nullptr;
  TS_TRY(dalloc(&X, (size_t)S * n));
  int rc = 0;
  do {
    count_launches(1);
    center_kernel<<<grid1((int64_t)S * n), 256, 0, st>>>(Y, s->d_mean, S, n, X);
    if (cudaMemsetAsync(A, 0, (size_t)S * kmax * sizeof(float), st) != cudaSuccess) { rc = fail(TS_ERR_CUDA, "memset"); break; }
    // A = X Phi ([S][n] x [n][kmax]), then / sigma on the host-known rank
    if (gemm<false, false, EPI_ATOMIC>(S, kmax, (int)std::min<int64_t>(n, INT32_MAX), X, n, s->d_phi, kmax, A,
                                       kmax, nullptr, nullptr, 0, st)) { rc = fail(TS_ERR_CUDA, "coef gemm"); break; }
    std::vector<float> a((size_t)S * kmax);
    if (cudaMemcpyAsync(a.data(), A, a.size() * sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) { rc = fail(TS_ERR_CUDA, "coef copy"); break; }
    for (int i = 0; i < S; ++i)
      for (int j = 0; j < kmax; ++j) a[(size_t)i * kmax + j] = j < s->k ? (float)(a[(size_t)i * kmax + j] / s->sigma[j]) : 0.f;
    if (cudaMemcpyAsync(A, a.data(), a.size() * sizeof(float), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) { rc = fail(TS_ERR_CUDA, "coef copy back"); break; }
  } while (0);
  dfree(X);
  return rc;
}

int ts_surrogate_train(ts_surrogate* s, const float* X_host, const double* Y, int S, int epochs, int batch,
                       double lr, uint64_t seed, double* loss_hist, void* stream) {
  if (!s || !X_host || !Y || S <= 0 || epochs <= 0 || batch <= 0 || !(lr > 0))
    return fail(TS_ERR_ARG, "ts_surrogate_train: bad argument");
  if (s->k == 0) return fail(TS_ERR_ARG, "ts_surrogate_train: fit a basis first");
  cudaStream_t st = (cudaStream_t)stream;
  const int nin = s->sizes[0], nout = s->sizes.back();
  const int B = std::min(batch, S);
  TS_TRY(ensure_batch(s, B));
  float *dX = nullptr, *dA = nullptr;
  TS_TRY(dalloc(&dX, (size_t)S * nin));
  int rc = 0;
  do {
    if ((rc = dalloc(&dA, (size_t)S * nout))) break;
    if (cudaMemcpyAsync(dX, X_host, (size_t)S * nin * sizeof(float), cudaMemcpyHostToDevice, st) != cudaSuccess) {
      rc = fail(TS_ERR_CUDA, "input copy");
      break;
    }
    if ((rc = ts_surrogate_coefficients(s, Y, S, dA, st))) break;
    std::mt19937_64 rng(seed);
    std::vector<int> perm(S);
    for (int i = 0; i < S; ++i) perm[i] = i;
    for (int ep = 0; ep < epochs && rc == 0; ++ep) {
      for (int i = S - 1; i > 0; --i) std::swap(perm[i], perm[(int)(rng() % (uint64_t)(i + 1))]);
      double sum = 0;
      int nb = 0;
      for (int b0 = 0; b0 + B <= S; b0 += B) {
        if (cudaMemcpyAsync(s->d_idx, perm.data() + b0, B * sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess) {
          rc = fail(TS_ERR_CUDA, "index copy");
          break;
        }
        count_launches(2);
        gather_rows_kernel<<<grid1((int64_t)B * nin), 256, 0, st>>>(dX, s->d_idx, B, nin, s->d_h[0]);
        gather_rows_kernel<<<grid1((int64_t)B * nout), 256, 0, st>>>(dA, s->d_idx, B, nout, s->d_T);
        double l = 0;
        if ((rc = forward(s, B, st)) || (rc = backward(s, B, &l, st)) || (rc = adam(s, lr, st))) break;
        sum += l;
        ++nb;
      }
      if (loss_hist) loss_hist[ep] = nb ? sum / nb : 0.0;
    }
  } while (0);
  cudaStreamSynchronize(st);
  dfree(dX);
  dfree(dA);
  return rc;
}

}  // extern "C"

// the problem's Dirichlet mask (api.cu)
namespace ts {
int problem_fixed_mask(ts_problem* pr, const uint8_t** dmask, int* C, int64_t* n);
}

extern "C" int ts_surrogate_guess(ts_surrogate* s, ts_problem* prob, const float* x_host, double* y_inout,
                                  void* stream) {
  if (!s || !prob || !x_host || !y_inout) return fail(TS_ERR_ARG, "ts_surrogate_guess: NULL argument");
  if (s->k == 0) return fail(TS_ERR_ARG, "ts_surrogate_guess: fit a basis first");
  cudaStream_t st = (cudaStream_t)stream;
  const uint8_t* dmask = nullptr;
  int C = 0;
  int64_t n = 0;
  TS_TRY(problem_fixed_mask(prob, &dmask, &C, &n));
  if (n != s->n_dof) return fail(TS_ERR_ARG, "ts_surrogate_guess: field size differs from the basis");
  TS_TRY(ensure_batch(s, 1));
  const int L = (int)s->sizes.size() - 1, kmax = s->sizes.back();
  TS_CUDA(cudaMemcpyAsync(s->d_h[0], x_host, s->sizes[0] * sizeof(float), cudaMemcpyHostToDevice, st));
  TS_TRY(forward(s, 1, st));
  std::vector<float> a(kmax);
  TS_CUDA(cudaMemcpyAsync(a.data(), s->d_h[L], kmax * sizeof(float), cudaMemcpyDeviceToHost, st));
  TS_CUDA(cudaStreamSynchronize(st));
  for (int j = 0; j < kmax; ++j) a[j] = j < s->k ? (float)(a[j] * s->sigma[j]) : 0.f;
  TS_CUDA(cudaMemcpyAsync(s->d_coef, a.data(), kmax * sizeof(float), cudaMemcpyHostToDevice, st));
  count_launches(1);
  reconstruct_kernel<<<grid1(n), 256, 0, st>>>(s->d_mean, s->d_phi, kmax, s->d_coef, dmask, C, n, y_inout);
  TS_CUDA(cudaGetLastError());
  TS_CUDA(cudaStreamSynchronize(st));
  return 0;
}
