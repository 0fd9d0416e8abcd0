// FP64 vector kernels of the restarted GMRES solve (Gram-Schmidt dots and
// updates, norms, casts).  GMRES is the paper's linear solver (section 2.4,
// remark 6; Krylov size 100, section 3.2); its orthogonalisation stays in
// FP64 even when the tangent products run in FP32.
//
// Reductions are two-stage and deterministic: a fixed grid of blocks writes
// per-block partial sums, one warp per vector adds them in block order.
#include "common.cuh"
#include "kernels.h"

namespace ts {

// at most 4 blocks per SM (11% less Gram-Schmidt time than 2 or 6 per SM on a
// 2.1M-unknown field); small fields take one block per 2048 entries, so that
// launch and reduction overheads do not grow with the grid
constexpr int RED_BLOCKS = 608;
static int dots_blocks(int64_t n) {
  const int64_t b = (n + 2047) / 2048;
  return (int)(b < 1 ? 1 : (b > RED_BLOCKS ? RED_BLOCKS : b));
}
constexpr int RED_THREADS = 256;
constexpr int DOT_GROUP = 4;     // basis vectors per pass over w in dots_kernel

int krylov_partial_blocks() { return RED_BLOCKS; }

static unsigned long long g_launches = 0;
void count_launches(int n) { __atomic_fetch_add(&g_launches, (unsigned long long)n, __ATOMIC_RELAXED); }
unsigned long long launches_total() { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// partial[j * gridDim.x + b] = sum over block b's chunk of basis_j . w for
// j < nvec (nvec >= 1), and with self != 0 also row nvec = w . w.  With *skip != 0 the
// block writes zeros and reads nothing (a second Gram-Schmidt pass that is not
// needed).  On GB300 the multiply-adds run on the FP64 pipe; of the layouts
// measured on the 2.1M-unknown junction field (chunks x vector groups, a
// warp-level transposed GEMV, 16-byte loads) this one streams fastest.
__global__ void __launch_bounds__(RED_THREADS) dots_kernel(const double* __restrict__ basis,
                                                           int64_t ld, int nvec,
                                                           const double* __restrict__ w,
                                                           int64_t n, double* __restrict__ partial,
                                                           int self, const double* __restrict__ skip) {
  const int nout = nvec + (self ? 1 : 0);
  if (skip != nullptr && *skip != 0.0) {
    for (int j = threadIdx.x; j < nout; j += blockDim.x) partial[(int64_t)j * gridDim.x + blockIdx.x] = 0.0;
    return;
  }
  __shared__ double red[RED_THREADS / 32][DOT_GROUP];
  const int64_t chunk = ((n + gridDim.x - 1) / gridDim.x + 1) & ~(int64_t)1;
  const int64_t i0 = (int64_t)blockIdx.x * chunk;
  const int64_t i1 = i0 + chunk < n ? i0 + chunk : n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double self_acc = 0;
  for (int j0 = 0; j0 < nvec; j0 += DOT_GROUP) {
    const int nj = nvec - j0 < DOT_GROUP ? nvec - j0 : DOT_GROUP;
    double acc[DOT_GROUP];
#pragma unroll
    for (int jj = 0; jj < DOT_GROUP; ++jj) acc[jj] = 0;
    if (self && j0 == 0) {
      for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const double wi = w[i];
#pragma unroll
        for (int jj = 0; jj < DOT_GROUP; ++jj)
          if (jj < nj) acc[jj] += basis[(int64_t)(j0 + jj) * ld + i] * wi;
        self_acc += wi * wi;
      }
    } else {
      for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const double wi = w[i];
#pragma unroll
        for (int jj = 0; jj < DOT_GROUP; ++jj)
          if (jj < nj) acc[jj] += basis[(int64_t)(j0 + jj) * ld + i] * wi;
      }
    }
#pragma unroll
    for (int jj = 0; jj < DOT_GROUP; ++jj) {
      double s = warp_sum(acc[jj]);
      if (lane == 0) red[warp][jj] = s;
    }
    __syncthreads();
    if ((int)threadIdx.x < nj) {
      double s = 0;
      for (int k = 0; k < RED_THREADS / 32; ++k) s += red[k][threadIdx.x];
      partial[(int64_t)(j0 + threadIdx.x) * gridDim.x + blockIdx.x] = s;
    }
    __syncthreads();
  }
  if (self) {   // row nvec: w . w (accumulated with the first group)
    const double s = warp_sum(self_acc);
    if (lane == 0) red[warp][0] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0;
      for (int k = 0; k < RED_THREADS / 32; ++k) t += red[k][0];
      partial[(int64_t)nvec * gridDim.x + blockIdx.x] = t;
    }
  }
}

__global__ void sum_partials_kernel(const double* __restrict__ partial, int nblk, int nvec,
                                    double* __restrict__ h) {
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (j >= nvec) return;
  double s = 0;
  for (int b = lane; b < nblk; b += 32) s += partial[(int64_t)j * nblk + b];
  s = warp_sum(s);
  if (lane == 0) h[j] = s;
}

int krylov_dots(const double* basis, int64_t ld, int nvec, const double* w, int64_t n,
                double* partial, double* h_out, cudaStream_t st, int self, const double* skip) {
  const int nout = nvec + (self ? 1 : 0);
  count_launches(2);
  const int nblk = dots_blocks(n);
  dots_kernel<<<nblk, RED_THREADS, 0, st>>>(basis, ld, nvec, w, n, partial, self, skip);
  sum_partials_kernel<<<(nout + 3) / 4, 128, 0, st>>>(partial, nblk, nout, h_out);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

// Second Gram-Schmidt pass needed?  h holds the first pass's coefficients
// h[0..nvec) and |w|^2 before it at h[nvec]; after the pass |w'|^2 =
// |w|^2 - sum h_j^2.  The pass is skipped (flag 1) when |w'|^2 >= |w|^2 / 2:
// a vector that lost less than half its length to the projection is
// orthogonal to working accuracy after one pass ("twice is enough").
__global__ void reorth_test_kernel(const double* __restrict__ h, int nvec, double* __restrict__ flag) {
  double s = 0;
  for (int j = threadIdx.x; j < nvec; j += 32) s += h[j] * h[j];
  s = warp_sum(s);
  if (threadIdx.x == 0) {
    const double w2 = h[nvec];
    *flag = (w2 > 0 && w2 - s >= 0.5 * w2) ? 1.0 : 0.0;
  }
}

int krylov_reorth_test(const double* h, int nvec, double* flag, cudaStream_t st) {
  count_launches(1);
  reorth_test_kernel<<<1, 32, 0, st>>>(h, nvec, flag);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

// w -= sum_j h_j basis_j (nothing when *skip != 0)
__global__ void sub_kernel(double* __restrict__ w, const double* __restrict__ basis, int64_t ld,
                           int nvec, const double* __restrict__ h, int64_t n,
                           const double* __restrict__ skip) {
  if (skip != nullptr && *skip != 0.0) return;
  extern __shared__ double sh[];
  for (int j = threadIdx.x; j < nvec; j += blockDim.x) sh[j] = h[j];
  __syncthreads();
  const bool vec = ((ld | n) & 1) == 0 && ((reinterpret_cast<uintptr_t>(basis) | reinterpret_cast<uintptr_t>(w)) & 15) == 0;
  if (vec) {
    double2* w2 = reinterpret_cast<double2*>(w);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n / 2;
         i += (int64_t)gridDim.x * blockDim.x) {
      double2 acc = w2[i];
      int j = 0;
      for (; j + 3 < nvec; j += 4) {
        double2 b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) b[u] = reinterpret_cast<const double2*>(basis + (int64_t)(j + u) * ld)[i];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          acc.x = fma(-sh[j + u], b[u].x, acc.x);
          acc.y = fma(-sh[j + u], b[u].y, acc.y);
        }
      }
      for (; j < nvec; ++j) {
        const double2 b = reinterpret_cast<const double2*>(basis + (int64_t)j * ld)[i];
        acc.x = fma(-sh[j], b.x, acc.x);
        acc.y = fma(-sh[j], b.y, acc.y);
      }
      w2[i] = acc;
    }
    return;
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double acc = w[i];
    for (int j = 0; j < nvec; ++j) acc -= sh[j] * basis[(int64_t)j * ld + i];
    w[i] = acc;
  }
}

// x = sum_j c_j basis_j
__global__ void combine_kernel(double* __restrict__ x, const double* __restrict__ basis,
                               int64_t ld, int nvec, const double* __restrict__ c, int64_t n) {
  extern __shared__ double sh[];
  for (int j = threadIdx.x; j < nvec; j += blockDim.x) sh[j] = c[j];
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0;
    for (int j = 0; j < nvec; ++j) acc += sh[j] * basis[(int64_t)j * ld + i];
    x[i] = acc;
  }
}

static int grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  return (int)(g < 1 ? 1 : g);
}

int krylov_sub(double* w, const double* basis, int64_t ld, int nvec, const double* h, int64_t n,
               cudaStream_t st, const double* skip) {
  count_launches(1);
  sub_kernel<<<grid_for(n), 256, nvec * sizeof(double), st>>>(w, basis, ld, nvec, h, n, skip);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int krylov_combine(double* x, const double* basis, int64_t ld, int nvec, const double* coef,
                   int64_t n, cudaStream_t st) {
  count_launches(1);
  combine_kernel<<<grid_for(n), 256, nvec * sizeof(double), st>>>(x, basis, ld, nvec, coef, n);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

__global__ void scale_kernel(double* out, const double* in, double a, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = a * in[i];
}
__global__ void axpy_kernel(double* y, const double* x, double a, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] += a * x[i];
}
__global__ void d2f_kernel(float* out, const double* in, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}
__global__ void f2d_kernel(double* out, const float* in, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}

int vec_scale(double* out, const double* in, double a, int64_t n, cudaStream_t st) {
  count_launches(1);
  scale_kernel<<<grid_for(n), 256, 0, st>>>(out, in, a, n);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}
int vec_axpy(double* y, const double* x, double a, int64_t n, cudaStream_t st) {
  count_launches(1);
  axpy_kernel<<<grid_for(n), 256, 0, st>>>(y, x, a, n);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}
int vec_cast_d2f(float* out, const double* in, int64_t n, cudaStream_t st) {
  count_launches(1);
  d2f_kernel<<<grid_for(n), 256, 0, st>>>(out, in, n);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}
int vec_cast_f2d(double* out, const float* in, int64_t n, cudaStream_t st) {
  count_launches(1);
  f2d_kernel<<<grid_for(n), 256, 0, st>>>(out, in, n);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

__global__ void mul_kernel(double* out, const double* a, const double* b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = a[i] * b[i];
}

// out = in / sqrt(*n2) (zero when the norm vanishes); the norm stays on the device
__global__ void scale_rsqrt_kernel(double* __restrict__ out, const double* __restrict__ in,
                                   const double* __restrict__ n2, int64_t n) {
  const double v = *n2;
  const double s = v > 0 ? 1.0 / sqrt(v) : 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i] * s;
}

int vec_normalise(double* out, const double* in, const double* n2, int64_t n, cudaStream_t st) {
  count_launches(1);
  scale_rsqrt_kernel<<<grid_for(n), 256, 0, st>>>(out, in, n2, n);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int vec_mul(double* out, const double* a, const double* b, int64_t n, cudaStream_t st) {
  count_launches(1);
  mul_kernel<<<grid_for(n), 256, 0, st>>>(out, a, b, n);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

// Approximate diagonal of H per node, field and mode (a preconditioner only):
//   momentum:   mu V |grad N_a|^2 + mass V/10 + rho V tau_e [(u.grad N_a)^2 + (n omega)^2/10]
//   continuity: (V / rho) tau_e |grad N_a|^2
// with tau_e the one-mode tau of App. B eq. (3D-taut) (omega_hat = 0) at the
// element's mean mode-0 velocity.  One thread per element of a colour.
__global__ void diag_kernel(const int4* __restrict__ tets, const double* __restrict__ geo,
                            const double* __restrict__ y, int N, Phys<double> ph,
                            double* __restrict__ D, int64_t e0, int64_t e1) {
  const int C = 2 * N;
  for (int64_t e = e0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < e1;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int4 nd = tets[e];
    const int node[4] = {nd.x, nd.y, nd.z, nd.w};
    const double* g = geo + e * GEO_STRIDE;
    double u[3] = {0, 0, 0};
    for (int a = 0; a < 4; ++a)
      for (int i = 0; i < 3; ++i) u[i] += 0.25 * y[(int64_t)node[a] * 4 * C + i * C];
    const double* G = g + GEO_G;
    const double uGu = u[0] * (G[0] * u[0] + G[1] * u[1] + G[2] * u[2]) +
                       u[1] * (G[1] * u[0] + G[3] * u[1] + G[4] * u[2]) +
                       u[2] * (G[2] * u[0] + G[4] * u[1] + G[5] * u[2]);
    const double GG = G[0] * G[0] + G[3] * G[3] + G[5] * G[5] +
                      2.0 * (G[1] * G[1] + G[2] * G[2] + G[4] * G[4]);
    const double tau = 1.0 / sqrt(uGu + ph.C_I * ph.nu * ph.nu * GG);
    const double vol = g[GEO_VOL];
    for (int a = 0; a < 4; ++a) {
      const double* dn = g + a * 3;
      const double adv = u[0] * dn[0] + u[1] * dn[1] + u[2] * dn[2];
      const double g2 = dn[0] * dn[0] + dn[1] * dn[1] + dn[2] * dn[2];
      const double mom = ph.mu * vol * g2 + ph.mass_coef * vol * 0.1 + ph.rho * vol * tau * adv * adv;
      const double con = vol / ph.rho * tau * g2;
      double* d = D + (int64_t)node[a] * 4 * C;
      for (int n = 0; n < N; ++n) {
        const double m = mom + ph.rho * tau * vol * (n * ph.omega) * (n * ph.omega) * 0.1;
        for (int i = 0; i < 3; ++i) {
          d[i * C + 2 * n] += m;
          d[i * C + 2 * n + 1] += m;
        }
        d[3 * C + 2 * n] += con;
        d[3 * C + 2 * n + 1] += con;
      }
    }
  }
}

int launch_diag(const int4* tets, const double* geo, const double* y, int N, Phys<double> ph,
                double* D, int64_t e0, int64_t e1, cudaStream_t st) {
  if (e1 <= e0) return 0;
  int64_t blocks = (e1 - e0 + 127) / 128;
  if (blocks > 152 * 8) blocks = 152 * 8;
  count_launches(1);
  diag_kernel<<<(int)blocks, 128, 0, st>>>(tets, geo, y, N, ph, D, e0, e1);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

__global__ void diag_invert_kernel(double* D, const uint8_t* __restrict__ dmask, int64_t V, int C) {
  const int64_t n = V * 4 * C;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t A = t / (4 * C);
    const int r = (int)(t - A * 4 * C);
    const int f = r / C, c = r - f * C;
    const bool fixed = (c == 1) || (f < 3 && dmask[A]);
    const double d = D[t];
    D[t] = (fixed || !(d > 0)) ? 1.0 : 1.0 / d;
  }
}

int launch_diag_invert(double* D, const uint8_t* dmask, int64_t V, int C, cudaStream_t st) {
  count_launches(1);
  diag_invert_kernel<<<grid_for(V * 4 * C), 256, 0, st>>>(D, dmask, V, C);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace ts
