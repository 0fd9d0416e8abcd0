// tau at every quadrature point, eq. (3D-tau):
//   tau = [A_i G_ij A_j + C_I nu^2 G_ij G_ij I]^{-1/2}
// computed, as the paper prescribes after eq. (3D-tau), from the eigenpairs
// of the matrix under the root (section 2.2), at every quadrature point
// (section 4).
//
// GB300 mapping: a group of N lanes owns one quadrature point; a warp holds
// floor(32/N) points.  With G = L L^T (3x3 Cholesky) the argument becomes
// M = sum_m C_m C_m + C_I nu^2 (G:G) I, C_m = A(w_m), w_m = sum_i L_im u_i,
// because the convolution matrix is linear in the velocity modes.  The
// symmetric eigenproblem of the real (2N-1)x(2N-1) form of M is solved by
// parallel cyclic Jacobi (round-robin ordering, N disjoint rotations per
// round, one per lane), padded with a decoupled dummy row to size 2N.
// tau = V diag(lambda^{-1/2}) V^T is written as a packed upper triangle.
#include "common.cuh"
#include "jacobi.cuh"
#include "kernels.h"

namespace ts {

template <int N>
struct TauLayout {
  using D = Dims<N>;
  static constexpr int NP = D::NP, NM = D::NM, C = D::C;
  static constexpr int LD = NP + 1;
  static constexpr int GPW = 32 / N;
  static constexpr int CM = 0;                       // [3][NM][NM]
  static constexpr int M = CM + 3 * NM * NM;         // [NP][LD]
  static constexpr int V = M + NP * LD;              // [NP][LD]
  static constexpr int W = V + NP * LD;              // [3][C]
  static constexpr int GROUP = ((W + 3 * C) + 1) & ~1;
  static constexpr int WARP = GPW * GROUP + 64;      // + reduction scratch
};

template <typename T, int N>
__global__ void __launch_bounds__(128) tau_kernel(const int4* __restrict__ tets,
                                                  const T* __restrict__ geo,
                                                  const T* __restrict__ y, int64_t n_qp,
                                                  T* __restrict__ tau_out, T nu, T C_I,
                                                  int max_sweeps, T tol2,
                                                  unsigned* __restrict__ n_unconverged,
                                                  float* __restrict__ eig_out) {
  using D = Dims<N>;
  using L = TauLayout<N>;
  constexpr int NP = D::NP, NM = D::NM, C = D::C, LD = L::LD, GPW = L::GPW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* smem = reinterpret_cast<T*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane / N, k = lane - (lane / N) * N;
  const bool in_group = g < GPW;
  T* wbase = smem + warp * L::WARP;
  T* base = wbase + (in_group ? g : 0) * L::GROUP;
  T* Cm = base + L::CM;
  T* M = base + L::M;
  T* Vv = base + L::V;
  T* w = base + L::W;
  T* red = wbase + GPW * L::GROUP;       // [32] partial sums, [32..] flags

  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t qb = ((int64_t)blockIdx.x * (blockDim.x >> 5) + warp) * GPW; qb < n_qp;
       qb += warps_total * GPW) {
    const int64_t gq = qb + g;
    const bool live = in_group && gq < n_qp;
    const int64_t e = live ? gq >> 2 : 0;
    const int q = (int)(gq & 3);
    T l00 = 0, l10 = 0, l20 = 0, l11 = 0, l21 = 0, l22 = 0, diff = 0;
    if (live) {
      const T* gg = geo + e * GEO_STRIDE + GEO_G;
      T gxx = gg[0], gxy = gg[1], gxz = gg[2], gyy = gg[3], gyz = gg[4], gzz = gg[5];
      l00 = Real<T>::sqrt(gxx);
      l10 = gxy / l00;
      l20 = gxz / l00;
      l11 = Real<T>::sqrt(gyy - l10 * l10);
      l21 = (gyz - l20 * l10) / l11;
      l22 = Real<T>::sqrt(gzz - l20 * l20 - l21 * l21);
      T GG = gxx * gxx + gyy * gyy + gzz * gzz + T(2) * (gxy * gxy + gxz * gxz + gyz * gyz);
      diff = C_I * nu * nu * GG;
      const int4 nd = tets[e];
      const int node[4] = {nd.x, nd.y, nd.z, nd.w};
      // velocity modes at the point, then w_m = sum_i L_im u_i
      for (int c = k; c < C; c += N) {
        T u[3] = {0, 0, 0};
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const T lam = (T)qp_bary(q, a);
          const T* ya = y + (int64_t)node[a] * 4 * C;
#pragma unroll
          for (int i = 0; i < 3; ++i) u[i] += lam * ya[i * C + c];
        }
        if (c == 1) u[0] = u[1] = u[2] = 0;
        w[0 * C + c] = l00 * u[0] + l10 * u[1] + l20 * u[2];
        w[1 * C + c] = l11 * u[1] + l21 * u[2];
        w[2 * C + c] = l22 * u[2];
      }
    }
    __syncwarp();
    if (live) {
      for (int t = k; t < 3 * NM * NM; t += N) {
        int m = t / (NM * NM), rs = t - m * NM * NM;
        int r = rs / NM, s = rs - r * NM;
        Cm[t] = conv_entry<T, N>(w + m * C, r, s);
      }
    }
    __syncwarp();
    if (live) {
      for (int t = k; t < NP * NP; t += N) {
        int r = t / NP, s = t - r * NP;
        if (r > s) continue;
        T acc = 0;
        if (r < NM && s < NM) {
#pragma unroll
          for (int m = 0; m < 3; ++m) {
            const T* cr = Cm + m * NM * NM + r * NM;
            const T* cs = Cm + m * NM * NM + s * NM;
            for (int j = 0; j < NM; ++j) acc += cr[j] * cs[j];
          }
          if (r == s) acc += diff;
        } else if (r == s) {
          acc = T(1);                      // decoupled dummy
        }
        M[r * LD + s] = acc;
        M[s * LD + r] = acc;
        Vv[r * LD + s] = (r == s) ? T(1) : T(0);
        Vv[s * LD + r] = (r == s) ? T(1) : T(0);
      }
    }
    __syncwarp();
    // parallel cyclic Jacobi
    const bool converged = jacobi_group<T, N>(M, Vv, k, g, lane, live, red, max_sweeps, tol2);
    if (live && k == 0 && !converged) atomicAdd(n_unconverged, 1u);
    // eigenpairs for the derivative of tau (exact tangent), when asked
    if (live && eig_out) {
      float* eo = eig_out + gq * D::EIG;
      for (int t = k; t < NM * NM; t += N) eo[t] = (float)Vv[(t / NM) * LD + t % NM];
      for (int j = k; j < NM; j += N) eo[NM * NM + j] = (float)M[j * LD + j];
    }
    // tau = V diag(lambda^{-1/2}) V^T, packed upper triangle
    if (live) {
      T* out = tau_out + gq * Dims<N>::NT_PAD;
      for (int t = k; t < NM * NM; t += N) {
        int r = t / NM, s = t - r * NM;
        if (r > s) continue;
        T acc = 0;
        for (int j = 0; j < NM; ++j) {
          T lam = M[j * LD + j];
          acc += Vv[r * LD + j] * Vv[s * LD + j] * Real<T>::rsqrt(lam);
        }
        out[packed_index(r, s, NM)] = acc;
      }
      if (k == 0)
        for (int t = Dims<N>::NT; t < Dims<N>::NT_PAD; ++t) out[t] = T(0);
    }
    __syncwarp();
  }
}

template <typename T, int N>
int launch_tau(const int4* tets, const T* geo, const T* y, int64_t n_elem, T* tau_out, T nu,
               T C_I, unsigned* n_unconverged, cudaStream_t st, float* eig_out) {
  using L = TauLayout<N>;
  const int warps = 4;
  size_t smem = (size_t)warps * L::WARP * sizeof(T);
  cudaFuncSetAttribute(tau_kernel<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int64_t n_qp = n_elem * 4;
  int64_t groups = (n_qp + L::GPW - 1) / L::GPW;
  int64_t blocks = (groups + warps - 1) / warps;
  if (blocks > 152 * 64) blocks = 152 * 64;
  if (blocks < 1) blocks = 1;
  const int sweeps = sizeof(T) == 4 ? 12 : 20;
  const T tol2 = sizeof(T) == 4 ? T(1e-12) : T(1e-28);
  count_launches(1);
  tau_kernel<T, N><<<(int)blocks, warps * 32, smem, st>>>(tets, geo, y, n_qp, tau_out, nu, C_I,
                                                          sweeps, tol2, n_unconverged, eig_out);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

// Loads tau_kernel<T, N> into the current device's context without launching
// it (with lazy module loading a kernel is otherwise loaded at its first launch).
template <typename T, int N>
int preload_tau() {
  using L = TauLayout<N>;
  cudaFuncAttributes a;
  if (cudaFuncGetAttributes(&a, tau_kernel<T, N>) != cudaSuccess) return -2;
  const size_t smem = (size_t)4 * L::WARP * sizeof(T);
  return cudaFuncSetAttribute(tau_kernel<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
                 cudaSuccess ? 0 : -2;
}

// ---------------------------------------------------------------------------
// FP64 tau from FP32 eigenvectors.  The FP32 Jacobi gives V32 with
// V32^T M V32 diagonal to about 1e-7 ||M||.  In FP64: one Newton-Schulz step
// (two) make V orthonormal to FP64 rounding, B = V^T M V, and f(B) = B^{-1/2} is
// expanded to second order around diag(B) with the Daleckii-Krein formulas
// (Frechet derivatives of a matrix function at a diagonal matrix are
// Hadamard-type sums with the divided differences of f).  For f = l^{-1/2}
// with s = sqrt(l) the divided differences have cancellation-free forms
//   f[a,b]   = -1 / (s_a s_b (s_a + s_b))
//   f[a,b,c] = (s_a + s_b + s_c) / (s_a s_b s_c (s_a+s_b)(s_b+s_c)(s_a+s_c)),
// which gives, with X_ik = E_ik / (s_i s_k (s_i + s_k)) and E = offdiag(B),
//   Z = diag(1/s) - X + X D_s X + (X D_{s^2} X) ./ (s_i + s_j),
// tau = V Z V^T, error third order in E.
template <int N>
struct PolishLayout {
  static constexpr int NP = 2 * N, NM = 2 * N - 1, C = 2 * N, LD = NP + 1;
  static constexpr int GPW = 32 / N;
  // in doubles
  static constexpr int CM = 0;                       // [3][NM][NM] scratch
  static constexpr int M64 = CM + 3 * NM * NM;       // [NP][LD]
  static constexpr int V64 = M64 + NP * LD;          // [NP][LD]
  static constexpr int W = V64 + NP * LD;            // [3][C]
  static constexpr int F32 = W + 3 * C;              // start of the float part
  static constexpr int GROUP = F32 + NP * LD;        // 2 [NP][LD] float matrices = NP*LD doubles
  static constexpr int WARP = GPW * GROUP + 64 + 32; // + double and float reduction scratch
};

template <int N>
__global__ void __launch_bounds__(128) tau_polish_kernel(const int4* __restrict__ tets,
                                                         const double* __restrict__ geo,
                                                         const double* __restrict__ y,
                                                         int64_t n_qp, double* __restrict__ tau_out,
                                                         double nu, double C_I,
                                                         unsigned* __restrict__ n_unconverged,
                                                         float* __restrict__ eig_out) {
  using L = PolishLayout<N>;
  constexpr int NP = L::NP, NM = L::NM, C = L::C, LD = L::LD, GPW = L::GPW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* smem = reinterpret_cast<double*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane / N, k = lane - (lane / N) * N;
  const bool in_group = g < GPW;
  double* wbase = smem + warp * L::WARP;
  double* base = wbase + (in_group ? g : 0) * L::GROUP;
  double* Cm = base + L::CM;
  double* M = base + L::M64;
  double* Vd = base + L::V64;
  double* w = base + L::W;
  float* Mf = reinterpret_cast<float*>(base + L::F32);
  float* Vf = Mf + NP * LD;
  double* red_d = wbase + GPW * L::GROUP;
  float* red_f = reinterpret_cast<float*>(red_d + 64);

  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t qb = ((int64_t)blockIdx.x * (blockDim.x >> 5) + warp) * GPW; qb < n_qp;
       qb += warps_total * GPW) {
    const int64_t gq = qb + g;
    const bool live = in_group && gq < n_qp;
    const int64_t e = live ? gq >> 2 : 0;
    const int q = (int)(gq & 3);
    double diff = 0;
    if (live) {
      const double* gg = geo + e * GEO_STRIDE + GEO_G;
      const double gxx = gg[0], gxy = gg[1], gxz = gg[2], gyy = gg[3], gyz = gg[4], gzz = gg[5];
      const double l00 = sqrt(gxx), l10 = gxy / l00, l20 = gxz / l00;
      const double l11 = sqrt(gyy - l10 * l10), l21 = (gyz - l20 * l10) / l11;
      const double l22 = sqrt(gzz - l20 * l20 - l21 * l21);
      const double GG = gxx * gxx + gyy * gyy + gzz * gzz + 2.0 * (gxy * gxy + gxz * gxz + gyz * gyz);
      diff = C_I * nu * nu * GG;
      const int4 nd = tets[e];
      const int node[4] = {nd.x, nd.y, nd.z, nd.w};
      for (int c = k; c < C; c += N) {
        double u[3] = {0, 0, 0};
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const double lam = qp_bary(q, a);
          const double* ya = y + (int64_t)node[a] * 4 * C;
#pragma unroll
          for (int i = 0; i < 3; ++i) u[i] += lam * ya[i * C + c];
        }
        if (c == 1) u[0] = u[1] = u[2] = 0;
        w[0 * C + c] = l00 * u[0] + l10 * u[1] + l20 * u[2];
        w[1 * C + c] = l11 * u[1] + l21 * u[2];
        w[2 * C + c] = l22 * u[2];
      }
    }
    __syncwarp();
    if (live)
      for (int t = k; t < 3 * NM * NM; t += N) {
        const int m = t / (NM * NM), rs = t - m * NM * NM;
        const int r = rs / NM, s = rs - r * NM;
        Cm[t] = conv_entry<double, N>(w + m * C, r, s);
      }
    __syncwarp();
    if (live)
      for (int t = k; t < NP * NP; t += N) {
        const int r = t / NP, s = t - r * NP;
        if (r > s) continue;
        double acc = 0;
        if (r < NM && s < NM) {
#pragma unroll
          for (int m = 0; m < 3; ++m) {
            const double* cr = Cm + m * NM * NM + r * NM;
            const double* cs = Cm + m * NM * NM + s * NM;
            for (int j = 0; j < NM; ++j) acc += cr[j] * cs[j];
          }
          if (r == s) acc += diff;
        } else if (r == s) {
          acc = 1.0;   // decoupled dummy
        }
        M[r * LD + s] = acc;
        M[s * LD + r] = acc;
        Mf[r * LD + s] = (float)acc;
        Mf[s * LD + r] = (float)acc;
        Vf[r * LD + s] = (r == s) ? 1.f : 0.f;
        Vf[s * LD + r] = (r == s) ? 1.f : 0.f;
      }
    __syncwarp();
    const bool conv32 = jacobi_group<float, N>(Mf, Vf, k, g, lane, live, red_f, 12, 1e-12f);
    if (live && k == 0 && !conv32) atomicAdd(n_unconverged, 1u);
    // V in FP64, re-orthonormalised by two Newton-Schulz steps V <- V (3I - V^T V) / 2
    // (the FP32 eigenvectors are orthonormal only to FP32 rounding)
    if (live)
      for (int t = k; t < NP * NP; t += N) Vd[(t / NP) * LD + t % NP] = (double)Vf[(t / NP) * LD + t % NP];
    __syncwarp();
    for (int it = 0; it < 2; ++it) {
      if (live)
        for (int t = k; t < NM * NM; t += N) {
          const int r = t / NM, s = t - r * NM;
          double acc = 0;
          for (int i = 0; i < NM; ++i) acc += Vd[i * LD + r] * Vd[i * LD + s];
          Cm[t] = ((r == s) ? 3.0 : 0.0) - acc;      // 3I - V^T V
        }
      __syncwarp();
      if (live)
        for (int t = k; t < NM * NM; t += N) {
          const int r = t / NM, s = t - r * NM;
          double acc = 0;
          for (int j = 0; j < NM; ++j) acc += Vd[r * LD + j] * Cm[j * NM + s];
          Cm[NM * NM + t] = 0.5 * acc;
        }
      __syncwarp();
      if (live)
        for (int t = k; t < NM * NM; t += N) Vd[(t / NM) * LD + t % NM] = Cm[NM * NM + t];
      __syncwarp();
    }
    // P = M V, then B = V^T M V over the NM x NM block of M (dummy row/column unchanged)
    if (live)
      for (int t = k; t < NM * NM; t += N) {
        const int r = t / NM, s = t - r * NM;
        double acc = 0;
        for (int j = 0; j < NM; ++j) acc += M[r * LD + j] * Vd[j * LD + s];
        Cm[t] = acc;
      }
    __syncwarp();
    if (live)
      for (int t = k; t < NM * NM; t += N) {
        const int r = t / NM, s = t - r * NM;
        if (r > s) continue;
        double acc = 0;
        for (int i = 0; i < NM; ++i) acc += Vd[i * LD + r] * Cm[i * NM + s];
        M[r * LD + s] = acc;
        M[s * LD + r] = acc;
      }
    __syncwarp();
    if (live && eig_out) {
      float* eo = eig_out + gq * Dims<N>::EIG;
      for (int t = k; t < NM * NM; t += N) eo[t] = (float)Vd[(t / NM) * LD + t % NM];
      for (int j = k; j < NM; j += N) eo[NM * NM + j] = (float)M[j * LD + j];
    }
    // s = sqrt(diag B) once per point (reusing the w rows: 3C >= 2 NM)
    double* sq = w;          // [NM] sqrt(b_ii)
    double* sq2 = w + NM;    // [NM] b_ii
    if (live)
      for (int i = k; i < NM; i += N) {
        sq[i] = sqrt(M[i * LD + i]);
        sq2[i] = M[i * LD + i];
      }
    __syncwarp();
    // X_ik = E_ik / (s_i s_k (s_i + s_k)), E = offdiag B
    if (live)
      for (int t = k; t < NM * NM; t += N) {
        const int r = t / NM, s = t - r * NM;
        const double sr = sq[r], ss = sq[s];
        Cm[t] = (r == s) ? 0.0 : M[r * LD + s] / (sr * ss * (sr + ss));
      }
    __syncwarp();
    // Z = diag(1/s) - X + sum_k X_ik X_kj (s_k + s_k^2 / (s_i + s_j))   (second order)
    if (live)
      for (int t = k; t < NM * NM; t += N) {
        const int r = t / NM, s = t - r * NM;
        const double sr = sq[r], ss = sq[s];
        const double inv_rs = 1.0 / (sr + ss);
        double acc = 0;
        for (int j = 0; j < NM; ++j) acc += Cm[r * NM + j] * Cm[j * NM + s] * (sq[j] + sq2[j] * inv_rs);
        Cm[NM * NM + t] = ((r == s) ? 1.0 / sr : 0.0) - Cm[t] + acc;
      }
    __syncwarp();
    // Q = Z V^T in the third scratch slot
    if (live)
      for (int t = k; t < NM * NM; t += N) {
        const int r = t / NM, s = t - r * NM;
        double acc = 0;
        for (int j = 0; j < NM; ++j) acc += Cm[NM * NM + r * NM + j] * Vd[s * LD + j];
        Cm[2 * NM * NM + t] = acc;
      }
    __syncwarp();
    if (live) {
      double* out = tau_out + gq * Dims<N>::NT_PAD;
      for (int t = k; t < NM * NM; t += N) {
        const int r = t / NM, s = t - r * NM;
        if (r > s) continue;
        double acc = 0;
        for (int j = 0; j < NM; ++j) acc += Vd[r * LD + j] * Cm[2 * NM * NM + j * NM + s];
        out[packed_index(r, s, NM)] = acc;
      }
      if (k == 0)
        for (int t = Dims<N>::NT; t < Dims<N>::NT_PAD; ++t) out[t] = 0.0;
    }
    __syncwarp();
  }
}

template <int N>
int launch_tau_polish(const int4* tets, const double* geo, const double* y, int64_t n_elem,
                      double* tau_out, double nu, double C_I, unsigned* n_unconverged,
                      cudaStream_t st, float* eig_out) {
  using L = PolishLayout<N>;
  int warps = 4;
  while (warps > 1 && (size_t)warps * L::WARP * sizeof(double) > 200 * 1024) --warps;
  const size_t smem = (size_t)warps * L::WARP * sizeof(double);
  if (smem > 227 * 1024) return -6;
  cudaFuncSetAttribute(tau_polish_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int64_t n_qp = n_elem * 4;
  const int64_t groups = (n_qp + L::GPW - 1) / L::GPW;
  int64_t blocks = (groups + warps - 1) / warps;
  if (blocks > 152 * 64) blocks = 152 * 64;
  if (blocks < 1) blocks = 1;
  count_launches(1);
  tau_polish_kernel<N><<<(int)blocks, warps * 32, smem, st>>>(tets, geo, y, n_qp, tau_out, nu, C_I,
                                                              n_unconverged, eig_out);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

#define TS_INST_POLISH(T, N)                                                                  \
  template int launch_tau_polish<N>(const int4*, const double*, const double*, int64_t,      \
                                    double*, double, double, unsigned*, cudaStream_t, float*);
TS_FOR_EACH_N(TS_INST_POLISH, double)


// ---------------------------------------------------------------------------
// Backflow stabilisation (section 2.6): at every point of a Neumann face,
// |A_n|_- = (A_n - |A_n|)/2 with A_n = A_i n_i = A(u . n), taken through the
// eigenpairs of A_n (remark 1 of section 2.6), stored like tau as a packed
// upper triangle in the orthonormal real basis.  Face points: the 3-point
// degree-2 rule (barycentric 2/3, 1/6, 1/6), weights area/3.
__host__ __device__ constexpr double face_bary(int g, int b) { return g == b ? 2.0 / 3.0 : 1.0 / 6.0; }

template <int N>
struct BackflowLayout {
  static constexpr int NP = 2 * N, C = 2 * N, LD = NP + 1, GPW = 32 / N;
  static constexpr int M = 0, V = M + NP * LD, W = V + NP * LD;
  static constexpr int GROUP = (W + C + 1) & ~1;
  static constexpr int WARP = GPW * GROUP + 64;
};

template <typename T, int N>
__global__ void __launch_bounds__(128) backflow_neg_kernel(const int32_t* __restrict__ faces,
                                                           const T* __restrict__ normals,
                                                           const T* __restrict__ y, int64_t n_pts,
                                                           T* __restrict__ bneg) {
  using L = BackflowLayout<N>;
  constexpr int NP = L::NP, NM = 2 * N - 1, C = L::C, LD = L::LD, GPW = L::GPW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* smem = reinterpret_cast<T*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane / N, k = lane - (lane / N) * N;
  const bool in_group = g < GPW;
  T* wbase = smem + warp * L::WARP;
  T* base = wbase + (in_group ? g : 0) * L::GROUP;
  T* M = base + L::M;
  T* Vv = base + L::V;
  T* w = base + L::W;
  T* red = wbase + GPW * L::GROUP;
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t pb = ((int64_t)blockIdx.x * (blockDim.x >> 5) + warp) * GPW; pb < n_pts;
       pb += warps_total * GPW) {
    const int64_t gp = pb + g;
    const bool live = in_group && gp < n_pts;
    const int64_t f = live ? gp / 3 : 0;
    const int gq = (int)(gp - (gp / 3) * 3);
    if (live) {
      const T nx = normals[f * 3], ny = normals[f * 3 + 1], nz = normals[f * 3 + 2];
      for (int c = k; c < C; c += N) {
        T un = 0;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          const T* yb = y + (int64_t)faces[f * 3 + b] * 4 * C;
          un += (T)face_bary(gq, b) * (nx * yb[c] + ny * yb[C + c] + nz * yb[2 * C + c]);
        }
        w[c] = (c == 1) ? T(0) : un;
      }
    }
    __syncwarp();
    if (live)
      for (int t = k; t < NP * NP; t += N) {
        const int r = t / NP, s2 = t - r * NP;
        T val;
        if (r < NM && s2 < NM) val = conv_entry<T, N>(w, r, s2);
        else val = (r == s2) ? T(1) : T(0);   // decoupled dummy
        M[r * LD + s2] = val;
        Vv[r * LD + s2] = (r == s2) ? T(1) : T(0);
      }
    __syncwarp();
    jacobi_group<T, N>(M, Vv, k, g, lane, live, red, sizeof(T) == 4 ? 12 : 20,
                       sizeof(T) == 4 ? T(1e-12) : T(1e-28));
    if (live) {
      T* out = bneg + gp * Dims<N>::NT_PAD;
      for (int t = k; t < NM * NM; t += N) {
        const int r = t / NM, s2 = t - r * NM;
        if (r > s2) continue;
        T acc = 0;
        for (int j = 0; j < NM; ++j) {
          const T lam = M[j * LD + j];
          if (lam < T(0)) acc += Vv[r * LD + j] * Vv[s2 * LD + j] * lam;
        }
        out[packed_index(r, s2, NM)] = acc;
      }
      if (k == 0)
        for (int t = Dims<N>::NT; t < Dims<N>::NT_PAD; ++t) out[t] = T(0);
    }
    __syncwarp();
  }
}

// out[A][i] += coef * sum_g (area/3) N_A(g) |A_n|_- u_i(g), one thread per (face, point, i)
template <typename T, int N>
__global__ void backflow_apply_kernel(const int32_t* __restrict__ faces, const T* __restrict__ area,
                                      const T* __restrict__ bneg, const T* __restrict__ v,
                                      const uint8_t* __restrict__ dmask, int mask_input, T coef,
                                      T* __restrict__ out, int64_t n_faces) {
  constexpr int C = 2 * N, NM = 2 * N - 1, NTP = Dims<N>::NT_PAD;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_faces * 9;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = t / 9;
    const int gi = (int)(t - f * 9), g = gi / 3, i = gi - (gi / 3) * 3;
    int nb[3];
    T u[C];
#pragma unroll
    for (int c = 0; c < C; ++c) u[c] = 0;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      nb[b] = faces[f * 3 + b];
      if (mask_input && dmask[nb[b]]) continue;
      const T* vb = v + (int64_t)nb[b] * 4 * C + i * C;
#pragma unroll
      for (int c = 0; c < C; ++c) u[c] += (T)face_bary(g, b) * vb[c];
    }
    u[1] = 0;
    const T* B = bneg + (f * 3 + g) * NTP;
    T z[C];
#pragma unroll
    for (int r = 0; r < NM; ++r) {
      T acc = 0;
#pragma unroll
      for (int kk = 0; kk < NM; ++kk) {
        const int a = r < kk ? r : kk, b = r < kk ? kk : r;
        T bv = B[packed_index(a, b, NM)];
        if (r == 0 && kk > 0) bv *= Real<T>::SQRT2;
        if (r > 0 && kk == 0) bv *= Real<T>::INV_SQRT2;
        acc += bv * u[stor_of(kk)];
      }
      z[stor_of(r)] = acc;
    }
    const T wq = coef * area[f] / T(3);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if (dmask[nb[b]]) continue;
      T* dst = out + (int64_t)nb[b] * 4 * C + i * C;
      const T s = wq * (T)face_bary(g, b);
#pragma unroll
      for (int c = 0; c < C; ++c)
        if (c != 1) atomicAdd(dst + c, s * z[c]);
    }
  }
}

template <typename T, int N>
int launch_backflow(const int32_t* faces, const T* normals, const T* area, int64_t n_faces,
                    const T* y_for_matrix, T* bneg, const T* v, const uint8_t* dmask, int mask_input,
                    T coef, T* out, cudaStream_t st) {
  if (n_faces <= 0) return 0;
  if (y_for_matrix) {
    using L = BackflowLayout<N>;
    const int warps = 4;
    const size_t smem = (size_t)warps * L::WARP * sizeof(T);
    cudaFuncSetAttribute(backflow_neg_kernel<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int64_t n_pts = n_faces * 3;
    int64_t blocks = ((n_pts + L::GPW - 1) / L::GPW + warps - 1) / warps;
    if (blocks > 152 * 32) blocks = 152 * 32;
    count_launches(1);
    backflow_neg_kernel<T, N><<<(int)blocks, warps * 32, smem, st>>>(faces, normals, y_for_matrix, n_pts, bneg);
  }
  int64_t blocks = (n_faces * 9 + 127) / 128;
  if (blocks > 152 * 16) blocks = 152 * 16;
  count_launches(1);
  backflow_apply_kernel<T, N><<<(int)blocks, 128, 0, st>>>(faces, area, bneg, v, dmask, mask_input, coef, out, n_faces);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

#define TS_INST_BACKFLOW(T, N)                                                                 \
  template int launch_backflow<T, N>(const int32_t*, const T*, const T*, int64_t, const T*, T*, \
                                     const T*, const uint8_t*, int, T, T*, cudaStream_t);
TS_FOR_EACH_N(TS_INST_BACKFLOW, float)
TS_FOR_EACH_N(TS_INST_BACKFLOW, double)

#define TS_INST_TAU(T, N)                                                                 \
  template int launch_tau<T, N>(const int4*, const T*, const T*, int64_t, T*, T, T,       \
                                unsigned*, cudaStream_t, float*);
#define TS_INST_PRELOAD_TAU(T, N) template int preload_tau<T, N>();
TS_FOR_EACH_N(TS_INST_PRELOAD_TAU, float)
TS_FOR_EACH_N(TS_INST_TAU, float)
TS_FOR_EACH_N(TS_INST_TAU, double)

}  // namespace ts
