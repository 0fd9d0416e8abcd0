// Derivative of tau (eq. 3D-tau) along a tangent direction: the term the
// paper's tangent (and the LIN_A tangent) leave out by freezing tau (section
// 2.4), needed for the exact derivative of the residual of eq. (Rmc).
//
// In the orthonormal real basis of a mode vector (x_0, sqrt2 Re x_n, sqrt2 Im
// x_n) M = sum_m C_m C_m + C_I nu^2 (G:G) I with C_m = A(w_m), w_m = sum_i
// L_im u_i and G = L L^T, so along v
//   dM = sum_m (C_m dC_m + dC_m C_m),   dC_m = A(sum_i L_im v_i),
// and for tau = f(M), f(l) = l^{-1/2}, with M = V diag(lambda) V^T the
// Daleckii-Krein formula gives
//   d tau = V [(V^T dM V) o Phi] V^T,  Phi_ij = -1 / (s_i s_j (s_i + s_j)),  s = sqrt(lambda)
// (the divided difference of f, also on the diagonal: f'(l) = -1/(2 s^3)).
// The kernel returns dT_i = d tau L_i(u0) for the three momentum components,
// with the eigenpairs of M and the strong residual L(u0) cached by the
// residual at the linearisation state.  FP32 throughout: this is a Jacobian
// term, its rounding changes the Newton path, not the converged field.
//
// GB300 mapping: one warp per quadrature point, the point's n x n matrices
// (n = 2N - 1) in shared memory, lanes over matrix entries.
#include "common.cuh"
#include "jacobi.cuh"
#include "kernels.h"

namespace ts {

namespace {

template <int N>
struct DtauLayout {
  static constexpr int C = 2 * N, NM = 2 * N - 1, NN = NM * NM;
  static constexpr int V = 0;              // eigenvectors [NM][NM]
  static constexpr int X = V + NN;         // sum_m C_m dC_m, later dM
  static constexpr int CM = X + NN;        // C_m, later Y = dM V
  static constexpr int DC = CM + NN;       // dC_m, later B o Phi
  static constexpr int LAM = DC + NN;      // eigenvalues [NM]
  static constexpr int U = LAM + NM;       // u0 at the point [3][C]
  static constexpr int DV = U + 3 * C;     // v at the point [3][C]
  static constexpr int W = DV + 3 * C;     // w_m [3][C]
  static constexpr int DW = W + 3 * C;     // dw_m [3][C]
  static constexpr int XI = DW + 3 * C;    // orthonormal L(u0) [3][NM], later F l
  static constexpr int ELL = XI + 3 * NM;  // V^T xi [3][NM]
  static constexpr int WARP = (ELL + 3 * NM + 3) & ~3;
};

}  // namespace

template <int N>
__global__ void __launch_bounds__(256)
    dtau_kernel(const int4* __restrict__ tets, const float* __restrict__ geo, const float* __restrict__ u0,
                const float* __restrict__ v, const uint8_t* __restrict__ dmask, const float* __restrict__ eig,
                const float* __restrict__ l0, float* __restrict__ dT, int64_t n_qp) {
  using L = DtauLayout<N>;
  using D = Dims<N>;
  constexpr int C = L::C, NM = L::NM, NN = L::NN;
  extern __shared__ __align__(16) float smem_f[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  float* ws = smem_f + warp * L::WARP;
  float* sV = ws + L::V;
  float* sX = ws + L::X;
  float* sC = ws + L::CM;
  float* sD = ws + L::DC;
  float* lam = ws + L::LAM;
  float* su = ws + L::U;
  float* sv = ws + L::DV;
  float* sw = ws + L::W;
  float* sdw = ws + L::DW;
  float* xi = ws + L::XI;
  float* ell = ws + L::ELL;
  for (int64_t gq = (int64_t)blockIdx.x * wpb + warp; gq < n_qp; gq += (int64_t)gridDim.x * wpb) {
    const int64_t e = gq >> 2;
    const int q = (int)(gq & 3);
    const int4 nd = tets[e];
    const int node[4] = {nd.x, nd.y, nd.z, nd.w};
    const float* ep = eig + gq * D::EIG;
    for (int t = lane; t < NN; t += 32) sV[t] = ep[t];
    for (int t = lane; t < NM; t += 32) lam[t] = ep[NN + t];
    // u0 and v (masked like a tangent input) at the point
    for (int t = lane; t < 3 * C; t += 32) {
      const int i = t / C, c = t - i * C;
      float au = 0.f, av = 0.f;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const float lamq = (float)qp_bary(q, a);
        au += lamq * u0[(int64_t)node[a] * 4 * C + i * C + c];
        if (!dmask[node[a]]) av += lamq * v[(int64_t)node[a] * 4 * C + i * C + c];
      }
      su[t] = c == 1 ? 0.f : au;
      sv[t] = c == 1 ? 0.f : av;
    }
    // the strong residual L_i(u0) at the point in the orthonormal basis
    for (int t = lane; t < 3 * NM; t += 32) {
      const int i = t / NM, r = t - i * NM;
      const float x = l0[((e * 4 + q) * 3 + i) * C + stor_of(r)];
      xi[t] = r == 0 ? x : Real<float>::SQRT2 * x;
    }
    __syncwarp();
    // w_m and dw_m with the Cholesky factor of G (lower: G = L L^T)
    {
      const float* gg = geo + e * GEO_STRIDE + GEO_G;
      const float l00 = sqrtf(gg[0]);
      const float l10 = gg[1] / l00, l20 = gg[2] / l00;
      const float l11 = sqrtf(gg[3] - l10 * l10);
      const float l21 = (gg[4] - l20 * l10) / l11;
      const float l22 = sqrtf(gg[5] - l20 * l20 - l21 * l21);
      for (int c = lane; c < C; c += 32) {
        sw[0 * C + c] = l00 * su[c] + l10 * su[C + c] + l20 * su[2 * C + c];
        sw[1 * C + c] = l11 * su[C + c] + l21 * su[2 * C + c];
        sw[2 * C + c] = l22 * su[2 * C + c];
        sdw[0 * C + c] = l00 * sv[c] + l10 * sv[C + c] + l20 * sv[2 * C + c];
        sdw[1 * C + c] = l11 * sv[C + c] + l21 * sv[2 * C + c];
        sdw[2 * C + c] = l22 * sv[2 * C + c];
      }
    }
    for (int t = lane; t < NN; t += 32) sX[t] = 0.f;
    __syncwarp();
    // X = sum_m C_m dC_m
    for (int m = 0; m < 3; ++m) {
      for (int t = lane; t < NN; t += 32) {
        const int r = t / NM, s = t - r * NM;
        sC[t] = conv_entry<float, N>(sw + m * C, r, s);
        sD[t] = conv_entry<float, N>(sdw + m * C, r, s);
      }
      __syncwarp();
      for (int t = lane; t < NN; t += 32) {
        const int r = t / NM, s = t - r * NM;
        float acc = sX[t];
#pragma unroll
        for (int k = 0; k < NM; ++k) acc = fmaf(sC[r * NM + k], sD[k * NM + s], acc);
        sX[t] = acc;
      }
      __syncwarp();
    }
    // dM = X + X^T (in sD), Y = dM V (in sC)
    for (int t = lane; t < NN; t += 32) {
      const int r = t / NM, s = t - r * NM;
      sD[t] = sX[t] + sX[s * NM + r];
    }
    __syncwarp();
    for (int t = lane; t < NN; t += 32) {
      const int r = t / NM, s = t - r * NM;
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < NM; ++k) acc = fmaf(sD[r * NM + k], sV[k * NM + s], acc);
      sC[t] = acc;
    }
    __syncwarp();
    // F = (V^T Y) o Phi (in sX); ell_i = V^T xi_i
    for (int t = lane; t < NN; t += 32) {
      const int r = t / NM, s = t - r * NM;
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < NM; ++k) acc = fmaf(sV[k * NM + r], sC[k * NM + s], acc);
      const float sr = sqrtf(fmaxf(lam[r], 1e-30f)), ss = sqrtf(fmaxf(lam[s], 1e-30f));
      sX[t] = -acc / (sr * ss * (sr + ss));
    }
    for (int t = lane; t < 3 * NM; t += 32) {
      const int i = t / NM, r = t - i * NM;
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < NM; ++k) acc = fmaf(sV[k * NM + r], xi[i * NM + k], acc);
      ell[t] = acc;
    }
    __syncwarp();
    // g_i = F ell_i (into xi)
    for (int t = lane; t < 3 * NM; t += 32) {
      const int i = t / NM, r = t - i * NM;
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < NM; ++k) acc = fmaf(sX[r * NM + k], ell[i * NM + k], acc);
      xi[t] = acc;
    }
    __syncwarp();
    // dT_i = V g_i, back to storage coordinates
    float* out = dT + (e * 4 + q) * 3 * C;
    for (int t = lane; t < 3 * C; t += 32) {
      const int i = t / C, c = t - i * C;
      float val = 0.f;
      if (c != 1) {
        const int r = c == 0 ? 0 : c - 1;
#pragma unroll
        for (int k = 0; k < NM; ++k) val = fmaf(sV[r * NM + k], xi[i * NM + k], val);
        if (r != 0) val *= Real<float>::INV_SQRT2;
      }
      out[t] = val;
    }
    __syncwarp();
  }
}

template <int N>
int launch_dtau(const int4* tets, const float* geo, const float* u0, const float* v, const uint8_t* dmask,
                const float* eig, const float* l0, float* dT, int64_t n_elem, cudaStream_t st) {
  using L = DtauLayout<N>;
  if (n_elem <= 0) return 0;
  const int warps = 8;
  const size_t smem = (size_t)warps * L::WARP * sizeof(float);
  if (smem > 227 * 1024) return -6;
  cudaFuncSetAttribute(dtau_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int64_t n_qp = 4 * n_elem;
  int64_t blocks = (n_qp + warps - 1) / warps;
  if (blocks > 152 * 64) blocks = 152 * 64;
  count_launches(1);
  dtau_kernel<N><<<(int)blocks, warps * 32, smem, st>>>(tets, geo, u0, v, dmask, eig, l0, dT, n_qp);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

#define TS_INST_DTAU(T, N)                                                                                   \
  template int launch_dtau<N>(const int4*, const float*, const float*, const float*, const uint8_t*,         \
                              const float*, const float*, float*, int64_t, cudaStream_t);
TS_FOR_EACH_N(TS_INST_DTAU, float)

}  // namespace ts
