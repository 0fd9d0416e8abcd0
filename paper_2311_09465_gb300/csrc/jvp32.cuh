// FP32 tangent product of eq. (K_mat), section 2.4 -- the GMRES hot loop.
//
// Same arithmetic as the element operator in apply.cu (see the formulas
// there): per quadrature point the convective products c_i = A_j dv_i/dx_j
// (+ A(v_j) du0_i/dx_j for the LIN_A variant) are formed on K = 3N-2 time
// samples and truncated back to |m| < N, L_i is multiplied by the cached
// tau_q, T_i is sampled again for the SUPG sum sum_q w A_j T_i.
//
// GB300 mapping (one launch per product):
//  * 3 lanes per element, lane i owns velocity component i: its transforms,
//    tau matvec, Galerkin/SUPG/viscous/mass rows; 10 elements per warp.
//  * The DFT matrices live in __constant__ memory and every index is a
//    compile-time constant, so each transform is a chain of FFMAs with a
//    constant-bank operand and register inputs.
//  * tau for the warp's 10 consecutive elements (a contiguous block of the
//    cache, the dominant HBM stream) is staged into shared memory with
//    16-byte loads; the three lanes of an element read it by broadcast.
//  * u0 at the nodes is read as precomputed time samples (one transform per
//    node per Newton step instead of one per element per product).
//  * Results are added to the nodes with 8-byte vector atomics (red), so
//    the whole product is one launch; Hv must be zero on entry.
// Included by the jvp32_n*.cu translation units, each of which defines
// J32_NLIST (the mode counts it instantiates) and J32_TAG (a name suffix).
#pragma once
#include "common.cuh"
#include "kernels.h"

namespace ts {
namespace {

// ---------------------------------------------------------------- DFT tables
// forward [K][C] then inverse [C][K] for each N of this unit, concatenated
__host__ __device__ constexpr int dft_size(int N) { return 2 * (3 * N - 2) * (2 * N); }
__host__ __device__ constexpr int dft_offset(int N) {
  const int list[] = {J32_NLIST};
  int off = 0;
  for (int n : list) {
    if (n == N) return off;
    off += dft_size(n);
  }
  return -1;
}
__host__ __device__ constexpr int dft_total() {
  const int list[] = {J32_NLIST};
  int off = 0;
  for (int n : list) off += dft_size(n);
  return off;
}

__constant__ float c_dft[dft_total()];

template <int N>
__device__ __forceinline__ float CF(int k, int c) {   // forward coefficient
  return c_dft[dft_offset(N) + k * (2 * N) + c];
}
template <int N>
__device__ __forceinline__ float CI(int c, int k) {   // inverse coefficient
  return c_dft[dft_offset(N) + (3 * N - 2) * (2 * N) + c * (3 * N - 2) + k];
}

// modes (storage coordinates) -> K samples
template <int N>
__device__ __forceinline__ void fwd(const float (&x)[2 * N], float (&y)[3 * N - 2]) {
#pragma unroll
  for (int k = 0; k < 3 * N - 2; ++k) {
    float acc = x[0] * CF<N>(k, 0);
#pragma unroll
    for (int c = 2; c < 2 * N; ++c) acc = fmaf(x[c], CF<N>(k, c), acc);
    y[k] = acc;
  }
}
// K samples -> modes |m| < N (the exact truncated product)
template <int N>
__device__ __forceinline__ void inv(const float (&x)[3 * N - 2], float (&y)[2 * N]) {
#pragma unroll
  for (int c = 0; c < 2 * N; ++c) {
    if (c == 1) {
      y[c] = 0.f;
      continue;
    }
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < 3 * N - 2; ++k) acc = fmaf(x[k], CI<N>(c, k), acc);
    y[c] = acc;
  }
}

template <int N>
__device__ __forceinline__ float om_apply(const float (&x)[2 * N], int c, float omega) {
  const int n = c >> 1;
  if (n == 0) return 0.f;
  return (c & 1) ? float(n) * omega * x[c - 1] : -float(n) * omega * x[c + 1];
}

constexpr int EPW = 10;   // elements per warp (3 lanes each)

template <int N, int MODE>
struct J32Layout {
  static constexpr int C = 2 * N, K = 3 * N - 2, NTP = Dims<N>::NT_PAD;
  static constexpr bool LINA = MODE == MODE_JVP_LIN_A;
  static constexpr int TS = 4 * NTP + 4;              // tau stride per element (16 B multiple)
  static constexpr int US = (12 * K) | 1;             // u0 samples per element, odd stride
  static constexpr int TAU = 0;
  static constexpr int U = TAU + EPW * TS;
  static constexpr int VS = U + EPW * US;             // LIN_A: v samples at the points
  static constexpr int OUT = VS + (LINA ? EPW * US : 0);   // per lane [4*C][32]
  static constexpr int GT = OUT + 4 * C * 32;                 // per lane [3][C][32]: SUPG sums (modes)
  // per-warp stride rounded to 16 bytes: the tau block at offset 0 of every
  // warp's workspace is written with 16-byte stores
  static constexpr int WARP = (GT + 3 * C * 32 + 3) & ~3;
  static_assert(TAU % 4 == 0 && TS % 4 == 0 && WARP % 4 == 0, "16-byte alignment of the tau block");
};

template <int N, int MODE>
__global__ void __launch_bounds__(32 * 6, 1)
    jvp32_kernel(const int4* __restrict__ tets, const float* __restrict__ geo,
                 const float* __restrict__ v, const float* __restrict__ u0t,
                 const float* __restrict__ tau, const float* __restrict__ t0cache,
                 const uint8_t* __restrict__ dmask, float* __restrict__ out, Phys<float> ph,
                 int64_t n_elem) {
  constexpr int C = 2 * N, K = 3 * N - 2, NM = 2 * N - 1, NTP = Dims<N>::NT_PAD;
  using L = J32Layout<N, MODE>;
  constexpr bool PAPER = MODE == MODE_JVP_PAPER;
  constexpr bool LINA = MODE == MODE_JVP_LIN_A;
  constexpr float QA = 0.5854101966249685f, QB = 0.1381966011250105f;
  extern __shared__ __align__(16) float smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* ws = smem + warp * L::WARP;
  float* s_tau = ws + L::TAU;
  float* s_u = ws + L::U;
  float* s_v = ws + L::VS;
  float* s_out = ws + L::OUT;
  float* s_gt = ws + L::GT;   // [(j*C + c)*32 + lane]
  const bool active = lane < 3 * EPW;
  const int el = active ? lane / 3 : 0, ci = active ? lane - 3 * (lane / 3) : 0;
  const int wpb = blockDim.x >> 5;
  const float rho = ph.rho, omega = ph.omega;

  for (int64_t base = ((int64_t)blockIdx.x * wpb + warp) * EPW; base < n_elem;
       base += (int64_t)gridDim.x * wpb * EPW) {
    const int nvalid = (int)((n_elem - base) < EPW ? (n_elem - base) : EPW);
    const int64_t e = base + el;
    const bool live = active && el < nvalid;
    __syncwarp();
    // ---- stage tau of the warp's elements (contiguous in the cache)
    {
      const float4* src = reinterpret_cast<const float4*>(tau + base * 4 * NTP);
      const int n4 = nvalid * NTP;   // float4 count (4*NTP floats per element)
      for (int t = lane; t < n4; t += 32) {
        const int ee = t / NTP, r = t - ee * NTP;
        reinterpret_cast<float4*>(s_tau + ee * L::TS)[r] = src[t];
      }
    }
    // ---- per-lane element data
    int node[4] = {0, 0, 0, 0};
    float dN[12], vol = 0.f;
#pragma unroll
    for (int j = 0; j < 12; ++j) dN[j] = 0.f;
    if (live) {
      const int4 nd = tets[e];
      node[0] = nd.x;
      node[1] = nd.y;
      node[2] = nd.z;
      node[3] = nd.w;
      const float* g = geo + e * GEO_STRIDE;
#pragma unroll
      for (int j = 0; j < 12; ++j) dN[j] = g[j];
      vol = g[GEO_VOL];
    }
    // velocity component ci at the nodes (masked) and the pressure gradient
    float S[C], dp[C];
    float gt[3][K];   // dv_ci/dx_j on samples
    {
      float gi[3][C];
#pragma unroll
      for (int c = 0; c < C; ++c) {
        S[c] = 0.f;
        dp[c] = 0.f;
        gi[0][c] = gi[1][c] = gi[2][c] = 0.f;
      }
      if (live) {
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const float* va = v + (int64_t)node[a] * 4 * C;
          const bool fixed = dmask[node[a]] != 0;
#pragma unroll
          for (int c = 0; c < C; ++c) {
            const float x = (c == 1 || fixed) ? 0.f : va[ci * C + c];
            const float p = (c == 1) ? 0.f : va[3 * C + c];
            S[c] += x;
            gi[0][c] = fmaf(dN[a * 3 + 0], x, gi[0][c]);
            gi[1][c] = fmaf(dN[a * 3 + 1], x, gi[1][c]);
            gi[2][c] = fmaf(dN[a * 3 + 2], x, gi[2][c]);
            dp[c] = fmaf(dN[a * 3 + ci], p, dp[c]);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < 3; ++j) fwd<N>(gi[j], gt[j]);
    }
    // u0 component ci at the points (samples) -> shared; LIN_A also du0_ci/dx_j
    float gu[3][K];
    {
      float un[4][K];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int k = 0; k < K; ++k)
          un[a][k] = live ? u0t[((int64_t)node[a] * 3 + ci) * K + k] : 0.f;
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const float s = un[0][k] + un[1][k] + un[2][k] + un[3][k];
          if (live) s_u[el * L::US + (q * 3 + ci) * K + k] = QB * s + (QA - QB) * un[q][k];
        }
      if (LINA) {
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
          for (int k = 0; k < K; ++k)
            gu[j][k] = dN[0 * 3 + j] * un[0][k] + dN[1 * 3 + j] * un[1][k] +
                       dN[2 * 3 + j] * un[2][k] + dN[3 * 3 + j] * un[3][k];
      }
    }
    if (LINA) {
      // v component ci at each point, sampled -> shared
#pragma unroll 1
      for (int q = 0; q < 4; ++q) {
        float vq[C], vt[K];
        const float* vqn = v + (int64_t)node[q] * 4 * C;
        const bool fixed = live ? dmask[node[q]] != 0 : true;
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const float x = (!live || c == 1 || fixed) ? 0.f : vqn[ci * C + c];
          vq[c] = QB * S[c] + (QA - QB) * x;
        }
        fwd<N>(vq, vt);
        if (live)
#pragma unroll
          for (int k = 0; k < K; ++k) s_v[el * L::US + (q * 3 + ci) * K + k] = vt[k];
      }
    }
    // zero the per-lane output rows
#pragma unroll
    for (int t = 0; t < 4 * C; ++t) s_out[t * 32 + lane] = 0.f;
    __syncwarp();

    float W[3][K], sumTc[C];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int k = 0; k < K; ++k) W[j][k] = 0.f;
#pragma unroll
    for (int c = 0; c < C; ++c) sumTc[c] = 0.f;
    const float* tq_base = s_tau + el * L::TS;
    const float* u_base = s_u + el * L::US;
    const float* v_base = s_v + el * L::US;

#pragma unroll 1
    for (int q = 0; q < 4; ++q) {
      // c_ci = u0_j dv_ci/dx_j (+ v_j du0_ci/dx_j) on samples, truncated to modes
      float ct[K], cm[C];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        float acc = 0.f;
#pragma unroll
        for (int j = 0; j < 3; ++j) acc = fmaf(u_base[(q * 3 + j) * K + k], gt[j][k], acc);
        if (LINA) {
#pragma unroll
          for (int j = 0; j < 3; ++j) acc = fmaf(v_base[(q * 3 + j) * K + k], gu[j][k], acc);
        }
        ct[k] = acc;
      }
      inv<N>(ct, cm);
      // v_ci at the point (modes) and rho (Omega v + c)
      float vq[C], G[C], Lm[C];
      {
        const float* vqn = v + (int64_t)node[q] * 4 * C;
        const bool fixed = live ? dmask[node[q]] != 0 : true;
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const float x = (!live || c == 1 || fixed) ? 0.f : vqn[ci * C + c];
          vq[c] = QB * S[c] + (QA - QB) * x;
        }
      }
#pragma unroll
      for (int c = 0; c < C; ++c) {
        G[c] = (c == 1) ? 0.f : rho * (om_apply<N>(vq, c, omega) + cm[c]);
        Lm[c] = PAPER ? G[c] : G[c] + dp[c];
      }
      // T = tau_q L (packed symmetric tau in the orthonormal basis; storage scaling)
      const float* tp = tq_base + q * NTP;
      float T[C], Tc[C];
#pragma unroll
      for (int r = 0; r < NM; ++r) {
        float acc = 0.f, accp = 0.f;
#pragma unroll
        for (int kk = 0; kk < NM; ++kk) {
          const int a = r < kk ? r : kk, b = r < kk ? kk : r;
          float t = tp[packed_index(a, b, NM)];
          if (r == 0 && kk > 0) t *= Real<float>::SQRT2;
          if (r > 0 && kk == 0) t *= Real<float>::INV_SQRT2;
          acc = fmaf(t, Lm[stor_of(kk)], acc);
          if (PAPER) accp = fmaf(t, dp[stor_of(kk)], accp);
        }
        T[stor_of(r)] = acc;
        Tc[stor_of(r)] = accp;
      }
      T[1] = 0.f;
      Tc[1] = 0.f;
#pragma unroll
      for (int c = 0; c < C; ++c) sumTc[c] += PAPER ? Tc[c] : T[c];
      // Galerkin + (-Omega N_a) LS terms: sum_q w N_a(q) [G - Omega T]
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const float X = G[c] - om_apply<N>(T, c, omega);
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const float lam = (a == q) ? QA : QB;
          s_out[(a * C + c) * 32 + lane] += lam * X;
        }
      }
      // SUPG on samples: W_j += u0_j T (+ v_j T0)
      float Tt[K];
      fwd<N>(T, Tt);
      float T0t[K];
      if (LINA) {
        float T0m[C];
        const float* t0p = t0cache + ((e * 4 + q) * 3 + ci) * C;
#pragma unroll
        for (int c = 0; c < C; ++c) T0m[c] = live ? t0p[c] : 0.f;
        fwd<N>(T0m, T0t);
      }
#pragma unroll
      for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < K; ++k) {
          float acc = fmaf(u_base[(q * 3 + j) * K + k], Tt[k], W[j][k]);
          if (LINA) acc = fmaf(v_base[(q * 3 + j) * K + k], T0t[k], acc);
          W[j][k] = acc;
        }
    }
    // SUPG sums to modes, kept in this lane's shared rows (reusing the gradient rows)
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float Wm[C];
      inv<N>(W[j], Wm);
#pragma unroll
      for (int c = 0; c < C; ++c) s_gt[(j * C + c) * 32 + lane] = Wm[c];
    }
    // dv_ci/dx_ci (this lane's share of the divergence) and the mean pressure
    float divc[C], pbar[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      divc[c] = 0.f;
      pbar[c] = 0.f;
    }
    if (live) {
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const float* vb = v + (int64_t)node[b] * 4 * C;
        const bool fixed = dmask[node[b]] != 0;
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const float x = (c == 1 || fixed) ? 0.f : vb[ci * C + c];
          divc[c] = fmaf(dN[b * 3 + ci], x, divc[c]);
          pbar[c] += (c == 1) ? 0.f : 0.25f * vb[3 * C + c];
        }
      }
    }
    const float w4 = 0.25f * vol;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      // viscous term through the element stiffness: sum_b (grad N_a . grad N_b) v_b
      float vis[C], va_own[C];
#pragma unroll
      for (int c = 0; c < C; ++c) {
        vis[c] = 0.f;
        va_own[c] = 0.f;
      }
      if (live) {
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const float kab = dN[a * 3] * dN[b * 3] + dN[a * 3 + 1] * dN[b * 3 + 1] + dN[a * 3 + 2] * dN[b * 3 + 2];
          const float* vb = v + (int64_t)node[b] * 4 * C;
          const bool fixed = dmask[node[b]] != 0;
#pragma unroll
          for (int c = 0; c < C; ++c) {
            const float x = (c == 1 || fixed) ? 0.f : vb[ci * C + c];
            vis[c] = fmaf(kab, x, vis[c]);
            if (b == a) va_own[c] = x;
          }
        }
      }
      float m[C], cont[C];
#pragma unroll
      for (int c = 0; c < C; ++c) {
        if (c == 1) {
          m[c] = 0.f;
          cont[c] = 0.f;
          continue;
        }
        float x = w4 * s_out[(a * C + c) * 32 + lane];
        x += w4 * (dN[a * 3 + 0] * s_gt[(0 * C + c) * 32 + lane] + dN[a * 3 + 1] * s_gt[(1 * C + c) * 32 + lane] +
                   dN[a * 3 + 2] * s_gt[(2 * C + c) * 32 + lane]);
        x += ph.mu * vol * vis[c];
        x -= dN[a * 3 + ci] * vol * pbar[c];
        if (ph.mass_coef != 0.f) x += ph.mass_coef * vol * 0.05f * (S[c] + va_own[c]);
        m[c] = x;
        // continuity: this lane's share of w div + (w/rho) dN_a/dx_ci sum_q Tc_ci
        cont[c] = w4 * divc[c] + (w4 / rho) * dN[a * 3 + ci] * sumTc[c];
      }
      // reduce the continuity row over the element's three lanes
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const float x1 = __shfl_down_sync(0xffffffffu, cont[c], 1);
        const float x2 = __shfl_down_sync(0xffffffffu, cont[c], 2);
        cont[c] += x1 + x2;
      }
      // scatter-add (8-byte vector atomics); fixed rows are skipped
      if (live) {
        float* dst = out + (int64_t)node[a] * 4 * C;
        if (!dmask[node[a]]) {
#pragma unroll
          for (int c = 0; c < C; c += 2) atomicAdd(reinterpret_cast<float2*>(dst + ci * C + c), make_float2(m[c], m[c + 1]));
        }
        if (ci == 0) {
#pragma unroll
          for (int c = 0; c < C; c += 2)
            atomicAdd(reinterpret_cast<float2*>(dst + 3 * C + c), make_float2(cont[c], cont[c + 1]));
        }
      }
    }
  }
}

// u0 at the nodes sampled in time: u0t[V][3][K]
template <int N>
__global__ void node_samples_kernel(const float* __restrict__ u0, float* __restrict__ u0t,
                                    int64_t V) {
  constexpr int C = 2 * N, K = 3 * N - 2;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < V * 3;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t node = t / 3;
    const int i = (int)(t - node * 3);
    float x[C], y[K];
#pragma unroll
    for (int c = 0; c < C; ++c) x[c] = (c == 1) ? 0.f : u0[node * 4 * C + i * C + c];
    fwd<N>(x, y);
#pragma unroll
    for (int k = 0; k < K; ++k) u0t[t * K + k] = y[k];
  }
}

template <int N>
static int launch_node_samples_impl(const float* u0, float* u0t, int64_t V, cudaStream_t st) {
  int64_t blocks = (V * 3 + 127) / 128;
  if (blocks > 152 * 16) blocks = 152 * 16;
  count_launches(1);
  node_samples_kernel<N><<<(int)blocks, 128, 0, st>>>(u0, u0t, V);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

template <int N, int MODE>
static int launch_j32_mode(const int4* tets, const float* geo, const float* v, const float* u0t,
                           const float* tau, const float* t0, const uint8_t* dmask, float* out,
                           Phys<float> ph, int64_t n_elem, cudaStream_t st) {
  using L = J32Layout<N, MODE>;
  int warps = 6;
  while (warps > 1 && (size_t)warps * L::WARP * sizeof(float) > 220 * 1024) --warps;
  const size_t smem = (size_t)warps * L::WARP * sizeof(float);
  cudaFuncSetAttribute(jvp32_kernel<N, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int64_t warps_needed = (n_elem + EPW - 1) / EPW;
  int64_t blocks = (warps_needed + warps - 1) / warps;
  if (blocks > 152 * 4) blocks = 152 * 4;
  if (blocks < 1) blocks = 1;
  count_launches(1);
  jvp32_kernel<N, MODE><<<(int)blocks, warps * 32, smem, st>>>(tets, geo, v, u0t, tau, t0, dmask,
                                                               out, ph, n_elem);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

template <int N>
static int launch_jvp32_impl(int mode, const int4* tets, const float* geo, const float* v, const float* u0t,
                 const float* tau, const float* t0, const uint8_t* dmask, float* out,
                 Phys<float> ph, int64_t n_elem, cudaStream_t st) {
  switch (mode) {
    case MODE_JVP_PAPER:
      return launch_j32_mode<N, MODE_JVP_PAPER>(tets, geo, v, u0t, tau, t0, dmask, out, ph, n_elem, st);
    case MODE_JVP_FROZEN:
      return launch_j32_mode<N, MODE_JVP_FROZEN>(tets, geo, v, u0t, tau, t0, dmask, out, ph, n_elem, st);
    case MODE_JVP_LIN_A:
      return launch_j32_mode<N, MODE_JVP_LIN_A>(tets, geo, v, u0t, tau, t0, dmask, out, ph, n_elem, st);
  }
  return -1;
}

}  // namespace

// copies this unit's tables (sliced from the table of all compiled N)
static int j32_upload_impl(const float* host_all, int (*global_offset)(int)) {
  static int device_mask = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 31 && ((device_mask >> dev) & 1)) return 0;
  float local[dft_total()];
  const int list[] = {J32_NLIST};
  for (int n : list) {
    const float* src = host_all + global_offset(n);
    for (int t = 0; t < dft_size(n); ++t) local[dft_offset(n) + t] = src[t];
  }
  if (cudaMemcpyToSymbol(c_dft, local, sizeof(local)) != cudaSuccess) return -2;
  if (dev < 31) device_mask |= 1 << dev;
  return 0;
}

template <int N>
int launch_jvp32(int mode, const int4* tets, const float* geo, const float* v, const float* u0t,
                 const float* tau, const float* t0, const uint8_t* dmask, float* out,
                 Phys<float> ph, int64_t n_elem, cudaStream_t st) {
  return launch_jvp32_impl<N>(mode, tets, geo, v, u0t, tau, t0, dmask, out, ph, n_elem, st);
}

template <int N>
int launch_node_samples(const float* u0, float* u0t, int64_t V, cudaStream_t st) {
  return launch_node_samples_impl<N>(u0, u0t, V, st);
}

}  // namespace ts
