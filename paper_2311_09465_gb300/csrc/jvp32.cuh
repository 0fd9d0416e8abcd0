// FP32 tangent product of eq. (K_mat), section 2.4 -- the GMRES hot loop.
//
// Same arithmetic as the element operator in apply.cu (see the formulas
// there): per quadrature point the convective products c_i = A_j dv_i/dx_j
// (+ A(v_j) du0_i/dx_j for the LIN_A variant) are formed on K = 3N-2 time
// samples and truncated back to |m| < N, L_i is multiplied by the cached
// tau_q, T_i is sampled again for the SUPG sum sum_q w A_j T_i.
//
// GB300 mapping (one launch per product):
//  * 16 lanes per element (velocity component or pressure x quadrature
//    point / node), two elements per warp; see the mapping note below.
//  * The DFT matrices live in __constant__ memory and every index is a
//    compile-time constant, so each transform is a chain of FFMAs with a
//    constant-bank operand and register inputs.
//  * tau of a quadrature point (the dominant HBM stream) is read with 16-byte
//    loads straight into the registers of the three lanes of that point.
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

// ---------------------------------------------------------------- mapping
// 16 lanes per element, two elements per warp.  Lane (f, q): f = lane/4
// within the element's half warp (0..2 a velocity component, 3 the
// pressure/continuity lane), q = lane%4 (the quadrature point in the point
// phase, the node in the node phases).  Node-level reductions go through
// shared memory; sums over the four points are xor butterflies over q in
// converged code.  tau of point q sits in the registers of the three
// velocity lanes of that point.
constexpr int EPW = 2;    // elements per warp (16 lanes each)

template <int N, int MODE>
struct J32Layout {
  static constexpr int C = 2 * N, K = 3 * N - 2;
  static constexpr bool LINA = MODE == MODE_JVP_LIN_A;
  // per element (floats)
  static constexpr int VN = 0;                       // v at the nodes [4 a][4 f][C]
  static constexpr int GM = VN + 16 * C;             // gradients [4 f][3 j][C]
  static constexpr int GT = GM + 12 * C;             // dv_i/dx_j samples [3 i][3 j][K]
  static constexpr int UQ = GT + 9 * K;              // u0 samples: nodes, then points [4][3 j][K]
  static constexpr int WM = UQ + 12 * K;             // SUPG sums, modes [3 j][3 i][C]
  static constexpr int GU = WM + 9 * C;              // LIN_A: du0_i/dx_j samples [3 i][3 j][K]
  static constexpr int VQ = GU + (LINA ? 9 * K : 0); // LIN_A: v at the points, samples [4 q][3 j][K]
  static constexpr int ELEM = (VQ + (LINA ? 12 * K : 0) + 3) & ~3;
  static constexpr int WARP = EPW * ELEM;
};

// The EPW elements base, base + 1 of instance I on one warp; wsm is the
// warp's shared-memory region (J32Layout<N, MODE>::WARP floats).
template <int N, int MODE>
__device__ __forceinline__ void j32_pass(const J32Inst& I, int64_t base, float* wsm, int lane) {
  constexpr int C = 2 * N, K = 3 * N - 2, NM = 2 * N - 1, NTP = Dims<N>::NT_PAD;
  using L = J32Layout<N, MODE>;
  constexpr bool PAPER = MODE == MODE_JVP_PAPER;
  constexpr bool LINA = MODE == MODE_JVP_LIN_A;
  constexpr float QA = 0.5854101966249685f, QB = 0.1381966011250105f, QD = QA - QB;
  constexpr unsigned FULL = 0xffffffffu;
  const int4* __restrict__ tets = I.tets;
  const float* __restrict__ geo = I.geo;
  const float* __restrict__ v = I.v;
  const float* __restrict__ u0t = I.u0t;
  const float* __restrict__ tau = I.tau;
  const float* __restrict__ t0cache = I.t0cache;
  const uint8_t* __restrict__ dmask = I.dmask;
  float* __restrict__ out = I.out;
  const Phys<float>& ph = I.ph;
  const int64_t n_elem = I.n_elem;
  const int slot = lane >> 4, f = (lane >> 2) & 3, q = lane & 3;
  float* es = wsm + slot * L::ELEM;
  float* s_vn = es + L::VN;
  float* s_gm = es + L::GM;
  float* s_gt = es + L::GT;
  float* s_uq = es + L::UQ;
  float* s_wm = es + L::WM;
  float* s_gu = es + L::GU;
  float* s_vq = es + L::VQ;
  const float rho = ph.rho, omega = ph.omega;
  {
    const int64_t e = base + slot;
    const bool live = e < n_elem;
    __syncwarp();
    // ---- element data (all lanes of the element read the same record)
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
    const int my_node = q == 0 ? node[0] : q == 1 ? node[1] : q == 2 ? node[2] : node[3];
    const bool my_fixed = live ? dmask[my_node] != 0 : true;
    // tau of point q into registers (velocity lanes)
    float tv[NTP];
    if (live && f < 3) {
      const float4* tp = reinterpret_cast<const float4*>(tau + (e * 4 + q) * NTP);
#pragma unroll
      for (int t = 0; t < NTP / 4; ++t) {
        const float4 x = tp[t];
        tv[4 * t] = x.x;
        tv[4 * t + 1] = x.y;
        tv[4 * t + 2] = x.z;
        tv[4 * t + 3] = x.w;
      }
    } else {
#pragma unroll
      for (int t = 0; t < NTP; ++t) tv[t] = 0.f;
    }
    // ---- P0: lane (f, a = q) stores field f of node a; velocity lanes store u0 samples of node a
    {
      const float* src = v + (int64_t)my_node * 4 * C + f * C;
#pragma unroll
      for (int c = 0; c < C; ++c)
        s_vn[(q * 4 + f) * C + c] = (!live || c == 1 || (f < 3 && my_fixed)) ? 0.f : src[c];
      if (f < 3) {
        const float* us = u0t + ((int64_t)my_node * 3 + f) * K;
#pragma unroll
        for (int k = 0; k < K; ++k) s_uq[(q * 3 + f) * K + k] = live ? us[k] : 0.f;
      }
    }
    __syncwarp();
    // ---- P1: gradients (lane (f, j = q < 3)); u0 at the points (lane (j = f < 3, q))
    if (q < 3) {
#pragma unroll
      for (int c = 0; c < C; ++c) {
        float acc = 0.f;
#pragma unroll
        for (int a = 0; a < 4; ++a) acc = fmaf(dN[a * 3 + q], s_vn[(a * 4 + f) * C + c], acc);
        s_gm[(f * 3 + q) * C + c] = acc;
      }
    }
    float uq[K];
    if (f < 3) {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float u0k = s_uq[(0 * 3 + f) * K + k], u1k = s_uq[(1 * 3 + f) * K + k];
        const float u2k = s_uq[(2 * 3 + f) * K + k], u3k = s_uq[(3 * 3 + f) * K + k];
        const float uqk = s_uq[(q * 3 + f) * K + k];
        uq[k] = QB * (u0k + u1k + u2k + u3k) + QD * uqk;
        if (LINA && q < 3)   // du0_f/dx_q on samples
          s_gu[(f * 3 + q) * K + k] = dN[0 * 3 + q] * u0k + dN[1 * 3 + q] * u1k + dN[2 * 3 + q] * u2k +
                                      dN[3 * 3 + q] * u3k;
      }
    }
    __syncwarp();
    if (f < 3) {
#pragma unroll
      for (int k = 0; k < K; ++k) s_uq[(q * 3 + f) * K + k] = uq[k];   // now u0 at point q
    }
    // ---- P2: gradient samples (lane (i = f < 3, j = q < 3)); LIN_A: v at the points sampled
    if (f < 3 && q < 3) {
      float gm[C], gt[K];
#pragma unroll
      for (int c = 0; c < C; ++c) gm[c] = s_gm[(f * 3 + q) * C + c];
      fwd<N>(gm, gt);
#pragma unroll
      for (int k = 0; k < K; ++k) s_gt[(f * 3 + q) * K + k] = gt[k];
    }
    if (LINA && f < 3) {
      float vm[C], vt[K];
#pragma unroll
      for (int c = 0; c < C; ++c)
        vm[c] = QB * (s_vn[(0 * 4 + f) * C + c] + s_vn[(1 * 4 + f) * C + c] + s_vn[(2 * 4 + f) * C + c] +
                      s_vn[(3 * 4 + f) * C + c]) +
                QD * s_vn[(q * 4 + f) * C + c];
      fwd<N>(vm, vt);
#pragma unroll
      for (int k = 0; k < K; ++k) s_vq[(q * 3 + f) * K + k] = vt[k];
    }
    __syncwarp();
    // ---- P3: point phase, lane (i = f < 3, q)
    float Wp[3][K], X[C], sX[C], sT[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      X[c] = 0.f;
      sT[c] = 0.f;
    }
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int k = 0; k < K; ++k) Wp[j][k] = 0.f;
    if (f < 3) {
      const int i = f;
      // c_i = u0_j dv_i/dx_j (+ v_j du0_i/dx_j) on samples, truncated to modes
      float ct[K], cm[C];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        float acc = 0.f;
#pragma unroll
        for (int j = 0; j < 3; ++j) acc = fmaf(s_uq[(q * 3 + j) * K + k], s_gt[(i * 3 + j) * K + k], acc);
        if (LINA) {
#pragma unroll
          for (int j = 0; j < 3; ++j) acc = fmaf(s_vq[(q * 3 + j) * K + k], s_gu[(i * 3 + j) * K + k], acc);
        }
        ct[k] = acc;
      }
      inv<N>(ct, cm);
      float G[C], Lm[C], dp[C];
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const float vq = QB * (s_vn[(0 * 4 + i) * C + c] + s_vn[(1 * 4 + i) * C + c] +
                               s_vn[(2 * 4 + i) * C + c] + s_vn[(3 * 4 + i) * C + c]) +
                         QD * s_vn[(q * 4 + i) * C + c];
        X[c] = vq;   // temporarily v_i at the point
        dp[c] = s_gm[(3 * 3 + i) * C + c];
      }
#pragma unroll
      for (int c = 0; c < C; ++c) {
        G[c] = (c == 1) ? 0.f : rho * (om_apply<N>(X, c, omega) + cm[c]);
        Lm[c] = PAPER ? G[c] : G[c] + dp[c];
      }
      // T = tau_q L, Tc = tau_q dp (PAPER); packed symmetric tau, storage scaling
      float T[C], Tc[C];
#pragma unroll
      for (int r = 0; r < NM; ++r) {
        float acc = 0.f, accp = 0.f;
#pragma unroll
        for (int kk = 0; kk < NM; ++kk) {
          const int a = r < kk ? r : kk, b = r < kk ? kk : r;
          float t = tv[packed_index(a, b, NM)];
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
      for (int c = 0; c < C; ++c) {
        sT[c] = PAPER ? Tc[c] : T[c];
        X[c] = G[c] - om_apply<N>(T, c, omega);
      }
      // SUPG products on samples: Wp_j = u0_j T (+ v_j T0)
      float Tt[K];
      fwd<N>(T, Tt);
      float T0t[K];
      if (LINA) {
        float T0m[C];
        const float* t0p = t0cache + ((e * 4 + q) * 3 + i) * C;
#pragma unroll
        for (int c = 0; c < C; ++c) T0m[c] = live ? t0p[c] : 0.f;
        fwd<N>(T0m, T0t);
      }
#pragma unroll
      for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < K; ++k) {
          float acc = s_uq[(q * 3 + j) * K + k] * Tt[k];
          if (LINA) acc = fmaf(s_vq[(q * 3 + j) * K + k], T0t[k], acc);
          Wp[j][k] = acc;
        }
    }
    // ---- P4: sums over the four points (xor butterflies over q, converged code)
#pragma unroll
    for (int c = 0; c < C; ++c) {
      float x = X[c];
      x += __shfl_xor_sync(FULL, x, 1);
      x += __shfl_xor_sync(FULL, x, 2);
      sX[c] = x;
      float t = sT[c];
      t += __shfl_xor_sync(FULL, t, 1);
      t += __shfl_xor_sync(FULL, t, 2);
      sT[c] = t;
    }
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int k = 0; k < K; ++k) {
        float w = Wp[j][k];
        w += __shfl_xor_sync(FULL, w, 1);
        w += __shfl_xor_sync(FULL, w, 2);
        Wp[j][k] = w;
      }
    // ---- P5: SUPG sums to modes, lane (i = f < 3, j = q < 3)
    if (f < 3 && q < 3) {
      float wt[K], wm[C];
#pragma unroll
      for (int k = 0; k < K; ++k) wt[k] = (q == 0) ? Wp[0][k] : (q == 1) ? Wp[1][k] : Wp[2][k];
      inv<N>(wt, wm);
#pragma unroll
      for (int c = 0; c < C; ++c) s_wm[(q * 3 + f) * C + c] = wm[c];
    }
    // continuity lanes fetch sum_q Tc_i from the velocity lanes (i, q) of their node
    float sTi[3][C];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int c = 0; c < C; ++c) sTi[i][c] = __shfl_sync(FULL, sT[c], (lane & 16) | (i << 2) | q);
    __syncwarp();
    // ---- P6: node phase, lane (f, a = q): the row of field f at node a
    const int a = q;
    const float w4 = 0.25f * vol;
    float row[C];
    if (f < 3) {
      const int i = f;
#pragma unroll
      for (int c = 0; c < C; ++c) {
        float m = w4 * (QB * sX[c] + QD * X[c]);                         // Galerkin + (-Omega N_a) LS
        float supg = 0.f, visc = 0.f;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          supg = fmaf(dN[a * 3 + j], s_wm[(j * 3 + i) * C + c], supg);
          visc = fmaf(dN[a * 3 + j], s_gm[(i * 3 + j) * C + c], visc);
        }
        m += w4 * supg + ph.mu * vol * visc;
        const float pbar = 0.25f * (s_vn[(0 * 4 + 3) * C + c] + s_vn[(1 * 4 + 3) * C + c] +
                                    s_vn[(2 * 4 + 3) * C + c] + s_vn[(3 * 4 + 3) * C + c]);
        m -= dN[a * 3 + i] * vol * pbar;
        if (ph.mass_coef != 0.f) {
          const float sum = s_vn[(0 * 4 + i) * C + c] + s_vn[(1 * 4 + i) * C + c] + s_vn[(2 * 4 + i) * C + c] +
                            s_vn[(3 * 4 + i) * C + c];
          m += ph.mass_coef * vol * 0.05f * (sum + s_vn[(a * 4 + i) * C + c]);
        }
        row[c] = (c == 1 || my_fixed) ? 0.f : m;
      }
    } else {
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const float div = s_gm[(0 * 3 + 0) * C + c] + s_gm[(1 * 3 + 1) * C + c] + s_gm[(2 * 3 + 2) * C + c];
        const float ls = dN[a * 3 + 0] * sTi[0][c] + dN[a * 3 + 1] * sTi[1][c] + dN[a * 3 + 2] * sTi[2][c];
        row[c] = (c == 1) ? 0.f : w4 * div + (w4 / rho) * ls;
      }
    }
    // scatter-add: 8-byte vector atomics of this lane's row (zero rows skipped)
    if (live && !(f < 3 && my_fixed)) {
      float* dst = out + (int64_t)my_node * 4 * C + f * C;
#pragma unroll
      for (int c = 0; c < C; c += 2) atomicAdd(reinterpret_cast<float2*>(dst + c), make_float2(row[c], row[c + 1]));
    }
  }
}

template <int N, int MODE>
__global__ void __launch_bounds__(128) jvp32_kernel(J32Inst I) {
  using L = J32Layout<N, MODE>;
  extern __shared__ __align__(16) float smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  for (int64_t base = ((int64_t)blockIdx.x * wpb + warp) * EPW; base < I.n_elem;
       base += (int64_t)gridDim.x * wpb * EPW)
    j32_pass<N, MODE>(I, base, smem + warp * L::WARP, lane);
}

__host__ __device__ constexpr bool j32_has(int N) { return dft_offset(N) >= 0; }

// Tangent products of many instances in one launch.  Tile t (EPW elements)
// belongs to the instance b with tile_off[b] <= t < tile_off[b + 1]; the
// instance and tile counts are read from the device (counts[0], counts[1]) so
// that a captured launch follows later changes of the tables; each warp
// takes tiles grid-stride and runs the body compiled for that instance's N
// (warp-uniform branch); shared memory is sized for the largest N.
template <int MODE, int NMAX>
__global__ void __launch_bounds__(128) jvp32_batch_kernel(const J32Inst* __restrict__ insts,
                                                          const int64_t* __restrict__ tile_off,
                                                          const int64_t* __restrict__ counts) {
  extern __shared__ __align__(16) float smem[];
  const int n_inst = (int)counts[0];
  const int64_t n_tiles = counts[1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  float* wsm = smem + warp * J32Layout<NMAX, MODE>::WARP;
  for (int64_t t = (int64_t)blockIdx.x * wpb + warp; t < n_tiles; t += (int64_t)gridDim.x * wpb) {
    int lo = 0, hi = n_inst - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tile_off[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const J32Inst I = insts[lo];
    const int64_t base = (t - tile_off[lo]) * EPW;
    switch (I.N) {
      case 1: if constexpr (j32_has(1)) j32_pass<1, MODE>(I, base, wsm, lane); break;
      case 2: if constexpr (j32_has(2)) j32_pass<2, MODE>(I, base, wsm, lane); break;
      case 3: if constexpr (j32_has(3)) j32_pass<3, MODE>(I, base, wsm, lane); break;
      case 4: if constexpr (j32_has(4)) j32_pass<4, MODE>(I, base, wsm, lane); break;
      case 5: if constexpr (j32_has(5)) j32_pass<5, MODE>(I, base, wsm, lane); break;
      case 7: if constexpr (j32_has(7)) j32_pass<7, MODE>(I, base, wsm, lane); break;
      default: break;
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
  const int warps = 4;
  const size_t smem = (size_t)warps * L::WARP * sizeof(float);
  cudaFuncSetAttribute(jvp32_kernel<N, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int64_t blocks = (n_elem + warps * EPW - 1) / (warps * EPW);
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  count_launches(1);
  J32Inst I{tets, geo, v, u0t, tau, t0, dmask, out, ph, n_elem, N};
  jvp32_kernel<N, MODE><<<(int)blocks, warps * 32, smem, st>>>(I);
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
