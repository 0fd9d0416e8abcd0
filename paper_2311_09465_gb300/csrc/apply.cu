// Element operator of the time-spectral GLS method: the residual of eq. (Rmc)
// and the tangent products of eq. (K_mat), section 2.4.
//
// Per element and quadrature point q (weights V/4, N_a = barycentric):
//   c_i   = A_j du_i/dx_j  formed on K = 3N-2 time samples:
//           modes -> samples (u_j at q, du_i/dx_j), pointwise product,
//           samples -> modes (exact truncated convolution, eq. phi-def)
//   L_i   = rho (Omega u_i + c_i) + dp/dx_i       (second derivatives dropped)
//   T_i   = tau_q L_i                              (tau from the cache, eq. 3D-tau)
//   r^m_ai += w [N_a rho(Omega u_i + c_i) - N_a Omega T_i] - dN_a/dx_i int p
//           + mu V dN_a/dx_j du_i/dx_j + dN_a/dx_j sum_q w A_j T_i
//   r^c_a  += w N_a du_i/dx_i + (w / rho) dN_a/dx_i T_i
// The SUPG sum sum_q w A_j T_i is formed on samples and transformed once.
// Modes: RESIDUAL (A, tau at the state itself; also stores T_i per point
// for the LIN_A product), JVP_PAPER (least-squares parts of G_i and D_j
// dropped, section 2.5.2: momentum LS sees tau rho(Omega v + A dv), continuity
// LS sees tau dp), JVP_FROZEN (all of eq. K_mat), JVP_LIN_A (FROZEN plus the
// derivative of A_j: rho A(v_j) du0_i/dx_j in c_i and dN_a/dx_j A(v_j) T0_i).
// Pseudo-time adds mass_coef * M v on momentum rows (section 2.5.3).
//
// GB300 mapping: one warp per element, all per-element arrays in a per-warp
// shared-memory workspace, lanes over output entries of each batched small
// contraction (DFT tables shared per CTA).  Elements of one colour share no
// node, so each warp adds its 4x4xC results to the nodes without atomics;
// the host launches the colours in order (deterministic).
#include <type_traits>

#include "common.cuh"
#include "ddfloat.cuh"
#include "kernels.h"

namespace ts {

template <int N, int MODE>
struct ApplyLayout {
  using D = Dims<N>;
  static constexpr int C = D::C, K = D::K, NM = D::NM;
  static constexpr bool LINA = MODE == MODE_JVP_LIN_A;
  static constexpr bool PAPER = MODE == MODE_JVP_PAPER;
  static constexpr int LDF = C | 1;   // odd strides: conflict-free row access
  static constexpr int LDI = K | 1;
  static constexpr int TABLES = K * LDF + C * LDI;
  // per-warp workspace offsets (elements of T)
  static constexpr int SG = 0;                       // geometry 20 (+4)
  static constexpr int SV = SG + 24;                 // v at nodes [4][4][C]
  static constexpr int SU = SV + 16 * C;             // u0 velocity at nodes [4][3][C]
  static constexpr int GV = SU + 12 * C;             // grad v [4 f][3 j][C]
  static constexpr int VQ = GV + 12 * C;             // v velocity at points [4][3][C]
  static constexpr int UQ = VQ + 12 * C;             // u0 velocity at points [4][3][C]
  static constexpr int PB = UQ + 12 * C;             // mean pressure [C]
  static constexpr int UQT = PB + C;                 // u0 at points, samples [4][3][K]
  static constexpr int GVT = UQT + 12 * K;           // grad v samples [3][3][K], later W samples
  static constexpr int CT = GVT + 9 * K;             // c samples [4][3][K], later T samples
  static constexpr int CQ = CT + 12 * K;             // rho(Omega v + c) modes [4][3][C]
  static constexpr int TQ = CQ + 12 * C;             // T modes [4][3][C]
  static constexpr int TC = TQ + 12 * C;             // PAPER: tau dp [4][3][C]
  static constexpr int WM = TC + (PAPER ? 12 * C : 0);   // W modes [3][3][C]
  static constexpr int TAU = WM + 9 * C;             // tau in storage coords [4][NM][NM]
  static constexpr int OUT = TAU + 4 * NM * NM;      // [4][4][C]
  static constexpr int GU = OUT + 16 * C;            // LIN_A: grad u0 [3][3][C]
  static constexpr int VQT = GU + (LINA ? 9 * C : 0);    // LIN_A: v at points samples
  static constexpr int GUT = VQT + (LINA ? 12 * K : 0);  // LIN_A: grad u0 samples
  static constexpr int T0 = GUT + (LINA ? 9 * K : 0);    // LIN_A: T0 modes
  static constexpr int T0T = T0 + (LINA ? 12 * C : 0);   // LIN_A: T0 samples
  static constexpr int END = T0T + (LINA ? 12 * K : 0);
  static constexpr int WARP = (END + 3) & ~3;
};

__device__ __forceinline__ float mad(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double mad(double a, double b, double c) { return ::fma(a, b, c); }
__device__ __forceinline__ ddv mad(ddv a, ddv b, ddv c) { return ddv(dd_fma(a.v, b.v, c.v)); }

// out[b*os + r] = sum_c M[r*ld + c] in[b*is + c]
template <typename T, int R, int CN>
__device__ __forceinline__ void warp_bmv(const T* __restrict__ M, int ld, const T* in, int is,
                                         T* out, int os, int B, int lane) {
  for (int t = lane; t < B * R; t += 32) {
    const int b = t / R, r = t - (t / R) * R;
    const T* mr = M + r * ld;
    const T* x = in + b * is;
    T acc = 0;
#pragma unroll
    for (int c = 0; c < CN; ++c) acc = mad(mr[c], x[c], acc);
    out[b * os + r] = acc;
  }
}

// (Omega x) in storage coordinates: mode n -> i n omega x_n
template <typename T>
__device__ __forceinline__ T omega_apply(const T* x, int c, T omega) {
  const int n = c >> 1;
  return (c & 1) ? T(n) * omega * x[c - 1] : -T(n) * omega * x[c + 1];
}

template <>
struct Real<ddv> {
  static __device__ __forceinline__ ddv sqrt2() { return ddv(dd{1.41421353816986083984375f, 2.4203234101944225e-08f}); }
  static __device__ __forceinline__ ddv inv_sqrt2() { return ddv(dd{0.707106769084930419921875f, 1.2101617050972112e-08f}); }
};
template <typename T>
__device__ __forceinline__ T sqrt2_of() { return Real<T>::SQRT2; }
template <>
__device__ __forceinline__ ddv sqrt2_of<ddv>() { return Real<ddv>::sqrt2(); }
template <typename T>
__device__ __forceinline__ T inv_sqrt2_of() { return Real<T>::INV_SQRT2; }
template <>
__device__ __forceinline__ ddv inv_sqrt2_of<ddv>() { return Real<ddv>::inv_sqrt2(); }

// T: arithmetic type (float, double, or the double-float ddv); S: storage type
// of every global array (T, or double for ddv)
template <typename T, int N, int MODE, typename S = T>
__global__ void __launch_bounds__(128)
    apply_kernel(const int4* __restrict__ tets, const S* __restrict__ geo,
                 const S* __restrict__ v, const S* __restrict__ u0, const S* __restrict__ tau,
                 S* __restrict__ t0cache, const uint8_t* __restrict__ dmask, S* __restrict__ out,
                 const S* __restrict__ dft, Phys<T> ph, int64_t e0, int64_t e1, S* __restrict__ l0cache) {
  using D = Dims<N>;
  using L = ApplyLayout<N, MODE>;
  constexpr int C = D::C, K = D::K, NM = D::NM, NT = D::NT, NTP = D::NT_PAD;
  constexpr bool RES = MODE == MODE_RESIDUAL;
  constexpr bool PAPER = MODE == MODE_JVP_PAPER;
  constexpr bool LINA = MODE == MODE_JVP_LIN_A;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sF = reinterpret_cast<T*>(smem_raw);   // forward DFT [K][LDF]
  T* sI = sF + K * L::LDF;                  // inverse DFT [C][LDI]
  for (int t = threadIdx.x; t < K * C; t += blockDim.x) {
    const int kk = t / C, c = t - kk * C;
    sF[kk * L::LDF + c] = T(dft[t]);
  }
  for (int t = threadIdx.x; t < C * K; t += blockDim.x) {
    const int c = t / K, kk = t - c * K;
    sI[c * L::LDI + kk] = T(dft[K * C + t]);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* ws = sF + L::TABLES + warp * L::WARP;
  T* sg = ws + L::SG;
  T* sv = ws + L::SV;
  T* su = ws + L::SU;
  T* gv = ws + L::GV;
  T* vq = ws + L::VQ;
  T* uq = ws + L::UQ;
  T* pb = ws + L::PB;
  T* uqt = ws + L::UQT;
  T* gvt = ws + L::GVT;
  T* ct = ws + L::CT;
  T* cq = ws + L::CQ;
  T* tq = ws + L::TQ;
  T* tc = PAPER ? ws + L::TC : tq;
  T* wm = ws + L::WM;
  T* st = ws + L::TAU;
  T* so = ws + L::OUT;
  T* gu = ws + L::GU;
  T* vqt = ws + L::VQT;
  T* gut = ws + L::GUT;
  T* t0 = ws + L::T0;
  T* t0t = ws + L::T0T;
  const T rho = ph.rho, omega = ph.omega;
  const int wpb = blockDim.x >> 5;

  for (int64_t e = e0 + (int64_t)blockIdx.x * wpb + warp; e < e1;
       e += (int64_t)gridDim.x * wpb) {
    const int4 nd = tets[e];
    const int node[4] = {nd.x, nd.y, nd.z, nd.w};
    if (lane < GEO_STRIDE) sg[lane] = T(geo[e * GEO_STRIDE + lane]);
    for (int t = lane; t < 16 * C; t += 32) {
      const int a = t / (4 * C), r = t - a * 4 * C;
      const int f = r / C, c = r - f * C;
      T val = T(v[(int64_t)node[a] * 4 * C + r]);
      if (c == 1) val = T(0);
      if (!RES && f < 3 && dmask[node[a]]) val = T(0);
      sv[t] = val;
    }
    for (int t = lane; t < 12 * C; t += 32) {
      const int a = t / (3 * C), r = t - a * 3 * C;
      const int c = r % C;
      T val = T(u0[(int64_t)node[a] * 4 * C + r]);
      su[t] = (c == 1) ? T(0) : val;
    }
    // tau: packed symmetric (orthonormal basis) -> full matrix in storage scaling
    {
      const S* tp = tau + e * 4 * NTP;
      for (int t = lane; t < 4 * NTP; t += 32) {
        const int q = t / NTP, p = t - q * NTP;
        if (p >= NT) continue;
        int r = 0, rem = p;
        while (rem >= NM - r) {
          rem -= NM - r;
          ++r;
        }
        const int s = r + rem;
        const T val = T(tp[t]);
        // T_s[r] = (1/d_r) sum_k tau[r][k] d_k L_s[k], d_0 = 1, d_k = sqrt2
        const T drs = (r == 0 && s > 0) ? sqrt2_of<T>() : T(1);
        const T dsr = (r == 0 && s > 0) ? inv_sqrt2_of<T>() : T(1);
        st[q * NM * NM + r * NM + s] = val * drs;
        st[q * NM * NM + s * NM + r] = val * dsr;
      }
    }
    if (LINA) {
      const S* tp = t0cache + e * 12 * C;
      for (int t = lane; t < 12 * C; t += 32) t0[t] = T(tp[t]);
    }
    __syncwarp();
    const T vol = sg[GEO_VOL];
    // ---- phase 1: gradients, point values (modes)
    for (int t = lane; t < 12 * C; t += 32) {
      const int f = t / (3 * C), r = t - f * 3 * C;
      const int j = r / C, c = r - j * C;
      T acc = 0;
#pragma unroll
      for (int a = 0; a < 4; ++a) acc += sg[a * 3 + j] * sv[a * 4 * C + f * C + c];
      gv[t] = acc;
    }
    for (int t = lane; t < 12 * C; t += 32) {
      const int q = t / (3 * C), r = t - q * 3 * C;   // r = i*C + c
      T av = 0, au = 0;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const T lam = (T)qp_bary(q, a);
        av += lam * sv[a * 4 * C + r];
        au += lam * su[a * 3 * C + r];
      }
      vq[t] = av;
      uq[t] = au;
    }
    for (int c = lane; c < C; c += 32)
      pb[c] = T(0.25) * (sv[3 * C + c] + sv[7 * C + c] + sv[11 * C + c] + sv[15 * C + c]);
    if (LINA) {
      for (int t = lane; t < 9 * C; t += 32) {
        const int i = t / (3 * C), r = t - i * 3 * C;
        const int j = r / C, c = r - j * C;
        T acc = 0;
#pragma unroll
        for (int a = 0; a < 4; ++a) acc += sg[a * 3 + j] * su[a * 3 * C + i * C + c];
        gu[t] = acc;   // du0_i/dx_j at [i][j][c]
      }
    }
    __syncwarp();
    // ---- phase 2: modes -> samples
    warp_bmv<T, K, C>(sF, L::LDF, uq, C, uqt, K, 12, lane);
    warp_bmv<T, K, C>(sF, L::LDF, gv, C, gvt, K, 9, lane);   // velocity gradients only
    if (LINA) {
      warp_bmv<T, K, C>(sF, L::LDF, vq, C, vqt, K, 12, lane);
      warp_bmv<T, K, C>(sF, L::LDF, gu, C, gut, K, 9, lane);
    }
    __syncwarp();
    // ---- phase 3: convective products on samples: c_i = u0_j dv_i/dx_j (+ v_j du0_i/dx_j)
    for (int t = lane; t < 12 * K; t += 32) {
      const int q = t / (3 * K), r = t - q * 3 * K;
      const int i = r / K, kk = r - i * K;
      T acc = 0;
#pragma unroll
      for (int j = 0; j < 3; ++j) acc += uqt[(q * 3 + j) * K + kk] * gvt[(i * 3 + j) * K + kk];
      if (LINA) {
#pragma unroll
        for (int j = 0; j < 3; ++j) acc += vqt[(q * 3 + j) * K + kk] * gut[(i * 3 + j) * K + kk];
      }
      ct[t] = acc;
    }
    __syncwarp();
    // ---- phase 4: samples -> modes (truncation to |m| < N)
    warp_bmv<T, C, K>(sI, L::LDI, ct, K, cq, C, 12, lane);
    __syncwarp();
    // ---- phase 5: rho (Omega v + c) at each point (in place)
    for (int t = lane; t < 12 * C; t += 32) {
      const int c = t % C;
      const T om = (c == 1) ? T(0) : omega_apply(vq + (t - c), c, omega);
      cq[t] = (c == 1) ? T(0) : rho * (om + cq[t]);
    }
    __syncwarp();
    // ---- phase 6: T = tau L (storage coordinates)
    for (int t = lane; t < 12 * NM; t += 32) {
      const int qi = t / NM, r = t - qi * NM;
      const int q = qi / 3, i = qi - q * 3;
      const T* tr = st + q * NM * NM + r * NM;
      const T* lu = cq + qi * C;
      const T* lp = gv + (9 + i) * C;     // dp/dx_i
      T acc = 0, accp = 0;
#pragma unroll
      for (int kk = 0; kk < NM; ++kk) {
        const int cs = stor_of(kk);
        if (PAPER) {
          acc += tr[kk] * lu[cs];
          accp += tr[kk] * lp[cs];
        } else {
          acc += tr[kk] * (lu[cs] + lp[cs]);
        }
      }
      tq[qi * C + stor_of(r)] = acc;
      if (PAPER) tc[qi * C + stor_of(r)] = accp;
      // the strong residual itself (the exact tangent's tau derivative acts on it)
      if (RES && l0cache) {
        const int cs = stor_of(r);
        l0cache[(e * 12 + qi) * C + cs] = static_cast<S>(lu[cs] + lp[cs]);
      }
    }
    for (int qi = lane; qi < 12; qi += 32) {
      tq[qi * C + 1] = T(0);
      if (PAPER) tc[qi * C + 1] = T(0);
      if (RES && l0cache) l0cache[(e * 12 + qi) * C + 1] = S(0);
    }
    __syncwarp();
    if (RES) {
      S* tp = t0cache + e * 12 * C;
      for (int t = lane; t < 12 * C; t += 32) tp[t] = static_cast<S>(tq[t]);
    }
    // ---- phase 7: T (and T0) to samples
    warp_bmv<T, K, C>(sF, L::LDF, tq, C, ct, K, 12, lane);
    if (LINA) warp_bmv<T, K, C>(sF, L::LDF, t0, C, t0t, K, 12, lane);
    __syncwarp();
    // ---- phase 8: SUPG sums on samples W_ji = sum_q u0_j T_i (+ v_j T0_i)
    for (int t = lane; t < 9 * K; t += 32) {
      const int ji = t / K, kk = t - ji * K;
      const int j = ji / 3, i = ji - j * 3;
      T acc = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) acc += uqt[(q * 3 + j) * K + kk] * ct[(q * 3 + i) * K + kk];
      if (LINA) {
#pragma unroll
        for (int q = 0; q < 4; ++q) acc += vqt[(q * 3 + j) * K + kk] * t0t[(q * 3 + i) * K + kk];
      }
      gvt[t] = acc;
    }
    __syncwarp();
    // ---- phase 9: W to modes
    warp_bmv<T, C, K>(sI, L::LDI, gvt, K, wm, C, 9, lane);
    __syncwarp();
    // ---- phase 10: element contributions per node
    const T w4 = T(0.25) * vol;
    for (int t = lane; t < 16 * C; t += 32) {
      const int a = t / (4 * C), r = t - a * 4 * C;
      const int f = r / C, c = r - f * C;
      T acc = 0;
      if (c != 1) {
        if (f < 3) {
          const int i = f;
          T gal = 0;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const T lam = (T)qp_bary(q, a);
            const T* tqi = tq + (q * 3 + i) * C;
            gal += lam * (cq[(q * 3 + i) * C + c] - omega_apply(tqi, c, omega));
          }
          acc = w4 * gal - sg[a * 3 + i] * vol * pb[c];
          T visc = 0, supg = 0;
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            visc += sg[a * 3 + j] * gv[(i * 3 + j) * C + c];
            supg += sg[a * 3 + j] * wm[(j * 3 + i) * C + c];
          }
          acc += ph.mu * vol * visc + w4 * supg;
          if (!RES && ph.mass_coef != T(0)) {
            T sum = sv[a * 4 * C + i * C + c];
#pragma unroll
            for (int b = 0; b < 4; ++b) sum += sv[b * 4 * C + i * C + c];
            acc += ph.mass_coef * vol * T(0.05) * sum;
          }
        } else {
          const T div = gv[(0 * 3 + 0) * C + c] + gv[(1 * 3 + 1) * C + c] + gv[(2 * 3 + 2) * C + c];
          T ls = 0;
#pragma unroll
          for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int i = 0; i < 3; ++i) ls += sg[a * 3 + i] * tc[(q * 3 + i) * C + c];
          acc = w4 * div + (w4 / rho) * ls;
        }
      }
      so[t] = acc;
    }
    __syncwarp();
    // ---- phase 11: colour-exclusive scatter-add
    for (int t = lane; t < 16 * C; t += 32) {
      const int a = t / (4 * C), r = t - a * 4 * C;
      const int f = r / C, c = r - f * C;
      if (c == 1) continue;
      if (f < 3 && dmask[node[a]]) continue;
      S* dst = out + (int64_t)node[a] * 4 * C + r;
      *dst += static_cast<S>(so[t]);
    }
    __syncwarp();
  }
}

// warps (elements in flight) per block of the double-float element operator
constexpr int APPLY_DD_WARPS = 4;

template <typename T, int N, int MODE, typename S = T>
static int launch_mode(const int4* tets, const S* geo, const S* v, const S* u0, const S* tau,
                       S* t0cache, const uint8_t* dmask, S* out, const S* dft, Phys<T> ph,
                       int64_t e0, int64_t e1, cudaStream_t st, S* l0cache = nullptr) {
  using L = ApplyLayout<N, MODE>;
  static_assert(sizeof(T) == sizeof(S) || sizeof(T) == 8, "workspace sized by T");
  if (e1 <= e0) return 0;
  int warps = std::is_same<T, ddv>::value ? APPLY_DD_WARPS : 4;
  while (warps > 1 && (size_t)(L::TABLES + warps * L::WARP) * sizeof(T) > 200 * 1024) --warps;
  const size_t smem = (size_t)(L::TABLES + warps * L::WARP) * sizeof(T);
  if (smem > 227 * 1024) return -6;
  cudaFuncSetAttribute(apply_kernel<T, N, MODE, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)smem);
  int64_t blocks = (e1 - e0 + warps - 1) / warps;
  if (blocks > 152 * 32) blocks = 152 * 32;
  count_launches(1);
  apply_kernel<T, N, MODE, S><<<(int)blocks, warps * 32, smem, st>>>(tets, geo, v, u0, tau, t0cache,
                                                                     dmask, out, dft, ph, e0, e1, l0cache);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

// Loads the residual's element kernel into the current device's context
// without launching it (lazy module loading would load it at its first launch).
template <typename T, int N>
int preload_apply_residual() {
  using L = ApplyLayout<N, MODE_RESIDUAL>;
  int warps = 4;
  while (warps > 1 && (size_t)(L::TABLES + warps * L::WARP) * sizeof(T) > 200 * 1024) --warps;
  const size_t smem = (size_t)(L::TABLES + warps * L::WARP) * sizeof(T);
  if (smem > 227 * 1024) return -6;
  cudaFuncAttributes a;
  if (cudaFuncGetAttributes(&a, apply_kernel<T, N, MODE_RESIDUAL>) != cudaSuccess) return -2;
  return cudaFuncSetAttribute(apply_kernel<T, N, MODE_RESIDUAL>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess
             ? 0 : -2;
}

template <typename T, int N>
int launch_apply(int mode, const int4* tets, const T* geo, const T* v, const T* u0,
                 const T* tau, T* t0cache, const uint8_t* dmask, T* out, const T* dft,
                 Phys<T> ph, int64_t e0, int64_t e1, cudaStream_t st, T* l0cache) {
  switch (mode) {
    case MODE_RESIDUAL:
      return launch_mode<T, N, MODE_RESIDUAL>(tets, geo, v, u0, tau, t0cache, dmask, out, dft,
                                              ph, e0, e1, st, l0cache);
    case MODE_JVP_PAPER:
      return launch_mode<T, N, MODE_JVP_PAPER>(tets, geo, v, u0, tau, t0cache, dmask, out, dft,
                                               ph, e0, e1, st);
    case MODE_JVP_FROZEN:
      return launch_mode<T, N, MODE_JVP_FROZEN>(tets, geo, v, u0, tau, t0cache, dmask, out, dft,
                                                ph, e0, e1, st);
    case MODE_JVP_LIN_A:
      return launch_mode<T, N, MODE_JVP_LIN_A>(tets, geo, v, u0, tau, t0cache, dmask, out, dft,
                                               ph, e0, e1, st);
  }
  return -1;
}

// The FP64 operator with its arithmetic in double-float (FP64 storage)
template <int N>
int launch_apply_dd(int mode, const int4* tets, const double* geo, const double* v, const double* u0,
                    const double* tau, double* t0cache, const uint8_t* dmask, double* out, const double* dft,
                    Phys<double> p, int64_t e0, int64_t e1, cudaStream_t st, double* l0cache) {
  Phys<ddv> ph{ddv(p.rho), ddv(p.mu), ddv(p.omega), ddv(p.nu), ddv(p.C_I), ddv(p.mass_coef)};
  switch (mode) {
    case MODE_RESIDUAL:
      return launch_mode<ddv, N, MODE_RESIDUAL, double>(tets, geo, v, u0, tau, t0cache, dmask, out, dft,
                                                        ph, e0, e1, st, l0cache);
    case MODE_JVP_PAPER:
      return launch_mode<ddv, N, MODE_JVP_PAPER, double>(tets, geo, v, u0, tau, t0cache, dmask, out, dft,
                                                         ph, e0, e1, st);
    case MODE_JVP_FROZEN:
      return launch_mode<ddv, N, MODE_JVP_FROZEN, double>(tets, geo, v, u0, tau, t0cache, dmask, out, dft,
                                                          ph, e0, e1, st);
    case MODE_JVP_LIN_A:
      return launch_mode<ddv, N, MODE_JVP_LIN_A, double>(tets, geo, v, u0, tau, t0cache, dmask, out, dft,
                                                         ph, e0, e1, st);
  }
  return -1;
}

// ---------------------------------------------------------------- tracer
// Time-spectral GLS convection-diffusion of a scalar phi (eq. 3D-weak with
// eq. 3D-weak-def, section 2.2) advected by a given velocity a: per element
// and quadrature point (weights V/4)
//   res  = Omega phi + A_j dphi/dx_j          (A_j = A(a_j), eq. phi-def)
//   T    = tau res                            (tau of eq. 3D-tau with kappa)
//   r_a += w [N_a res - N_a Omega T + dN_a/dx_j A_j T] + kappa V dN_a/dx_j dphi/dx_j
// The products A_j x are formed on K = 3N - 2 time samples, as in the flow
// operator; the SUPG sum sum_q w A_j T is transformed once per element.
template <int N>
struct TracerLayout {
  using D = Dims<N>;
  static constexpr int C = D::C, K = D::K, NM = D::NM;
  static constexpr int LDF = C | 1, LDI = K | 1;
  static constexpr int TABLES = K * LDF + C * LDI;
  static constexpr int SG = 0;              // geometry 20 (+4)
  static constexpr int PH = 24;             // phi at nodes [4][C]
  static constexpr int AN = PH + 4 * C;     // a at nodes [4][3][C]
  static constexpr int GP = AN + 12 * C;    // grad phi [3][C]
  static constexpr int PQ = GP + 3 * C;     // phi at points [4][C]
  static constexpr int AQ = PQ + 4 * C;     // a at points [4][3][C]
  static constexpr int AQT = AQ + 12 * C;   // a samples [4][3][K]
  static constexpr int GPT = AQT + 12 * K;  // grad phi samples [3][K], later W samples
  static constexpr int CT = GPT + 3 * K;    // c samples [4][K], later T samples
  static constexpr int RES = CT + 4 * K;    // res modes [4][C]
  static constexpr int TQ = RES + 4 * C;    // T modes [4][C]
  static constexpr int WM = TQ + 4 * C;     // W modes [3][C]
  static constexpr int TAU = WM + 3 * C;    // tau [4][NM][NM] (storage scaling)
  static constexpr int OUT = TAU + 4 * NM * NM;   // [4][C]
  static constexpr int WARP = (OUT + 4 * C + 3) & ~3;
};

template <typename T, int N, typename S = T>
__global__ void __launch_bounds__(128)
    tracer_kernel(const int4* __restrict__ tets, const S* __restrict__ geo, const S* __restrict__ a4,
                  const S* __restrict__ phi, const S* __restrict__ tau, const uint8_t* __restrict__ dmask,
                  S* __restrict__ out, const S* __restrict__ dft, T kappa, T omega, int64_t e0, int64_t e1,
                  int gls) {
  using D = Dims<N>;
  using L = TracerLayout<N>;
  constexpr int C = D::C, K = D::K, NM = D::NM, NT = D::NT, NTP = D::NT_PAD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sF = reinterpret_cast<T*>(smem_raw);
  T* sI = sF + K * L::LDF;
  for (int t = threadIdx.x; t < K * C; t += blockDim.x) {
    const int kk = t / C, c = t - kk * C;
    sF[kk * L::LDF + c] = T(dft[t]);
  }
  for (int t = threadIdx.x; t < C * K; t += blockDim.x) {
    const int c = t / K, kk = t - c * K;
    sI[c * L::LDI + kk] = T(dft[K * C + t]);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* ws = sF + L::TABLES + warp * L::WARP;
  T* sg = ws + L::SG;
  T* ph = ws + L::PH;
  T* an = ws + L::AN;
  T* gp = ws + L::GP;
  T* pq = ws + L::PQ;
  T* aq = ws + L::AQ;
  T* aqt = ws + L::AQT;
  T* gpt = ws + L::GPT;
  T* ct = ws + L::CT;
  T* res = ws + L::RES;
  T* tq = ws + L::TQ;
  T* wm = ws + L::WM;
  T* st = ws + L::TAU;
  T* so = ws + L::OUT;
  const int wpb = blockDim.x >> 5;
  for (int64_t e = e0 + (int64_t)blockIdx.x * wpb + warp; e < e1; e += (int64_t)gridDim.x * wpb) {
    const int4 nd = tets[e];
    const int node[4] = {nd.x, nd.y, nd.z, nd.w};
    if (lane < GEO_STRIDE) sg[lane] = T(geo[e * GEO_STRIDE + lane]);
    for (int t = lane; t < 4 * C; t += 32) {
      const int a = t / C, c = t - a * C;
      ph[t] = c == 1 ? T(0) : T(phi[(int64_t)node[a] * C + c]);
    }
    for (int t = lane; t < 12 * C; t += 32) {
      const int a = t / (3 * C), r = t - a * 3 * C;
      const int c = r % C;
      an[t] = c == 1 ? T(0) : T(a4[(int64_t)node[a] * 4 * C + r]);
    }
    {
      const S* tp = tau + e * 4 * NTP;
      for (int t = lane; t < 4 * NTP; t += 32) {
        const int q = t / NTP, p = t - q * NTP;
        if (p >= NT) continue;
        int r = 0, rem = p;
        while (rem >= NM - r) {
          rem -= NM - r;
          ++r;
        }
        const int s2 = r + rem;
        const T val = T(tp[t]);
        const T drs = (r == 0 && s2 > 0) ? sqrt2_of<T>() : T(1);
        const T dsr = (r == 0 && s2 > 0) ? inv_sqrt2_of<T>() : T(1);
        st[q * NM * NM + r * NM + s2] = val * drs;
        st[q * NM * NM + s2 * NM + r] = val * dsr;
      }
    }
    __syncwarp();
    const T vol = sg[GEO_VOL], w4 = T(0.25) * vol;
    for (int t = lane; t < 3 * C; t += 32) {
      const int j = t / C, c = t - j * C;
      T acc = 0;
#pragma unroll
      for (int a = 0; a < 4; ++a) acc += sg[a * 3 + j] * ph[a * C + c];
      gp[t] = acc;
    }
    for (int t = lane; t < 4 * C; t += 32) {
      const int q = t / C, c = t - q * C;
      T acc = 0;
#pragma unroll
      for (int a = 0; a < 4; ++a) acc += T(qp_bary(q, a)) * ph[a * C + c];
      pq[t] = acc;
    }
    for (int t = lane; t < 12 * C; t += 32) {
      const int q = t / (3 * C), r = t - q * 3 * C;
      T acc = 0;
#pragma unroll
      for (int a = 0; a < 4; ++a) acc += T(qp_bary(q, a)) * an[a * 3 * C + r];
      aq[t] = acc;
    }
    __syncwarp();
    warp_bmv<T, K, C>(sF, L::LDF, aq, C, aqt, K, 12, lane);
    warp_bmv<T, K, C>(sF, L::LDF, gp, C, gpt, K, 3, lane);
    __syncwarp();
    // convective product on samples c(q, t) = sum_j a_j(q, t) dphi/dx_j(t)
    for (int t = lane; t < 4 * K; t += 32) {
      const int q = t / K, kk = t - q * K;
      T acc = 0;
#pragma unroll
      for (int j = 0; j < 3; ++j) acc += aqt[(q * 3 + j) * K + kk] * gpt[j * K + kk];
      ct[t] = acc;
    }
    __syncwarp();
    warp_bmv<T, C, K>(sI, L::LDI, ct, K, res, C, 4, lane);
    __syncwarp();
    for (int t = lane; t < 4 * C; t += 32) {
      const int c = t % C;
      res[t] = c == 1 ? T(0) : omega_apply(pq + (t - c), c, omega) + res[t];
    }
    __syncwarp();
    // T = tau res (storage coordinates)
    for (int t = lane; t < 4 * NM; t += 32) {
      const int q = t / NM, r = t - q * NM;
      const T* tr = st + q * NM * NM + r * NM;
      const T* rq = res + q * C;
      T acc = 0;
#pragma unroll
      for (int kk = 0; kk < NM; ++kk) acc = mad(tr[kk], rq[stor_of(kk)], acc);
      tq[q * C + stor_of(r)] = gls ? acc : T(0);   // Galerkin only: no least-squares term
    }
    for (int q = lane; q < 4; q += 32) tq[q * C + 1] = T(0);
    __syncwarp();
    warp_bmv<T, K, C>(sF, L::LDF, tq, C, ct, K, 4, lane);
    __syncwarp();
    // SUPG sums on samples W_j(t) = sum_q a_j(q, t) T(q, t)
    for (int t = lane; t < 3 * K; t += 32) {
      const int j = t / K, kk = t - j * K;
      T acc = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) acc += aqt[(q * 3 + j) * K + kk] * ct[q * K + kk];
      gpt[t] = acc;
    }
    __syncwarp();
    warp_bmv<T, C, K>(sI, L::LDI, gpt, K, wm, C, 3, lane);
    __syncwarp();
    for (int t = lane; t < 4 * C; t += 32) {
      const int a = t / C, c = t - a * C;
      T acc = 0;
      if (c != 1) {
        T gal = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const T lam = T(qp_bary(q, a));
          gal += lam * (res[q * C + c] - omega_apply(tq + q * C, c, omega));
        }
        T supg = 0, diff = 0;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          supg += sg[a * 3 + j] * wm[j * C + c];
          diff += sg[a * 3 + j] * gp[j * C + c];
        }
        acc = w4 * (gal + supg) + kappa * vol * diff;
      }
      so[t] = acc;
    }
    __syncwarp();
    for (int t = lane; t < 4 * C; t += 32) {
      const int a = t / C, c = t - a * C;
      if (c == 1 || dmask[node[a]]) continue;
      out[(int64_t)node[a] * C + c] += static_cast<S>(so[t]);
    }
    __syncwarp();
  }
}

template <typename T, int N, typename S>
static int launch_tracer_t(const int4* tets, const S* geo, const S* a4, const S* phi, const S* tau,
                           const uint8_t* dmask, S* out, const S* dft, double kappa, double omega,
                           int64_t e0, int64_t e1, cudaStream_t st, int gls) {
  using L = TracerLayout<N>;
  if (e1 <= e0) return 0;
  int warps = 4;
  while (warps > 1 && (size_t)(L::TABLES + warps * L::WARP) * sizeof(T) > 200 * 1024) --warps;
  const size_t smem = (size_t)(L::TABLES + warps * L::WARP) * sizeof(T);
  if (smem > 227 * 1024) return -6;
  cudaFuncSetAttribute(tracer_kernel<T, N, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int64_t blocks = (e1 - e0 + warps - 1) / warps;
  if (blocks > 152 * 32) blocks = 152 * 32;
  count_launches(1);
  tracer_kernel<T, N, S><<<(int)blocks, warps * 32, smem, st>>>(tets, geo, a4, phi, tau, dmask, out, dft,
                                                                T(kappa), T(omega), e0, e1, gls);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

template <typename T, int N>
int launch_tracer(const int4* tets, const T* geo, const T* a4, const T* phi, const T* tau,
                  const uint8_t* dmask, T* out, const T* dft, double kappa, double omega, int64_t e0,
                  int64_t e1, cudaStream_t st, int gls) {
  return launch_tracer_t<T, N, T>(tets, geo, a4, phi, tau, dmask, out, dft, kappa, omega, e0, e1, st, gls);
}

// a [V][3][C] -> a4 [V][4][C] (the flow layout the tau kernels read; pressure zero)
template <typename T>
__global__ void repack_velocity_kernel(const T* __restrict__ a, T* __restrict__ a4, int64_t V, int C) {
  const int64_t total = V * 4 * C;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = t / (4 * C), r = t - v * 4 * C;
    a4[t] = r < 3 * C ? a[v * 3 * C + r] : T(0);
  }
}

template <typename T>
int launch_repack_velocity(const T* a, T* a4, int64_t V, int C, cudaStream_t st) {
  if (V <= 0) return 0;
  int64_t blocks = (V * 4 * C + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  count_launches(1);
  repack_velocity_kernel<T><<<(int)blocks, 256, 0, st>>>(a, a4, V, C);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}
template int launch_repack_velocity<float>(const float*, float*, int64_t, int, cudaStream_t);
template int launch_repack_velocity<double>(const double*, double*, int64_t, int, cudaStream_t);

// ---------------------------------------------------------------- outlets
// One block per call: Q_c = sum_A sum_i w_Ai v[A][i][c]; out[A][i][c] += R w_Ai Q_c.
// Thread t owns the outlet nodes t, t + blockDim, ... and keeps its partial
// flow rates of all C coefficients in its own column of part[C][blockDim]
// (the loads of a node are independent, so one node costs one memory round
// trip, not one per coefficient); warp w then sums the columns of the
// coefficients c = w, w + nw, ... in a fixed order (deterministic), and the
// threads scatter to their own nodes.
template <typename T>
__global__ void __launch_bounds__(256) outlet_kernel(const int32_t* __restrict__ nodes,
                                                     const T* __restrict__ w, int n, T R,
                                                     const T* __restrict__ v,
                                                     const uint8_t* __restrict__ dmask, int mask_input,
                                                     T* __restrict__ out, int C) {
  extern __shared__ __align__(16) unsigned char outlet_smem[];
  T* part = reinterpret_cast<T*>(outlet_smem);   // [C][blockDim.x]
  T* Q = part + (int64_t)C * blockDim.x;         // [C]
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
  for (int c = 0; c < C; ++c) part[c * nt + tid] = T(0);
  for (int b = tid; b < n; b += nt) {
    const int A = nodes[b];
    if (mask_input && dmask[A]) continue;
    const T w0 = w[b * 3 + 0], w1 = w[b * 3 + 1], w2 = w[b * 3 + 2];
    const T* va = v + (int64_t)A * 4 * C;
    for (int c = 0; c < C; ++c) part[c * nt + tid] += w0 * va[c] + w1 * va[C + c] + w2 * va[2 * C + c];
  }
  __syncthreads();
  for (int c = warp; c < C; c += nw) {
    T acc = 0;
    for (int k = lane; k < nt; k += 32) acc += part[c * nt + k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) Q[c] = (c == 1) ? T(0) : acc;
  }
  __syncthreads();
  for (int b = tid; b < n; b += nt) {
    const int A = nodes[b];
    if (dmask[A]) continue;
    T* oa = out + (int64_t)A * 4 * C;
    for (int i = 0; i < 3; ++i) {
      const T s = R * w[b * 3 + i];
      for (int c = 0; c < C; ++c)
        if (c != 1) oa[i * C + c] += s * Q[c];
    }
  }
}

template <typename T>
int launch_outlet(const int32_t* nodes, const T* w, int n_nodes, T R, const T* v,
                  const uint8_t* dmask, int mask_input, T* out, int C, cudaStream_t st) {
  if (n_nodes <= 0) return 0;
  if (C > 128) return -1;
  const int threads = 256;
  const size_t smem = ((size_t)C * threads + C) * sizeof(T);
  if (smem > 227 * 1024) return -1;
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(outlet_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return -2;
  count_launches(1);
  outlet_kernel<T><<<1, threads, smem, st>>>(nodes, w, n_nodes, R, v, dmask, mask_input, out, C);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

template <typename T>
__global__ void inlet_fill_kernel(const int32_t* __restrict__ nodes, const double* __restrict__ vals,
                                  int64_t n, int C, T* __restrict__ y) {
  const int64_t total = n * 3 * C;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = t / (3 * C), r = t - k * 3 * C;
    y[(int64_t)nodes[k] * 4 * C + r] = (T)vals[t];
  }
}

template <typename T>
int launch_inlet_fill(const int32_t* nodes, const double* vals, int64_t n, int C, T* y, cudaStream_t st) {
  if (n <= 0) return 0;
  int64_t blocks = (n * 3 * C + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  count_launches(1);
  inlet_fill_kernel<T><<<(int)blocks, 256, 0, st>>>(nodes, vals, n, C, y);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}
template int launch_inlet_fill<float>(const int32_t*, const double*, int64_t, int, float*, cudaStream_t);
template int launch_inlet_fill<double>(const int32_t*, const double*, int64_t, int, double*, cudaStream_t);

template int launch_outlet<float>(const int32_t*, const float*, int, float, const float*,
                                  const uint8_t*, int, float*, int, cudaStream_t);
template int launch_outlet<double>(const int32_t*, const double*, int, double, const double*,
                                   const uint8_t*, int, double*, int, cudaStream_t);

#define TS_INST_APPLY(T, N)                                                                  \
  template int launch_apply<T, N>(int, const int4*, const T*, const T*, const T*, const T*, \
                                  T*, const uint8_t*, T*, const T*, Phys<T>, int64_t,        \
                                  int64_t, cudaStream_t, T*);
TS_FOR_EACH_N(TS_INST_APPLY, float)
#define TS_INST_PRELOAD_APPLY(T, N) template int preload_apply_residual<T, N>();
TS_FOR_EACH_N(TS_INST_PRELOAD_APPLY, float)
TS_FOR_EACH_N(TS_INST_APPLY, double)
#define TS_INST_APPLY_DD(T, N)                                                                         \
  template int launch_apply_dd<N>(int, const int4*, const double*, const double*, const double*,      \
                                  const double*, double*, const uint8_t*, double*, const double*,     \
                                  Phys<double>, int64_t, int64_t, cudaStream_t, double*);
TS_FOR_EACH_N(TS_INST_APPLY_DD, double)
#define TS_INST_TRACER(T, N)                                                                        \
  template int launch_tracer<T, N>(const int4*, const T*, const T*, const T*, const T*, const uint8_t*, \
                                   T*, const T*, double, double, int64_t, int64_t, cudaStream_t, int);
TS_FOR_EACH_N(TS_INST_TRACER, float)
TS_FOR_EACH_N(TS_INST_TRACER, double)

}  // namespace ts
