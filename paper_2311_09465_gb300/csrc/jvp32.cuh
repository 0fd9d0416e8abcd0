// FP32 tangent product of eq. (K_mat), section 2.4 -- the GMRES hot loop.
//
// Same arithmetic as the element operator in apply.cu (see the formulas
// there): per quadrature point the convective products c_i = A_j dv_i/dx_j
// (+ A(v_j) du0_i/dx_j for the LIN_A variant) are formed on K = 3N-2 time
// samples and truncated back to |m| < N, L_i is multiplied by the cached
// tau_q, T_i is sampled again for the SUPG sum sum_q w A_j T_i.
//
// GB300 mapping (one element pass per product, plus a node pre-pass):
//  * Node pre-pass: v (Dirichlet and Im(mode 0) inputs masked) and the
//    linearisation velocity u0 are sampled in time once per node, stored as
//    [V][K] float4 (x, y, z, 0), so an element reads the velocity of its four
//    nodes at sample k with four 16-byte loads and no element-level forward
//    transform of v or u0 is needed.  The pre-pass also zeroes Hv.
//  * Element pass: one warp owns two elements at a time.  Work that is
//    pointwise in time (gradients and point values at a sample, the
//    convective and SUPG products) runs one lane per (element, sample); work
//    per point or per node (transforms, tau, the node rows) runs on 16 lanes
//    per element, lane (f, q) = (field, point or node).
//  * tau of the four points and the cached tau L(u0) of both elements, the
//    dominant HBM streams, are staged in shared memory by bulk asynchronous
//    copies (cp.async.bulk + mbarrier), issued one element pair ahead.
//  * Transforms use the symmetry of the real DFT (samples k and K-k share the
//    cosines and negate the sines), with coefficients in __constant__ memory
//    and compile-time indices: about half the multiply-adds of the plain
//    matrix form.
//  * Node rows are added with 16-byte vector atomics (red.global.add.v4.f32
//    through atomicAdd(float4*)), so Hv needs no colouring.
// Included by the jvp32_n*.cu translation units, each of which defines
// J32_NLIST (the mode counts it instantiates).
#pragma once
#include "common.cuh"
#include "kernels.h"

namespace ts {

namespace {

__device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

// shared-memory rows: M floats from a 16-byte aligned row padded to a multiple
// of 4 (ld4/st4: 16-byte accesses, st4 writes zeros into the padding), or an
// even count from an 8-byte aligned row (ld2)
template <int M>
__device__ __forceinline__ void ld4(const float* p, float (&x)[M]) {
  const float4* p4 = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int c4 = 0; c4 < (M + 3) / 4; ++c4) {
    const float4 v = p4[c4];
    const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (4 * c4 + u < M) x[4 * c4 + u] = e[u];
  }
}
template <int M>
__device__ __forceinline__ void st4(float* p, const float (&x)[M]) {
  float4* p4 = reinterpret_cast<float4*>(p);
#pragma unroll
  for (int c4 = 0; c4 < (M + 3) / 4; ++c4) {
    float e[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) e[u] = 4 * c4 + u < M ? x[4 * c4 + u] : 0.f;
    p4[c4] = make_float4(e[0], e[1], e[2], e[3]);
  }
}
template <int M>
__device__ __forceinline__ void ld2(const float* p, float (&x)[M]) {
  const float2* p2 = reinterpret_cast<const float2*>(p);
#pragma unroll
  for (int c2 = 0; c2 < M / 2; ++c2) {
    const float2 v = p2[c2];
    x[2 * c2] = v.x;
    x[2 * c2 + 1] = v.y;
  }
}
template <int M>
__device__ __forceinline__ void st2(float* p, const float (&x)[M]) {
  float2* p2 = reinterpret_cast<float2*>(p);
#pragma unroll
  for (int c2 = 0; c2 < M / 2; ++c2) p2[c2] = make_float2(x[2 * c2], x[2 * c2 + 1]);
}

// ---------------------------------------------------------------- DFT tables
// forward [K][C] then inverse [C][K] for each N of this unit, concatenated:
// forward (k, 2n) = 2 cos(2 pi n k / K), (k, 2n+1) = -2 sin(2 pi n k / K),
// inverse (2n, k) = cos(2 pi n k / K) / K, (2n+1, k) = -sin(2 pi n k / K) / K.
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

// modes (storage coordinates, slot 1 ignored) -> K samples.  Sample K-k has
// the same cosine part as sample k and the opposite sine part.
template <int N>
__device__ __forceinline__ void fwd(const float (&x)[2 * N], float (&y)[3 * N - 2]) {
  constexpr int K = 3 * N - 2, KH = (K - 1) / 2;
  float y0 = x[0];
#pragma unroll
  for (int n = 1; n < N; ++n) y0 = fmaf(x[2 * n], CF<N>(0, 2 * n), y0);
  y[0] = y0;
#pragma unroll
  for (int k = 1; k <= KH; ++k) {
    float cc = x[0], ss = 0.f;
#pragma unroll
    for (int n = 1; n < N; ++n) {
      cc = fmaf(x[2 * n], CF<N>(k, 2 * n), cc);
      ss = fmaf(x[2 * n + 1], CF<N>(k, 2 * n + 1), ss);
    }
    y[k] = cc + ss;
    y[K - k] = cc - ss;
  }
  if constexpr (K % 2 == 0) {   // the Nyquist sample: cosines only
    constexpr int k = K / 2;
    float cc = x[0];
#pragma unroll
    for (int n = 1; n < N; ++n) cc = fmaf(x[2 * n], CF<N>(k, 2 * n), cc);
    y[k] = cc;
  }
}

// K samples -> modes |m| < N (the exact truncated product); slot 1 = 0.
// Cosine coefficients see u_k + u_{K-k}, sine coefficients u_k - u_{K-k}.
template <int N>
__device__ __forceinline__ void inv(const float (&u)[3 * N - 2], float (&x)[2 * N]) {
  constexpr int K = 3 * N - 2, KH = (K - 1) / 2, KP = KH > 0 ? KH : 1;
  float P[KP], M[KP];
  float tot = u[0];
#pragma unroll
  for (int k = 1; k <= KH; ++k) {
    P[k - 1] = u[k] + u[K - k];
    M[k - 1] = u[k] - u[K - k];
    tot += P[k - 1];
  }
  if constexpr (K % 2 == 0) tot += u[K / 2];
  x[0] = tot * CI<N>(0, 0);
  x[1] = 0.f;
#pragma unroll
  for (int n = 1; n < N; ++n) {
    float a = u[0] * CI<N>(2 * n, 0), b = 0.f;
#pragma unroll
    for (int k = 1; k <= KH; ++k) {
      a = fmaf(P[k - 1], CI<N>(2 * n, k), a);
      b = fmaf(M[k - 1], CI<N>(2 * n + 1, k), b);
    }
    if constexpr (K % 2 == 0) a = fmaf(u[K / 2], CI<N>(2 * n, K / 2), a);
    x[2 * n] = a;
    x[2 * n + 1] = b;
  }
}

template <int N>
__device__ __forceinline__ float om_apply(const float (&x)[2 * N], int c, float omega) {
  const int n = c >> 1;
  if (n == 0) return 0.f;
  return (c & 1) ? float(n) * omega * x[c - 1] : -float(n) * omega * x[c + 1];
}

// T = tau L in storage coordinates, tau packed (upper triangle, orthonormal
// basis xi = (x_0, sqrt2 Re x_n, sqrt2 Im x_n)) in shared memory.  With
// z_0 = x_0 / sqrt2 and z_r = x_r the product is t = tau z, T_0 = sqrt2 t_0.
template <int N>
__device__ __forceinline__ void tau_apply(const float* __restrict__ tp, const float (&L)[2 * N],
                                          float (&T)[2 * N]) {
  constexpr int NM = 2 * N - 1, NTP = Dims<N>::NT_PAD;
  float z[NM], t[NM], tv[NTP];
  z[0] = L[0] * Real<float>::INV_SQRT2;
#pragma unroll
  for (int r = 1; r < NM; ++r) z[r] = L[r + 1];
  const float4* tp4 = reinterpret_cast<const float4*>(tp);
#pragma unroll
  for (int c4 = 0; c4 < NTP / 4; ++c4) {
    const float4 x = tp4[c4];
    tv[4 * c4] = x.x;
    tv[4 * c4 + 1] = x.y;
    tv[4 * c4 + 2] = x.z;
    tv[4 * c4 + 3] = x.w;
  }
#pragma unroll
  for (int r = 0; r < NM; ++r) t[r] = tv[packed_index(r, r, NM)] * z[r];
#pragma unroll
  for (int r = 0; r < NM; ++r)
#pragma unroll
    for (int s = r + 1; s < NM; ++s) {
      const float x = tv[packed_index(r, s, NM)];
      t[r] = fmaf(x, z[s], t[r]);
      t[s] = fmaf(x, z[r], t[s]);
    }
  T[0] = t[0] * Real<float>::SQRT2;
  T[1] = 0.f;
#pragma unroll
  for (int r = 1; r < NM; ++r) T[r + 1] = t[r];
}

// ---------------------------------------------------------------- bulk copies
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}
// waits for the barrier phase with the given parity; gives up after about a
// second of polling (each try_wait suspends for a bounded time) and returns false
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (int it = 0; it < (1 << 20); ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}

// ---------------------------------------------------------------- layout
constexpr int EPW = 2;    // elements per warp pass
constexpr float QA = 0.5854101966249685f, QB = 0.1381966011250105f, QD = QA - QB;
constexpr unsigned FULL = 0xffffffffu;

// Staging (bulk-copy destination) of one element pair, then two element
// workspaces.  All region offsets are multiples of 4 floats.
template <int N, int MODE>
struct J32Layout {
  static constexpr int C = 2 * N, K = 3 * N - 2, NTP = Dims<N>::NT_PAD;
  static constexpr int KP = (K + 3) & ~3;   // sample rows padded to 16 bytes
  static constexpr bool LINA = MODE == MODE_JVP_LIN_A || MODE == MODE_JVP_EXACT;
  static constexpr int STG_TAU = 0;                               // [2][4][NTP]
  static constexpr int STG_T0 = STG_TAU + EPW * 4 * NTP;          // [2][4][3][C] (LIN_A)
  static constexpr int STG = STG_T0 + (LINA ? EPW * 12 * C : 0);
  // one element's workspace
  static constexpr int VM = 0;                         // v modes at the nodes [4 a][4 f][C]
  static constexpr int GM = VM + 16 * C;               // gradients [4 f][3 j][C]
  static constexpr int VS = GM + 12 * C;               // sum over nodes [4 f][C]
  static constexpr int GE = VS + 4 * C;                // dN_a/dx_j [12], volume, pad, node ids [4]
  static constexpr int CT = GE + 20;                    // c, later T samples [4 q][3 i][KP]
  static constexpr int TS = CT + 12 * KP;               // T0 samples [4 q][3 i][KP] (LIN_A)
  // SUPG sums [3 j][3 i][KP], then Z modes; they take the place of v at the nodes
  // (dead after the point phase) when that is large enough
  static constexpr bool WS_IN_VM = 9 * KP <= 16 * C;
  static constexpr int END = TS + (LINA ? 12 * KP : 0);
  static constexpr int WS = WS_IN_VM ? VM : END;
  static constexpr int ELEM = WS_IN_VM ? END : END + 9 * KP;
  static constexpr int WORK = EPW * ELEM;
  static constexpr int WARP = STG + WORK;
};

// bytes of the staged tau / tau L of elements [base, base + n)
template <int N, bool LINA>
__device__ __forceinline__ void stage_issue(const float* tau, const float* t0, int64_t base, int n,
                                            float* stg, uint32_t bar) {
  constexpr int C = 2 * N, NTP = Dims<N>::NT_PAD;
  const uint32_t bt = (uint32_t)n * 4 * NTP * 4, b0 = LINA ? (uint32_t)n * 12 * C * 4 : 0u;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  mbar_expect(bar, bt + b0);
  bulk_g2s(smem_addr(stg), tau + base * 4 * NTP, bt, bar);
  if (LINA) bulk_g2s(smem_addr(stg + EPW * 4 * NTP), t0 + base * 12 * C, b0, bar);
}

// 16-byte vector atomics of one node row (C floats, 8-byte aligned start)
template <int C>
__device__ __forceinline__ void row_atomics(float* dst, const float (&row)[C]) {
  if ((reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
#pragma unroll
    for (int c = 0; c + 3 < C; c += 4)
      atomicAdd(reinterpret_cast<float4*>(dst + c), make_float4(row[c], row[c + 1], row[c + 2], row[c + 3]));
    if constexpr (C % 4 == 2)
      atomicAdd(reinterpret_cast<float2*>(dst + C - 2), make_float2(row[C - 2], row[C - 1]));
  } else {
    atomicAdd(reinterpret_cast<float2*>(dst), make_float2(row[0], row[1]));
#pragma unroll
    for (int c = 2; c + 3 < C; c += 4)
      atomicAdd(reinterpret_cast<float4*>(dst + c), make_float4(row[c], row[c + 1], row[c + 2], row[c + 3]));
    if constexpr (C % 4 == 0)
      atomicAdd(reinterpret_cast<float2*>(dst + C - 2), make_float2(row[C - 2], row[C - 1]));
  }
}

// One warp pass over the elements base, base + 1 of instance I.  stg holds
// their staged tau (and tau L) once the barrier phase 'parity' completes; the
// warp then calls issue_next() (lane 0 only) to stage the next pair.  work is
// the warp's two element workspaces.  Returns false if the staging wait gave up.
template <int N, int MODE, typename Issue>
__device__ __forceinline__ bool j32_pass(const J32Inst I, int64_t base, const float* stg, float* work,
                                         uint32_t bar, uint32_t parity, int lane, Issue issue_next) {
  using L = J32Layout<N, MODE>;
  constexpr int C = L::C, K = L::K, NTP = L::NTP;
  constexpr bool PAPER = MODE == MODE_JVP_PAPER;
  constexpr bool LINA = L::LINA;
  const int slot = lane >> 4, f = (lane >> 2) & 3, q = lane & 3, t16 = lane & 15;
  const int64_t e = base + slot;
  const bool live = e < I.n_elem;
  float* es = work + slot * L::ELEM;
  const float rho = I.ph.rho, omega = I.ph.omega;

  // ---- P0: element record and v modes of the nodes; lane (f, a = q) loads field f of node a
  {
    int4 nd = make_int4(0, 0, 0, 0);
    if (live) nd = I.tets[e];
    if (t16 < 13) es[L::GE + t16] = live ? I.geo[e * GEO_STRIDE + t16] : 0.f;
    if (t16 == 15) *reinterpret_cast<int4*>(es + L::GE + 16) = nd;
    const int node = q == 0 ? nd.x : q == 1 ? nd.y : q == 2 ? nd.z : nd.w;
    const bool zero = !live || (f < 3 && I.dmask[node] != 0);
    const float2* src = reinterpret_cast<const float2*>(I.v + ((int64_t)node * 4 + f) * C);
    float2* dst = reinterpret_cast<float2*>(es + L::VM + (q * 4 + f) * C);
#pragma unroll
    for (int c2 = 0; c2 < C / 2; ++c2) {
      float2 x = zero ? make_float2(0.f, 0.f) : src[c2];
      if (c2 == 0) x.y = 0.f;   // Im(mode 0) input ignored
      dst[c2] = x;
    }
  }
  __syncwarp();
  // ---- P1: lane (f, j < 3) the gradient of field f; lane (f, 3) the sum over the nodes
  {
    const float* vm = es + L::VM;
    float d[4] = {1.f, 1.f, 1.f, 1.f};   // lane (f, 3): plain sum over the nodes
    if (q < 3) {
#pragma unroll
      for (int a = 0; a < 4; ++a) d[a] = es[L::GE + a * 3 + q];
    }
    float acc[C], x[C];
    ld2<C>(vm + (0 * 4 + f) * C, x);
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = d[0] * x[c];
#pragma unroll
    for (int a = 1; a < 4; ++a) {
      ld2<C>(vm + (a * 4 + f) * C, x);
#pragma unroll
      for (int c = 0; c < C; ++c) acc[c] = fmaf(d[a], x[c], acc[c]);
    }
    st2<C>(es + (q < 3 ? L::GM + (f * 3 + q) * C : L::VS + f * C), acc);
  }
  // ---- A: one lane per (element, sample): convective products c_i(q, t_k)
  const float4* __restrict__ u0t = reinterpret_cast<const float4*>(I.u0t);
  const float4* __restrict__ vt = reinterpret_cast<const float4*>(I.vt);
#pragma unroll 1
  for (int t = lane; t < EPW * K; t += 32) {
    const int s = t >= K ? 1 : 0, k = t - s * K;
    const float* g = work + s * L::ELEM + L::GE;
    const int4 nd = *reinterpret_cast<const int4*>(g + 16);
    float dN[12];
    ld4<12>(g, dN);
    const int na[4] = {nd.x, nd.y, nd.z, nd.w};
    float ua[4][3], va[4][3];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const float4 x = u0t[(int64_t)na[a] * K + k];
      ua[a][0] = x.x;
      ua[a][1] = x.y;
      ua[a][2] = x.z;
      const float4 y = vt[(int64_t)na[a] * K + k];
      va[a][0] = y.x;
      va[a][1] = y.y;
      va[a][2] = y.z;
    }
    float gv[3][3], gu[3][3];   // dv_i/dx_j, du0_i/dx_j at t_k
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        gv[i][j] = dN[j] * va[0][i] + dN[3 + j] * va[1][i] + dN[6 + j] * va[2][i] + dN[9 + j] * va[3][i];
        if (LINA)
          gu[i][j] = dN[j] * ua[0][i] + dN[3 + j] * ua[1][i] + dN[6 + j] * ua[2][i] + dN[9 + j] * ua[3][i];
      }
    float su[3], sv[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      su[j] = QB * (ua[0][j] + ua[1][j] + ua[2][j] + ua[3][j]);
      sv[j] = QB * (va[0][j] + va[1][j] + va[2][j] + va[3][j]);
    }
    float* ct = work + s * L::ELEM + L::CT + k;
#pragma unroll
    for (int qq = 0; qq < 4; ++qq)
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        float acc = 0.f;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          acc = fmaf(fmaf(QD, ua[qq][j], su[j]), gv[i][j], acc);
          if (LINA) acc = fmaf(fmaf(QD, va[qq][j], sv[j]), gu[i][j], acc);
        }
        ct[(qq * 3 + i) * L::KP] = acc;
      }
  }
  __syncwarp();
  // ---- B: point phase, lane (i = f < 3, q)
  float rowp[C];   // node-row part known after this phase (lane (f, a = q))
  float sT[C];
  float X[C];
  float extra[C];  // velocity row a = q: consistent mass and pressure terms
#pragma unroll
  for (int c = 0; c < C; ++c) {
    X[c] = 0.f;
    sT[c] = 0.f;
    extra[c] = 0.f;
  }
  if (!__all_sync(FULL, mbar_wait(bar, parity))) return false;   // nothing added yet
  if (f < 3) {
    const int i = f;
    float cm[C];
    {
      float ctv[K];
      ld4<K>(es + L::CT + (q * 3 + i) * L::KP, ctv);
      inv<N>(ctv, cm);
    }
    float G[C], Lm[C], dp[C];
    {
      float vq[C], vs[C];
      ld2<C>(es + L::VM + (q * 4 + i) * C, vq);
      ld2<C>(es + L::VS + i * C, vs);
      ld2<C>(es + L::GM + (3 * 3 + i) * C, dp);
#pragma unroll
      for (int c = 0; c < C; ++c) vq[c] = fmaf(QD, vq[c], QB * vs[c]);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        G[c] = (c == 1) ? 0.f : rho * (om_apply<N>(vq, c, omega) + cm[c]);
        Lm[c] = PAPER ? G[c] : G[c] + dp[c];
      }
    }
    const float* tq = stg + L::STG_TAU + (slot * 4 + q) * NTP;
    float T[C];
    tau_apply<N>(tq, Lm, T);
    if (MODE == MODE_JVP_EXACT && live) {
      // + d tau[v] L(u0): the derivative of tau, computed per point beforehand
      float dt[C];
      ld2<C>(I.dT + ((e * 4 + q) * 3 + i) * C, dt);
#pragma unroll
      for (int c = 0; c < C; ++c) T[c] += dt[c];
    }
    if (PAPER) {
      float Tc[C];
      tau_apply<N>(tq, dp, Tc);
#pragma unroll
      for (int c = 0; c < C; ++c) sT[c] = Tc[c];
    } else {
#pragma unroll
      for (int c = 0; c < C; ++c) sT[c] = T[c];
    }
#pragma unroll
    for (int c = 0; c < C; ++c) X[c] = G[c] - om_apply<N>(T, c, omega);
    {
      float Tt[K];
      fwd<N>(T, Tt);
      st4<K>(es + L::CT + (q * 3 + i) * L::KP, Tt);
    }
    if (LINA) {
      float T0m[C], T0t[K];
      ld2<C>(stg + L::STG_T0 + ((slot * 4 + q) * 3 + i) * C, T0m);
      fwd<N>(T0m, T0t);
      st4<K>(es + L::TS + (q * 3 + i) * L::KP, T0t);
    }
    {
      // row (a = q, i): mass_coef V/20 (sum_b v_ib + v_ia) - dN_a/dx_i V pbar
      float vs[C], vm[C], ps[C];
      ld2<C>(es + L::VS + i * C, vs);
      ld2<C>(es + L::VM + (q * 4 + i) * C, vm);
      ld2<C>(es + L::VS + 3 * C, ps);
      const float vol = es[L::GE + GEO_VOL];
      const float mc = I.ph.mass_coef * vol * 0.05f, pv = 0.25f * es[L::GE + q * 3 + i] * vol;
#pragma unroll
      for (int c = 0; c < C; ++c) extra[c] = fmaf(mc, vs[c] + vm[c], -pv * ps[c]);
    }
  }
  __syncwarp();
  if (lane == 0) issue_next();   // the staging buffer is free again
  // sums over the four points (xor butterflies over q)
  const float w4 = 0.25f * es[L::GE + GEO_VOL];
#pragma unroll
  for (int c = 0; c < C; ++c) {
    float x = X[c];
    x += __shfl_xor_sync(FULL, x, 1);
    x += __shfl_xor_sync(FULL, x, 2);
    rowp[c] = fmaf(w4, fmaf(QD, X[c], QB * x), extra[c]);   // Galerkin + (-Omega N_a) LS, velocity lanes
    float y = sT[c];
    y += __shfl_xor_sync(FULL, y, 1);
    y += __shfl_xor_sync(FULL, y, 2);
    sT[c] = y;
  }
  {
    // continuity lanes (3, a): (w/rho) dN_a/dx_i sum_q T_i
    const float da0 = es[L::GE + q * 3 + 0], da1 = es[L::GE + q * 3 + 1], da2 = es[L::GE + q * 3 + 2];
    const float wr = w4 / rho;
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const float t0 = __shfl_sync(FULL, sT[c], (lane & 16) | (0 << 2) | q);
      const float t1 = __shfl_sync(FULL, sT[c], (lane & 16) | (1 << 2) | q);
      const float t2 = __shfl_sync(FULL, sT[c], (lane & 16) | (2 << 2) | q);
      if (f == 3) rowp[c] = wr * (da0 * t0 + da1 * t1 + da2 * t2);
    }
  }
  // ---- C: one lane per (element, sample): SUPG products W_ji = sum_q u0_j T_i (+ v_j T0_i)
#pragma unroll 1
  for (int t = lane; t < EPW * K; t += 32) {
    const int s = t >= K ? 1 : 0, k = t - s * K;
    const float* ew = work + s * L::ELEM;
    const int4 nd = *reinterpret_cast<const int4*>(ew + L::GE + 16);
    const int na[4] = {nd.x, nd.y, nd.z, nd.w};
    float ua[4][3], va[4][3];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const float4 x = u0t[(int64_t)na[a] * K + k];
      ua[a][0] = x.x;
      ua[a][1] = x.y;
      ua[a][2] = x.z;
      if (LINA) {
        const float4 y = vt[(int64_t)na[a] * K + k];
        va[a][0] = y.x;
        va[a][1] = y.y;
        va[a][2] = y.z;
      }
    }
    float su[3], sv[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      su[j] = QB * (ua[0][j] + ua[1][j] + ua[2][j] + ua[3][j]);
      if (LINA) sv[j] = QB * (va[0][j] + va[1][j] + va[2][j] + va[3][j]);
    }
    float W[3][3];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int i = 0; i < 3; ++i) W[j][i] = 0.f;
#pragma unroll
    for (int qq = 0; qq < 4; ++qq) {
      float uq[3], vq[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        uq[j] = fmaf(QD, ua[qq][j], su[j]);
        if (LINA) vq[j] = fmaf(QD, va[qq][j], sv[j]);
      }
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const float Ti = ew[L::CT + (qq * 3 + i) * L::KP + k];
        const float T0i = LINA ? ew[L::TS + (qq * 3 + i) * L::KP + k] : 0.f;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          W[j][i] = fmaf(uq[j], Ti, W[j][i]);
          if (LINA) W[j][i] = fmaf(vq[j], T0i, W[j][i]);
        }
      }
    }
    float* ws = work + s * L::ELEM + L::WS + k;
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int i = 0; i < 3; ++i) ws[(j * 3 + i) * L::KP] = W[j][i];
  }
  __syncwarp();
  // ---- D: SUPG sums to modes, one lane per (element, j, i), in place, with the
  // viscous gradient folded in: Z_ji = w W_ji + mu V dv_i/dx_j
  if (lane < EPW * 9) {
    const int s = lane >= 9 ? 1 : 0, ji = lane - 9 * s;
    const int j = ji / 3, i = ji - 3 * j;
    const float* ew = work + s * L::ELEM;
    float* p = work + s * L::ELEM + L::WS + ji * L::KP;
    float wt[K], wm[C], gm[C];
    ld4<K>(p, wt);
    inv<N>(wt, wm);
    ld2<C>(ew + L::GM + (i * 3 + j) * C, gm);
    const float vol_s = ew[L::GE + GEO_VOL], w4_s = 0.25f * vol_s, mv = I.ph.mu * vol_s;
#pragma unroll
    for (int c = 0; c < C; ++c) wm[c] = fmaf(w4_s, wm[c], mv * gm[c]);
    st2<C>(p, wm);
  }
  __syncwarp();
  // ---- E: node rows, lane (f, a = q)
  {
    const int a = q;
    const int4 nd = *reinterpret_cast<const int4*>(es + L::GE + 16);
    const int node = a == 0 ? nd.x : a == 1 ? nd.y : a == 2 ? nd.z : nd.w;
    const float da[3] = {es[L::GE + a * 3 + 0], es[L::GE + a * 3 + 1], es[L::GE + a * 3 + 2]};
    const bool fixed = live ? I.dmask[node] != 0 : true;
    float row[C], x[C];
#pragma unroll
    for (int c = 0; c < C; ++c) row[c] = rowp[c];
    if (f < 3) {
      const int i = f;
#pragma unroll
      for (int j = 0; j < 3; ++j) {   // SUPG + viscous
        ld2<C>(es + L::WS + (j * 3 + i) * L::KP, x);
#pragma unroll
        for (int c = 0; c < C; ++c) row[c] = fmaf(da[j], x[c], row[c]);
      }
    } else {
#pragma unroll
      for (int d = 0; d < 3; ++d) {   // w div v
        ld2<C>(es + L::GM + (d * 3 + d) * C, x);
#pragma unroll
        for (int c = 0; c < C; ++c) row[c] = fmaf(w4, x[c], row[c]);
      }
    }
    row[1] = 0.f;
    if (live && !(f < 3 && fixed)) row_atomics<C>(I.out + ((int64_t)node * 4 + f) * C, row);
  }
  __syncwarp();
  return true;
}

// after a staging wait gave up: flag the failure by a NaN in the output (the
// solver's norms then return TS_ERR_NAN) and wait once more, bounded, for the
// copy in flight so that none lands after the warp has left
__device__ __forceinline__ void j32_abort(float* out, uint32_t bar, uint32_t parity, int lane) {
  if (lane == 0 && out) out[0] = __int_as_float(0x7fc00000);
  mbar_wait(bar, parity);
}

template <int N, int MODE>
__global__ void __launch_bounds__(128) jvp32_kernel(J32Inst I) {
  using L = J32Layout<N, MODE>;
  extern __shared__ __align__(128) float smem[];
  __shared__ __align__(8) uint64_t s_bar[4];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  float* wsm = smem + warp * L::WARP;
  float* stg = wsm;
  float* work = wsm + L::STG;
  const uint32_t bar = smem_addr(&s_bar[warp]);
  const int64_t stride = (int64_t)gridDim.x * wpb * EPW;
  int64_t base = ((int64_t)blockIdx.x * wpb + warp) * EPW;
  if (base >= I.n_elem) return;
  if (lane == 0) {
    mbar_init(bar);
    stage_issue<N, L::LINA>(I.tau, I.t0cache, base, (int)min64(EPW, I.n_elem - base), stg, bar);
  }
  __syncwarp();
  uint32_t parity = 0;
  for (; base < I.n_elem; base += stride) {
    const int64_t next = base + stride;
    const float* tau = I.tau;
    const float* t0 = I.t0cache;
    const int64_t n_elem = I.n_elem;
    auto issue = [=]() {
      if (next < n_elem) stage_issue<N, L::LINA>(tau, t0, next, (int)min64(EPW, n_elem - next), stg, bar);
    };
    if (!j32_pass<N, MODE>(I, base, stg, work, bar, parity, lane, issue)) {
      j32_abort(I.out, bar, parity, lane);
      return;
    }
    parity ^= 1u;
  }
}

__host__ __device__ constexpr bool j32_has(int N) { return dft_offset(N) >= 0; }

__device__ __forceinline__ int ntp_of(int N) {
  const int nm = 2 * N - 1;
  return ((nm * (nm + 1) / 2) + 3) & ~3;
}

// instance of tile t (binary search over the tile prefix)
__device__ __forceinline__ int tile_instance(const int64_t* __restrict__ tile_off, int n_inst, int64_t t) {
  int lo = 0, hi = n_inst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tile_off[mid] <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// stages tile t's tau / tau L (LIN_A) with the instance's own sizes
__device__ __forceinline__ void batch_issue(const J32Inst* __restrict__ insts, const int64_t* __restrict__ tile_off,
                                            int n_inst, int64_t t, float* stg, uint32_t bar) {
  const int b = tile_instance(tile_off, n_inst, t);
  const J32Inst& I = insts[b];
  const int64_t base = (t - tile_off[b]) * EPW;
  const int n = (int)min64(EPW, I.n_elem - base);
  const int ntp = ntp_of(I.N), C = 2 * I.N;
  const uint32_t bt = (uint32_t)n * 4 * ntp * 4, b0 = (uint32_t)n * 12 * C * 4;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  mbar_expect(bar, bt + b0);
  bulk_g2s(smem_addr(stg), I.tau + base * 4 * ntp, bt, bar);
  bulk_g2s(smem_addr(stg + EPW * 4 * ntp), I.t0cache + base * 12 * C, b0, bar);
}

// Tangent products of many instances in one launch.  Tile t (EPW elements)
// belongs to the instance b with tile_off[b] <= t < tile_off[b + 1]; the
// instance and tile counts are read from the device (counts[0], counts[1]) so
// that a captured launch follows later changes of the tables; each warp
// takes tiles grid-stride and runs the body compiled for that instance's N
// (warp-uniform branch).  The staging and workspace regions are sized for
// the largest N, the workspace starting after the largest staging region, so
// staging the next tile never overlaps the current tile's workspace.
template <int MODE, int NMAX>
__global__ void __launch_bounds__(128) jvp32_batch_kernel(const J32Inst* __restrict__ insts,
                                                          const int64_t* __restrict__ tile_off,
                                                          const int64_t* __restrict__ counts) {
  using LM = J32Layout<NMAX, MODE>;
  extern __shared__ __align__(128) float smem[];
  __shared__ __align__(8) uint64_t s_bar[4];
  const int n_inst = (int)counts[0];
  const int64_t n_tiles = counts[1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  float* stg = smem + warp * LM::WARP;
  float* work = stg + LM::STG;
  const uint32_t bar = smem_addr(&s_bar[warp]);
  const int64_t stride = (int64_t)gridDim.x * wpb;
  int64_t t = (int64_t)blockIdx.x * wpb + warp;
  if (t >= n_tiles) return;
  if (lane == 0) {
    mbar_init(bar);
    batch_issue(insts, tile_off, n_inst, t, stg, bar);
  }
  __syncwarp();
  uint32_t parity = 0;
  for (; t < n_tiles; t += stride) {
    const int b = tile_instance(tile_off, n_inst, t);
    const J32Inst I = insts[b];
    const int64_t base = (t - tile_off[b]) * EPW;
    const int64_t next = t + stride;
    auto issue = [=]() {
      if (next < n_tiles) batch_issue(insts, tile_off, n_inst, next, stg, bar);
    };
    bool ok = true;
    switch (I.N) {
      case 1: if constexpr (j32_has(1)) ok = j32_pass<1, MODE>(I, base, stg, work, bar, parity, lane, issue); break;
      case 2: if constexpr (j32_has(2)) ok = j32_pass<2, MODE>(I, base, stg, work, bar, parity, lane, issue); break;
      case 3: if constexpr (j32_has(3)) ok = j32_pass<3, MODE>(I, base, stg, work, bar, parity, lane, issue); break;
      case 4: if constexpr (j32_has(4)) ok = j32_pass<4, MODE>(I, base, stg, work, bar, parity, lane, issue); break;
      case 5: if constexpr (j32_has(5)) ok = j32_pass<5, MODE>(I, base, stg, work, bar, parity, lane, issue); break;
      case 7: if constexpr (j32_has(7)) ok = j32_pass<7, MODE>(I, base, stg, work, bar, parity, lane, issue); break;
      default:
        // not compiled here (the host admits no such instance): keep the staging chain intact
        ok = __all_sync(FULL, mbar_wait(bar, parity));
        __syncwarp();
        if (ok && lane == 0) issue();
        break;
    }
    if (!ok) {
      j32_abort(I.out, bar, parity, lane);
      return;
    }
    parity ^= 1u;
  }
}

// Node pre-pass: x (velocity fields of a modal field [V][4][C]) sampled in
// time into xt[V][K] float4 (x, y, z, 0).  With dmask, Dirichlet nodes'
// velocities are taken as zero (tangent inputs); Im(mode 0) is ignored.
// With zero_out, the node's row of zero_out is cleared.
template <int N>
__device__ __forceinline__ void node_samples_one(const float* __restrict__ x, const uint8_t* __restrict__ dmask,
                                                 float4* __restrict__ xt, float* __restrict__ zero_out,
                                                 int64_t node) {
  constexpr int C = 2 * N, K = 3 * N - 2;
  const bool fixed = dmask != nullptr && dmask[node] != 0;
  float y[3][K];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float m[C];
    const float2* src = reinterpret_cast<const float2*>(x + (node * 4 + i) * C);
#pragma unroll
    for (int c2 = 0; c2 < C / 2; ++c2) {
      const float2 p = fixed ? make_float2(0.f, 0.f) : src[c2];
      m[2 * c2] = p.x;
      m[2 * c2 + 1] = p.y;
    }
    fwd<N>(m, y[i]);
  }
  float4* dst = xt + node * K;
#pragma unroll
  for (int k = 0; k < K; ++k) dst[k] = make_float4(y[0][k], y[1][k], y[2][k], 0.f);
  if (zero_out) {
    float4* z = reinterpret_cast<float4*>(zero_out + node * 4 * C);
#pragma unroll
    for (int c4 = 0; c4 < C; ++c4) z[c4] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

template <int N>
__global__ void __launch_bounds__(128) node_samples_kernel(const float* __restrict__ x,
                                                           const uint8_t* __restrict__ dmask,
                                                           float4* __restrict__ xt, float* __restrict__ zero_out,
                                                           int64_t V) {
  for (int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; node < V;
       node += (int64_t)gridDim.x * blockDim.x)
    node_samples_one<N>(x, dmask, xt, zero_out, node);
}

// the pre-pass of every instance of a batch: v sampled into each instance's vt
__global__ void __launch_bounds__(128) node_samples_batch_kernel(const J32Inst* __restrict__ insts,
                                                                 const int64_t* __restrict__ node_off,
                                                                 const int64_t* __restrict__ counts) {
  const int n_inst = (int)counts[0];
  const int64_t total = counts[2];
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int b = tile_instance(node_off, n_inst, g);
    const J32Inst& I = insts[b];
    const int64_t node = g - node_off[b];
    float4* vt = reinterpret_cast<float4*>(I.vt);
    switch (I.N) {
      case 1: if constexpr (j32_has(1)) node_samples_one<1>(I.v, I.dmask, vt, nullptr, node); break;
      case 2: if constexpr (j32_has(2)) node_samples_one<2>(I.v, I.dmask, vt, nullptr, node); break;
      case 3: if constexpr (j32_has(3)) node_samples_one<3>(I.v, I.dmask, vt, nullptr, node); break;
      case 4: if constexpr (j32_has(4)) node_samples_one<4>(I.v, I.dmask, vt, nullptr, node); break;
      case 5: if constexpr (j32_has(5)) node_samples_one<5>(I.v, I.dmask, vt, nullptr, node); break;
      case 7: if constexpr (j32_has(7)) node_samples_one<7>(I.v, I.dmask, vt, nullptr, node); break;
      default: break;
    }
  }
}

template <int N>
static int launch_node_samples_impl(const float* x, const uint8_t* dmask, float* xt, float* zero_out,
                                    int64_t V, cudaStream_t st) {
  int64_t blocks = (V + 127) / 128;
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (blocks < 1) blocks = 1;
  count_launches(1);
  node_samples_kernel<N><<<(int)blocks, 128, 0, st>>>(x, dmask, reinterpret_cast<float4*>(xt), zero_out, V);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

template <int N, int MODE>
static int launch_j32_mode(const J32Inst& I, cudaStream_t st) {
  using L = J32Layout<N, MODE>;
  const int warps = 4;
  const size_t smem = (size_t)warps * L::WARP * sizeof(float);
  static bool configured[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !configured[dev]) {
    if (cudaFuncSetAttribute(jvp32_kernel<N, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return -2;
    configured[dev] = true;
  }
  const int64_t pairs = (I.n_elem + EPW - 1) / EPW;
  int64_t blocks = (pairs + warps - 1) / warps;
  // resident blocks per SM times the SM count (152 on GB300) bounds the grid;
  // every warp then loops over its pairs with the staging one pair ahead
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jvp32_kernel<N, MODE>, warps * 32, smem) !=
          cudaSuccess || per_sm < 1)
    per_sm = 1;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (blocks > (int64_t)sms * per_sm) blocks = (int64_t)sms * per_sm;
  if (blocks < 1) blocks = 1;
  count_launches(1);
  jvp32_kernel<N, MODE><<<(int)blocks, warps * 32, smem, st>>>(I);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

template <int N>
static int launch_jvp32_impl(int mode, const J32Inst& I, cudaStream_t st) {
  switch (mode) {
    case MODE_JVP_PAPER: return launch_j32_mode<N, MODE_JVP_PAPER>(I, st);
    case MODE_JVP_FROZEN: return launch_j32_mode<N, MODE_JVP_FROZEN>(I, st);
    case MODE_JVP_LIN_A: return launch_j32_mode<N, MODE_JVP_LIN_A>(I, st);
    case MODE_JVP_EXACT: return launch_j32_mode<N, MODE_JVP_EXACT>(I, st);
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
int launch_jvp32(int mode, const J32Inst& I, cudaStream_t st, cudaEvent_t e_before, cudaEvent_t e_after) {
  // the node pre-pass samples v and clears out; the element pass adds to out
  if (launch_node_samples_impl<N>(I.v, I.dmask, I.vt, I.out, I.n_nodes, st)) return -2;
  if (e_before && cudaEventRecord(e_before, st) != cudaSuccess) return -2;
  const int rc = launch_jvp32_impl<N>(mode, I, st);
  if (rc) return rc;
  if (e_after && cudaEventRecord(e_after, st) != cudaSuccess) return -2;
  return 0;
}

template <int N>
int launch_node_samples(const float* u0, float* u0t, int64_t V, cudaStream_t st) {
  return launch_node_samples_impl<N>(u0, nullptr, u0t, nullptr, V, st);
}

}  // namespace ts
