// Assembled block-structured tangent of the paper's variant (section 2.5.2) and
// its sparse matrix-vector product.
//
// With A and tau frozen (eq. K_mat) and the least-squares parts dropped from
// G_i and D_j, the tangent of eq. (tangent) between nodes A and B is
//   [[K, 0, 0, G_1], [0, K, 0, G_2], [0, 0, K, G_3], [D_1, D_2, D_3, L]]
// where K_AB and L_AB are full mode matrices, but G_i = -int dN_A/dx_i N_B I
// and D_j = int N_A dN_B/dx_j I are scalars times the identity: per mesh
// connection the paper stores K once (reused for the three velocity fields),
// L, and six scalars (section 2.5.2), instead of the 16 full blocks.  Per
// element and quadrature point (weight w = V/4), in storage coordinates:
//   K_AB += w rho (lambda_qa S_qb + W_qa tau_q S_qb) + (mu V grad N_a . grad N_b
//           + c1 rho/dt V (1 + delta_ab)/20) I
//   L_AB += (w / rho) grad N_a . grad N_b tau_q
//   G_AB,i += -(V/4) dN_a/dx_i,   D_AB,j += (V/4) dN_b/dx_j
// with S_qb = lambda_qb Omega + Conv(beta_qb), W_qa = -lambda_qa Omega +
// Conv(beta_qa), beta_qb = sum_j dN_b/dx_j u0_j(q) (see precond.cu).
//
// Storage: the node graph in CSR (row A, sorted columns B, A itself
// included); per connection one record of HB = 2 C^2 + 8 floats:
// K [C][C], L [C][C], G_1..3, D_1..3, two pad floats (16-byte records).
//
// GB300 mapping.  Assembly: one warp per row gathers the row's (element,
// local node) pairs from the node-to-element list and adds every element
// contribution to the row's records (the warp owns the row: no atomics,
// deterministic).  Product: one warp per row streams the row's records
// (1.6 KB each at N = 7) through shared memory with 16-byte loads, lanes over
// the 8N outputs; the records are the only large HBM stream, so the product
// is bound by HBM bandwidth.
#include "common.cuh"
#include "kernels.h"

namespace ts {

namespace {

template <int N>
struct AsmLayout {
  static constexpr int C = 2 * N, CC = C * C;
  static constexpr int HB = 2 * CC + 8;
  // assembly workspace per warp (floats)
  static constexpr int TAU = 0, WM = CC, YM = 2 * CC, SM = 3 * CC, TSUM = 4 * CC;
  static constexpr int ZACC = 5 * CC;            // [4][C][C] LS + Galerkin parts of K_ab
  static constexpr int GEO = ZACC + 4 * CC;      // 20 (+4)
  static constexpr int UN = GEO + 24;            // u0 velocity at the 4 nodes [4][3][C]
  static constexpr int BET = UN + 12 * C;        // beta_qb [4][C] for the current q
  static constexpr int WARP = (BET + 4 * C + 3) & ~3;
  // product workspace per warp: the record and x_B
  static constexpr int PWARP = HB + 4 * C;
};

template <int N>
__device__ __forceinline__ float2 amode(const float* b, int k) {
  if (k <= -N || k >= N) return make_float2(0.f, 0.f);
  if (k >= 0) return make_float2(b[2 * k], k == 0 ? 0.f : b[2 * k + 1]);
  return make_float2(b[-2 * k], -b[-2 * k + 1]);
}

// Conv(beta) on storage coordinates (the truncated convolution of eq. phi-def)
template <int N>
__device__ __forceinline__ float aconv(const float* beta, int r, int s) {
  if (s == 1) return 0.f;
  const int m = r >> 1, n = s >> 1;
  const bool im_row = r & 1;
  if (n == 0) {
    const float2 b = amode<N>(beta, m);
    return im_row ? b.y : b.x;
  }
  const float2 lo = amode<N>(beta, m - n), hi = amode<N>(beta, m + n);
  if (!(s & 1)) return im_row ? lo.y + hi.y : lo.x + hi.x;
  return im_row ? lo.x - hi.x : hi.y - lo.y;
}

__device__ __forceinline__ float aomega(int r, int s, float omega) {
  const int n = r >> 1;
  if (n == 0 || (r ^ 1) != s) return 0.f;
  return (r & 1) ? n * omega : -n * omega;
}

}  // namespace

template <typename T, int N>
__global__ void __launch_bounds__(128)
    assemble_paper_kernel(const int32_t* __restrict__ node_off, const int32_t* __restrict__ node_elem,
                          const int32_t* __restrict__ row_off, const int32_t* __restrict__ cols,
                          const int4* __restrict__ tets, const T* __restrict__ geo, const T* __restrict__ u0,
                          const T* __restrict__ tau, Phys<float> ph, float* __restrict__ H, int64_t n_nodes) {
  using L = AsmLayout<N>;
  using D = Dims<N>;
  constexpr int C = L::C, CC = L::CC, HB = L::HB, NM = D::NM, NT = D::NT, NTP = D::NT_PAD;
  extern __shared__ __align__(16) float smem_f[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  float* ws = smem_f + warp * L::WARP;
  float* tq = ws + L::TAU;
  float* Wm = ws + L::WM;
  float* Ym = ws + L::YM;
  float* Sm = ws + L::SM;
  float* Ts = ws + L::TSUM;
  float* Z = ws + L::ZACC;
  float* sg = ws + L::GEO;
  float* un = ws + L::UN;
  float* bet = ws + L::BET;
  const float rho = ph.rho, omega = ph.omega;

  for (int64_t A = (int64_t)blockIdx.x * wpb + warp; A < n_nodes; A += (int64_t)gridDim.x * wpb) {
    const int r0 = row_off[A], r1 = row_off[A + 1];
    for (int64_t t = (int64_t)r0 * HB + lane; t < (int64_t)r1 * HB; t += 32) H[t] = 0.f;
    __syncwarp();
    for (int p = node_off[A]; p < node_off[A + 1]; ++p) {
      const int packed = node_elem[p];
      const int64_t e = packed >> 2;
      const int a = packed & 3;
      const int4 nd = tets[e];
      const int node[4] = {nd.x, nd.y, nd.z, nd.w};
      if (lane < GEO_STRIDE) sg[lane] = (float)geo[e * GEO_STRIDE + lane];
      for (int t = lane; t < 12 * C; t += 32) {
        const int b = t / (3 * C), r = t - b * 3 * C;
        const int c = r % C;
        un[t] = c == 1 ? 0.f : (float)u0[(int64_t)node[b] * 4 * C + r];
      }
      for (int t = lane; t < 4 * CC; t += 32) Z[t] = 0.f;
      for (int t = lane; t < CC; t += 32) Ts[t] = 0.f;
      // slot of each column node[b] in row A (lane b searches)
      int slot = -1;
      if (lane < 4) {
        const int Bn = node[lane];
        for (int s = r0; s < r1; ++s)
          if (cols[s] == Bn) {
            slot = s;
            break;
          }
      }
      __syncwarp();
      const float vol = sg[GEO_VOL], w4 = 0.25f * vol;
      for (int q = 0; q < 4; ++q) {
        const float laq = (float)qp_bary(q, a);
        // beta_qb for b = 0..3
        for (int t = lane; t < 4 * C; t += 32) {
          const int b = t / C, c = t - b * C;
          float acc = 0.f;
#pragma unroll
          for (int bb = 0; bb < 4; ++bb) {
            const float lam = (float)qp_bary(q, bb);
            acc += lam * (sg[b * 3 + 0] * un[(bb * 3 + 0) * C + c] + sg[b * 3 + 1] * un[(bb * 3 + 1) * C + c] +
                          sg[b * 3 + 2] * un[(bb * 3 + 2) * C + c]);
          }
          bet[t] = acc;
        }
        for (int t = lane; t < CC; t += 32) tq[t] = 0.f;
        __syncwarp();
        const T* tp = tau + (e * 4 + q) * NTP;
        for (int t = lane; t < NT; t += 32) {
          int r = 0, rem = t;
          while (rem >= NM - r) {
            rem -= NM - r;
            ++r;
          }
          const int s = r + rem;
          const float val = (float)tp[t];
          const float drs = (r == 0 && s > 0) ? Real<float>::SQRT2 : 1.f;
          const float dsr = (r == 0 && s > 0) ? Real<float>::INV_SQRT2 : 1.f;
          tq[stor_of(r) * C + stor_of(s)] = val * drs;
          tq[stor_of(s) * C + stor_of(r)] = val * dsr;
        }
        for (int t = lane; t < CC; t += 32) {
          const int r = t / C, s = t - r * C;
          Wm[t] = -laq * aomega(r, s, omega) + aconv<N>(bet + a * C, r, s);
        }
        __syncwarp();
        // Y = W_qa tau_q; Tsum += tau_q
        for (int t = lane; t < CC; t += 32) {
          const int r = t / C, s = t - r * C;
          float acc = 0.f;
#pragma unroll
          for (int k = 0; k < C; ++k) acc = fmaf(Wm[r * C + k], tq[k * C + s], acc);
          Ym[t] = acc;
          Ts[t] += tq[t];
        }
        for (int b = 0; b < 4; ++b) {
          const float lbq = (float)qp_bary(q, b);
          __syncwarp();
          for (int t = lane; t < CC; t += 32) {
            const int r = t / C, s = t - r * C;
            Sm[t] = lbq * aomega(r, s, omega) + aconv<N>(bet + b * C, r, s);
          }
          __syncwarp();
          // Z_b += laq S_qb + Y S_qb  (times w rho at the end)
          for (int t = lane; t < CC; t += 32) {
            const int r = t / C, s = t - r * C;
            float acc = laq * Sm[t];
#pragma unroll
            for (int k = 0; k < C; ++k) acc = fmaf(Ym[r * C + k], Sm[k * C + s], acc);
            Z[b * CC + t] += acc;
          }
        }
        __syncwarp();
      }
      // add the element's contributions to the four records of row A
      const float da0 = sg[a * 3 + 0], da1 = sg[a * 3 + 1], da2 = sg[a * 3 + 2];
      for (int b = 0; b < 4; ++b) {
        const int sb = __shfl_sync(0xffffffffu, slot, b);
        if (sb < 0) continue;   // cannot happen for a consistent graph
        float* rec = H + (int64_t)sb * HB;
        const float gab = da0 * sg[b * 3 + 0] + da1 * sg[b * 3 + 1] + da2 * sg[b * 3 + 2];
        const float diag = ph.mu * vol * gab + ph.mass_coef * vol * (a == b ? 0.1f : 0.05f);
        for (int t = lane; t < CC; t += 32) {
          const int r = t / C, s = t - r * C;
          rec[t] += w4 * rho * Z[b * CC + t] + (r == s ? diag : 0.f);
          rec[CC + t] += (w4 / rho) * gab * Ts[t];
        }
        if (lane < 3) rec[2 * CC + lane] += -w4 * sg[a * 3 + lane];
        else if (lane < 6) rec[2 * CC + lane] += w4 * sg[b * 3 + lane - 3];
        __syncwarp();
      }
    }
  }
}

// 16-byte asynchronous global -> shared copies (LDGSTS), grouped per stage
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(PENDING) : "memory"); }

// y = H x on the assembled records; Dirichlet velocity and Im(mode 0) inputs
// are ignored and the same rows of y are zero.  The record and x_B of the
// next connection are copied into shared memory (double buffer) while the
// current one is multiplied, so a warp keeps one record in flight.
constexpr int SPMV_WARPS = 8;   // warps (rows in flight) per block

template <int N>
__global__ void __launch_bounds__(256)
    spmv_paper_kernel(const int32_t* __restrict__ row_off, const int32_t* __restrict__ cols,
                      const float* __restrict__ H, const uint8_t* __restrict__ dmask,
                      const float* __restrict__ x, float* __restrict__ y, int64_t n_nodes) {
  using L = AsmLayout<N>;
  constexpr int C = L::C, CC = L::CC, HB = L::HB, NB = 4 * C;
  constexpr int R = (NB + 31) / 32;
  extern __shared__ __align__(16) float smem_f[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  float* buf0 = smem_f + warp * 2 * L::PWARP;   // [2][HB + NB]
  auto stage = [&](int p, float* dst) {
    const float4* src = reinterpret_cast<const float4*>(H + (int64_t)p * HB);
    for (int t = lane; t < HB / 4; t += 32) cp_async16(dst + 4 * t, src + t);
    const float4* xb = reinterpret_cast<const float4*>(x + (int64_t)cols[p] * NB);
    for (int t = lane; t < NB / 4; t += 32) cp_async16(dst + HB + 4 * t, xb + t);
    cp_async_commit();
  };
  for (int64_t A = (int64_t)blockIdx.x * wpb + warp; A < n_nodes; A += (int64_t)gridDim.x * wpb) {
    float acc[R];
#pragma unroll
    for (int k = 0; k < R; ++k) acc[k] = 0.f;
    const int r0 = row_off[A], r1 = row_off[A + 1];
    if (r0 < r1) stage(r0, buf0);
    for (int p = r0; p < r1; ++p) {
      float* rec = buf0 + ((p - r0) & 1) * L::PWARP;
      float* xs = rec + HB;
      if (p + 1 < r1) {
        stage(p + 1, buf0 + ((p + 1 - r0) & 1) * L::PWARP);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncwarp();
      const bool dirB = dmask[cols[p]] != 0;
      for (int t = lane; t < NB; t += 32) {
        const int f = t / C, c = t - f * C;
        if (c == 1 || (dirB && f < 3)) xs[t] = 0.f;
      }
      __syncwarp();
#pragma unroll
      for (int k = 0; k < R; ++k) {
        const int o = lane + 32 * k;
        if (o < NB) {
          const int f = o / C, r = o - f * C;
          float s = acc[k];
          // rows and x slices start at multiples of 2 floats: 8-byte shared loads
          if (f < 3) {
            const float2* Kr = reinterpret_cast<const float2*>(rec + r * C);
            const float2* xi = reinterpret_cast<const float2*>(xs + f * C);
#pragma unroll
            for (int c = 0; c < C / 2; ++c) {
              const float2 a = Kr[c], b = xi[c];
              s = fmaf(a.x, b.x, fmaf(a.y, b.y, s));
            }
            s = fmaf(rec[2 * CC + f], xs[3 * C + r], s);
          } else {
            const float2* Lr = reinterpret_cast<const float2*>(rec + CC + r * C);
            const float2* xp = reinterpret_cast<const float2*>(xs + 3 * C);
#pragma unroll
            for (int c = 0; c < C / 2; ++c) {
              const float2 a = Lr[c], b = xp[c];
              s = fmaf(a.x, b.x, fmaf(a.y, b.y, s));
            }
            s = fmaf(rec[2 * CC + 3], xs[r], s);
            s = fmaf(rec[2 * CC + 4], xs[C + r], s);
            s = fmaf(rec[2 * CC + 5], xs[2 * C + r], s);
          }
          acc[k] = s;
        }
      }
      __syncwarp();
    }
    const bool dirA = dmask[A] != 0;
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int o = lane + 32 * k;
      if (o < NB) {
        const int f = o / C, r = o - f * C;
        y[A * NB + o] = (r == 1 || (dirA && f < 3)) ? 0.f : acc[k];
      }
    }
  }
}

// One colour of a symmetric block Gauss-Seidel sweep with the assembled
// records: for each node A of the colour (rows[0..n_rows)),
//   z_A = Binv_A (r_A - sum_{B != A} H_AB z_B)
// with z read as it stands (earlier colours of this sweep already updated).
// Binv: inverted nodal diagonal blocks, column-major (precond.cu).  One warp
// per row.  A colour holds only a few thousand rows (a few warps per SM), so
// each warp keeps SGS_STAGES - 1 copies in flight through a ring of
// SGS_STAGES shared-memory slots: first the row's connections (one record
// plus z_B per slot), then its inverted block in chunks of whole columns, so
// that the block is already on its way while the last connections are
// multiplied.  The terms of every output are added in the same order as a
// plain loop over the connections and then over the block's columns.
constexpr int SGS_STAGES = 2;
constexpr int SGS_WARPS = 2;   // warps (rows in flight) per block

template <int N>
struct SgsChunks {
  static constexpr int NB = 8 * N;
  static constexpr int CPC = AsmLayout<N>::PWARP / NB;     // block columns per slot
  static constexpr int NCH = (NB + CPC - 1) / CPC;         // chunks per block
};

template <int N>
__global__ void __launch_bounds__(256)
    sgs_colour_kernel(const int32_t* __restrict__ rows, int64_t n_rows, const int32_t* __restrict__ row_off,
                      const int32_t* __restrict__ cols, const float* __restrict__ H,
                      const float* __restrict__ binv, const uint8_t* __restrict__ dmask,
                      const float* __restrict__ r, float* __restrict__ z, int diag_only) {
  using L = AsmLayout<N>;
  using K = SgsChunks<N>;
  constexpr int C = L::C, CC = L::CC, HB = L::HB, NB = 4 * C, S = SGS_STAGES;
  constexpr int CPC = K::CPC, NCH = K::NCH;
  constexpr int R = (NB + 31) / 32;
  static_assert(CPC >= 1 && (CPC * NB) % 4 == 0, "block chunk must be whole 16-byte copies");
  extern __shared__ __align__(16) float smem_f[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  float* buf0 = smem_f + warp * S * L::PWARP;   // [S][PWARP]
  for (int64_t k = (int64_t)blockIdx.x * wpb + warp; k < n_rows; k += (int64_t)gridDim.x * wpb) {
    const int A = rows[k];
    const bool dirA = dmask[A] != 0;
    float acc[R], rv[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int o = lane + 32 * j;
      acc[j] = 0.f;
      rv[j] = o < NB ? r[(int64_t)A * NB + o] : 0.f;
    }
    const int r0 = row_off[A], r1 = row_off[A + 1];
    // position of the diagonal connection in the row (rows hold at most a
    // few dozen connections): the i-th off-diagonal one is r0 + i, or
    // r0 + i + 1 from the diagonal on
    int pd = r1;
    for (int b = r0; b < r1; b += 32) {
      const unsigned hit = __ballot_sync(0xffffffffu, b + lane < r1 && cols[b + lane] == A);
      if (hit) {
        pd = b + __ffs(hit) - 1;
        break;
      }
    }
    // diag_only: every z_B is zero (the sweep's first colour), so is the sum
    const int n_off = diag_only ? 0 : (r1 - r0) - (pd < r1 ? 1 : 0);
    const int n_items = n_off + NCH;
    auto conn = [&](int i) { return r0 + i + (r0 + i >= pd ? 1 : 0); };
    const float* Bi = binv + (int64_t)A * NB * NB;
    // one commit group per ring position, empty past the row's end, so that
    // waiting for all but the newest S - 1 groups always means "slot i landed"
    auto stage = [&](int i) {
      float* dst = buf0 + (i % S) * L::PWARP;
      if (i < n_off) {
        const int p = conn(i);
        const float4* src = reinterpret_cast<const float4*>(H + (int64_t)p * HB);
        for (int t = lane; t < HB / 4; t += 32) cp_async16(dst + 4 * t, src + t);
        const float4* zb = reinterpret_cast<const float4*>(z + (int64_t)cols[p] * NB);
        for (int t = lane; t < NB / 4; t += 32) cp_async16(dst + HB + 4 * t, zb + t);
      } else if (i < n_items) {
        const int c0 = (i - n_off) * CPC;
        const int ncol = NB - c0 < CPC ? NB - c0 : CPC;
        const float4* src = reinterpret_cast<const float4*>(Bi + (int64_t)c0 * NB);
        for (int t = lane; t < ncol * NB / 4; t += 32) cp_async16(dst + 4 * t, src + t);
      }
      cp_async_commit();
    };
#pragma unroll
    for (int i = 0; i < S - 1; ++i) stage(i);
    float tv[R], out[R];
#pragma unroll
    for (int j = 0; j < R; ++j) tv[j] = out[j] = 0.f;
    for (int i = 0; i < n_items; ++i) {
      // slot (i + S - 1) % S was used in iteration i - 1 (synced below)
      stage(i + S - 1);
      cp_async_wait<S - 1>();
      __syncwarp();
      float* rec = buf0 + (i % S) * L::PWARP;
      if (i < n_off) {
        float* xs = rec + HB;
        const bool dirB = dmask[cols[conn(i)]] != 0;
        for (int t = lane; t < NB; t += 32) {
          const int f = t / C, c = t - f * C;
          if (c == 1 || (dirB && f < 3)) xs[t] = 0.f;
        }
        __syncwarp();
#pragma unroll
        for (int j = 0; j < R; ++j) {
          const int o = lane + 32 * j;
          if (o < NB) {
            const int f = o / C, rr = o - f * C;
            float s = acc[j];
            if (f < 3) {
              const float2* Kr = reinterpret_cast<const float2*>(rec + rr * C);
              const float2* xi = reinterpret_cast<const float2*>(xs + f * C);
#pragma unroll
              for (int c = 0; c < C / 2; ++c) {
                const float2 a = Kr[c], b = xi[c];
                s = fmaf(a.x, b.x, fmaf(a.y, b.y, s));
              }
              s = fmaf(rec[2 * CC + f], xs[3 * C + rr], s);
            } else {
              const float2* Lr = reinterpret_cast<const float2*>(rec + CC + rr * C);
              const float2* xp = reinterpret_cast<const float2*>(xs + 3 * C);
#pragma unroll
              for (int c = 0; c < C / 2; ++c) {
                const float2 a = Lr[c], b = xp[c];
                s = fmaf(a.x, b.x, fmaf(a.y, b.y, s));
              }
              s = fmaf(rec[2 * CC + 3], xs[rr], s);
              s = fmaf(rec[2 * CC + 4], xs[C + rr], s);
              s = fmaf(rec[2 * CC + 5], xs[2 * C + rr], s);
            }
            acc[j] = s;
          }
        }
      } else {
        // t = r_A - (off-diagonal sum), kept in registers; each block column
        // takes its entry of t from the lane that holds it
        if (i == n_off) {
#pragma unroll
          for (int j = 0; j < R; ++j) {
            const int o = lane + 32 * j;
            const int f = o / C, c = o - f * C;
            tv[j] = (o >= NB || c == 1 || (dirA && f < 3)) ? 0.f : rv[j] - acc[j];
          }
        }
        const int c0 = (i - n_off) * CPC;
        const int ncol = NB - c0 < CPC ? NB - c0 : CPC;
        for (int u = 0; u < ncol; ++u) {
          const int col = c0 + u;
          float xc = 0.f;
#pragma unroll
          for (int j = 0; j < R; ++j) {
            const float v = __shfl_sync(0xffffffffu, tv[j], col & 31);
            if ((col >> 5) == j) xc = v;
          }
#pragma unroll
          for (int j = 0; j < R; ++j) {
            const int o = lane + 32 * j;
            if (o < NB) out[j] = fmaf(rec[u * NB + o], xc, out[j]);
          }
        }
      }
      __syncwarp();
    }
    // the groups still open are empty (positions past the row's end)
    cp_async_wait<0>();
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int o = lane + 32 * j;
      if (o < NB) z[(int64_t)A * NB + o] = out[j];
    }
    __syncwarp();
  }
}

template <int N>
int launch_sgs_colour(const int32_t* rows, int64_t n_rows, const int32_t* row_off, const int32_t* cols,
                      const float* H, const float* binv, const uint8_t* dmask, const float* r, float* z,
                      int diag_only, cudaStream_t st) {
  using L = AsmLayout<N>;
  if (n_rows <= 0) return 0;
  int warps = SGS_WARPS;
  while (warps > 1 && (size_t)warps * SGS_STAGES * L::PWARP * sizeof(float) > 200 * 1024) --warps;
  const size_t smem = (size_t)warps * SGS_STAGES * L::PWARP * sizeof(float);
  if (smem > 227 * 1024) return -6;
  cudaFuncSetAttribute(sgs_colour_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int64_t blocks = (n_rows + warps - 1) / warps;
  if (blocks > 152 * 64) blocks = 152 * 64;
  count_launches(1);
  sgs_colour_kernel<N><<<(int)blocks, warps * 32, smem, st>>>(rows, n_rows, row_off, cols, H, binv, dmask, r, z,
                                                               diag_only);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

template <typename T, int N>
int launch_assemble_paper(const int32_t* node_off, const int32_t* node_elem, const int32_t* row_off,
                          const int32_t* cols, const int4* tets, const T* geo, const T* u0, const T* tau,
                          Phys<float> ph, float* H, int64_t n_nodes, cudaStream_t st) {
  using L = AsmLayout<N>;
  if (n_nodes <= 0) return 0;
  int warps = 4;
  while (warps > 1 && (size_t)warps * L::WARP * sizeof(float) > 200 * 1024) --warps;
  const size_t smem = (size_t)warps * L::WARP * sizeof(float);
  if (smem > 227 * 1024) return -6;
  cudaFuncSetAttribute(assemble_paper_kernel<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int64_t blocks = (n_nodes + warps - 1) / warps;
  if (blocks > 152 * 32) blocks = 152 * 32;
  count_launches(1);
  assemble_paper_kernel<T, N><<<(int)blocks, warps * 32, smem, st>>>(node_off, node_elem, row_off, cols, tets,
                                                                    geo, u0, tau, ph, H, n_nodes);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

template <int N>
int launch_spmv_paper(const int32_t* row_off, const int32_t* cols, const float* H, const uint8_t* dmask,
                      const float* x, float* y, int64_t n_nodes, cudaStream_t st) {
  using L = AsmLayout<N>;
  if (n_nodes <= 0) return 0;
  const int warps = SPMV_WARPS;
  const size_t smem = (size_t)warps * 2 * L::PWARP * sizeof(float);
  if (smem > 227 * 1024) return -6;
  cudaFuncSetAttribute(spmv_paper_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int64_t blocks = (n_nodes + warps - 1) / warps;
  if (blocks > 152 * 64) blocks = 152 * 64;
  count_launches(1);
  spmv_paper_kernel<N><<<(int)blocks, warps * 32, smem, st>>>(row_off, cols, H, dmask, x, y, n_nodes);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int assembled_record_floats(int N) { return 2 * (2 * N) * (2 * N) + 8; }

#define TS_INST_ASM(T, N)                                                                                   \
  template int launch_assemble_paper<T, N>(const int32_t*, const int32_t*, const int32_t*, const int32_t*,  \
                                           const int4*, const T*, const T*, const T*, Phys<float>, float*,    \
                                           int64_t, cudaStream_t);
TS_FOR_EACH_N(TS_INST_ASM, float)
TS_FOR_EACH_N(TS_INST_ASM, double)
#define TS_INST_SGS(T, N)                                                                                  \
  template int launch_sgs_colour<N>(const int32_t*, int64_t, const int32_t*, const int32_t*, const float*, \
                                    const float*, const uint8_t*, const float*, float*, int, cudaStream_t);
TS_FOR_EACH_N(TS_INST_SGS, float)
#define TS_INST_SPMV(T, N)                                                                          \
  template int launch_spmv_paper<N>(const int32_t*, const int32_t*, const float*, const uint8_t*, \
                                    const float*, float*, int64_t, cudaStream_t);
TS_FOR_EACH_N(TS_INST_SPMV, float)

}  // namespace ts
