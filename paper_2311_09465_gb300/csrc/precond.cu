// Nodal block-Jacobi preconditioner of the tangent H (eq. tangent, eq. K_mat,
// section 2.4): for every node A the 8N x 8N block H_AA that couples the node's
// own unknowns (3 velocity fields and pressure, modes 0..N-1, re/im), summed
// over the elements around the node, then inverted.
//
// With A and tau frozen (eq. K_mat), per element, quadrature point q (weight
// w = V/4) and local node a, in the real storage coordinates of a mode vector:
//   S_qa = lambda_qa Omega + Conv(beta_qa),  W_qa = -lambda_qa Omega + Conv(beta_qa),
//   beta_qa = sum_j dN_a/dx_j u0_j(q)   (so Conv(beta_qa) = A_j dN_a/dx_j)
//   K_aa += w rho (lambda_qa S_qa + W_qa tau_q S_qa) + mu V |grad N_a|^2 I + m_aa I
//   G_i  += -V/4 dN_a/dx_i I + w dN_a/dx_i W_qa tau_q        (LS part: FROZEN)
//   D_j  +=  w dN_a/dx_j I   + w dN_a/dx_j tau_q S_qa         (LS part: FROZEN)
//   L    += (w / rho) |grad N_a|^2 tau_q
// with m_aa = c1 rho/dt V/10 (the consistent mass, section 2.5.3) and, on a
// resistance outlet, R (int N_A n_i)(int N_A n_j) per mode.  K is the same
// for the three velocity fields; the paper's variant drops the LS parts of G
// and D (section 2.5.2).  The derivative of A_j (LIN_A) is not part of the
// block: the blocks of a LIN_A problem are those of the frozen tangent.
//
// Conv(beta) is the truncated convolution of eq. (phi-def) written on the
// storage coordinates (x_0, Re x_n, Im x_n): with y_m = sum_n beta_{m-n} x_n
// and x_{-n} = conj(x_n), the column of Re x_n (n >= 1) is beta_{m-n} +
// beta_{m+n} and the column of Im x_n is i (beta_{m-n} - beta_{m+n}).
//
// GB300 mapping: one warp per node gathers its (element, local node) pairs
// from a node-to-element list, so each block is summed in shared memory and
// written once (no atomics, deterministic).  The warp then inverts the block
// in place (Gauss-Jordan, partial pivoting, FP32) and stores it column-major;
// the apply kernel (one warp per node, coalesced column reads) multiplies it
// with the node's slice of a Krylov vector.
#include "common.cuh"
#include "kernels.h"

namespace ts {

template <int N>
struct BlockLayout {
  static constexpr int C = 2 * N;
  static constexpr int NB = 4 * C;              // block size (unknowns per node)
  static constexpr int CC = C * C;
  // per-warp workspace (floats): the final block F [NB][NB] (its first 5 CC
  // also serve as per-point temporaries while summing), the accumulators
  // K, G_0..2, D_0..2, L [8][C][C], and small per-element arrays
  static constexpr int F = 0;
  static constexpr int TAU = 0, SM = CC, WM = 2 * CC, XM = 3 * CC, YM = 4 * CC;
  static constexpr int ACC = NB * NB;           // K at ACC, G_i at ACC+(1+i)CC, D_j at ACC+(4+j)CC, L at ACC+7CC
  static constexpr int GEO = ACC + 8 * CC;      // 20 (+4)
  static constexpr int UN = GEO + 24;           // u0 velocity at the 4 nodes [4][3][C]
  static constexpr int GAM = UN + 12 * C;       // gamma_b = sum_j dN_a/dx_j u0_bj [4][C]
  static constexpr int BET = GAM + 4 * C;       // beta_q [C]
  static constexpr int PIV = BET + C;           // pivot rows [NB]
  static constexpr int WARP = (PIV + NB + 3) & ~3;
};

// (re, im) of mode k of a conjugate-symmetric vector stored as (x_0, re/im of 1..N-1)
template <int N>
__device__ __forceinline__ float2 mode_of(const float* b, int k) {
  if (k <= -N || k >= N) return make_float2(0.f, 0.f);
  if (k >= 0) return make_float2(b[2 * k], k == 0 ? 0.f : b[2 * k + 1]);
  return make_float2(b[-2 * k], -b[-2 * k + 1]);
}

// entry (row r, column s) of Conv(beta) on storage coordinates
template <int N>
__device__ __forceinline__ float conv_entry(const float* beta, int r, int s) {
  if (s == 1) return 0.f;
  const int m = r >> 1, n = s >> 1;
  const bool im_row = r & 1;
  if (n == 0) {
    const float2 b = mode_of<N>(beta, m);
    return im_row ? b.y : b.x;
  }
  const float2 lo = mode_of<N>(beta, m - n), hi = mode_of<N>(beta, m + n);
  if (!(s & 1)) return im_row ? lo.y + hi.y : lo.x + hi.x;
  return im_row ? lo.x - hi.x : hi.y - lo.y;
}

// Omega on storage coordinates: (Omega x)_{2n} = -n w x_{2n+1}, (Omega x)_{2n+1} = n w x_{2n}
__device__ __forceinline__ float omega_entry(int r, int s, float omega) {
  const int n = r >> 1;
  if (n == 0 || (r ^ 1) != s) return 0.f;
  return (r & 1) ? n * omega : -n * omega;
}

// C = A B for C x C matrices in shared memory (row-major), lanes over outputs
template <int C>
__device__ __forceinline__ void warp_mm(const float* A, const float* B, float* out, int lane) {
  for (int t = lane; t < C * C; t += 32) {
    const int r = t / C, s = t - r * C;
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < C; ++k) acc = fmaf(A[r * C + k], B[k * C + s], acc);
    out[t] = acc;
  }
}

template <typename T, int N, bool PAPER, bool INVERT>
__global__ void __launch_bounds__(128)
    block_diag_kernel(const int32_t* __restrict__ node_off, const int32_t* __restrict__ node_elem,
                      const int4* __restrict__ tets, const T* __restrict__ geo, const T* __restrict__ u0,
                      const T* __restrict__ tau, const uint8_t* __restrict__ dmask,
                      const float* __restrict__ outdiag, Phys<float> ph, float* __restrict__ out,
                      int64_t n_nodes, unsigned* __restrict__ n_singular) {
  using L = BlockLayout<N>;
  using D = Dims<N>;
  constexpr int C = L::C, NB = L::NB, CC = L::CC, NM = D::NM, NT = D::NT, NTP = D::NT_PAD;
  extern __shared__ __align__(16) float smem_f[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  float* ws = smem_f + warp * L::WARP;
  float* F = ws + L::F;
  float* tq = ws + L::TAU;
  float* Sm = ws + L::SM;
  float* Wm = ws + L::WM;
  float* Xm = ws + L::XM;
  float* Ym = ws + L::YM;
  float* Kacc = ws + L::ACC;
  float* Gacc = Kacc + CC;
  float* Dacc = Kacc + 4 * CC;
  float* Lacc = Kacc + 7 * CC;
  float* sg = ws + L::GEO;
  float* un = ws + L::UN;
  float* gam = ws + L::GAM;
  float* bet = ws + L::BET;
  int* piv = reinterpret_cast<int*>(ws + L::PIV);
  const float rho = ph.rho, omega = ph.omega;

  for (int64_t A = (int64_t)blockIdx.x * wpb + warp; A < n_nodes; A += (int64_t)gridDim.x * wpb) {
    for (int t = lane; t < 8 * CC; t += 32) Kacc[t] = 0.f;
    __syncwarp();
    const int p0 = node_off[A], p1 = node_off[A + 1];
    for (int p = p0; p < p1; ++p) {
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
      __syncwarp();
      const float vol = sg[GEO_VOL], w4 = 0.25f * vol;
      const float da0 = sg[a * 3 + 0], da1 = sg[a * 3 + 1], da2 = sg[a * 3 + 2];
      for (int t = lane; t < 4 * C; t += 32) {
        const int b = t / C, c = t - b * C;
        gam[t] = da0 * un[(b * 3 + 0) * C + c] + da1 * un[(b * 3 + 1) * C + c] + da2 * un[(b * 3 + 2) * C + c];
      }
      for (int q = 0; q < 4; ++q) {
        const float laq = (float)qp_bary(q, a);
        __syncwarp();
        for (int c = lane; c < C; c += 32) {
          float acc = 0.f;
#pragma unroll
          for (int b = 0; b < 4; ++b) acc += (float)qp_bary(q, b) * gam[b * C + c];
          bet[c] = acc;
        }
        // tau_q: packed upper triangle in the orthonormal basis -> storage coordinates
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
          const float cv = conv_entry<N>(bet, r, s), om = omega_entry(r, s, omega);
          Sm[t] = laq * om + cv;
          Wm[t] = -laq * om + cv;
        }
        __syncwarp();
        warp_mm<C>(tq, Sm, Xm, lane);   // X = tau S
        warp_mm<C>(Wm, tq, Ym, lane);   // Y = W tau
        __syncwarp();
        for (int t = lane; t < CC; t += 32) {
          const int r = t / C, s = t - r * C;
          float wx = 0.f;
#pragma unroll
          for (int k = 0; k < C; ++k) wx = fmaf(Wm[r * C + k], Xm[k * C + s], wx);
          Kacc[t] += w4 * rho * (laq * Sm[t] + wx);
          Lacc[t] += (w4 / rho) * (da0 * da0 + da1 * da1 + da2 * da2) * tq[t];
          if (!PAPER) {
            Gacc[t] += w4 * da0 * Ym[t];
            Gacc[CC + t] += w4 * da1 * Ym[t];
            Gacc[2 * CC + t] += w4 * da2 * Ym[t];
            Dacc[t] += w4 * da0 * Xm[t];
            Dacc[CC + t] += w4 * da1 * Xm[t];
            Dacc[2 * CC + t] += w4 * da2 * Xm[t];
          }
        }
      }
      __syncwarp();
      // identity parts: viscous, consistent mass, Galerkin pressure and divergence
      const float g2 = da0 * da0 + da1 * da1 + da2 * da2;
      for (int c = lane; c < C; c += 32) {
        Kacc[c * C + c] += ph.mu * vol * g2 + ph.mass_coef * vol * 0.1f;
        Gacc[c * C + c] += -0.25f * vol * da0;
        Gacc[CC + c * C + c] += -0.25f * vol * da1;
        Gacc[2 * CC + c * C + c] += -0.25f * vol * da2;
        Dacc[c * C + c] += w4 * da0;
        Dacc[CC + c * C + c] += w4 * da1;
        Dacc[2 * CC + c * C + c] += w4 * da2;
      }
      __syncwarp();
    }
    // ---- the full block F [NB][NB], rows/columns (field, storage coordinate)
    const bool dir = dmask[A] != 0;
    const float* od = outdiag + A * 6;   // R w_i w_j (xx, xy, xz, yy, yz, zz)
    for (int t = lane; t < NB * NB; t += 32) {
      const int row = t / NB, col = t - row * NB;
      const int f = row / C, c = row - f * C, g = col / C, d = col - g * C;
      float val;
      if (f < 3 && g < 3) {
        val = f == g ? Kacc[c * C + d] : 0.f;
        if (c == d) {
          const int lo = f < g ? f : g, hi = f < g ? g : f;
          const int k = lo == 0 ? hi : (lo == 1 ? 2 + hi : 5);
          val += od[k];
        }
      } else if (f < 3) {
        val = Gacc[f * CC + c * C + d];
      } else if (g < 3) {
        val = Dacc[g * CC + c * C + d];
      } else {
        val = Lacc[c * C + d];
      }
      // fixed unknowns: Im(mode 0) of every field, velocity of a Dirichlet node
      const bool fr = c == 1 || (dir && f < 3), fc = d == 1 || (dir && g < 3);
      if (fr || fc) val = (INVERT && row == col) ? 1.f : 0.f;
      F[t] = val;
    }
    __syncwarp();
    float* dst = out + A * NB * NB;
    if (!INVERT) {
      for (int t = lane; t < NB * NB; t += 32) dst[t] = F[t];
      __syncwarp();
      continue;
    }
    // ---- in-place Gauss-Jordan inversion with partial pivoting
    bool singular = false;
    for (int k = 0; k < NB; ++k) {
      float best = -1.f;
      int bi = k;
      for (int i = k + lane; i < NB; i += 32) {
        const float v = fabsf(F[i * NB + k]);
        if (v > best) {
          best = v;
          bi = i;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) {
          best = ov;
          bi = oi;
        }
      }
      if (!(best > 0.f) || !isfinite(best)) {
        singular = true;
        break;
      }
      if (lane == 0) piv[k] = bi;
      if (bi != k)
        for (int j = lane; j < NB; j += 32) {
          const float tmp = F[k * NB + j];
          F[k * NB + j] = F[bi * NB + j];
          F[bi * NB + j] = tmp;
        }
      __syncwarp();
      const float inv = 1.f / F[k * NB + k];
      __syncwarp();
      for (int j = lane; j < NB; j += 32) F[k * NB + j] = j == k ? inv : F[k * NB + j] * inv;
      __syncwarp();
      for (int t = lane; t < NB * NB; t += 32) {
        const int i = t / NB, j = t - i * NB;
        if (i == k) continue;
        const float fik = F[i * NB + k];
        if (j == k) continue;
        F[t] = fmaf(-fik, F[k * NB + j], F[t]);
      }
      __syncwarp();
      for (int i = lane; i < NB; i += 32)
        if (i != k) F[i * NB + k] = -F[i * NB + k] * inv;
      __syncwarp();
    }
    if (singular) {
      if (lane == 0) atomicAdd(n_singular, 1u);
      for (int t = lane; t < NB * NB; t += 32) dst[t] = (t / NB == t % NB) ? 1.f : 0.f;
      __syncwarp();
      continue;
    }
    // undo the row exchanges as column exchanges, in reverse order
    for (int k = NB - 1; k >= 0; --k) {
      const int pk = piv[k];
      if (pk != k)
        for (int i = lane; i < NB; i += 32) {
          const float tmp = F[i * NB + k];
          F[i * NB + k] = F[i * NB + pk];
          F[i * NB + pk] = tmp;
        }
      __syncwarp();
    }
    // column-major store for the apply kernel
    for (int t = lane; t < NB * NB; t += 32) {
      const int col = t / NB, row = t - col * NB;
      dst[t] = F[row * NB + col];
    }
    __syncwarp();
  }
}

// z[A] = Binv[A] x[A] per node (column-major FP32 blocks, FP64 vectors)
template <int N>
__global__ void __launch_bounds__(256)
    block_apply_kernel(const float* __restrict__ binv, const double* __restrict__ x, double* __restrict__ z,
                       int64_t n_nodes) {
  constexpr int NB = 8 * N;
  constexpr int R = (NB + 31) / 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  for (int64_t A = (int64_t)blockIdx.x * wpb + warp; A < n_nodes; A += (int64_t)gridDim.x * wpb) {
    const double* xa = x + A * NB;
    float xr[R];
#pragma unroll
    for (int s = 0; s < R; ++s) xr[s] = lane + 32 * s < NB ? (float)xa[lane + 32 * s] : 0.f;
    float acc[R];
#pragma unroll
    for (int s = 0; s < R; ++s) acc[s] = 0.f;
    const float* B = binv + A * NB * NB;
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      const float xj = __shfl_sync(0xffffffffu, xr[j >> 5], j & 31);
#pragma unroll
      for (int s = 0; s < R; ++s)
        if (lane + 32 * s < NB) acc[s] = fmaf(B[j * NB + lane + 32 * s], xj, acc[s]);
    }
    double* za = z + A * NB;
#pragma unroll
    for (int s = 0; s < R; ++s)
      if (lane + 32 * s < NB) za[lane + 32 * s] = (double)acc[s];
  }
}

template <typename T, int N>
int launch_block_diag(int variant_paper, int invert, const int32_t* node_off, const int32_t* node_elem,
                      const int4* tets, const T* geo, const T* u0, const T* tau, const uint8_t* dmask,
                      const float* outdiag, Phys<float> ph, float* out, int64_t n_nodes,
                      unsigned* n_singular, cudaStream_t st) {
  using L = BlockLayout<N>;
  if (n_nodes <= 0) return 0;
  int warps = 4;
  while (warps > 1 && (size_t)warps * L::WARP * sizeof(float) > 200 * 1024) --warps;
  const size_t smem = (size_t)warps * L::WARP * sizeof(float);
  if (smem > 227 * 1024) return -6;
  int64_t blocks = (n_nodes + warps - 1) / warps;
  if (blocks > 152 * 16) blocks = 152 * 16;
  auto go = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    count_launches(1);
    kern<<<(int)blocks, warps * 32, smem, st>>>(node_off, node_elem, tets, geo, u0, tau, dmask, outdiag, ph,
                                               out, n_nodes, n_singular);
  };
  if (variant_paper) {
    if (invert) go(block_diag_kernel<T, N, true, true>);
    else go(block_diag_kernel<T, N, true, false>);
  } else {
    if (invert) go(block_diag_kernel<T, N, false, true>);
    else go(block_diag_kernel<T, N, false, false>);
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

template <int N>
int launch_block_apply(const float* binv, const double* x, double* z, int64_t n_nodes, cudaStream_t st) {
  if (n_nodes <= 0) return 0;
  const int threads = 256;
  int64_t blocks = (n_nodes + 7) / 8;
  if (blocks > 152 * 8) blocks = 152 * 8;
  count_launches(1);
  block_apply_kernel<N><<<(int)blocks, threads, 0, st>>>(binv, x, z, n_nodes);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

#define TS_INST_BLOCK(T, N)                                                                          \
  template int launch_block_diag<T, N>(int, int, const int32_t*, const int32_t*, const int4*, const T*, \
                                       const T*, const T*, const uint8_t*, const float*, Phys<float>,  \
                                       float*, int64_t, unsigned*, cudaStream_t);
TS_FOR_EACH_N(TS_INST_BLOCK, float)
TS_FOR_EACH_N(TS_INST_BLOCK, double)
#define TS_INST_BAPPLY(T, N) template int launch_block_apply<N>(const float*, const double*, double*, int64_t, cudaStream_t);
TS_FOR_EACH_N(TS_INST_BAPPLY, float)

}  // namespace ts
