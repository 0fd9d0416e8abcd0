// tau of eq. (3D-tau) to near-FP64 accuracy with the arithmetic in
// double-float (pairs of FP32 numbers, ddfloat.cuh) instead of FP64.
//
// Same refinement as tau_polish_kernel (tau.cu): FP32 Jacobi eigenvectors V,
// two Newton-Schulz steps V <- V (3I - V^T V)/2, B = V^T M V, the second-order
// Daleckii-Krein expansion of B^{-1/2} around diag(B), tau = V Z V^T.  GB300
// issues FP32 at 64 times its FP64 rate, and a double-float multiply-add is
// about 15 FP32 instructions, so this form does the O(n_m^3) work several
// times faster.  A double-float sum carries an absolute error near 2^-46 of
// its largest term (FP64: 2^-53), so tau is about a hundred times less
// accurate than the FP64 refinement in the directions of the smallest
// eigenvalues of M; entries stay within ~1e-14 * cond(M) of the exact value.
//
// Each point's matrix is scaled by an even power of two so that its entries
// are near 1 (FP32 exponent range); the scale is undone exactly at the end.
#include "common.cuh"
#include "ddfloat.cuh"
#include "jacobi.cuh"
#include "kernels.h"

namespace ts {

namespace {

template <int N>
__device__ __forceinline__ dd conv_entry_dd(const dd* a, int r, int s) {
  constexpr float S2H = 1.41421353816986083984375f;  // sqrt(2) = S2H + S2L
  constexpr float S2L = (float)(1.41421356237309504880 - 1.41421353816986083984375);
  auto ar = [&](int kk) -> dd {
    const int m = kk < 0 ? -kk : kk;
    return m < N ? a[2 * m] : dd{0.f, 0.f};
  };
  auto ai = [&](int kk) -> dd {
    const int m = kk < 0 ? -kk : kk;
    if (m >= N || m == 0) return dd{0.f, 0.f};
    return kk > 0 ? a[2 * m + 1] : dd_neg(a[2 * m + 1]);
  };
  if (r == 0 && s == 0) return a[0];
  if (r == 0 || s == 0) {
    const int o = r == 0 ? s : r;
    const int n = (o + 1) >> 1;
    return dd_mul((o & 1) ? ar(n) : ai(n), dd{S2H, S2L});
  }
  const int m = (r + 1) >> 1, n = (s + 1) >> 1;
  const bool rre = r & 1, sre = s & 1;
  if (rre && sre) return dd_add(ar(m - n), ar(m + n));
  if (rre && !sre) return dd_add(ai(m + n), dd_neg(ai(m - n)));
  if (!rre && sre) return dd_add(ai(m - n), ai(m + n));
  return dd_add(ar(m - n), dd_neg(ar(m + n)));
}

// (r, s), r <= s, of the packed row-major upper-triangle index t of an
// n x n symmetric matrix (the inverse of packed_index)
template <int NM>
__device__ __forceinline__ void tri_rs(int t, int& r, int& s) {
  r = 0;
  while (t >= NM - r) {
    t -= NM - r;
    ++r;
  }
  s = r + t;
}

// The double-float multiply-add is a chain of about ten dependent FP32
// operations, and the point's shared footprint leaves only a few warps per
// SM, so one accumulation per lane leaves the FP32 pipe idle most of the
// time.  Each lane therefore computes CH outputs of a phase at once (t,
// t + N, ..., t + (CH - 1) N of its group's outputs; a slot past the phase's
// end repeats t and is not stored), CH independent chains.  Within an output
// the terms are added in the same order as a plain loop would, so the
// results do not depend on this grouping (2 to 6 chains gave bit-identical
// residuals; 3 was the fastest at N = 7).
constexpr int CH = 3;   // outputs (accumulation chains) per lane pass

struct DotN {
  dd c[CH];
};

__device__ __forceinline__ void dot_zero(DotN& d) {
#pragma unroll
  for (int x = 0; x < CH; ++x) d.c[x] = dd{0.f, 0.f};
}

// c_x += sum_j fa(x)[j * as] fb(x)[j * bs], j = 0..cnt-1, x < CH
template <bool FF, typename FA, typename FB>
__device__ __forceinline__ void dotn(DotN& d, FA fa, int as, FB fb, int bs, int cnt) {
#pragma unroll 1
  for (int j = 0; j < cnt; ++j) {
    const int ia = j * as, ib = j * bs;
#pragma unroll
    for (int x = 0; x < CH; ++x) {
      if (FF)
        d.c[x] = dd_fma_ff(fa(x)[ia].hi, fb(x)[ib].hi, d.c[x]);
      else
        d.c[x] = dd_fma(fa(x)[ia], fb(x)[ib], d.c[x]);
    }
  }
}

}  // namespace

template <int N>
struct DDLayout {
  static constexpr int NP = 2 * N, NM = 2 * N - 1, C = 2 * N, LD = NP + 1;
  static constexpr int GPW = 32 / N;
  static constexpr int NN = NM * NM;
  // in 8-byte words (one dd per word).  The scratch holds one C_m at a time,
  // then the two FP32 Jacobi matrices (and, for a warm start, an FP32 n x n
  // product), then the refinement's temporaries (at most two n x n matrices).
  static constexpr int JAC = NP * LD + (NN + 1) / 2;
  static constexpr int SCR = (2 * NN > JAC) ? 2 * NN : JAC;
  static constexpr int CM = 0;
  static constexpr int M = CM + SCR;        // [NM][NM] M, later B
  static constexpr int V = M + NN;          // [NM][NM] eigenvectors
  static constexpr int W = V + NN;          // [3][C] w_m, later sqrt(b_ii), 1/sqrt(b_ii), floats
  // a point's block, padded to N (mod 16) words of 8 bytes: the N lanes of a
  // group read N consecutive words of a row, and consecutive groups then
  // start 2N banks apart, so the groups of a warp do not share banks
  static constexpr int GROUP_RAW = W + 3 * C;
  static constexpr int GROUP = GROUP_RAW + ((N - GROUP_RAW) % 16 + 16) % 16;
  static constexpr int WARP = GROUP * GPW + 32;   // + 64 floats of reduction scratch
};

template <int N>
__global__ void __launch_bounds__(128) tau_dd_kernel(const int4* __restrict__ tets,
                                                    const double* __restrict__ geo,
                                                    const double* __restrict__ y, int64_t n_qp,
                                                    double* __restrict__ tau_out, double nu,
                                                    double C_I,
                                                    unsigned* __restrict__ n_unconverged,
                                                    float* __restrict__ eig_out,
                                                    float* __restrict__ vcache, int warm) {
  using L = DDLayout<N>;
  constexpr int NP = L::NP, NM = L::NM, C = L::C, LD = L::LD, NN = L::NN, GPW = L::GPW;
  constexpr int NT = NM * (NM + 1) / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  dd* smem = reinterpret_cast<dd*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane / N, k = lane - (lane / N) * N;
  const bool in_group = g < GPW;
  dd* wbase = smem + warp * L::WARP;
  dd* base = wbase + (in_group ? g : 0) * L::GROUP;
  dd* S = base + L::CM;
  dd* M = base + L::M;
  dd* V = base + L::V;
  dd* w = base + L::W;
  float* Mf = reinterpret_cast<float*>(S);
  float* Vf = Mf + NP * LD;
  float* red = reinterpret_cast<float*>(wbase + GPW * L::GROUP);

  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t qb = ((int64_t)blockIdx.x * (blockDim.x >> 5) + warp) * GPW; qb < n_qp;
       qb += warps_total * GPW) {
    const int64_t gq = qb + g;
    const bool live = in_group && gq < n_qp;
    const int64_t e = live ? gq >> 2 : 0;
    const int q = (int)(gq & 3);
    // w_m = sum_i L_im u_i for this lane's two storage coordinates k, k + N
    dd wl[2][3];
    double diff = 0;
    float part = 0.f;
    if (live) {
      const double* gg = geo + e * GEO_STRIDE + GEO_G;
      const dd gxx = dd_from_double(gg[0]), gxy = dd_from_double(gg[1]),
               gxz = dd_from_double(gg[2]), gyy = dd_from_double(gg[3]),
               gyz = dd_from_double(gg[4]), gzz = dd_from_double(gg[5]);
      const double GG = gg[0] * gg[0] + gg[3] * gg[3] + gg[5] * gg[5] +
                        2.0 * (gg[1] * gg[1] + gg[2] * gg[2] + gg[4] * gg[4]);
      diff = C_I * nu * nu * GG;
      // G = L L^T (Cholesky) in double-float
      const dd l00 = dd_sqrt(gxx), r00 = dd_rcp(l00);
      const dd l10 = dd_mul(gxy, r00), l20 = dd_mul(gxz, r00);
      const dd l11 = dd_sqrt(dd_fma(dd_neg(l10), l10, gyy)), r11 = dd_rcp(l11);
      const dd l21 = dd_mul(dd_fma(dd_neg(l20), l10, gyz), r11);
      const dd l22 = dd_sqrt(dd_fma(dd_neg(l21), l21, dd_fma(dd_neg(l20), l20, gzz)));
      const int4 nd = tets[e];
      const int node[4] = {nd.x, nd.y, nd.z, nd.w};
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = k + h * N;
        double u[3] = {0, 0, 0};
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const double lam = qp_bary(q, a);
          const double* ya = y + (int64_t)node[a] * 4 * C;
#pragma unroll
          for (int i = 0; i < 3; ++i) u[i] += lam * ya[i * C + c];
        }
        if (c == 1) u[0] = u[1] = u[2] = 0;
        const dd u0 = dd_from_double(u[0]), u1 = dd_from_double(u[1]), u2 = dd_from_double(u[2]);
        wl[h][0] = dd_fma(l00, u0, dd_fma(l10, u1, dd_mul(l20, u2)));
        wl[h][1] = dd_fma(l11, u1, dd_mul(l21, u2));
        wl[h][2] = dd_mul(l22, u2);
#pragma unroll
        for (int m = 0; m < 3; ++m) part += wl[h][m].hi * wl[h][m].hi;
      }
    }
    red[lane] = part;
    __syncwarp();
    // scale the point's M by 2^(-2 h2) (w by 2^-h2) so that it is near 1
    double unscale = 1.0;
    dd diffd = dd{0.f, 0.f};
    if (live) {
      float est = 0.f;
      for (int j = 0; j < N; ++j) est += red[g * N + j];
      est = 4.f * est + (float)diff;
      int ex = 0;
      if (est > 0.f && isfinite(est)) frexpf(est, &ex);
      const int h2 = ex >> 1;
      const float sw = ldexpf(1.f, -h2);
      unscale = ldexp(1.0, -h2);
      diffd = dd_from_double(diff * unscale * unscale);
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int m = 0; m < 3; ++m) w[m * C + k + h * N] = dd_scale(wl[h][m], sw);
    }
    __syncwarp();
    // M = sum_m C_m C_m + C_I nu^2 (G:G) I, one convolution matrix C_m = A(w_m)
    // (symmetric) at a time; M carries the running sum of an entry from one m
    // to the next exactly (a double-float store), so every entry adds its
    // terms in the order m = 0, 1, 2, j = 0..n-1
#pragma unroll 1
    for (int m = 0; m < 3; ++m) {
      if (live)
        for (int t = k; t < NT; t += N) {
          int r, s;
          tri_rs<NM>(t, r, s);
          const dd v = conv_entry_dd<N>(w + m * C, r, s);
          S[r * NM + s] = v;
          S[s * NM + r] = v;
        }
      __syncwarp();
      if (live)
#pragma unroll 1
        for (int t0 = k; t0 < NT; t0 += CH * N) {
          int r[CH], c[CH];
#pragma unroll
          for (int x = 0; x < CH; ++x) tri_rs<NM>(t0 + x * N < NT ? t0 + x * N : t0, r[x], c[x]);
          DotN d;
#pragma unroll
          for (int x = 0; x < CH; ++x)
            d.c[x] = m == 0 ? (r[x] == c[x] ? diffd : dd{0.f, 0.f}) : M[r[x] * NM + c[x]];
          dotn<false>(
            d, [&](int x) { return S + r[x] * NM; }, 1, [&](int x) { return S + c[x] * NM; }, 1, NM);
#pragma unroll
          for (int x = 0; x < CH; ++x)
            if (t0 + x * N < NT) {
              M[r[x] * NM + c[x]] = d.c[x];
              M[c[x] * NM + r[x]] = d.c[x];
            }
        }
      __syncwarp();
    }
    // FP32 Jacobi on the leading part (the scratch now holds Mf, Vf)
    if (!warm) {
      if (live)
        for (int t = k; t < NP * NP; t += N) {
          const int r = t / NP, s = t - r * NP;
          Mf[r * LD + s] = (r < NM && s < NM) ? M[r * NM + s].hi : (r == s ? 1.f : 0.f);
          Vf[r * LD + s] = (r == s) ? 1.f : 0.f;
        }
      __syncwarp();
    } else {
      // warm start: the point's eigenvectors W of the previous evaluation
      // (vcache) start the rotations (Vf = W) on Mf = W^T M W, which is nearly
      // diagonal when the state moved little, so the sweeps stop early; the
      // refinement below makes tau independent of the start up to rounding
      float* Tf = Vf + NP * LD;   // [NM][NM]
      const float* wc = vcache + gq * NN;
      if (live)
        for (int t = k; t < NP * NP; t += N) {
          const int r = t / NP, s = t - r * NP;
          Vf[r * LD + s] = (r < NM && s < NM) ? wc[r * NM + s] : (r == s ? 1.f : 0.f);
        }
      __syncwarp();
      if (live)
        for (int t = k; t < NN; t += N) {
          const int r = t / NM, s = t - r * NM;
          float acc = 0.f;
          for (int j = 0; j < NM; ++j) acc = fmaf(M[r * NM + j].hi, Vf[j * LD + s], acc);
          Tf[t] = acc;
        }
      __syncwarp();
      if (live) {
        for (int t = k; t < NT; t += N) {
          int r, s;
          tri_rs<NM>(t, r, s);
          float acc = 0.f;
          for (int j = 0; j < NM; ++j) acc = fmaf(Vf[j * LD + r], Tf[j * NM + s], acc);
          Mf[r * LD + s] = acc;
          Mf[s * LD + r] = acc;
        }
        for (int t = k; t < 2 * NP - 1; t += N) {   // the padding row and column
          const int r = t < NP ? NM : t - NP, s = t < NP ? t : NM;
          Mf[r * LD + s] = (r == s) ? 1.f : 0.f;
          Mf[s * LD + r] = (r == s) ? 1.f : 0.f;
        }
      }
      __syncwarp();
    }
    const bool conv32 = jacobi_group<float, N>(Mf, Vf, k, g, lane, live, red, 12, 1e-12f);
    if (live && k == 0 && !conv32) atomicAdd(n_unconverged, 1u);
    if (live)
      for (int t = k; t < NN; t += N) V[t] = dd_make(Vf[(t / NM) * LD + t % NM]);
    __syncwarp();
    // two Newton-Schulz steps: H = 1.5 I - 0.5 V^T V, V <- V H
    dd* H = S;
    dd* T = S + NN;
#pragma unroll 1
    for (int it = 0; it < 2; ++it) {
      if (live)
#pragma unroll 1
        for (int t0 = k; t0 < NT; t0 += CH * N) {
          int r[CH], c[CH];
#pragma unroll
          for (int x = 0; x < CH; ++x) tri_rs<NM>(t0 + x * N < NT ? t0 + x * N : t0, r[x], c[x]);
          DotN d;
        dot_zero(d);
          if (it == 0)
            dotn<true>(
            d, [&](int x) { return V + r[x]; }, NM, [&](int x) { return V + c[x]; }, NM, NM);
          else
            dotn<false>(
            d, [&](int x) { return V + r[x]; }, NM, [&](int x) { return V + c[x]; }, NM, NM);
#pragma unroll
          for (int x = 0; x < CH; ++x)
            if (t0 + x * N < NT) {
              dd h = dd_scale(dd_neg(d.c[x]), 0.5f);
              if (r[x] == c[x]) h = dd_add_f(h, 1.5f);
              H[r[x] * NM + c[x]] = h;
              H[c[x] * NM + r[x]] = h;
            }
        }
      __syncwarp();
      if (live)
#pragma unroll 1
        for (int t0 = k; t0 < NN; t0 += CH * N) {
          int r[CH], c[CH];
#pragma unroll
          for (int x = 0; x < CH; ++x) {
            const int t = t0 + x * N < NN ? t0 + x * N : t0;
            r[x] = t / NM;
            c[x] = t - r[x] * NM;
          }
          DotN d;
        dot_zero(d);
          dotn<false>(
            d, [&](int x) { return V + r[x] * NM; }, 1, [&](int x) { return H + c[x]; }, NM, NM);
#pragma unroll
          for (int x = 0; x < CH; ++x)
            if (t0 + x * N < NN) T[t0 + x * N] = d.c[x];
        }
      __syncwarp();
      if (live)
        for (int t = k; t < NN; t += N) V[t] = T[t];
      __syncwarp();
    }
    // P = M V, B = V^T P (into M)
    dd* P = S;
    if (live)
#pragma unroll 1
      for (int t0 = k; t0 < NN; t0 += CH * N) {
        int r[CH], c[CH];
#pragma unroll
        for (int x = 0; x < CH; ++x) {
          const int t = t0 + x * N < NN ? t0 + x * N : t0;
          r[x] = t / NM;
          c[x] = t - r[x] * NM;
        }
        DotN d;
        dot_zero(d);
        dotn<false>(
            d, [&](int x) { return M + r[x] * NM; }, 1, [&](int x) { return V + c[x]; }, NM, NM);
#pragma unroll
        for (int x = 0; x < CH; ++x)
          if (t0 + x * N < NN) P[t0 + x * N] = d.c[x];
      }
    __syncwarp();
    if (live)
#pragma unroll 1
      for (int t0 = k; t0 < NT; t0 += CH * N) {
        int r[CH], c[CH];
#pragma unroll
        for (int x = 0; x < CH; ++x) tri_rs<NM>(t0 + x * N < NT ? t0 + x * N : t0, r[x], c[x]);
        DotN d;
        dot_zero(d);
        dotn<false>(
            d, [&](int x) { return V + r[x]; }, NM, [&](int x) { return P + c[x]; }, NM, NM);
#pragma unroll
        for (int x = 0; x < CH; ++x)
          if (t0 + x * N < NT) {
            M[r[x] * NM + c[x]] = d.c[x];
            M[c[x] * NM + r[x]] = d.c[x];
          }
      }
    __syncwarp();
    // eigenpairs for the derivative of tau (exact tangent), when asked: the
    // refined vectors and diag(B) with the point's scale undone
    if (live && vcache)
      for (int t = k; t < NN; t += N) vcache[gq * NN + t] = V[t].hi;
    if (live && eig_out) {
      float* eo = eig_out + gq * Dims<N>::EIG;
      const float back = (float)(1.0 / (unscale * unscale));
      for (int t = k; t < NN; t += N) eo[t] = V[t].hi;
      for (int j = k; j < NM; j += N) eo[NN + j] = M[j * NM + j].hi * back;
    }
    // s_i = sqrt(b_ii), 1/s_i (double-float), and FP32 copies for the small terms
    dd* sq = w;
    dd* isq = w + NM;
    float* sf = reinterpret_cast<float*>(w + 2 * NM);
    float* s2f = sf + NM;
    if (live)
      for (int i = k; i < NM; i += N) {
        const dd b = M[i * NM + i];
        const dd si = dd_sqrt(b);
        sq[i] = si;
        isq[i] = dd_rcp(si);
        sf[i] = si.hi;
        s2f[i] = b.hi;
      }
    __syncwarp();
    // X_ik = E_ik / (s_i s_k (s_i + s_k)) in FP32 (first order in E)
    float* X = reinterpret_cast<float*>(S);
    dd* Z = S + NN;
    dd* Q = S;   // over X, which only the Z phase reads
    if (live)
      for (int t = k; t < NN; t += N) {
        const int r = t / NM, s = t - r * NM;
        const float sr = sf[r], ss = sf[s];
        X[t] = (r == s) ? 0.f : M[r * NM + s].hi / (sr * ss * (sr + ss));
      }
    __syncwarp();
    // Z = diag(1/s) - X + sum_j X_rj X_js (s_j + s_j^2 / (s_r + s_s))
    if (live)
      for (int t = k; t < NN; t += N) {
        const int r = t / NM, s = t - r * NM;
        const float inv_rs = 1.f / (sf[r] + sf[s]);
        float acc = 0.f;
        for (int j = 0; j < NM; ++j) acc += X[r * NM + j] * X[j * NM + s] * (sf[j] + s2f[j] * inv_rs);
        const dd z0 = (r == s) ? isq[r] : dd{0.f, 0.f};
        Z[t] = dd_add_f(z0, acc - X[t]);
      }
    __syncwarp();
    // Q = Z V^T, tau = V Q (upper triangle), undo the scale
    if (live)
#pragma unroll 1
      for (int t0 = k; t0 < NN; t0 += CH * N) {
        int r[CH], c[CH];
#pragma unroll
        for (int x = 0; x < CH; ++x) {
          const int t = t0 + x * N < NN ? t0 + x * N : t0;
          r[x] = t / NM;
          c[x] = t - r[x] * NM;
        }
        DotN d;
        dot_zero(d);
        dotn<false>(
            d, [&](int x) { return Z + r[x] * NM; }, 1, [&](int x) { return V + c[x] * NM; }, 1, NM);
#pragma unroll
        for (int x = 0; x < CH; ++x)
          if (t0 + x * N < NN) Q[t0 + x * N] = d.c[x];
      }
    __syncwarp();
    if (live) {
      double* out = tau_out + gq * Dims<N>::NT_PAD;
#pragma unroll 1
      for (int t0 = k; t0 < NT; t0 += CH * N) {
        int r[CH], c[CH];
#pragma unroll
        for (int x = 0; x < CH; ++x) tri_rs<NM>(t0 + x * N < NT ? t0 + x * N : t0, r[x], c[x]);
        DotN d;
        dot_zero(d);
        dotn<false>(
            d, [&](int x) { return V + r[x] * NM; }, 1, [&](int x) { return Q + c[x]; }, NM, NM);
#pragma unroll
        for (int x = 0; x < CH; ++x)
          if (t0 + x * N < NT) out[t0 + x * N] = dd_to_double(d.c[x]) * unscale;
      }
      if (k == 0)
        for (int t = Dims<N>::NT; t < Dims<N>::NT_PAD; ++t) out[t] = 0.0;
    }
    __syncwarp();
  }
}

template <int N>
int launch_tau_dd(const int4* tets, const double* geo, const double* y, int64_t n_elem,
                  double* tau_out, double nu, double C_I, unsigned* n_unconverged,
                  cudaStream_t st, float* eig_out, float* vcache, int warm) {
  using L = DDLayout<N>;
  // warps per block (1..4) that keep the most warps resident per SM: the
  // shared footprint is the limit (228 KB per SM, 1 KB of it reserved per block)
  int warps = 1, best = 0;
  for (int wb = 1; wb <= 4; ++wb) {
    const size_t per_block = (size_t)wb * L::WARP * sizeof(dd);
    if (per_block > 227 * 1024) break;
    const int resident = wb * (int)((228 * 1024) / (per_block + 1024));
    if (resident > best) {
      best = resident;
      warps = wb;
    }
  }
  const size_t smem = (size_t)warps * L::WARP * sizeof(dd);
  if (smem > 227 * 1024) return -6;
  cudaFuncSetAttribute(tau_dd_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int64_t n_qp = n_elem * 4;
  const int64_t groups = (n_qp + L::GPW - 1) / L::GPW;
  int64_t blocks = (groups + warps - 1) / warps;
  if (blocks > 152 * 128) blocks = 152 * 128;
  if (blocks < 1) blocks = 1;
  count_launches(1);
  tau_dd_kernel<N><<<(int)blocks, warps * 32, smem, st>>>(tets, geo, y, n_qp, tau_out, nu, C_I,
                                                          n_unconverged, eig_out, vcache,
                                                          vcache != nullptr && warm);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

#define TS_INST_TAU_DD(T, N)                                                              \
  template int launch_tau_dd<N>(const int4*, const double*, const double*, int64_t, double*, \
                                double, double, unsigned*, cudaStream_t, float*, float*, int);
TS_FOR_EACH_N(TS_INST_TAU_DD, double)

}  // namespace ts
