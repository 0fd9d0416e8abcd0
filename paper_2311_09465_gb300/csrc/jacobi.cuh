// Shared by the tau kernels: the real symmetric convolution matrix entry and
// the parallel cyclic Jacobi eigensolver on a group of N lanes.
#pragma once
#include "common.cuh"

namespace ts {

// entry (r, s) of the real symmetric convolution matrix of a (storage
// coordinates a[0..C-1]) in the orthonormal basis (x0, sqrt2 Re, sqrt2 Im)
template <typename T, int N>
__device__ __forceinline__ T conv_entry(const T* a, int r, int s) {
  auto ar = [&](int k) -> T {
    int m = k < 0 ? -k : k;
    return m < N ? a[2 * m] : T(0);
  };
  auto ai = [&](int k) -> T {
    int m = k < 0 ? -k : k;
    if (m >= N || m == 0) return T(0);
    return k > 0 ? a[2 * m + 1] : -a[2 * m + 1];
  };
  if (r == 0 && s == 0) return a[0];
  const T s2 = Real<T>::SQRT2;
  if (r == 0 || s == 0) {
    int o = r == 0 ? s : r;
    int n = (o + 1) >> 1;
    return (o & 1) ? s2 * ar(n) : s2 * ai(n);
  }
  int m = (r + 1) >> 1, n = (s + 1) >> 1;
  bool rre = r & 1, sre = s & 1;
  if (rre && sre) return ar(m - n) + ar(m + n);
  if (rre && !sre) return ai(m + n) - ai(m - n);
  if (!rre && sre) return ai(m - n) + ai(m + n);
  return ar(m - n) - ar(m + n);
}


// Parallel cyclic Jacobi on the symmetric NP x NP matrix M (row stride NP+1)
// owned by a group of N lanes; rotations accumulate into V (V <- V J).
// Round-robin ordering: in each of the NP-1 rounds the N lanes rotate N
// disjoint pairs, rows first then columns.  Every lane of the warp must call
// this function (it synchronises the warp); lanes with live == false only
// take part in the synchronisation.  Returns whether this group reached
// sum_{i<j} M_ij^2 <= tol2 * sum_i M_ii^2 within max_sweeps.
template <typename T, int N>
__device__ bool jacobi_group(T* M, T* Vv, int k, int g, int lane, bool live, T* red,
                             int max_sweeps, T tol2) {
  constexpr int NP = 2 * N, NM = 2 * N - 1, LD = NP + 1, P = NP - 1;
  bool converged = false;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    for (int rr = 0; rr < P; ++rr) {
      int p, qq;
      if (k == 0) {
        p = 0;
        qq = 1 + rr % P;
      } else {
        p = 1 + (rr + k) % P;
        qq = 1 + (rr - k + P) % P;
      }
      T c = 1, s = 0;
      if (live) {
        T app = M[p * LD + p], aqq = M[qq * LD + qq], apq = M[p * LD + qq];
        if (apq != T(0)) {
          T zeta = (aqq - app) / (T(2) * apq);
          T t = T(1) / (fabs(zeta) + Real<T>::sqrt(T(1) + zeta * zeta));
          if (zeta < T(0)) t = -t;
          c = Real<T>::rsqrt(T(1) + t * t);
          s = t * c;
        }
      }
      __syncwarp();
      // each rotation reads the two rows (columns) into registers before it
      // writes any of them back: the loads of a lane are then independent and
      // in flight together (a load after a store to the same array would have
      // to wait for it)
      if (live && s != T(0)) {
        T mp[NP], mq[NP];
#pragma unroll
        for (int j = 0; j < NP; ++j) {
          mp[j] = M[p * LD + j];
          mq[j] = M[qq * LD + j];
        }
#pragma unroll
        for (int j = 0; j < NP; ++j) {
          M[p * LD + j] = c * mp[j] - s * mq[j];
          M[qq * LD + j] = s * mp[j] + c * mq[j];
        }
      }
      __syncwarp();
      if (live && s != T(0)) {
        T ap[NP], aq[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) {
          ap[i] = M[i * LD + p];
          aq[i] = M[i * LD + qq];
        }
#pragma unroll
        for (int i = 0; i < NP; ++i) {
          M[i * LD + p] = c * ap[i] - s * aq[i];
          M[i * LD + qq] = s * ap[i] + c * aq[i];
        }
#pragma unroll
        for (int i = 0; i < NP; ++i) {
          ap[i] = Vv[i * LD + p];
          aq[i] = Vv[i * LD + qq];
        }
#pragma unroll
        for (int i = 0; i < NP; ++i) {
          Vv[i * LD + p] = c * ap[i] - s * aq[i];
          Vv[i * LD + qq] = s * ap[i] + c * aq[i];
        }
        M[p * LD + qq] = T(0);
        M[qq * LD + p] = T(0);
      }
      __syncwarp();
    }
    // convergence: sum of squared off-diagonals vs squared diagonal
    T off = 0, dg = 0;
    if (live) {
      for (int r = k; r < NM; r += N) {
        dg += M[r * LD + r] * M[r * LD + r];
        for (int s = r + 1; s < NM; ++s) off += M[r * LD + s] * M[r * LD + s];
      }
    }
    red[lane] = off;
    red[32 + lane] = dg;
    __syncwarp();
    bool mine = true;
    if (live) {
      T so = 0, sd = 0;
      for (int j = 0; j < N; ++j) {
        so += red[g * N + j];
        sd += red[32 + g * N + j];
      }
      mine = so <= tol2 * sd;
    }
    __syncwarp();
    converged = mine;
    if (__all_sync(0xffffffffu, !live || mine)) break;
  }
  return converged;
}

}  // namespace ts
