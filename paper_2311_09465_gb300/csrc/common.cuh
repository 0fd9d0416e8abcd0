// Shared definitions of the GB300 time-spectral GLS kernels.
//
// Representation on the device (see include/tsgls.h): a modal field is
// [V][4][C] with C = 2N storage coordinates per field (re, im of modes
// 0..N-1; slot 1 = Im(mode 0) is always zero).  Inside the kernels the
// convective products are formed on K = 3N-2 time samples: the product of
// two trigonometric polynomials of degree N-1 has degree 2N-2, and K > 3N-3
// samples recover its modes |m| < N without aliasing, i.e. exactly the
// truncated convolution A_{mn} = u_{m-n}, |m-n| < N of eq. (phi-def).
//
// tau (eq. 3D-tau) is stored per quadrature point as the packed upper
// triangle of the real symmetric (2N-1)x(2N-1) matrix it becomes in the
// orthonormal real basis xi = (x_0, sqrt2 Re x_n, sqrt2 Im x_n): a Hermitian
// matrix that maps conjugate-symmetric mode vectors to conjugate-symmetric
// ones is real symmetric there, with the same eigenvalues.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ts {

// element geometry record: dN_a/dx_j at [a*3+j] (0..11), volume at 12,
// metric G (xx,xy,xz,yy,yz,zz) at 13..18, pad to 20
constexpr int GEO_STRIDE = 20;
constexpr int GEO_VOL = 12;
constexpr int GEO_G = 13;

template <int N>
struct Dims {
  static constexpr int C = 2 * N;               // storage coordinates per field
  static constexpr int NM = 2 * N - 1;          // real dimension of a mode vector
  static constexpr int K = 3 * N - 2;           // time samples per product
  static constexpr int NT = NM * (NM + 1) / 2;  // packed tau entries
  static constexpr int NT_PAD = (NT + 3) & ~3;  // per quadrature point, 16-byte multiple
  static constexpr int NP = 2 * N;              // Jacobi size (NM + 1 decoupled dummy)
  // eigenpair cache per point: eigenvectors [NM][NM] (column j = vector j,
  // orthonormal basis) then eigenvalues [NM], padded to a 16-byte multiple
  static constexpr int EIG = (NM * NM + NM + 3) & ~3;
};

// barycentric coordinates of the symmetric degree-2 rule (weights V/4)
__host__ __device__ constexpr double qp_bary(int q, int a) {
  return q == a ? 0.5854101966249685 : 0.1381966011250105;
}

// storage coordinate of compact real index r (skips the Im(mode 0) slot)
__host__ __device__ constexpr int stor_of(int r) { return r == 0 ? 0 : r + 1; }

// packed upper-triangle index, r <= s, n = matrix size
__host__ __device__ constexpr int packed_index(int r, int s, int n) {
  return r * n - (r * (r - 1)) / 2 + (s - r);
}

template <typename T>
struct Real;
template <>
struct Real<float> {
  static __device__ __forceinline__ float rsqrt(float x) { return rsqrtf(x); }
  static __device__ __forceinline__ float sqrt(float x) { return sqrtf(x); }
  static constexpr float SQRT2 = 1.41421356237309505f;
  static constexpr float INV_SQRT2 = 0.70710678118654752f;
};
template <>
struct Real<double> {
  static __device__ __forceinline__ double rsqrt(double x) { return 1.0 / ::sqrt(x); }
  static __device__ __forceinline__ double sqrt(double x) { return ::sqrt(x); }
  static constexpr double SQRT2 = 1.41421356237309505;
  static constexpr double INV_SQRT2 = 0.70710678118654752;
};

struct ddv;   // double-float value type (ddfloat.cuh)

// kernel-side view of the problem constants
template <typename T>
struct Phys {
  T rho, mu, omega, nu, C_I, mass_coef;
};

enum ApplyMode { MODE_RESIDUAL = 0, MODE_JVP_PAPER = 1, MODE_JVP_FROZEN = 2, MODE_JVP_LIN_A = 3,
                 MODE_JVP_EXACT = 4 /* LIN_A + the derivative of tau, passed in as dT */ };

}  // namespace ts
