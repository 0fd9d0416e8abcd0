// Kernel launchers of the GB300 time-spectral GLS library (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

// Mode counts with compiled kernels.  Each entry instantiates the tau,
// operator and boundary kernels in FP32 and FP64.
#define TS_FOR_EACH_N(X, T) X(T, 1) X(T, 2) X(T, 3) X(T, 4) X(T, 5) X(T, 7) X(T, 10) X(T, 15)
#define TS_N_LIST 1, 2, 3, 4, 5, 7, 10, 15

namespace ts {

// process-wide count of kernel launches issued by this library
void count_launches(int n);
unsigned long long launches_total();

template <typename T, int N>
int launch_tau(const int4* tets, const T* geo, const T* y, int64_t n_elem, T* tau_out, T nu,
               T C_I, unsigned* n_unconverged, cudaStream_t st, float* eig_out = nullptr);

// load a kernel into the current device's context without launching it
// (instantiated for T = float only)
template <typename T, int N>
int preload_tau();
template <typename T, int N>
int preload_apply_residual();

// FP64 tau from FP32 Jacobi eigenvectors plus an FP64 polish (tau.cu)
template <int N>
int launch_tau_polish(const int4* tets, const double* geo, const double* y, int64_t n_elem,
                      double* tau_out, double nu, double C_I, unsigned* n_unconverged,
                      cudaStream_t st, float* eig_out = nullptr);

// the same refinement in double-float arithmetic (tau_dd.cu); with vcache
// ((2N-1)^2 floats per point) the refined eigenvectors are stored there, and
// with warm the Jacobi sweeps start from the ones stored by the last launch
template <int N>
int launch_tau_dd(const int4* tets, const double* geo, const double* y, int64_t n_elem,
                  double* tau_out, double nu, double C_I, unsigned* n_unconverged,
                  cudaStream_t st, float* eig_out = nullptr, float* vcache = nullptr, int warm = 0);

// Backflow stabilisation on one Neumann face set (tau.cu): when y_for_matrix
// is given, first |A_n|_- at the 3 points of every face into bneg; then
// out[A][i] += coef * int N_A |A_n|_- v_i over the faces (atomics).
template <typename T, int N>
int launch_backflow(const int32_t* faces, const T* normals, const T* area, int64_t n_faces,
                    const T* y_for_matrix, T* bneg, const T* v, const uint8_t* dmask, int mask_input,
                    T coef, T* out, cudaStream_t st);

// One colour range [e0, e1) of the element operator (see apply.cu).
template <typename T, int N>
int launch_apply(int mode, const int4* tets, const T* geo, const T* v, const T* u0,
                 const T* tau, T* t0cache, const uint8_t* dmask, T* out, const T* dft,
                 Phys<T> ph, int64_t e0, int64_t e1, cudaStream_t st, T* l0cache = nullptr);

// y[node][i][c] = vals[k][i][c] for the k-th listed node, velocity fields i < 3
// (the inlet Dirichlet data of the initial guess)
template <typename T>
int launch_inlet_fill(const int32_t* nodes, const double* vals, int64_t n, int C, T* y, cudaStream_t st);

// The same element operator on FP64 data with double-float arithmetic
// (FP32-pipe pairs, ~48 significant bits; see ddfloat.cuh)
template <int N>
int launch_apply_dd(int mode, const int4* tets, const double* geo, const double* v, const double* u0,
                    const double* tau, double* t0cache, const uint8_t* dmask, double* out, const double* dft,
                    Phys<double> ph, int64_t e0, int64_t e1, cudaStream_t st, double* l0cache = nullptr);

// Tracer residual of eq. (3D-weak) on one colour range [e0, e1) (apply.cu):
// phi [V][C], a4 the advecting velocity in the flow layout [V][4][C], tau the
// tracer's tau cache; out += element rows (Dirichlet rows and Im(mode 0) skipped)
template <typename T, int N>
int launch_tracer(const int4* tets, const T* geo, const T* a4, const T* phi, const T* tau,
                  const uint8_t* dmask, T* out, const T* dft, double kappa, double omega, int64_t e0,
                  int64_t e1, cudaStream_t st, int gls = 1);
template <typename T>
int launch_repack_velocity(const T* a, T* a4, int64_t V, int C, cudaStream_t st);

// Resistance outlets: out[A][i][c] += R w_Ai Q_c with Q_c = sum_B w_Bi v[B][i][c]
template <typename T>
int launch_outlet(const int32_t* nodes, const T* w, int n_nodes, T R, const T* v,
                  const uint8_t* dmask, int mask_input, T* out, int C, cudaStream_t st);

// One instance's operands of an FP32 tangent product (jvp32.cuh); also the
// per-instance entry of the batched launch.
struct J32Inst {
  const int4* tets;
  const float* geo;
  const float* v;
  const float* u0t;      // [V][K] float4: u0 velocity sampled in time (x, y, z, 0)
  float* vt;             // [V][K] float4 scratch: masked v sampled in time (node pre-pass)
  const float* tau;
  const float* t0cache;
  const uint8_t* dmask;
  float* out;
  Phys<float> ph;
  int64_t n_elem;
  int64_t n_nodes;
  int N;
  const float* dT = nullptr;   // [E][4][3][C] d tau[v] L(u0) (exact tangent only)
};

// Batched LIN_A tangent products of instances with N <= J32_MAX_N in one
// element launch after one node pre-pass (jvp32_batch.cu); every out must be
// zero on entry.  d_counts holds {n_inst, n_tiles, n_nodes} on the device,
// tile_off n_inst + 1 prefix sums of ceil(n_elem / 2), node_off n_inst + 1
// prefix sums of the node counts.  Shared memory per warp: j32_batch_warp_bytes().
int launch_jvp32_batch(const J32Inst* d_insts, const int64_t* d_tile_off, const int64_t* d_node_off,
                       const int64_t* d_counts, int warps_per_block, int blocks, cudaStream_t st);
size_t j32_batch_warp_bytes();
int j32_batch_configure();
int j32_upload_batch(const float* host_all);

// FP32 tangent product (jvp32.cuh): a node pre-pass (v sampled into I.vt,
// I.out cleared) and one element launch
// (with e_before / e_after: events recorded around the element launch)
template <int N>
int launch_jvp32(int mode, const J32Inst& I, cudaStream_t st, cudaEvent_t e_before = nullptr,
                 cudaEvent_t e_after = nullptr);
// d tau[v] L_i(u0) at every quadrature point (dtau.cu): the Frechet derivative of
// tau = M^{-1/2} (eq. 3D-tau) in the direction of v, from the cached eigenpairs
// of M (eig [E*4][EIG]) and strong residual L(u0) (l0 [E][4][3][C]);
// dT [E][4][3][C], storage coordinates
template <int N>
int launch_dtau(const int4* tets, const float* geo, const float* u0, const float* v, const uint8_t* dmask,
                const float* eig, const float* l0, float* dT, int64_t n_elem, cudaStream_t st);

// u0 velocity at the nodes as time samples [V][K] float4 (x, y, z, 0)
template <int N>
int launch_node_samples(const float* u0, float* u0t, int64_t V, cudaStream_t st);
// the table of all compiled N (forward [K][C] then inverse [C][K] each)
int dft_constant_total();
int dft_constant_offset(int N);
// each fast-path translation unit copies its slice into its constant bank
int j32_upload_n123(const float* host_all);
int j32_upload_n45(const float* host_all);
int j32_upload_n7(const float* host_all);
constexpr int J32_MAX_N = 7;   // largest N with the single-launch FP32 kernel

// Nodal diagonal blocks H_AA of the tangent (precond.cu): one 8N x 8N block per
// node from the node-to-element list (packed element * 4 + local node); with
// invert the inverse, column-major, else H_AA row-major.  Fixed unknowns
// (Im(mode 0), Dirichlet velocity) have zero rows and columns (identity when
// inverted); n_singular counts blocks that could not be inverted (stored as I).
template <typename T, int N>
int launch_block_diag(int variant_paper, int invert, const int32_t* node_off, const int32_t* node_elem,
                      const int4* tets, const T* geo, const T* u0, const T* tau, const uint8_t* dmask,
                      const float* outdiag, Phys<float> ph, float* out, int64_t n_nodes,
                      unsigned* n_singular, cudaStream_t st);
// z[A] = Binv[A] x[A] for every node (FP32 blocks, FP64 vectors)
template <int N>
int launch_block_apply(const float* binv, const double* x, double* z, int64_t n_nodes, cudaStream_t st);

// Assembled tangent of the paper's variant (assembled.cu): per node-graph
// connection a record of assembled_record_floats(N) floats (K, L, G_1..3, D_1..3)
template <typename T, int N>
int launch_assemble_paper(const int32_t* node_off, const int32_t* node_elem, const int32_t* row_off,
                          const int32_t* cols, const int4* tets, const T* geo, const T* u0, const T* tau,
                          Phys<float> ph, float* H, int64_t n_nodes, cudaStream_t st);
template <int N>
int launch_spmv_paper(const int32_t* row_off, const int32_t* cols, const float* H, const uint8_t* dmask,
                      const float* x, float* y, int64_t n_nodes, cudaStream_t st);
int assembled_record_floats(int N);
// one colour of a block Gauss-Seidel sweep: z_A = Binv_A (r_A - sum_{B != A} H_AB z_B)
template <int N>
int launch_sgs_colour(const int32_t* rows, int64_t n_rows, const int32_t* row_off, const int32_t* cols,
                      const float* H, const float* binv, const uint8_t* dmask, const float* r, float* z,
                      int diag_only, cudaStream_t st);

// FP64 Krylov helpers (krylov.cu)
// h_out[j] = basis_j . w (j < nvec), with self also h_out[nvec] = w . w;
// with *skip != 0 (device flag) every h_out is 0 and nothing is read
int krylov_dots(const double* basis, int64_t ld, int nvec, const double* w, int64_t n,
                double* partial, double* h_out, cudaStream_t st, int self = 0,
                const double* skip = nullptr);
// w -= sum_j h_j basis_j, nothing when *skip != 0
int krylov_sub(double* w, const double* basis, int64_t ld, int nvec, const double* h, int64_t n,
               cudaStream_t st, const double* skip = nullptr);
// flag = 1 when the second Gram-Schmidt pass can be skipped (see krylov.cu)
int krylov_reorth_test(const double* h, int nvec, double* flag, cudaStream_t st);
int krylov_combine(double* x, const double* basis, int64_t ld, int nvec, const double* coef,
                   int64_t n, cudaStream_t st);
int vec_scale(double* out, const double* in, double a, int64_t n, cudaStream_t st);
int vec_axpy(double* y, const double* x, double a, int64_t n, cudaStream_t st);
int vec_cast_d2f(float* out, const double* in, int64_t n, cudaStream_t st);
int vec_cast_f2d(double* out, const float* in, int64_t n, cudaStream_t st);
int krylov_partial_blocks();
int vec_mul(double* out, const double* a, const double* b, int64_t n, cudaStream_t st);
// out = in / sqrt(*n2) with the squared norm read on the device
int vec_normalise(double* out, const double* in, const double* n2, int64_t n, cudaStream_t st);
// approximate diagonal of the tangent for right preconditioning (one colour range)
int launch_diag(const int4* tets, const double* geo, const double* y, int N, Phys<double> ph,
                double* D, int64_t e0, int64_t e1, cudaStream_t st);
// D <- 1/D on free unknowns, 1 on fixed ones
int launch_diag_invert(double* D, const uint8_t* dmask, int64_t V, int C, cudaStream_t st);

}  // namespace ts
