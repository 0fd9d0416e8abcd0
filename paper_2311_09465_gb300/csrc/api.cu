// C ABI of the GB300 time-spectral GLS library: mesh and problem set-up,
// residual and tangent dispatch, and the pseudo-time Newton-GMRES solve
// (sections 2.4-2.5 of Esmaily & Jia, arXiv 2311.09465).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <complex>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/tsgls.h"
#include "abi_util.h"
#include "kernels.h"

using namespace ts;

namespace ts {
thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}
}  // namespace ts

namespace {

// loads the allocation-free residual's arrays and kernels on the current
// device (defined with that entry point below)
int noalloc_setup(int N);

bool n_supported(int N) {
  const int list[] = {TS_N_LIST};
  for (int n : list)
    if (n == N) return true;
  return false;
}

}  // namespace

struct ts_mesh {
  int device = 0;
  int64_t V = 0, E = 0, F = 0;
  std::vector<double> xyz;
  std::vector<int32_t> tets;          // colour-sorted, [E][4]
  std::vector<int32_t> bfaces;        // [F][3], outward
  std::vector<int32_t> btag;
  std::vector<int64_t> colour_off;    // colour c: [off[c], off[c+1])
  int4* d_tets = nullptr;
  double* d_geo64 = nullptr;
  float* d_geo32 = nullptr;
  int32_t* d_node_off = nullptr;      // [V + 1] node-to-element list offsets
  int32_t* d_node_elem = nullptr;     // [4E] element * 4 + local node (colour-sorted ids)
  int64_t nnzb = 0;                   // node-graph connections (A itself included)
  int32_t* d_row_off = nullptr;       // [V + 1] node graph in CSR
  int32_t* d_cols = nullptr;          // [nnzb] sorted neighbour ids per row
  std::vector<int32_t> node_colour;   // colour of each node (host)
  std::vector<int64_t> ncolour_off;   // node colouring of the node graph: colour c holds
  int32_t* d_node_perm = nullptr;     // d_node_perm[ncolour_off[c] .. ncolour_off[c+1])
};

template <typename T>
struct LinState {
  T* u0 = nullptr;      // [V][4][C] linearisation state
  T* tau = nullptr;     // [E][4][NT_PAD]
  T* t0 = nullptr;      // [E][4][3][C] tau L at the state
  T* dft = nullptr;     // forward [K][C] then inverse [C][K]
  T* u0t = nullptr;     // [V][K][4] u0 velocity sampled in time (FP32 fast path)
  T* vt = nullptr;      // [V][K][4] scratch of the FP32 fast path: the product's input sampled
  T* bneg = nullptr;    // [backflow points][NT_PAD] |A_n|_- (section 2.6)
  T* l0 = nullptr;      // [E][4][3][C] strong residual L(u0) (exact tangent)
  bool exact_valid = false;   // l0 and the eigenpair cache belong to this state
  int64_t bneg_points = 0;
  bool valid = false;
};

struct Outlet {
  int tag;
  double R;
  std::vector<int32_t> nodes;
  std::vector<double> w;        // [n][3] int N_A n_i over the outlet
  int32_t* d_nodes = nullptr;
  double* d_w64 = nullptr;
  float* d_w32 = nullptr;
};

// inflow boundary data of one inlet tag (section 2.4, eq. upgh_def)
struct Inlet {
  int tag = 0;
  int profile = 0;
  double centre[3] = {0, 0, 0}, dir[3] = {0, 0, 0}, R = 0;   // dir: unit inflow direction
  std::vector<int32_t> nodes;   // every node of the tag (rim nodes get zero velocity)
  std::vector<double> vals;     // [n][3][C] Dirichlet velocity modes
  int32_t* d_nodes = nullptr;
  double* d_vals = nullptr;
};

struct BackflowSet {
  int tag;
  double beta;
  int64_t n = 0;                 // faces
  int64_t offset = 0;            // first point in the |A_n|_- cache
  int32_t* d_faces = nullptr;    // [n][3] outward
  double *d_n64 = nullptr, *d_a64 = nullptr;
  float *d_n32 = nullptr, *d_a32 = nullptr;
};

struct ts_problem {
  const ts_mesh* mesh = nullptr;
  ts_params p{};
  int C = 0, K = 0, NTP = 0;
  std::vector<uint8_t> dmask;
  uint8_t* d_dmask = nullptr;
  bool dmask_dirty = true;
  std::vector<Outlet> outlets;
  std::vector<BackflowSet> backflow;
  std::vector<Inlet> inlets;
  int64_t bf_points = 0;         // 3 per backflow face
  LinState<float> l32;
  LinState<double> l64;
  unsigned* d_counter = nullptr;
  // solver workspace (FP64)
  double* d_basis = nullptr;
  int basis_m = 0;
  double *d_w = nullptr, *d_r = nullptr, *d_dy = nullptr, *d_partial = nullptr, *d_h = nullptr;
  float *d_v32 = nullptr, *d_w32 = nullptr;
  double *d_D = nullptr, *d_t = nullptr;      // preconditioner diagonal (inverted), temp
  float* d_binv = nullptr;                    // inverted nodal blocks [V][8N][8N] (block Jacobi)
  int tau_warm = 0;                           // TS_OPT_TAU_WARM
  float* d_vcache = nullptr;                  // eigenvectors of M per point [E*4][(2N-1)^2] (warm start)
  bool vcache_valid = false;
  bool binv_valid = false;                    // d_binv built at the current linearisation state
  float* d_eig = nullptr;                     // eigenpairs of M per point [E*4][EIG] (exact tangent)
  float* d_dT = nullptr;                      // d tau[v] L(u0) per point [E][4][3][C] (exact tangent)
  float* d_hasm = nullptr;                    // assembled PAPER tangent records [nnzb][2C^2 + 8]
  float *d_r32 = nullptr, *d_z32 = nullptr;   // block Gauss-Seidel work vectors
  bool hasm_valid = false;
  float* d_outdiag = nullptr;                 // [V][6] outlet R w_i w_j per node
  bool outdiag_dirty = true;
  cudaEvent_t ev_a = nullptr, ev_b = nullptr; // time of the tangent products in a solve
  // stage times (ts_stage_times): tau start/end and element pass end of the
  // last residual; element kernel start/end of the last FP32 tangent product
  cudaEvent_t sev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  bool sev_res = false, sev_jvp = false;
  bool fast32 = true;    // FP32 products with the single-launch kernel (jvp32.cu)
  int tau64 = TS_TAU64_DOUBLEFLOAT;  // how the FP64 residual computes tau
  int elem64 = TS_ELEMENT64_DOUBLEFLOAT;  // arithmetic of the FP64 element operator
};

// ------------------------------------------------------------------ helpers

static int64_t field_len(const ts_problem* pr) { return pr->mesh->V * 4 * (int64_t)pr->C; }

namespace ts {
int dft_constant_total() {
  const int list[] = {TS_N_LIST};
  int off = 0;
  for (int n : list) off += 2 * (3 * n - 2) * (2 * n);
  return off;
}
int dft_constant_offset(int N) {
  const int list[] = {TS_N_LIST};
  int off = 0;
  for (int n : list) {
    if (n == N) return off;
    off += 2 * (3 * n - 2) * (2 * n);
  }
  return -1;
}
}  // namespace ts

static void dft_tables(int N, std::vector<double>& out) {
  const int C = 2 * N, K = 3 * N - 2;
  out.assign((size_t)2 * K * C, 0.0);
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < K; ++k) {
    out[k * C + 0] = 1.0;
    for (int n = 1; n < N; ++n) {
      double th = 2.0 * pi * n * k / K;
      out[k * C + 2 * n] = 2.0 * std::cos(th);
      out[k * C + 2 * n + 1] = -2.0 * std::sin(th);
    }
  }
  double* inv = out.data() + K * C;
  for (int k = 0; k < K; ++k) {
    inv[0 * K + k] = 1.0 / K;
    for (int n = 1; n < N; ++n) {
      double th = 2.0 * pi * n * k / K;
      inv[(2 * n) * K + k] = std::cos(th) / K;
      inv[(2 * n + 1) * K + k] = -std::sin(th) / K;
    }
  }
}

template <typename T>
static int lin_alloc(ts_problem* pr, LinState<T>& l) {
  if (l.u0) return 0;
  const ts_mesh* m = pr->mesh;
  TS_TRY(dalloc(&l.u0, (size_t)field_len(pr)));
  TS_TRY(dalloc(&l.tau, (size_t)m->E * 4 * pr->NTP));
  TS_TRY(dalloc(&l.t0, (size_t)m->E * 12 * pr->C));
  std::vector<double> tab;
  dft_tables(pr->p.N, tab);
  std::vector<T> tt(tab.begin(), tab.end());
  TS_TRY(dalloc(&l.dft, tt.size()));
  TS_CUDA(cudaMemcpy(l.dft, tt.data(), tt.size() * sizeof(T), cudaMemcpyHostToDevice));
  if (sizeof(T) == 4) {
    TS_TRY(dalloc(&l.u0t, (size_t)m->V * 4 * pr->K));
    TS_TRY(dalloc(&l.vt, (size_t)m->V * 4 * pr->K));
  }
  // constant-memory DFT tables of every compiled N (used by the FP32 fast path)
  std::vector<float> all(dft_constant_total());
  const int list[] = {TS_N_LIST};
  for (int n : list) {
    std::vector<double> tn;
    dft_tables(n, tn);
    std::copy(tn.begin(), tn.end(), all.begin() + dft_constant_offset(n));
  }
  if (j32_upload_n123(all.data()) || j32_upload_n45(all.data()) || j32_upload_n7(all.data()) ||
      j32_upload_batch(all.data()))
    return fail(TS_ERR_CUDA, "DFT constant upload failed");
  return 0;
}

template <typename T>
static void lin_free(LinState<T>& l) {
  dfree(l.u0);
  dfree(l.tau);
  dfree(l.t0);
  dfree(l.dft);
  dfree(l.u0t);
  dfree(l.vt);
  dfree(l.bneg);
  dfree(l.l0);
  l.bneg_points = 0;
  l.valid = false;
}

static int sync_dmask(ts_problem* pr) {
  if (!pr->dmask_dirty) return 0;
  TS_CUDA(cudaMemcpy(pr->d_dmask, pr->dmask.data(), pr->dmask.size(), cudaMemcpyHostToDevice));
  pr->dmask_dirty = false;
  return 0;
}

template <typename T>
static const T* geo_of(const ts_mesh* m);
template <>
const float* geo_of<float>(const ts_mesh* m) { return m->d_geo32; }
template <>
const double* geo_of<double>(const ts_mesh* m) { return m->d_geo64; }

template <typename T>
static LinState<T>& lin_of(ts_problem* pr);
template <>
LinState<float>& lin_of<float>(ts_problem* pr) { return pr->l32; }
template <>
LinState<double>& lin_of<double>(ts_problem* pr) { return pr->l64; }

template <typename T>
static const T* outlet_w(const Outlet& o);
template <>
const float* outlet_w<float>(const Outlet& o) { return o.d_w32; }
template <>
const double* outlet_w<double>(const Outlet& o) { return o.d_w64; }

template <typename T>
static Phys<T> phys_of(const ts_problem* pr, bool with_mass) {
  Phys<T> ph;
  ph.rho = (T)pr->p.rho;
  ph.mu = (T)pr->p.mu;
  ph.omega = (T)pr->p.omega;
  ph.nu = (T)(pr->p.mu / pr->p.rho);
  ph.C_I = (T)pr->p.C_I;
  double dt = pr->p.dt_pseudo;
  ph.mass_coef = (with_mass && dt > 0 && std::isfinite(dt)) ? (T)(pr->p.c1 * pr->p.rho / dt) : T(0);
  return ph;
}

// dispatch on the compiled mode counts
template <typename T, int N>
static int apply_colours(ts_problem* pr, int mode, const T* v, const T* u0, LinState<T>& l,
                         T* out, bool with_mass, cudaStream_t st, T* l0 = nullptr) {
  const ts_mesh* m = pr->mesh;
  Phys<T> ph = phys_of<T>(pr, with_mass);
  for (size_t c = 0; c + 1 < m->colour_off.size(); ++c) {
    int rc;
    if constexpr (sizeof(T) == 8) {
      if (pr->elem64 == TS_ELEMENT64_DOUBLEFLOAT)
        rc = launch_apply_dd<N>(mode, m->d_tets, m->d_geo64, (const double*)v, (const double*)u0,
                                (const double*)l.tau, (double*)l.t0, pr->d_dmask, (double*)out,
                                (const double*)l.dft, phys_of<double>(pr, with_mass), m->colour_off[c],
                                m->colour_off[c + 1], st, (double*)l0);
      else
        rc = launch_apply<T, N>(mode, m->d_tets, geo_of<T>(m), v, u0, l.tau, l.t0, pr->d_dmask,
                                out, l.dft, ph, m->colour_off[c], m->colour_off[c + 1], st, l0);
    } else {
      rc = launch_apply<T, N>(mode, m->d_tets, geo_of<T>(m), v, u0, l.tau, l.t0, pr->d_dmask,
                              out, l.dft, ph, m->colour_off[c], m->colour_off[c + 1], st, l0);
    }
    if (rc) return fail(rc == -6 ? TS_ERR_UNSUPPORTED : TS_ERR_CUDA, "element kernel launch failed");
  }
  const bool mask_input = mode != MODE_RESIDUAL;
  for (auto& o : pr->outlets) {
    int rc = launch_outlet<T>(o.d_nodes, outlet_w<T>(o), (int)o.nodes.size(), (T)o.R, v,
                              pr->d_dmask, mask_input ? 1 : 0, out, pr->C, st);
    if (rc) return fail(TS_ERR_CUDA, "outlet kernel launch failed");
  }
  return 0;
}

template <typename T>
static const T* bf_normals(const BackflowSet& b);
template <>
const float* bf_normals<float>(const BackflowSet& b) { return b.d_n32; }
template <>
const double* bf_normals<double>(const BackflowSet& b) { return b.d_n64; }
template <typename T>
static const T* bf_area(const BackflowSet& b);
template <>
const float* bf_area<float>(const BackflowSet& b) { return b.d_a32; }
template <>
const double* bf_area<double>(const BackflowSet& b) { return b.d_a64; }

template <typename T>
static int bneg_alloc(ts_problem* pr, LinState<T>& l) {
  if (l.bneg_points == pr->bf_points) return 0;
  dfree(l.bneg);
  l.bneg_points = 0;
  if (pr->bf_points == 0) return 0;
  TS_TRY(dalloc(&l.bneg, (size_t)pr->bf_points * pr->NTP));
  l.bneg_points = pr->bf_points;
  return 0;
}

// backflow stabilisation: -int N_A (rho/2) beta |A_n|_- v_i; with_matrix
// refreshes |A_n|_- from v (the residual), otherwise the cached one is used
template <typename T, int N>
static int backflow_terms(ts_problem* pr, LinState<T>& l, const T* v, bool with_matrix,
                          int mask_input, T* out, cudaStream_t st) {
  for (auto& b : pr->backflow) {
    const T coef = (T)(-0.5 * pr->p.rho * b.beta);
    int rc = launch_backflow<T, N>(b.d_faces, bf_normals<T>(b), bf_area<T>(b), b.n,
                                   with_matrix ? v : nullptr, l.bneg + b.offset * pr->NTP, v,
                                   pr->d_dmask, mask_input, coef, out, st);
    if (rc) return fail(TS_ERR_CUDA, "backflow kernel launch failed");
  }
  return 0;
}

template <typename T, int N>
static int residual_impl(ts_problem* pr, const T* y, T* r, cudaStream_t st) {
  const ts_mesh* m = pr->mesh;
  LinState<T>& l = lin_of<T>(pr);
  TS_TRY(lin_alloc(pr, l));
  const int64_t n = field_len(pr);
  TS_CUDA(cudaMemcpyAsync(l.u0, y, n * sizeof(T), cudaMemcpyDeviceToDevice, st));
  // the exact tangent also needs the eigenpairs of M and the strong residual
  const bool exact = pr->p.jvp_variant == TS_JVP_EXACT;
  float* eig = nullptr;
  if (exact) {
    if (!pr->d_eig) TS_TRY(dalloc(&pr->d_eig, (size_t)m->E * 4 * Dims<N>::EIG));
    if (!l.l0) TS_TRY(dalloc(&l.l0, (size_t)m->E * 12 * pr->C));
    eig = pr->d_eig;
  }
  TS_CUDA(cudaEventRecord(pr->sev[0], st));
  int rc;
  if constexpr (sizeof(T) == 8) {
    if (pr->tau64 == TS_TAU64_JACOBI)
      rc = launch_tau<T, N>(m->d_tets, geo_of<T>(m), y, m->E, l.tau, (T)(pr->p.mu / pr->p.rho),
                            (T)pr->p.C_I, pr->d_counter, st, eig);
    else if (pr->tau64 == TS_TAU64_DOUBLEFLOAT) {
      float* vc = nullptr;
      if (pr->tau_warm) {
        constexpr int64_t NMN = (2 * N - 1) * (2 * N - 1);
        if (!pr->d_vcache) TS_TRY(dalloc(&pr->d_vcache, (size_t)(m->E * 4 * NMN)));
        vc = pr->d_vcache;
      }
      rc = launch_tau_dd<N>(m->d_tets, m->d_geo64, (const double*)y, m->E, (double*)l.tau,
                            pr->p.mu / pr->p.rho, pr->p.C_I, pr->d_counter, st, eig, vc,
                            pr->vcache_valid ? 1 : 0);
      if (vc && rc == 0) pr->vcache_valid = true;
    }
    else
      rc = launch_tau_polish<N>(m->d_tets, m->d_geo64, (const double*)y, m->E, (double*)l.tau,
                                pr->p.mu / pr->p.rho, pr->p.C_I, pr->d_counter, st, eig);
  } else {
    rc = launch_tau<T, N>(m->d_tets, geo_of<T>(m), y, m->E, l.tau, (T)(pr->p.mu / pr->p.rho),
                          (T)pr->p.C_I, pr->d_counter, st, eig);
  }
  if (rc) return fail(TS_ERR_CUDA, "tau kernel launch failed");
  TS_CUDA(cudaEventRecord(pr->sev[1], st));
  TS_CUDA(cudaMemsetAsync(r, 0, n * sizeof(T), st));
  TS_TRY(apply_colours<T, N>(pr, MODE_RESIDUAL, y, y, l, r, false, st, exact ? l.l0 : nullptr));
  TS_CUDA(cudaEventRecord(pr->sev[2], st));
  pr->sev_res = true;
  TS_TRY(bneg_alloc(pr, l));
  TS_TRY(backflow_terms<T, N>(pr, l, y, true, 0, r, st));
  if constexpr (sizeof(T) == 4 && N <= J32_MAX_N) {
    if (launch_node_samples<N>((const float*)l.u0, (float*)l.u0t, m->V, st))
      return fail(TS_ERR_CUDA, "node sample kernel failed");
  }
  l.valid = true;
  l.exact_valid = exact;
  pr->hasm_valid = false;
  pr->binv_valid = false;
  // the other precision's state is now stale
  if (sizeof(T) == 4) pr->l64.valid = false; else pr->l32.valid = false;
  return 0;
}

template <typename D, typename S, int N>
static int convert_lin(ts_problem* pr, LinState<D>& dst, LinState<S>& src, cudaStream_t st) {
  TS_TRY(lin_alloc(pr, dst));
  const ts_mesh* m = pr->mesh;
  const int64_t n_u = field_len(pr), n_tau = m->E * 4 * pr->NTP, n_t0 = m->E * 12 * pr->C;
  int rc = 0;
  dst.exact_valid = src.exact_valid && src.l0;
  if (src.l0) {
    if (!dst.l0) TS_TRY(dalloc(&dst.l0, (size_t)n_t0));
    if (sizeof(D) == 4) rc |= vec_cast_d2f((float*)dst.l0, (const double*)src.l0, n_t0, st);
    else rc |= vec_cast_f2d((double*)dst.l0, (const float*)src.l0, n_t0, st);
  }
  if (sizeof(D) == 4) {
    rc |= vec_cast_d2f((float*)dst.u0, (const double*)src.u0, n_u, st);
    rc |= vec_cast_d2f((float*)dst.tau, (const double*)src.tau, n_tau, st);
    rc |= vec_cast_d2f((float*)dst.t0, (const double*)src.t0, n_t0, st);
    if constexpr (N <= J32_MAX_N)
      rc |= launch_node_samples<N>((const float*)dst.u0, (float*)dst.u0t, m->V, st);
  } else {
    rc |= vec_cast_f2d((double*)dst.u0, (const float*)src.u0, n_u, st);
    rc |= vec_cast_f2d((double*)dst.tau, (const float*)src.tau, n_tau, st);
    rc |= vec_cast_f2d((double*)dst.t0, (const float*)src.t0, n_t0, st);
  }
  TS_TRY(bneg_alloc(pr, dst));
  if (pr->bf_points > 0) {
    const int64_t nb = pr->bf_points * pr->NTP;
    if (sizeof(D) == 4) rc |= vec_cast_d2f((float*)dst.bneg, (const double*)src.bneg, nb, st);
    else rc |= vec_cast_f2d((double*)dst.bneg, (const float*)src.bneg, nb, st);
  }
  if (rc) return fail(TS_ERR_CUDA, "state conversion failed");
  dst.valid = true;
  return 0;
}

static int mode_of_variant(int v) {
  switch (v) {
    case TS_JVP_PAPER: return MODE_JVP_PAPER;
    case TS_JVP_FROZEN: return MODE_JVP_FROZEN;
    case TS_JVP_LIN_A: return MODE_JVP_LIN_A;
    case TS_JVP_EXACT: return MODE_JVP_EXACT;
  }
  return -1;
}

template <typename T, int N>
static int jvp_impl(ts_problem* pr, const T* v, T* hv, cudaStream_t st) {
  LinState<T>& l = lin_of<T>(pr);
  if (!l.valid) {
    if (sizeof(T) == 4 && pr->l64.valid)
      TS_TRY(convert_lin<float, double, N>(pr, pr->l32, pr->l64, st));
    else if (sizeof(T) == 8 && pr->l32.valid)
      TS_TRY(convert_lin<double, float, N>(pr, pr->l64, pr->l32, st));
    else
      return fail(TS_ERR_ARG, "ts_jvp: no linearisation state (call ts_residual first)");
  }
  const int mode = mode_of_variant(pr->p.jvp_variant);
  if (mode < 0) return fail(TS_ERR_ARG, "unknown jvp variant");
  if (mode == MODE_JVP_EXACT) {
    if (sizeof(T) != 4 || N > J32_MAX_N || !pr->fast32)
      return fail(TS_ERR_UNSUPPORTED, "ts_jvp: the exact tangent runs in FP32 with N <= 7 (single launch)");
    if (!pr->d_eig || !l.l0 || !l.exact_valid)
      return fail(TS_ERR_ARG, "ts_jvp: the exact tangent needs a residual computed with TS_JVP_EXACT set");
  }
  if constexpr (sizeof(T) == 4 && N <= J32_MAX_N) if (pr->fast32) {
    // the node pre-pass of the product clears hv
    const ts_mesh* m = pr->mesh;
    J32Inst I{m->d_tets, m->d_geo32, (const float*)v, (const float*)l.u0t, (float*)l.vt,
              (const float*)l.tau, (const float*)l.t0, pr->d_dmask, (float*)hv,
              phys_of<float>(pr, true), m->E, m->V, N};
    if (mode == MODE_JVP_EXACT) {
      if (!pr->d_dT) TS_TRY(dalloc(&pr->d_dT, (size_t)m->E * 12 * pr->C));
      if (launch_dtau<N>(m->d_tets, m->d_geo32, (const float*)l.u0, (const float*)v, pr->d_dmask, pr->d_eig,
                         (const float*)l.l0, pr->d_dT, m->E, st))
        return fail(TS_ERR_CUDA, "tau derivative kernel launch failed");
      I.dT = pr->d_dT;
    }
    int rc = launch_jvp32<N>(mode, I, st, pr->sev[3], pr->sev[4]);
    if (rc) return fail(TS_ERR_CUDA, "FP32 tangent kernel launch failed");
    pr->sev_jvp = true;
    for (auto& o : pr->outlets)
      if (launch_outlet<T>(o.d_nodes, outlet_w<T>(o), (int)o.nodes.size(), (T)o.R, v, pr->d_dmask, 1,
                           hv, pr->C, st))
        return fail(TS_ERR_CUDA, "outlet kernel launch failed");
    return backflow_terms<T, N>(pr, l, v, false, 1, hv, st);
  }
  TS_CUDA(cudaMemsetAsync(hv, 0, field_len(pr) * sizeof(T), st));
  TS_TRY(apply_colours<T, N>(pr, mode, v, l.u0, l, hv, true, st));
  return backflow_terms<T, N>(pr, l, v, false, 1, hv, st);
}

#define TS_DISPATCH(N_, CALL)                                                   \
  switch (N_) {                                                                 \
    case 1: { constexpr int NN = 1; return CALL; }                              \
    case 2: { constexpr int NN = 2; return CALL; }                              \
    case 3: { constexpr int NN = 3; return CALL; }                              \
    case 4: { constexpr int NN = 4; return CALL; }                              \
    case 5: { constexpr int NN = 5; return CALL; }                              \
    case 7: { constexpr int NN = 7; return CALL; }                              \
    case 10: { constexpr int NN = 10; return CALL; }                            \
    case 15: { constexpr int NN = 15; return CALL; }                            \
    default: return fail(TS_ERR_UNSUPPORTED, "no kernel compiled for this N");  \
  }

static int residual_any(ts_problem* pr, const void* y, void* r, int precision, cudaStream_t st) {
  if (precision == 32) {
    TS_DISPATCH(pr->p.N, (residual_impl<float, NN>(pr, (const float*)y, (float*)r, st)));
  } else {
    TS_DISPATCH(pr->p.N, (residual_impl<double, NN>(pr, (const double*)y, (double*)r, st)));
  }
}

static int jvp_any(ts_problem* pr, const void* v, void* hv, int precision, cudaStream_t st) {
  if (precision == 32) {
    TS_DISPATCH(pr->p.N, (jvp_impl<float, NN>(pr, (const float*)v, (float*)hv, st)));
  } else {
    TS_DISPATCH(pr->p.N, (jvp_impl<double, NN>(pr, (const double*)v, (double*)hv, st)));
  }
}

// ------------------------------------------------------------------ C ABI

template <int N>
static int j32_inst_impl(ts_problem* pr, J32Inst* I, cudaStream_t st) {
  if constexpr (N > J32_MAX_N) {
    return fail(TS_ERR_UNSUPPORTED, "batched tangent: no single-launch kernel for this N");
  } else {
    if (pr->p.jvp_variant != TS_JVP_LIN_A) return fail(TS_ERR_UNSUPPORTED, "batched tangent: LIN_A only");
    TS_TRY(sync_dmask(pr));
    LinState<float>& l = pr->l32;
    if (!l.valid) {
      if (!pr->l64.valid) return fail(TS_ERR_ARG, "batched tangent: no linearisation state");
      TS_TRY(convert_lin<float, double, N>(pr, pr->l32, pr->l64, st));
    }
    const ts_mesh* m = pr->mesh;
    *I = J32Inst{m->d_tets, m->d_geo32, nullptr, (const float*)l.u0t, (float*)l.vt, (const float*)l.tau,
                 (const float*)l.t0, pr->d_dmask, nullptr, phys_of<float>(pr, true), m->E, m->V, N};
    return 0;
  }
}

template <int N>
static int j32_boundary_impl(ts_problem* pr, const float* v, float* hv, cudaStream_t st) {
  for (auto& o : pr->outlets)
    if (launch_outlet<float>(o.d_nodes, outlet_w<float>(o), (int)o.nodes.size(), (float)o.R, v,
                             pr->d_dmask, 1, hv, pr->C, st))
      return fail(TS_ERR_CUDA, "outlet kernel launch failed");
  return backflow_terms<float, N>(pr, pr->l32, v, false, 1, hv, st);
}

static int precond_diag(ts_problem* pr, const double* y, double* D, cudaStream_t st) {
  TS_TRY(sync_dmask(pr));
  TS_CUDA(cudaMemsetAsync(D, 0, field_len(pr) * sizeof(double), st));
  const ts_mesh* msh = pr->mesh;
  Phys<double> ph = phys_of<double>(pr, true);
  for (size_t c = 0; c + 1 < msh->colour_off.size(); ++c)
    if (launch_diag(msh->d_tets, msh->d_geo64, y, pr->p.N, ph, D, msh->colour_off[c], msh->colour_off[c + 1], st))
      return fail(TS_ERR_CUDA, "diag kernel");
  if (launch_diag_invert(D, pr->d_dmask, msh->V, pr->C, st)) return fail(TS_ERR_CUDA, "diag invert");
  return 0;
}

// per-node outlet couplings R w_i w_j (the diagonal part of the resistance term)
static int sync_outdiag(ts_problem* pr) {
  if (!pr->d_outdiag) TS_TRY(dalloc(&pr->d_outdiag, (size_t)pr->mesh->V * 6));
  if (!pr->outdiag_dirty) return 0;
  std::vector<float> od((size_t)pr->mesh->V * 6, 0.f);
  for (auto& o : pr->outlets)
    for (size_t k = 0; k < o.nodes.size(); ++k) {
      const double* w = &o.w[3 * k];
      float* d = &od[(size_t)o.nodes[k] * 6];
      d[0] += (float)(o.R * w[0] * w[0]);
      d[1] += (float)(o.R * w[0] * w[1]);
      d[2] += (float)(o.R * w[0] * w[2]);
      d[3] += (float)(o.R * w[1] * w[1]);
      d[4] += (float)(o.R * w[1] * w[2]);
      d[5] += (float)(o.R * w[2] * w[2]);
    }
  TS_CUDA(cudaMemcpy(pr->d_outdiag, od.data(), od.size() * 4, cudaMemcpyHostToDevice));
  pr->outdiag_dirty = false;
  return 0;
}

template <typename T, int N>
static int block_diag_impl(ts_problem* pr, LinState<T>& l, int invert, float* out, cudaStream_t st) {
  const ts_mesh* m = pr->mesh;
  Phys<double> p64 = phys_of<double>(pr, true);
  Phys<float> ph{(float)p64.rho, (float)p64.mu, (float)p64.omega, (float)p64.nu, (float)p64.C_I,
                 (float)p64.mass_coef};
  const int paper = pr->p.jvp_variant == TS_JVP_PAPER;
  int rc = launch_block_diag<T, N>(paper, invert, m->d_node_off, m->d_node_elem, m->d_tets, geo_of<T>(m),
                                   l.u0, l.tau, pr->d_dmask, pr->d_outdiag, ph, out, m->V, pr->d_counter, st);
  if (rc) return fail(rc == -6 ? TS_ERR_UNSUPPORTED : TS_ERR_CUDA, "block diagonal kernel launch failed");
  return 0;
}

// nodal diagonal blocks of the tangent at the last residual's state
static int block_diag_any(ts_problem* pr, int invert, float* out, cudaStream_t st) {
  TS_TRY(sync_dmask(pr));
  TS_TRY(sync_outdiag(pr));
  if (pr->l64.valid) {
    TS_DISPATCH(pr->p.N, (block_diag_impl<double, NN>(pr, pr->l64, invert, out, st)));
  }
  if (pr->l32.valid) {
    TS_DISPATCH(pr->p.N, (block_diag_impl<float, NN>(pr, pr->l32, invert, out, st)));
  }
  return fail(TS_ERR_ARG, "block diagonal: no linearisation state (call ts_residual first)");
}

static int block_apply_any(ts_problem* pr, const double* x, double* z, cudaStream_t st) {
  int rc = 0;
  switch (pr->p.N) {
#define TS_BAPPLY_CASE(NV) case NV: rc = launch_block_apply<NV>(pr->d_binv, x, z, pr->mesh->V, st); break;
    TS_BAPPLY_CASE(1) TS_BAPPLY_CASE(2) TS_BAPPLY_CASE(3) TS_BAPPLY_CASE(4) TS_BAPPLY_CASE(5)
    TS_BAPPLY_CASE(7) TS_BAPPLY_CASE(10) TS_BAPPLY_CASE(15)
#undef TS_BAPPLY_CASE
    default: return fail(TS_ERR_UNSUPPORTED, "no kernel compiled for this N");
  }
  return rc ? fail(TS_ERR_CUDA, "block apply kernel launch failed") : 0;
}

static int block_precond_setup(ts_problem* pr, cudaStream_t st) {
  const int64_t nb = 8 * (int64_t)pr->p.N;
  if (!pr->d_binv) TS_TRY(dalloc(&pr->d_binv, (size_t)pr->mesh->V * nb * nb));
  TS_TRY(block_diag_any(pr, 1, pr->d_binv, st));
  pr->binv_valid = true;
  return 0;
}

template <typename T, int N>
static int assemble_impl(ts_problem* pr, LinState<T>& l, cudaStream_t st) {
  const ts_mesh* m = pr->mesh;
  if (!pr->d_hasm) TS_TRY(dalloc(&pr->d_hasm, (size_t)m->nnzb * assembled_record_floats(N)));
  Phys<double> p64 = phys_of<double>(pr, true);
  Phys<float> ph{(float)p64.rho, (float)p64.mu, (float)p64.omega, (float)p64.nu, (float)p64.C_I,
                 (float)p64.mass_coef};
  int rc = launch_assemble_paper<T, N>(m->d_node_off, m->d_node_elem, m->d_row_off, m->d_cols, m->d_tets,
                                       geo_of<T>(m), l.u0, l.tau, ph, pr->d_hasm, m->V, st);
  if (rc) return fail(rc == -6 ? TS_ERR_UNSUPPORTED : TS_ERR_CUDA, "assembly kernel launch failed");
  pr->hasm_valid = true;
  return 0;
}

static int assemble_any(ts_problem* pr, cudaStream_t st) {
  if (!pr->backflow.empty()) return fail(TS_ERR_UNSUPPORTED, "assembled tangent: backflow faces not supported");
  if (pr->l64.valid) {
    TS_DISPATCH(pr->p.N, (assemble_impl<double, NN>(pr, pr->l64, st)));
  }
  if (pr->l32.valid) {
    TS_DISPATCH(pr->p.N, (assemble_impl<float, NN>(pr, pr->l32, st)));
  }
  return fail(TS_ERR_ARG, "assembled tangent: no linearisation state (call ts_residual first)");
}

template <int N>
static int spmv_impl(ts_problem* pr, const float* v, float* hv, cudaStream_t st) {
  const ts_mesh* m = pr->mesh;
  int rc = launch_spmv_paper<N>(m->d_row_off, m->d_cols, pr->d_hasm, pr->d_dmask, v, hv, m->V, st);
  if (rc) return fail(rc == -6 ? TS_ERR_UNSUPPORTED : TS_ERR_CUDA, "assembled product kernel launch failed");
  for (auto& o : pr->outlets)
    if (launch_outlet<float>(o.d_nodes, outlet_w<float>(o), (int)o.nodes.size(), (float)o.R, v, pr->d_dmask, 1,
                             hv, pr->C, st))
      return fail(TS_ERR_CUDA, "outlet kernel launch failed");
  return 0;
}

static int spmv_any(ts_problem* pr, const float* v, float* hv, cudaStream_t st) {
  if (!pr->hasm_valid) return fail(TS_ERR_ARG, "ts_spmv: no assembled tangent (call ts_assemble first)");
  TS_DISPATCH(pr->p.N, (spmv_impl<NN>(pr, v, hv, st)));
}

// Symmetric block Gauss-Seidel with the assembled records (precond 3): a
// forward sweep over the node colours from z = 0, then a backward sweep.
// Two updates are left out because their result is known exactly: the first
// colour of the forward sweep sees z = 0 everywhere else (its off-diagonal
// sum is zero: z_A = Binv_A r_A), and the first colour of the backward sweep
// is the forward sweep's last, whose neighbours have not changed since.
template <int N>
static int sgs_impl(ts_problem* pr, cudaStream_t st) {
  const ts_mesh* m = pr->mesh;
  const int nc = (int)m->ncolour_off.size() - 1;
  for (int pass = 0; pass < 2; ++pass)
    for (int k = pass; k < nc; ++k) {
      const int c = pass == 0 ? k : nc - 1 - k;
      const int64_t o0 = m->ncolour_off[c], o1 = m->ncolour_off[c + 1];
      if (launch_sgs_colour<N>(m->d_node_perm + o0, o1 - o0, m->d_row_off, m->d_cols, pr->d_hasm, pr->d_binv,
                               pr->d_dmask, pr->d_r32, pr->d_z32, pass == 0 && k == 0, st))
        return fail(TS_ERR_CUDA, "block Gauss-Seidel kernel launch failed");
    }
  return 0;
}

static int sgs_apply_any(ts_problem* pr, const double* x, double* z, cudaStream_t st) {
  const int64_t n = field_len(pr);
  if (vec_cast_d2f(pr->d_r32, x, n, st)) return fail(TS_ERR_CUDA, "cast");
  TS_CUDA(cudaMemsetAsync(pr->d_z32, 0, n * sizeof(float), st));
  TS_DISPATCH(pr->p.N, ([&]() -> int {
    TS_TRY(sgs_impl<NN>(pr, st));
    if (vec_cast_f2d(z, pr->d_z32, n, st)) return fail(TS_ERR_CUDA, "cast");
    return 0;
  }()));
}

static int sgs_setup(ts_problem* pr, cudaStream_t st) {
  const int64_t n = field_len(pr);
  if (!pr->d_r32) TS_TRY(dalloc(&pr->d_r32, (size_t)n));
  if (!pr->d_z32) TS_TRY(dalloc(&pr->d_z32, (size_t)n));
  TS_TRY(block_precond_setup(pr, st));
  return assemble_any(pr, st);
}

namespace ts {
// operands of the problem's FP32 LIN_A tangent for the batched launch (v, out unset)
int problem_j32_inst(ts_problem* pr, J32Inst* I, cudaStream_t st) {
  TS_DISPATCH(pr->p.N, (j32_inst_impl<NN>(pr, I, st)));
}
// boundary terms of the FP32 tangent (resistance outlets, backflow), added to hv
int problem_j32_boundary(ts_problem* pr, const float* v, float* hv, cudaStream_t st) {
  TS_DISPATCH(pr->p.N, (j32_boundary_impl<NN>(pr, v, hv, st)));
}
// approximate inverse diagonal of the tangent at y (the right preconditioner of ts_solve)
int problem_precond(ts_problem* pr, const double* y, double* D, cudaStream_t st) {
  return precond_diag(pr, y, D, st);
}
int64_t problem_field_len(const ts_problem* pr) { return field_len(pr); }
const ts_params* problem_params(const ts_problem* pr) { return &pr->p; }

// the problem's Dirichlet mask on the device, storage coordinates per field, field length
int problem_fixed_mask(ts_problem* pr, const uint8_t** dmask, int* C, int64_t* n) {
  TS_TRY(sync_dmask(pr));
  *dmask = pr->d_dmask;
  *C = pr->C;
  *n = field_len(pr);
  return 0;
}
}  // namespace ts

extern "C" {

const char* ts_last_error(void) { return g_last_error.c_str(); }
const char* ts_version(void) { return "tsgls-gb300 0.1 (sm_103a)"; }

int64_t ts_launch_count(void) { return (int64_t)ts::launches_total(); }

int ts_stage_times(ts_problem* pr, double* out) {
  if (!pr || !out) return fail(TS_ERR_ARG, "ts_stage_times: NULL argument");
  out[0] = out[1] = out[2] = -1.0;
  float ms = 0.f;
  if (pr->sev_res) {
    TS_CUDA(cudaEventSynchronize(pr->sev[2]));
    TS_CUDA(cudaEventElapsedTime(&ms, pr->sev[0], pr->sev[1]));
    out[0] = ms;
    TS_CUDA(cudaEventElapsedTime(&ms, pr->sev[1], pr->sev[2]));
    out[1] = ms;
  }
  if (pr->sev_jvp) {
    TS_CUDA(cudaEventSynchronize(pr->sev[4]));
    TS_CUDA(cudaEventElapsedTime(&ms, pr->sev[3], pr->sev[4]));
    out[2] = ms;
  }
  return 0;
}

int ts_mesh_load(const double* xyz_host, int64_t n_nodes, const int32_t* tets_host,
                 int64_t n_tets, const int32_t* bfaces_host, const int32_t* btag_host,
                 int64_t n_bfaces, ts_mesh** out) {
  if (!out) return fail(TS_ERR_ARG, "ts_mesh_load: out is NULL");
  *out = nullptr;
  if (!xyz_host || !tets_host || n_nodes < 4 || n_tets < 1 || n_bfaces < 0 ||
      (n_bfaces > 0 && (!bfaces_host || !btag_host)))
    return fail(TS_ERR_ARG, "ts_mesh_load: bad sizes or NULL arrays");
  if (n_nodes >= (int64_t)1 << 31 || n_tets >= (int64_t)1 << 31)
    return fail(TS_ERR_ARG, "ts_mesh_load: mesh too large for 32-bit ids");
  for (int64_t i = 0; i < 4 * n_tets; ++i)
    if (tets_host[i] < 0 || tets_host[i] >= n_nodes)
      return fail(TS_ERR_ARG, "ts_mesh_load: tetrahedron node id out of range");
  for (int64_t i = 0; i < 3 * n_bfaces; ++i)
    if (bfaces_host[i] < 0 || bfaces_host[i] >= n_nodes)
      return fail(TS_ERR_ARG, "ts_mesh_load: boundary face node id out of range");

  ts_mesh* m = new ts_mesh();
  cudaGetDevice(&m->device);
  m->V = n_nodes;
  m->E = n_tets;
  m->F = n_bfaces;
  m->xyz.assign(xyz_host, xyz_host + 3 * n_nodes);
  // greedy colouring: the lowest colour unused at all four nodes
  std::vector<uint64_t> used(n_nodes, 0);
  std::vector<int> col(n_tets);
  int ncol = 0;
  for (int64_t e = 0; e < n_tets; ++e) {
    const int32_t* t = tets_host + 4 * e;
    uint64_t u = used[t[0]] | used[t[1]] | used[t[2]] | used[t[3]];
    if (u == ~0ull) {
      delete m;
      return fail(TS_ERR_ARG, "ts_mesh_load: more than 64 element colours needed");
    }
    int c = __builtin_ctzll(~u);
    col[e] = c;
    ncol = std::max(ncol, c + 1);
    for (int a = 0; a < 4; ++a) used[t[a]] |= 1ull << c;
  }
  std::vector<int64_t> cnt(ncol + 1, 0);
  for (int64_t e = 0; e < n_tets; ++e) cnt[col[e] + 1]++;
  for (int c = 0; c < ncol; ++c) cnt[c + 1] += cnt[c];
  m->colour_off = cnt;
  std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
  m->tets.resize(4 * n_tets);
  std::vector<double> geo(GEO_STRIDE * n_tets, 0.0);
  for (int64_t e = 0; e < n_tets; ++e) {
    int64_t d = pos[col[e]]++;
    const int32_t* t = tets_host + 4 * e;
    for (int a = 0; a < 4; ++a) m->tets[4 * d + a] = t[a];
    const double* x0 = &m->xyz[3 * t[0]];
    double J[3][3];   // J[i][k] = d x_i / d xi_k
    for (int k = 0; k < 3; ++k)
      for (int i = 0; i < 3; ++i) J[i][k] = m->xyz[3 * t[k + 1] + i] - x0[i];
    double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                 J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                 J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    double scale = 0;
    for (int i = 0; i < 3; ++i)
      for (int k = 0; k < 3; ++k) scale = std::max(scale, std::fabs(J[i][k]));
    if (!(std::fabs(det) > 1e-14 * scale * scale * scale)) {
      delete m;
      return fail(TS_ERR_ARG, "ts_mesh_load: degenerate tetrahedron");
    }
    double inv[3][3];  // inv[k][i] = d xi_k / d x_i
    inv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
    inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    inv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
    inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    inv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
    inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    double* g = &geo[GEO_STRIDE * d];
    for (int j = 0; j < 3; ++j) {
      g[0 * 3 + j] = -(inv[0][j] + inv[1][j] + inv[2][j]);
      for (int a = 1; a < 4; ++a) g[a * 3 + j] = inv[a - 1][j];
    }
    g[GEO_VOL] = std::fabs(det) / 6.0;
    auto G = [&](int i, int j) { return inv[0][i] * inv[0][j] + inv[1][i] * inv[1][j] + inv[2][i] * inv[2][j]; };
    g[GEO_G + 0] = G(0, 0);
    g[GEO_G + 1] = G(0, 1);
    g[GEO_G + 2] = G(0, 2);
    g[GEO_G + 3] = G(1, 1);
    g[GEO_G + 4] = G(1, 2);
    g[GEO_G + 5] = G(2, 2);
  }
  // boundary faces, oriented outward with the owning tetrahedron
  std::vector<std::vector<int32_t>> node_tets(n_nodes);
  for (int64_t e = 0; e < n_tets; ++e)
    for (int a = 0; a < 4; ++a) node_tets[tets_host[4 * e + a]].push_back((int32_t)e);
  m->bfaces.resize(3 * n_bfaces);
  m->btag.assign(btag_host, btag_host + n_bfaces);
  for (int64_t f = 0; f < n_bfaces; ++f) {
    int32_t a = bfaces_host[3 * f], b = bfaces_host[3 * f + 1], c = bfaces_host[3 * f + 2];
    int32_t opp = -1;
    for (int32_t e : node_tets[a]) {
      const int32_t* t = tets_host + 4 * e;
      int hits = 0, other = -1;
      for (int k = 0; k < 4; ++k) {
        if (t[k] == a || t[k] == b || t[k] == c) ++hits;
        else other = t[k];
      }
      if (hits == 3) {
        opp = other;
        break;
      }
    }
    if (opp < 0) {
      delete m;
      return fail(TS_ERR_ARG, "ts_mesh_load: boundary face not on any tetrahedron");
    }
    const double* pa = &m->xyz[3 * a];
    double u[3], v[3], w[3], n[3];
    for (int i = 0; i < 3; ++i) {
      u[i] = m->xyz[3 * b + i] - pa[i];
      v[i] = m->xyz[3 * c + i] - pa[i];
      w[i] = m->xyz[3 * opp + i] - pa[i];
    }
    n[0] = u[1] * v[2] - u[2] * v[1];
    n[1] = u[2] * v[0] - u[0] * v[2];
    n[2] = u[0] * v[1] - u[1] * v[0];
    if (n[0] * w[0] + n[1] * w[1] + n[2] * w[2] > 0) std::swap(b, c);
    m->bfaces[3 * f] = a;
    m->bfaces[3 * f + 1] = b;
    m->bfaces[3 * f + 2] = c;
  }
  std::vector<float> geo32(geo.begin(), geo.end());
  // node-to-element list over the colour-sorted elements (element * 4 + local node)
  std::vector<int32_t> noff(n_nodes + 1, 0), nel(4 * n_tets);
  for (int64_t i = 0; i < 4 * n_tets; ++i) noff[m->tets[i] + 1]++;
  for (int64_t v = 0; v < n_nodes; ++v) noff[v + 1] += noff[v];
  {
    std::vector<int32_t> fill(noff.begin(), noff.end() - 1);
    for (int64_t d = 0; d < n_tets; ++d)
      for (int a = 0; a < 4; ++a) nel[fill[m->tets[4 * d + a]]++] = (int32_t)(4 * d + a);
  }
  // node graph (nodes sharing an element, the node itself included), sorted rows
  std::vector<int32_t> roff(n_nodes + 1, 0), cols;
  {
    std::vector<int32_t> nb;
    for (int64_t v = 0; v < n_nodes; ++v) {
      nb.clear();
      for (int32_t p = noff[v]; p < noff[v + 1]; ++p) {
        const int32_t d = nel[p] >> 2;
        for (int a = 0; a < 4; ++a) nb.push_back(m->tets[4 * (int64_t)d + a]);
      }
      std::sort(nb.begin(), nb.end());
      nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
      cols.insert(cols.end(), nb.begin(), nb.end());
      roff[v + 1] = (int32_t)cols.size();
    }
  }
  m->nnzb = (int64_t)cols.size();
  // greedy colouring of the node graph: no two nodes of a colour share an element
  std::vector<int32_t> ncl(n_nodes, -1), perm(n_nodes);
  {
    std::vector<int64_t> mark;
    int nc = 0;
    for (int64_t v = 0; v < n_nodes; ++v) {
      mark.assign(nc + 1, -1);
      for (int32_t p = roff[v]; p < roff[v + 1]; ++p)
        if (ncl[cols[p]] >= 0) mark[ncl[cols[p]]] = v;
      int c = 0;
      while (c < nc && mark[c] == v) ++c;
      ncl[v] = c;
      if (c == nc) ++nc;
    }
    std::vector<int64_t> cnt(nc + 1, 0);
    for (int64_t v = 0; v < n_nodes; ++v) cnt[ncl[v] + 1]++;
    for (int c = 0; c < nc; ++c) cnt[c + 1] += cnt[c];
    m->ncolour_off = cnt;
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    for (int64_t v = 0; v < n_nodes; ++v) perm[fill[ncl[v]]++] = (int32_t)v;
    m->node_colour = ncl;
  }
  int rc = 0;
  rc |= dalloc(&m->d_tets, (size_t)n_tets);
  rc |= dalloc(&m->d_geo64, geo.size());
  rc |= dalloc(&m->d_geo32, geo32.size());
  rc |= dalloc(&m->d_node_off, noff.size());
  rc |= dalloc(&m->d_node_elem, nel.size());
  rc |= dalloc(&m->d_row_off, roff.size());
  rc |= dalloc(&m->d_cols, cols.size());
  rc |= dalloc(&m->d_node_perm, perm.size());
  if (rc) {
    ts_mesh_free(m);
    return TS_ERR_OOM;
  }
  if (cudaMemcpy(m->d_node_off, noff.data(), noff.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(m->d_node_elem, nel.data(), nel.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(m->d_row_off, roff.data(), roff.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(m->d_cols, cols.data(), cols.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(m->d_node_perm, perm.data(), perm.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
    ts_mesh_free(m);
    return fail(TS_ERR_CUDA, "ts_mesh_load: host-to-device copy failed");
  }
  cudaError_t e1 = cudaMemcpy(m->d_tets, m->tets.data(), 16 * n_tets, cudaMemcpyHostToDevice);
  cudaError_t e2 = cudaMemcpy(m->d_geo64, geo.data(), geo.size() * 8, cudaMemcpyHostToDevice);
  cudaError_t e3 = cudaMemcpy(m->d_geo32, geo32.data(), geo32.size() * 4, cudaMemcpyHostToDevice);
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
    ts_mesh_free(m);
    return fail(TS_ERR_CUDA, "ts_mesh_load: host-to-device copy failed");
  }
  *out = m;
  return 0;
}

void ts_mesh_free(ts_mesh* m) {
  if (!m) return;
  dfree(m->d_tets);
  dfree(m->d_geo64);
  dfree(m->d_geo32);
  dfree(m->d_node_off);
  dfree(m->d_node_elem);
  dfree(m->d_row_off);
  dfree(m->d_cols);
  dfree(m->d_node_perm);
  delete m;
}

int ts_mesh_colors(const ts_mesh* m) {
  if (!m) return fail(TS_ERR_ARG, "NULL mesh");
  return (int)m->colour_off.size() - 1;
}

int ts_problem_create(const ts_mesh* mesh, const ts_params* params, ts_problem** out) {
  if (!out || !mesh || !params) return fail(TS_ERR_ARG, "ts_problem_create: NULL argument");
  *out = nullptr;
  const ts_params& p = *params;
  if (!n_supported(p.N)) return fail(TS_ERR_UNSUPPORTED, "ts_problem_create: N not compiled");
  if (!(p.rho > 0) || !(p.mu > 0) || !(p.omega >= 0) || !(p.C_I > 0))
    return fail(TS_ERR_ARG, "ts_problem_create: rho, mu, C_I must be positive, omega >= 0");
  if (mode_of_variant(p.jvp_variant) < 0) return fail(TS_ERR_ARG, "unknown jvp variant");
  ts_problem* pr = new ts_problem();
  pr->mesh = mesh;
  pr->p = p;
  pr->C = 2 * p.N;
  pr->K = 3 * p.N - 2;
  const int nm = 2 * p.N - 1;
  pr->NTP = ((nm * (nm + 1) / 2) + 3) & ~3;
  pr->dmask.assign(mesh->V, 0);
  {
  }
  if (dalloc(&pr->d_dmask, (size_t)mesh->V) || dalloc(&pr->d_counter, 1) ||
      cudaEventCreate(&pr->ev_a) != cudaSuccess || cudaEventCreate(&pr->ev_b) != cudaSuccess ||
      cudaEventCreate(&pr->sev[0]) != cudaSuccess || cudaEventCreate(&pr->sev[1]) != cudaSuccess ||
      cudaEventCreate(&pr->sev[2]) != cudaSuccess || cudaEventCreate(&pr->sev[3]) != cudaSuccess ||
      cudaEventCreate(&pr->sev[4]) != cudaSuccess) {
    ts_problem_free(pr);
    return TS_ERR_OOM;
  }
  cudaMemset(pr->d_counter, 0, sizeof(unsigned));
  // the allocation-free residual must not load anything at call time
  if (int rc = noalloc_setup(p.N)) {
    ts_problem_free(pr);
    return rc;
  }
  *out = pr;
  return 0;
}

void ts_problem_free(ts_problem* pr) {
  if (!pr) return;
  if (pr->ev_a) cudaEventDestroy(pr->ev_a);
  if (pr->ev_b) cudaEventDestroy(pr->ev_b);
  for (auto& e : pr->sev)
    if (e) cudaEventDestroy(e);
  dfree(pr->d_dmask);
  dfree(pr->d_counter);
  for (auto& o : pr->outlets) {
    dfree(o.d_nodes);
    dfree(o.d_w64);
    dfree(o.d_w32);
  }
  for (auto& in : pr->inlets) {
    dfree(in.d_nodes);
    dfree(in.d_vals);
  }
  for (auto& b : pr->backflow) {
    dfree(b.d_faces);
    dfree(b.d_n64);
    dfree(b.d_a64);
    dfree(b.d_n32);
    dfree(b.d_a32);
  }
  lin_free(pr->l32);
  lin_free(pr->l64);
  dfree(pr->d_basis);
  dfree(pr->d_w);
  dfree(pr->d_r);
  dfree(pr->d_dy);
  dfree(pr->d_partial);
  dfree(pr->d_h);
  dfree(pr->d_v32);
  dfree(pr->d_w32);
  dfree(pr->d_D);
  dfree(pr->d_t);
  dfree(pr->d_binv);
  dfree(pr->d_vcache);
  dfree(pr->d_eig);
  dfree(pr->d_dT);
  dfree(pr->d_hasm);
  dfree(pr->d_r32);
  dfree(pr->d_z32);
  dfree(pr->d_outdiag);
  delete pr;
}

int ts_problem_set(ts_problem* pr, double dt_pseudo, int jvp_variant) {
  if (!pr) return fail(TS_ERR_ARG, "NULL problem");
  if (mode_of_variant(jvp_variant) < 0) return fail(TS_ERR_ARG, "unknown jvp variant");
  pr->p.dt_pseudo = dt_pseudo;
  pr->p.jvp_variant = jvp_variant;
  return 0;
}

int ts_problem_option(ts_problem* pr, int key, int value) {
  if (!pr) return fail(TS_ERR_ARG, "NULL problem");
  if (key == TS_OPT_TAU64) {
    if (value != TS_TAU64_REFINE && value != TS_TAU64_DOUBLEFLOAT && value != TS_TAU64_JACOBI)
      return fail(TS_ERR_ARG, "unknown TS_OPT_TAU64 value");
    pr->tau64 = value;
    return 0;
  }
  if (key == TS_OPT_ELEMENT64) {
    if (value != TS_ELEMENT64_NATIVE && value != TS_ELEMENT64_DOUBLEFLOAT)
      return fail(TS_ERR_ARG, "unknown TS_OPT_ELEMENT64 value");
    pr->elem64 = value;
    return 0;
  }
  if (key == TS_OPT_TAU_WARM) {
    if (value != 0 && value != 1) return fail(TS_ERR_ARG, "TS_OPT_TAU_WARM takes 0 or 1");
    pr->tau_warm = value;
    pr->vcache_valid = false;
    return 0;
  }
  if (key == TS_OPT_FP32_TANGENT) {
    if (value != 0 && value != 1) return fail(TS_ERR_ARG, "TS_OPT_FP32_TANGENT takes 0 or 1");
    pr->fast32 = value == 0;
    return 0;
  }
  return fail(TS_ERR_ARG, "unknown option key");
}

}  // extern "C"

namespace {

// J_nu(z), nu = 0 or 1, from its power series sum_k (-1)^k (z/2)^(2k+nu) / (k! (k+nu)!)
// (Abramowitz & Stegun 9.1.10); adequate for |z| up to about 30
std::complex<double> bessel_j_series(int nu, std::complex<double> z) {
  const std::complex<double> h = 0.5 * z, h2 = h * h;
  std::complex<double> term = nu == 0 ? std::complex<double>(1.0) : h;
  std::complex<double> sum = term;
  for (int k = 1; k < 400; ++k) {
    term *= -h2 / (double)(k * (k + nu));
    sum += term;
    if (std::abs(term) <= 1e-18 * std::abs(sum) && k > std::abs(h) + 2) break;
  }
  return sum;
}

// velocity mode n at radius r of a profile with flow-rate coefficient Q and mean
// velocity U = Q / (pi R^2): parabolic 2U(1 - r^2/R^2), or the Womersley mode
// U [1 - J0(L r/R) / J0(L)] / [1 - 2 J1(L) / (L J0(L))], L = i^{3/2} alpha_n,
// alpha_n = R sqrt(n omega / nu) (mode 0 of Womersley is the parabola)
std::complex<double> inlet_mode_value(int profile, int n, double r, double R, std::complex<double> Q,
                                      double omega, double nu) {
  const double pi = 3.14159265358979323846;
  const std::complex<double> U = Q / (pi * R * R);
  const double x = std::min(r / R, 1.0);
  if (profile == TS_PROFILE_PARABOLIC || n == 0) return 2.0 * U * (1.0 - x * x);
  const double alpha = R * std::sqrt(n * omega / nu);
  const std::complex<double> i32 = std::polar(1.0, 0.75 * pi);   // i^{3/2}
  const std::complex<double> L = i32 * alpha;
  const std::complex<double> j0 = bessel_j_series(0, L);
  const std::complex<double> shape = 1.0 - bessel_j_series(0, L * x) / j0;
  const std::complex<double> mean_shape = 1.0 - 2.0 * bessel_j_series(1, L) / (L * j0);
  return U * shape / mean_shape;
}

}  // namespace

extern "C" {

int ts_set_inlet(ts_problem* pr, int tag, const double* Qn_host, int profile, const double* geometry_host) {
  if (!pr || !Qn_host) return fail(TS_ERR_ARG, "ts_set_inlet: NULL argument");
  if (profile != TS_PROFILE_PARABOLIC && profile != TS_PROFILE_WOMERSLEY)
    return fail(TS_ERR_ARG, "ts_set_inlet: unknown profile");
  const ts_mesh* m = pr->mesh;
  const int N = pr->p.N, C = pr->C;
  for (int n = 0; n < N; ++n)
    if (!std::isfinite(Qn_host[2 * n]) || !std::isfinite(Qn_host[2 * n + 1]))
      return fail(TS_ERR_ARG, "ts_set_inlet: non-finite flow-rate coefficient");
  // outward normal (faces are oriented outward at ts_mesh_load), tag nodes, rim nodes
  double nrm[3] = {0, 0, 0};
  std::vector<uint8_t> on_tag(m->V, 0), on_other(m->V, 0);
  for (int64_t f = 0; f < m->F; ++f) {
    const int32_t* t = &m->bfaces[3 * f];
    if (m->btag[f] != tag) {
      for (int k = 0; k < 3; ++k) on_other[t[k]] = 1;
      continue;
    }
    const double* pa = &m->xyz[3 * t[0]];
    double u[3], v[3];
    for (int i = 0; i < 3; ++i) {
      u[i] = m->xyz[3 * t[1] + i] - pa[i];
      v[i] = m->xyz[3 * t[2] + i] - pa[i];
    }
    nrm[0] += u[1] * v[2] - u[2] * v[1];
    nrm[1] += u[2] * v[0] - u[0] * v[2];
    nrm[2] += u[0] * v[1] - u[1] * v[0];
    for (int k = 0; k < 3; ++k) on_tag[t[k]] = 1;
  }
  const double nl = std::sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
  if (!(nl > 0)) return fail(TS_ERR_ARG, "ts_set_inlet: no boundary face carries this tag");
  Inlet in;
  in.tag = tag;
  in.profile = profile;
  for (int i = 0; i < 3; ++i) in.dir[i] = -nrm[i] / nl;
  const double* d = in.dir;
  // centre: the area-weighted centroid of the tag's triangles; radius: the
  // largest distance of a rim node from the axis through the centre
  double cen[3] = {0, 0, 0}, atot = 0;
  for (int64_t f = 0; f < m->F; ++f) {
    if (m->btag[f] != tag) continue;
    const int32_t* t = &m->bfaces[3 * f];
    const double *pa = &m->xyz[3 * t[0]], *pb = &m->xyz[3 * t[1]], *pc = &m->xyz[3 * t[2]];
    double u[3], v[3];
    for (int i = 0; i < 3; ++i) {
      u[i] = pb[i] - pa[i];
      v[i] = pc[i] - pa[i];
    }
    const double cx = u[1] * v[2] - u[2] * v[1], cy = u[2] * v[0] - u[0] * v[2], cz = u[0] * v[1] - u[1] * v[0];
    const double ar = 0.5 * std::sqrt(cx * cx + cy * cy + cz * cz);
    for (int i = 0; i < 3; ++i) cen[i] += ar * (pa[i] + pb[i] + pc[i]) / 3.0;
    atot += ar;
  }
  for (int i = 0; i < 3; ++i) in.centre[i] = cen[i] / atot;
  int n_rim = 0;
  double rmax = 0;
  for (int64_t v = 0; v < m->V; ++v) {
    if (!on_tag[v]) continue;
    in.nodes.push_back((int32_t)v);
    if (!on_other[v]) continue;
    const double* x = &m->xyz[3 * v];
    double rel[3], ax = 0, r2 = 0;
    for (int i = 0; i < 3; ++i) rel[i] = x[i] - in.centre[i];
    for (int i = 0; i < 3; ++i) ax += rel[i] * d[i];
    for (int i = 0; i < 3; ++i) r2 += (rel[i] - ax * d[i]) * (rel[i] - ax * d[i]);
    rmax = std::max(rmax, std::sqrt(r2));
    ++n_rim;
  }
  if (n_rim < 3 || !(rmax > 0)) return fail(TS_ERR_ARG, "ts_set_inlet: the tag's rim (nodes shared with other tags) has < 3 nodes");
  in.R = rmax;
  if (geometry_host) {
    double dl = 0;
    for (int i = 0; i < 3; ++i) dl += geometry_host[3 + i] * geometry_host[3 + i];
    dl = std::sqrt(dl);
    if (!(dl > 0) || !(geometry_host[6] > 0)) return fail(TS_ERR_ARG, "ts_set_inlet: bad inlet geometry");
    for (int i = 0; i < 3; ++i) {
      in.centre[i] = geometry_host[i];
      in.dir[i] = geometry_host[3 + i] / dl;
    }
    in.R = geometry_host[6];
  }
  // Dirichlet velocity modes: profile x flow-rate coefficient along the inflow direction
  const double nu = pr->p.mu / pr->p.rho;
  in.vals.assign(in.nodes.size() * 3 * C, 0.0);
  for (size_t k = 0; k < in.nodes.size(); ++k) {
    const int32_t v = in.nodes[k];
    if (on_other[v]) continue;   // the rim belongs to the wall: no-slip
    const double* x = &m->xyz[3 * v];
    double rel[3], ax = 0;
    for (int i = 0; i < 3; ++i) rel[i] = x[i] - in.centre[i];
    for (int i = 0; i < 3; ++i) ax += rel[i] * d[i];
    double r2 = 0;
    for (int i = 0; i < 3; ++i) {
      const double pi_ = rel[i] - ax * d[i];
      r2 += pi_ * pi_;
    }
    const double r = std::sqrt(r2);
    for (int n = 0; n < N; ++n) {
      const std::complex<double> Q(Qn_host[2 * n], n == 0 ? 0.0 : Qn_host[2 * n + 1]);
      const std::complex<double> w = inlet_mode_value(profile, n, r, in.R, Q, pr->p.omega, nu);
      for (int i = 0; i < 3; ++i) {
        in.vals[(k * 3 + i) * C + 2 * n] = w.real() * d[i];
        in.vals[(k * 3 + i) * C + 2 * n + 1] = n == 0 ? 0.0 : w.imag() * d[i];
      }
    }
  }
  for (int32_t v : in.nodes) pr->dmask[v] = 1;
  pr->dmask_dirty = true;
  TS_TRY(dalloc(&in.d_nodes, in.nodes.size()));
  TS_TRY(dalloc(&in.d_vals, in.vals.size()));
  TS_CUDA(cudaMemcpy(in.d_nodes, in.nodes.data(), in.nodes.size() * 4, cudaMemcpyHostToDevice));
  TS_CUDA(cudaMemcpy(in.d_vals, in.vals.data(), in.vals.size() * 8, cudaMemcpyHostToDevice));
  // a second call for the same tag replaces the first
  for (auto it = pr->inlets.begin(); it != pr->inlets.end(); ++it)
    if (it->tag == tag) {
      dfree(it->d_nodes);
      dfree(it->d_vals);
      pr->inlets.erase(it);
      break;
    }
  pr->inlets.push_back(std::move(in));
  return 0;
}

int ts_inlet_info(const ts_problem* pr, int tag, double* out_host) {
  if (!pr || !out_host) return fail(TS_ERR_ARG, "ts_inlet_info: NULL argument");
  for (const auto& in : pr->inlets)
    if (in.tag == tag) {
      for (int i = 0; i < 3; ++i) {
        out_host[i] = in.centre[i];
        out_host[3 + i] = in.dir[i];
      }
      out_host[6] = in.R;
      return 0;
    }
  return fail(TS_ERR_ARG, "ts_inlet_info: no inlet with this tag");
}

int ts_initial_guess(ts_problem* pr, void* y, int precision, void* stream) {
  if (!pr || !y) return fail(TS_ERR_ARG, "ts_initial_guess: NULL argument");
  if (precision != 32 && precision != 64) return fail(TS_ERR_ARG, "precision must be 32 or 64");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t esz = precision == 64 ? 8 : 4;
  TS_CUDA(cudaMemsetAsync(y, 0, (size_t)field_len(pr) * esz, st));
  for (const auto& in : pr->inlets) {
    const int rc = precision == 64
                       ? launch_inlet_fill<double>(in.d_nodes, in.d_vals, (int64_t)in.nodes.size(), pr->C, (double*)y, st)
                       : launch_inlet_fill<float>(in.d_nodes, in.d_vals, (int64_t)in.nodes.size(), pr->C, (float*)y, st);
    if (rc) return fail(TS_ERR_CUDA, "inlet fill kernel launch failed");
  }
  return 0;
}

int ts_set_bc(ts_problem* pr, int tag, int kind, double value) {
  if (!pr) return fail(TS_ERR_ARG, "NULL problem");
  const ts_mesh* m = pr->mesh;
  if (kind == TS_BC_DIRICHLET) {
    for (int64_t f = 0; f < m->F; ++f)
      if (m->btag[f] == tag)
        for (int k = 0; k < 3; ++k) pr->dmask[m->bfaces[3 * f + k]] = 1;
    pr->dmask_dirty = true;
    return 0;
  }
  if (kind == TS_BC_TRACTION) return 0;
  if (kind == TS_BC_BACKFLOW) {
    if (!(value >= 0 && value <= 1)) return fail(TS_ERR_ARG, "ts_set_bc: backflow beta must be in [0, 1]");
    BackflowSet b;
    b.tag = tag;
    b.beta = value;
    std::vector<int32_t> fc;
    std::vector<double> nn, ar;
    for (int64_t f = 0; f < m->F; ++f) {
      if (m->btag[f] != tag) continue;
      const int32_t* t = &m->bfaces[3 * f];
      const double* pa = &m->xyz[3 * t[0]];
      double u[3], w[3], n[3];
      for (int i = 0; i < 3; ++i) {
        u[i] = m->xyz[3 * t[1] + i] - pa[i];
        w[i] = m->xyz[3 * t[2] + i] - pa[i];
      }
      n[0] = u[1] * w[2] - u[2] * w[1];
      n[1] = u[2] * w[0] - u[0] * w[2];
      n[2] = u[0] * w[1] - u[1] * w[0];
      const double len = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
      fc.insert(fc.end(), t, t + 3);
      for (int i = 0; i < 3; ++i) nn.push_back(n[i] / len);
      ar.push_back(0.5 * len);
    }
    if (fc.empty()) return fail(TS_ERR_ARG, "ts_set_bc: no boundary face carries this tag");
    b.n = (int64_t)ar.size();
    b.offset = pr->bf_points;
    std::vector<float> nn32(nn.begin(), nn.end()), ar32(ar.begin(), ar.end());
    int rc = dalloc(&b.d_faces, fc.size()) | dalloc(&b.d_n64, nn.size()) | dalloc(&b.d_a64, ar.size()) |
             dalloc(&b.d_n32, nn.size()) | dalloc(&b.d_a32, ar.size());
    if (rc) return TS_ERR_OOM;
    TS_CUDA(cudaMemcpy(b.d_faces, fc.data(), fc.size() * 4, cudaMemcpyHostToDevice));
    TS_CUDA(cudaMemcpy(b.d_n64, nn.data(), nn.size() * 8, cudaMemcpyHostToDevice));
    TS_CUDA(cudaMemcpy(b.d_a64, ar.data(), ar.size() * 8, cudaMemcpyHostToDevice));
    TS_CUDA(cudaMemcpy(b.d_n32, nn32.data(), nn32.size() * 4, cudaMemcpyHostToDevice));
    TS_CUDA(cudaMemcpy(b.d_a32, ar32.data(), ar32.size() * 4, cudaMemcpyHostToDevice));
    pr->bf_points += 3 * b.n;
    pr->backflow.push_back(b);
    // the cached state no longer matches the problem
    pr->l32.valid = false;
    pr->l64.valid = false;
    return 0;
  }
  if (kind != TS_BC_RESISTANCE) return fail(TS_ERR_ARG, "ts_set_bc: unknown kind");
  if (!(value >= 0)) return fail(TS_ERR_ARG, "ts_set_bc: resistance must be >= 0");
  Outlet o;
  o.tag = tag;
  o.R = value;
  std::vector<int64_t> slot(m->V, -1);
  for (int64_t f = 0; f < m->F; ++f) {
    if (m->btag[f] != tag) continue;
    const int32_t* t = &m->bfaces[3 * f];
    const double* pa = &m->xyz[3 * t[0]];
    double u[3], v[3], n6[3];
    for (int i = 0; i < 3; ++i) {
      u[i] = m->xyz[3 * t[1] + i] - pa[i];
      v[i] = m->xyz[3 * t[2] + i] - pa[i];
    }
    // (area / 3) * unit normal = cross / 6 per face vertex
    n6[0] = (u[1] * v[2] - u[2] * v[1]) / 6.0;
    n6[1] = (u[2] * v[0] - u[0] * v[2]) / 6.0;
    n6[2] = (u[0] * v[1] - u[1] * v[0]) / 6.0;
    for (int k = 0; k < 3; ++k) {
      int32_t A = t[k];
      if (slot[A] < 0) {
        slot[A] = (int64_t)o.nodes.size();
        o.nodes.push_back(A);
        o.w.insert(o.w.end(), {0.0, 0.0, 0.0});
      }
      for (int i = 0; i < 3; ++i) o.w[3 * slot[A] + i] += n6[i];
    }
  }
  if (o.nodes.empty()) return fail(TS_ERR_ARG, "ts_set_bc: no boundary face carries this tag");
  std::vector<float> w32(o.w.begin(), o.w.end());
  int rc = dalloc(&o.d_nodes, o.nodes.size()) | dalloc(&o.d_w64, o.w.size()) |
           dalloc(&o.d_w32, o.w.size());
  if (rc) return TS_ERR_OOM;
  TS_CUDA(cudaMemcpy(o.d_nodes, o.nodes.data(), o.nodes.size() * 4, cudaMemcpyHostToDevice));
  TS_CUDA(cudaMemcpy(o.d_w64, o.w.data(), o.w.size() * 8, cudaMemcpyHostToDevice));
  TS_CUDA(cudaMemcpy(o.d_w32, w32.data(), w32.size() * 4, cudaMemcpyHostToDevice));
  pr->outlets.push_back(std::move(o));
  pr->outdiag_dirty = true;
  return 0;
}

int ts_residual(ts_problem* pr, const void* y, void* r, int precision, void* stream) {
  if (!pr || !y || !r) return fail(TS_ERR_ARG, "ts_residual: NULL argument");
  if (precision != 32 && precision != 64) return fail(TS_ERR_ARG, "precision must be 32 or 64");
  if (y == r) return fail(TS_ERR_ARG, "ts_residual: y and r alias");
  TS_TRY(sync_dmask(pr));
  return residual_any(pr, y, r, precision, (cudaStream_t)stream);
}

int ts_assemble(ts_problem* pr, void* stream) {
  if (!pr) return fail(TS_ERR_ARG, "ts_assemble: NULL problem");
  TS_TRY(sync_dmask(pr));
  return assemble_any(pr, (cudaStream_t)stream);
}

int ts_spmv(ts_problem* pr, const float* v, float* hv, void* stream) {
  if (!pr || !v || !hv) return fail(TS_ERR_ARG, "ts_spmv: NULL argument");
  if ((const void*)v == (const void*)hv) return fail(TS_ERR_ARG, "ts_spmv: v and Hv alias");
  TS_TRY(sync_dmask(pr));
  return spmv_any(pr, v, hv, (cudaStream_t)stream);
}

int64_t ts_assembled_bytes(const ts_problem* pr) {
  if (!pr) return fail(TS_ERR_ARG, "ts_assembled_bytes: NULL problem");
  return pr->mesh->nnzb * (int64_t)assembled_record_floats(pr->p.N) * 4;
}

int64_t ts_mesh_connections(const ts_mesh* m) {
  if (!m) return fail(TS_ERR_ARG, "ts_mesh_connections: NULL mesh");
  return m->nnzb;
}

int ts_block_diagonal(ts_problem* pr, float* blocks, int invert, void* stream) {
  if (!pr || !blocks) return fail(TS_ERR_ARG, "ts_block_diagonal: NULL argument");
  if (invert != 0 && invert != 1) return fail(TS_ERR_ARG, "ts_block_diagonal: invert must be 0 or 1");
  return block_diag_any(pr, invert, blocks, (cudaStream_t)stream);
}

int ts_mesh_node_colours(const ts_mesh* m, int32_t* colour_host) {
  if (!m) return fail(TS_ERR_ARG, "ts_mesh_node_colours: NULL mesh");
  if (colour_host) std::copy(m->node_colour.begin(), m->node_colour.end(), colour_host);
  return (int)m->ncolour_off.size() - 1;
}

int ts_precond_setup(ts_problem* pr, int kind, void* stream) {
  if (!pr) return fail(TS_ERR_ARG, "ts_precond_setup: NULL problem");
  if (kind != 2 && kind != 3) return fail(TS_ERR_ARG, "ts_precond_setup: kind must be 2 or 3");
  if (!pr->l32.valid && !pr->l64.valid) return fail(TS_ERR_ARG, "ts_precond_setup: no residual computed yet");
  TS_TRY(sync_dmask(pr));
  return kind == 2 ? block_precond_setup(pr, (cudaStream_t)stream) : sgs_setup(pr, (cudaStream_t)stream);
}

int ts_precond_apply(ts_problem* pr, int kind, const double* x, double* z, void* stream) {
  if (!pr || !x || !z) return fail(TS_ERR_ARG, "ts_precond_apply: NULL argument");
  if (x == z) return fail(TS_ERR_ARG, "ts_precond_apply: x and z alias");
  if (kind != 2 && kind != 3) return fail(TS_ERR_ARG, "ts_precond_apply: kind must be 2 or 3");
  if (!pr->binv_valid || (kind == 3 && (!pr->hasm_valid || !pr->d_r32)))
    return fail(TS_ERR_ARG, "ts_precond_apply: preconditioner not set up at the current state");
  TS_TRY(sync_dmask(pr));
  const cudaStream_t st = (cudaStream_t)stream;
  return kind == 2 ? block_apply_any(pr, x, z, st) : sgs_apply_any(pr, x, z, st);
}

int ts_jvp(ts_problem* pr, const void* v, void* hv, int precision, void* stream) {
  if (!pr || !v || !hv) return fail(TS_ERR_ARG, "ts_jvp: NULL argument");
  if (precision != 32 && precision != 64) return fail(TS_ERR_ARG, "precision must be 32 or 64");
  if (v == hv) return fail(TS_ERR_ARG, "ts_jvp: v and Hv alias");
  TS_TRY(sync_dmask(pr));
  return jvp_any(pr, v, hv, precision, (cudaStream_t)stream);
}

}  // extern "C"

// ------------------------------------------------------------------ tracer (eq. 3D-weak)

struct ts_tracer {
  const ts_mesh* mesh = nullptr;
  int N = 0, C = 0, NTP = 0;
  double kappa = 0, omega = 0, C_I = 3;
  std::vector<uint8_t> dmask;
  uint8_t* d_dmask = nullptr;
  bool dirty = true;
  double *a4_64 = nullptr, *tau64 = nullptr, *dft64 = nullptr;
  float *a4_32 = nullptr, *tau32 = nullptr, *dft32 = nullptr;
  unsigned* d_counter = nullptr;
  int gls = 1;                       // 0: Galerkin terms only (no least-squares term)
  // solve workspace (FP64)
  double *basis = nullptr, *w = nullptr, *r = nullptr, *dphi = nullptr, *partial = nullptr, *h = nullptr;
  int basis_m = 0;
};

namespace {

template <typename T>
T*& tr_a4(ts_tracer* t);
template <>
double*& tr_a4<double>(ts_tracer* t) { return t->a4_64; }
template <>
float*& tr_a4<float>(ts_tracer* t) { return t->a4_32; }
template <typename T>
T*& tr_tau(ts_tracer* t);
template <>
double*& tr_tau<double>(ts_tracer* t) { return t->tau64; }
template <>
float*& tr_tau<float>(ts_tracer* t) { return t->tau32; }
template <typename T>
T*& tr_dft(ts_tracer* t);
template <>
double*& tr_dft<double>(ts_tracer* t) { return t->dft64; }
template <>
float*& tr_dft<float>(ts_tracer* t) { return t->dft32; }

// advecting velocity and tau of the tracer (once per velocity)
template <typename T, int N>
int tracer_prepare(ts_tracer* tr, const T* a, cudaStream_t st) {
  const ts_mesh* m = tr->mesh;
  T*& a4 = tr_a4<T>(tr);
  T*& tau = tr_tau<T>(tr);
  T*& dft = tr_dft<T>(tr);
  if (!a4) TS_TRY(dalloc(&a4, (size_t)m->V * 4 * tr->C));
  if (!tau) TS_TRY(dalloc(&tau, (size_t)m->E * 4 * tr->NTP));
  if (!dft) {
    std::vector<double> tab;
    dft_tables(N, tab);
    std::vector<T> tt(tab.begin(), tab.end());
    TS_TRY(dalloc(&dft, tt.size()));
    TS_CUDA(cudaMemcpy(dft, tt.data(), tt.size() * sizeof(T), cudaMemcpyHostToDevice));
  }
  if (tr->dirty) {
    TS_CUDA(cudaMemcpy(tr->d_dmask, tr->dmask.data(), tr->dmask.size(), cudaMemcpyHostToDevice));
    tr->dirty = false;
  }
  if (launch_repack_velocity<T>(a, a4, m->V, tr->C, st)) return fail(TS_ERR_CUDA, "repack kernel launch failed");
  int rc;
  if constexpr (sizeof(T) == 8)
    rc = launch_tau_dd<N>(m->d_tets, m->d_geo64, a4, m->E, tau, tr->kappa, tr->C_I, tr->d_counter, st);
  else
    rc = launch_tau<float, N>(m->d_tets, m->d_geo32, a4, m->E, tau, (float)tr->kappa, (float)tr->C_I,
                              tr->d_counter, st);
  if (rc) return fail(TS_ERR_CUDA, "tau kernel launch failed");
  return 0;
}

// r = r(phi) with the prepared velocity and tau
template <typename T, int N>
int tracer_apply(ts_tracer* tr, const T* phi, T* r, cudaStream_t st) {
  const ts_mesh* m = tr->mesh;
  TS_CUDA(cudaMemsetAsync(r, 0, (size_t)m->V * tr->C * sizeof(T), st));
  for (size_t c = 0; c + 1 < m->colour_off.size(); ++c)
    if (launch_tracer<T, N>(m->d_tets, geo_of<T>(m), tr_a4<T>(tr), phi, tr_tau<T>(tr), tr->d_dmask, r,
                            tr_dft<T>(tr), tr->kappa, tr->omega, m->colour_off[c], m->colour_off[c + 1], st,
                            tr->gls))
      return fail(TS_ERR_CUDA, "tracer kernel launch failed");
  return 0;
}

template <typename T, int N>
int tracer_residual_impl(ts_tracer* tr, const T* a, const T* phi, T* r, cudaStream_t st) {
  TS_TRY(tracer_prepare<T, N>(tr, a, st));
  return tracer_apply<T, N>(tr, phi, r, st);
}

double tracer_dnorm(ts_tracer* tr, const double* x, int64_t n, cudaStream_t st, int* rc) {
  *rc = krylov_dots(x, n, 1, x, n, tr->partial, tr->h + 300, st);
  double h = 0;
  if (!*rc) *rc = cudaMemcpyAsync(&h, tr->h + 300, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess;
  if (!*rc) *rc = cudaStreamSynchronize(st) != cudaSuccess;
  return std::sqrt(std::max(h, 0.0));
}

// restarted GMRES (classical Gram-Schmidt, two passes) on the linear tracer
// operator: phi += d with r(phi) + A d = 0, d zero on the Dirichlet nodes
template <int N>
int tracer_solve_impl(ts_tracer* tr, const double* a, double* phi, double tol, int m, int max_matvec,
                      int* matvecs, double* rel, cudaStream_t st) {
  const int64_t n = tr->mesh->V * (int64_t)tr->C;
  if (tr->basis_m < m + 1) {
    dfree(tr->basis);
    TS_TRY(dalloc(&tr->basis, (size_t)(m + 1) * n));
    tr->basis_m = m + 1;
  }
  if (!tr->w) {
    TS_TRY(dalloc(&tr->w, n));
    TS_TRY(dalloc(&tr->r, n));
    TS_TRY(dalloc(&tr->dphi, n));
    TS_TRY(dalloc(&tr->partial, (size_t)krylov_partial_blocks() * 130));
    TS_TRY(dalloc(&tr->h, 512));
  }
  TS_TRY(tracer_prepare<double, N>(tr, a, st));
  TS_TRY(tracer_apply<double, N>(tr, phi, tr->r, st));
  int rc = 0;
  const double bnorm = tracer_dnorm(tr, tr->r, n, st, &rc);
  if (rc) return fail(TS_ERR_CUDA, "tracer solve: norm");
  *matvecs = 0;
  *rel = 1.0;
  if (bnorm == 0) return 0;
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), yk(m);
  TS_CUDA(cudaMemsetAsync(tr->dphi, 0, n * sizeof(double), st));
  // the current linear residual b - A d (b = -r(phi0)) is -w
  TS_CUDA(cudaMemcpyAsync(tr->w, tr->r, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  double beta = bnorm;
  int nmv = 0;
  while (true) {
    if (vec_scale(tr->basis, tr->w, -1.0 / beta, n, st)) return fail(TS_ERR_CUDA, "scale");
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int k_used = 0;
    for (int k = 0; k < m; ++k) {
      TS_TRY(tracer_apply<double, N>(tr, tr->basis + (int64_t)k * n, tr->w, st));
      ++nmv;
      double* h1 = tr->h;
      double* h2 = tr->h + 130;
      if (krylov_dots(tr->basis, n, k + 1, tr->w, n, tr->partial, h1, st) ||
          krylov_sub(tr->w, tr->basis, n, k + 1, h1, n, st) ||
          krylov_dots(tr->basis, n, k + 1, tr->w, n, tr->partial, h2, st) ||
          krylov_sub(tr->w, tr->basis, n, k + 1, h2, n, st) ||
          krylov_dots(tr->w, n, 1, tr->w, n, tr->partial, tr->h + 260, st) ||
          vec_normalise(tr->basis + (int64_t)(k + 1) * n, tr->w, tr->h + 260, n, st))
        return fail(TS_ERR_CUDA, "tracer solve: Gram-Schmidt");
      double hh[391];
      TS_CUDA(cudaMemcpyAsync(hh, tr->h, 261 * sizeof(double), cudaMemcpyDeviceToHost, st));
      TS_CUDA(cudaStreamSynchronize(st));
      double hcol[130];
      for (int j = 0; j <= k; ++j) hcol[j] = hh[j] + hh[130 + j];
      const double hn = std::sqrt(std::max(hh[260], 0.0));
      hcol[k + 1] = hn;
      for (int j = 0; j < k; ++j) {
        const double t = cs[j] * hcol[j] + sn[j] * hcol[j + 1];
        hcol[j + 1] = -sn[j] * hcol[j] + cs[j] * hcol[j + 1];
        hcol[j] = t;
      }
      const double d = std::hypot(hcol[k], hcol[k + 1]);
      cs[k] = d > 0 ? hcol[k] / d : 1.0;
      sn[k] = d > 0 ? hcol[k + 1] / d : 0.0;
      hcol[k] = d;
      for (int j = 0; j <= k; ++j) H[(size_t)j * m + k] = hcol[j];
      g[k + 1] = -sn[k] * g[k];
      g[k] = cs[k] * g[k];
      k_used = k + 1;
      if (std::fabs(g[k + 1]) <= tol * bnorm || nmv >= max_matvec || hn == 0) break;
    }
    for (int i = k_used - 1; i >= 0; --i) {
      double sum = g[i];
      for (int j = i + 1; j < k_used; ++j) sum -= H[(size_t)i * m + j] * yk[j];
      yk[i] = sum / H[(size_t)i * m + i];
    }
    TS_CUDA(cudaMemcpyAsync(tr->h, yk.data(), k_used * sizeof(double), cudaMemcpyHostToDevice, st));
    if (krylov_combine(tr->w, tr->basis, n, k_used, tr->h, n, st)) return fail(TS_ERR_CUDA, "combine");
    if (vec_axpy(tr->dphi, tr->w, 1.0, n, st)) return fail(TS_ERR_CUDA, "axpy");
    // true linear residual: r(phi0) + A d = r(phi0 + d) (the operator is linear)
    if (vec_axpy(phi, tr->dphi, 1.0, n, st)) return fail(TS_ERR_CUDA, "axpy");
    TS_TRY(tracer_apply<double, N>(tr, phi, tr->w, st));
    ++nmv;
    beta = tracer_dnorm(tr, tr->w, n, st, &rc);
    if (rc) return fail(TS_ERR_CUDA, "tracer solve: norm");
    if (vec_axpy(phi, tr->dphi, -1.0, n, st)) return fail(TS_ERR_CUDA, "axpy");
    *rel = beta / bnorm;
    if (beta <= tol * bnorm || nmv >= max_matvec) break;
  }
  if (vec_axpy(phi, tr->dphi, 1.0, n, st)) return fail(TS_ERR_CUDA, "axpy");
  TS_CUDA(cudaStreamSynchronize(st));
  *matvecs = nmv;
  if (*rel > tol) return fail(TS_ERR_NOCONV, "ts_tracer_solve: matvec cap reached");
  return 0;
}

}  // namespace

extern "C" {

int ts_tracer_create(const ts_mesh* mesh, int N, double kappa, double omega, double C_I, ts_tracer** out) {
  if (!out || !mesh) return fail(TS_ERR_ARG, "ts_tracer_create: NULL argument");
  *out = nullptr;
  if (!n_supported(N)) return fail(TS_ERR_UNSUPPORTED, "ts_tracer_create: N not compiled");
  if (!(kappa > 0) || !(omega >= 0) || !(C_I > 0))
    return fail(TS_ERR_ARG, "ts_tracer_create: kappa and C_I must be positive, omega >= 0");
  ts_tracer* t = new ts_tracer();
  t->mesh = mesh;
  t->N = N;
  t->C = 2 * N;
  const int nm = 2 * N - 1;
  t->NTP = ((nm * (nm + 1) / 2) + 3) & ~3;
  t->kappa = kappa;
  t->omega = omega;
  t->C_I = C_I;
  t->dmask.assign(mesh->V, 0);
  if (dalloc(&t->d_dmask, (size_t)mesh->V) || dalloc(&t->d_counter, 1)) {
    ts_tracer_free(t);
    return TS_ERR_OOM;
  }
  cudaMemset(t->d_counter, 0, sizeof(unsigned));
  *out = t;
  return 0;
}

void ts_tracer_free(ts_tracer* t) {
  if (!t) return;
  dfree(t->basis);
  dfree(t->w);
  dfree(t->r);
  dfree(t->dphi);
  dfree(t->partial);
  dfree(t->h);
  dfree(t->d_dmask);
  dfree(t->d_counter);
  dfree(t->a4_64);
  dfree(t->tau64);
  dfree(t->dft64);
  dfree(t->a4_32);
  dfree(t->tau32);
  dfree(t->dft32);
  delete t;
}

int ts_tracer_set_dirichlet(ts_tracer* t, int tag) {
  if (!t) return fail(TS_ERR_ARG, "NULL tracer");
  const ts_mesh* m = t->mesh;
  for (int64_t f = 0; f < m->F; ++f)
    if (m->btag[f] == tag)
      for (int k = 0; k < 3; ++k) t->dmask[m->bfaces[3 * f + k]] = 1;
  t->dirty = true;
  return 0;
}

int ts_tracer_set_stabilised(ts_tracer* t, int gls) {
  if (!t) return fail(TS_ERR_ARG, "NULL tracer");
  if (gls != 0 && gls != 1) return fail(TS_ERR_ARG, "ts_tracer_set_stabilised: 0 or 1");
  t->gls = gls;
  return 0;
}

int ts_tracer_solve(ts_tracer* t, const double* a, double* phi_inout, double tol, int krylov, int max_matvec,
                    int* matvecs_out, double* rel_out, void* stream) {
  if (!t || !a || !phi_inout || !matvecs_out || !rel_out) return fail(TS_ERR_ARG, "ts_tracer_solve: NULL argument");
  if (!(tol > 0) || krylov < 1 || krylov > 128 || max_matvec < 1)
    return fail(TS_ERR_ARG, "ts_tracer_solve: tol > 0, 1 <= krylov <= 128, max_matvec >= 1");
  if (t->dirty) {
    TS_CUDA(cudaMemcpy(t->d_dmask, t->dmask.data(), t->dmask.size(), cudaMemcpyHostToDevice));
    t->dirty = false;
  }
  cudaStream_t st = (cudaStream_t)stream;
  TS_DISPATCH(t->N, (tracer_solve_impl<NN>(t, a, phi_inout, tol, krylov, max_matvec, matvecs_out, rel_out, st)));
}

int ts_tracer_residual(ts_tracer* t, const void* a, const void* phi, void* r, int precision, void* stream) {
  if (!t || !a || !phi || !r) return fail(TS_ERR_ARG, "ts_tracer_residual: NULL argument");
  if (precision != 32 && precision != 64) return fail(TS_ERR_ARG, "precision must be 32 or 64");
  if (phi == r || a == r) return fail(TS_ERR_ARG, "ts_tracer_residual: r aliases an input");
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == 64) {
    TS_DISPATCH(t->N, (tracer_residual_impl<double, NN>(t, (const double*)a, (const double*)phi, (double*)r, st)));
  }
  TS_DISPATCH(t->N, (tracer_residual_impl<float, NN>(t, (const float*)a, (const float*)phi, (float*)r, st)));
}

}  // extern "C"

// ------------------------------------------------------------------ allocation-free residual
// For callers that must not allocate device memory at call time (for example
// code running inside a real-time loop or under an allocator that forbids
// new device allocations): the FP32 residual with tau and tau L held in one
// file-scope device array and the DFT tables in a second, small one, instead
// of the problem's lazily allocated buffers.  Both arrays belong to this
// translation unit's module; ts_problem_create loads that module on the
// current device (looking up the arrays' addresses forces it, also under
// CUDA's lazy module loading), fills the tables once per device and loads the
// two kernels the entry point launches, so the entry point itself only
// launches kernels and clears r.
namespace {

constexpr size_t kNoAllocFloats = (32u << 20) / sizeof(float);   // 32 MiB per device
static __device__ __align__(256) float g_noalloc_scratch[kNoAllocFloats];

constexpr int dft_total_floats() {
  const int list[] = {TS_N_LIST};
  int off = 0;
  for (int n : list) off += 2 * (3 * n - 2) * (2 * n);
  return off;
}
// FP32 DFT tables of every compiled N, each at dft_constant_offset(N)
static __device__ __align__(16) float g_noalloc_dft[dft_total_floats()];

constexpr int kMaxDevices = 64;
struct NoAllocDevice {
  std::atomic<float*> scratch{nullptr};
  std::atomic<float*> dft{nullptr};
};
NoAllocDevice g_noalloc[kMaxDevices];
std::mutex g_noalloc_mutex;

// Device addresses of the two arrays for the current device; the first call
// on a device (made by ts_problem_create) resolves them with that device
// current and uploads the tables.
int noalloc_arrays(float** scratch, float** dft) {
  int dev = 0;
  TS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(TS_ERR_ARG, "allocation-free residual: device index >= 64");
  NoAllocDevice& d = g_noalloc[dev];
  float* s = d.scratch.load(std::memory_order_acquire);
  float* t = d.dft.load(std::memory_order_acquire);
  if (!s || !t) {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    s = d.scratch.load(std::memory_order_acquire);
    t = d.dft.load(std::memory_order_acquire);
    if (!s || !t) {
      void* ps = nullptr;
      void* pt = nullptr;
      TS_CUDA(cudaGetSymbolAddress(&ps, g_noalloc_scratch));
      TS_CUDA(cudaGetSymbolAddress(&pt, g_noalloc_dft));
      std::vector<float> all(dft_total_floats());
      const int list[] = {TS_N_LIST};
      for (int n : list) {
        std::vector<double> tn;
        dft_tables(n, tn);
        std::copy(tn.begin(), tn.end(), all.begin() + dft_constant_offset(n));
      }
      TS_CUDA(cudaMemcpy(pt, all.data(), all.size() * sizeof(float), cudaMemcpyHostToDevice));
      s = static_cast<float*>(ps);
      t = static_cast<float*>(pt);
      d.dft.store(t, std::memory_order_release);
      d.scratch.store(s, std::memory_order_release);
    }
  }
  *scratch = s;
  *dft = t;
  return 0;
}

template <int N>
int noalloc_preload_kernels() {
  if (preload_tau<float, N>() || preload_apply_residual<float, N>())
    return fail(TS_ERR_CUDA, "allocation-free residual: kernel preload failed");
  return 0;
}

// set-up done by ts_problem_create on the problem's device
int noalloc_setup(int N) {
  float *s = nullptr, *t = nullptr;
  TS_TRY(noalloc_arrays(&s, &t));
  TS_DISPATCH(N, (noalloc_preload_kernels<NN>()));
}

template <int N>
int residual_noalloc_impl(ts_problem* pr, const float* y, float* r, cudaStream_t st) {
  constexpr int C = 2 * N;
  const ts_mesh* m = pr->mesh;
  const size_t tau_n = (size_t)m->E * 4 * pr->NTP, tau_pad = (tau_n + 63) & ~(size_t)63;
  const size_t t0_n = (size_t)m->E * 12 * C;
  const size_t need = tau_pad + t0_n;
  if (need > kNoAllocFloats)
    return fail(TS_ERR_ARG, "ts_residual_noalloc: mesh needs " + std::to_string(need * 4) +
                                " bytes of scratch, the fixed array holds " +
                                std::to_string(kNoAllocFloats * 4));
  float *base = nullptr, *tables = nullptr;
  TS_TRY(noalloc_arrays(&base, &tables));
  LinState<float> l;
  l.dft = tables + dft_constant_offset(N);
  l.tau = base;
  l.t0 = l.tau + tau_pad;
  if (launch_tau<float, N>(m->d_tets, m->d_geo32, y, m->E, l.tau, (float)(pr->p.mu / pr->p.rho),
                           (float)pr->p.C_I, pr->d_counter, st))
    return fail(TS_ERR_CUDA, "tau kernel launch failed");
  TS_CUDA(cudaMemsetAsync(r, 0, (size_t)field_len(pr) * sizeof(float), st));
  return apply_colours<float, N>(pr, MODE_RESIDUAL, y, y, l, r, false, st);
}

}  // namespace

extern "C" {

int ts_residual_noalloc(ts_problem* pr, const float* y, float* r, void* stream) {
  if (!pr || !y || !r) return fail(TS_ERR_ARG, "ts_residual_noalloc: NULL argument");
  if ((const void*)y == (const void*)r) return fail(TS_ERR_ARG, "ts_residual_noalloc: y and r alias");
  if (!pr->backflow.empty())
    return fail(TS_ERR_ARG, "ts_residual_noalloc: backflow stabilisation needs ts_residual");
  TS_TRY(sync_dmask(pr));
  cudaStream_t st = (cudaStream_t)stream;
  TS_DISPATCH(pr->p.N, (residual_noalloc_impl<NN>(pr, y, r, st)));
}

// ------------------------------------------------------------------ solve

static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

static int dnorm(ts_problem* pr, const double* x, int64_t n, cudaStream_t st, double* out) {
  if (krylov_dots(x, n, 1, x, n, pr->d_partial, pr->d_h, st)) return fail(TS_ERR_CUDA, "norm");
  double h;
  TS_CUDA(cudaMemcpyAsync(&h, pr->d_h, sizeof(double), cudaMemcpyDeviceToHost, st));
  TS_CUDA(cudaStreamSynchronize(st));
  *out = std::sqrt(std::max(h, 0.0));
  return 0;
}

int ts_solve(ts_problem* pr, void* y_inout, const ts_solve_opts* opts, ts_solve_report* rep,
             void* stream) {
  if (!pr || !y_inout || !opts || !rep) return fail(TS_ERR_ARG, "ts_solve: NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  ts_solve_opts o = *opts;
  if (o.tol <= 0) o.tol = 1e-8;
  if (o.max_steps <= 0) o.max_steps = 200;
  if (o.krylov <= 0) o.krylov = 100;
  if (o.eps_ls <= 0) o.eps_ls = 0.05;
  if (o.max_matvec <= 0) o.max_matvec = 10000;
  if (o.precision != 32 && o.precision != 64) return fail(TS_ERR_ARG, "precision must be 32 or 64");
  if (o.precond < 0 || o.precond > 3) return fail(TS_ERR_ARG, "ts_solve: precond must be 0, 1, 2 or 3");
  std::memset(rep, 0, sizeof(*rep));
  TS_TRY(sync_dmask(pr));
  // the solve's own residuals start tau's eigensolve from the previous step's
  // eigenvectors (TS_OPT_TAU_WARM); the caller's setting returns on exit
  struct WarmGuard {
    ts_problem* p;
    int saved;
    ~WarmGuard() {
      p->tau_warm = saved;
      if (!saved) p->vcache_valid = false;
    }
  } warm_guard{pr, pr->tau_warm};
  pr->tau_warm = 1;
  const int64_t n = field_len(pr);
  const int m = o.krylov;
  if (pr->basis_m < m + 1) {
    dfree(pr->d_basis);
    TS_TRY(dalloc(&pr->d_basis, (size_t)(m + 1) * n));
    pr->basis_m = m + 1;
  }
  if (!pr->d_w) {
    TS_TRY(dalloc(&pr->d_w, n));
    TS_TRY(dalloc(&pr->d_r, n));
    TS_TRY(dalloc(&pr->d_dy, n));
    TS_TRY(dalloc(&pr->d_partial, (size_t)krylov_partial_blocks() * 130));
    TS_TRY(dalloc(&pr->d_h, 3 * 130 + 2));
    TS_TRY(dalloc(&pr->d_v32, n));
    TS_TRY(dalloc(&pr->d_w32, n));
    TS_TRY(dalloc(&pr->d_D, n));
    TS_TRY(dalloc(&pr->d_t, n));
  }
  if (o.krylov > 128) return fail(TS_ERR_ARG, "ts_solve: krylov must be <= 128");
  double* y = (double*)y_inout;
  double* V = pr->d_basis;
  const double t_start = now_s();
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), yk(m);
  double r_ref = o.r_ref;
  int status = TS_ERR_NOCONV;
  int step = 0;
  const double dt0 = pr->p.dt_pseudo;
  const bool ser = o.ser > 0 && dt0 > 0 && std::isfinite(dt0);
  double r_first = -1;
  // step rejection: the last accepted norm, the pseudo-time step factor, and
  // whether the coming residual is the re-evaluation at a restored state
  const bool rejecting = o.reject > 1 && dt0 > 0 && std::isfinite(dt0);
  double rel_acc = -1, backoff = 1.0;
  int n_rej = 0;
  bool retry = false;
  for (step = 0; step <= o.max_steps; ++step) {
    double t0 = now_s();
    TS_TRY(ts_residual(pr, y, pr->d_r, 64, st));
    double rn;
    TS_TRY(dnorm(pr, pr->d_r, n, st, &rn));   // synchronises: the residual's events are complete
    rep->t_residual += now_s() - t0;
    {
      float ms = 0.f;
      if (pr->sev_res && cudaEventElapsedTime(&ms, pr->sev[0], pr->sev[1]) == cudaSuccess) rep->t_tau += ms * 1e-3;
      ++rep->n_residual;
    }
    if (!std::isfinite(rn)) {
      status = fail(TS_ERR_NAN, "ts_solve: non-finite residual norm");
      break;
    }
    if (r_ref <= 0) r_ref = rn;
    double rel = rn / r_ref;
    if (rep->hist_len < 512) rep->hist[rep->hist_len++] = rel;
    rep->r_final = rel;
    if (o.verbose) fprintf(stderr, "[tsgls] step %d |r|/r_ref = %.3e matvecs %d\n", step, rel, rep->matvecs);
    if (rel <= o.tol) {
      status = 0;
      break;
    }
    if (step == o.max_steps) break;
    if (rejecting && !retry && rel_acc > 0 && rel > o.reject * rel_acc && n_rej < 8) {
      // undo the last update; the next pass re-evaluates the residual there
      // and retries with a smaller pseudo-time step
      if (vec_axpy(y, pr->d_dy, -1.0, n, st)) return fail(TS_ERR_CUDA, "axpy");
      backoff *= 0.25;
      ++n_rej;
      ++rep->rejected;
      retry = true;
      continue;
    }
    if (!retry) {
      n_rej = 0;
      if (rel_acc > 0) backoff = std::min(1.0, 2.0 * backoff);
    }
    retry = false;
    rel_acc = rel;
    if (ser) {
      // growth measured from the reference norm: a start closer to the root
      // (a learned guess) begins with the step the plain start would have there
      if (r_first < 0) r_first = o.r_ref > 0 ? o.r_ref : rn;
      double dt = dt0 * std::pow(r_first / rn, o.ser);
      if (o.dt_max > 0 && dt > o.dt_max) dt = o.dt_max;
      dt *= backoff;
      pr->p.dt_pseudo = dt > 1e8 * dt0 ? INFINITY : dt;
    } else if (rejecting) {
      pr->p.dt_pseudo = dt0 * backoff;
    }
    // right preconditioner: approximate inverse diagonal of the tangent, or the
    // inverted nodal diagonal blocks of the tangent at this state
    if (o.precond) {
      const double tp = now_s();
      if (o.precond == 1) TS_TRY(precond_diag(pr, y, pr->d_D, st));
      else if (o.precond == 2) TS_TRY(block_precond_setup(pr, st));
      else TS_TRY(sgs_setup(pr, st));
      TS_CUDA(cudaStreamSynchronize(st));
      rep->t_precond += now_s() - tp;
    }
    // GMRES(m) on (H + c1 rho/dt M) D d' = -r, d = D d', from d = 0
    TS_CUDA(cudaMemsetAsync(pr->d_dy, 0, n * sizeof(double), st));
    double bnorm = rn;
    double beta = rn;
    TS_CUDA(cudaMemcpyAsync(pr->d_w, pr->d_r, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    int nmv = 0;
    bool done = false;
    double lin_res = bnorm;   // last estimate of the linear residual
    while (!done && nmv < o.max_matvec) {
      // V0 = -(current linear residual) / beta ; the residual lives in d_w
      if (vec_scale(V, pr->d_w, -1.0 / beta, n, st)) return fail(TS_ERR_CUDA, "scale");
      std::fill(g.begin(), g.end(), 0.0);
      g[0] = beta;
      int k_used = 0;
      for (int k = 0; k < m; ++k) {
        const double tj = now_s();
        TS_CUDA(cudaEventRecord(pr->ev_a, st));
        double* vk = V + (int64_t)k * n;
        if (o.precond == 1) {
          if (vec_mul(pr->d_t, pr->d_D, vk, n, st)) return fail(TS_ERR_CUDA, "mul");
          vk = pr->d_t;
        } else if (o.precond == 2) {
          TS_TRY(block_apply_any(pr, vk, pr->d_t, st));
          vk = pr->d_t;
        } else if (o.precond == 3) {
          TS_TRY(sgs_apply_any(pr, vk, pr->d_t, st));
          vk = pr->d_t;
        }
        if (o.precision == 32) {
          if (vec_cast_d2f(pr->d_v32, vk, n, st)) return fail(TS_ERR_CUDA, "cast");
          TS_TRY(ts_jvp(pr, pr->d_v32, pr->d_w32, 32, st));
          if (vec_cast_f2d(pr->d_w, pr->d_w32, n, st)) return fail(TS_ERR_CUDA, "cast");
        } else {
          TS_TRY(ts_jvp(pr, vk, pr->d_w, 64, st));
        }
        TS_CUDA(cudaEventRecord(pr->ev_b, st));
        ++nmv;
        // classical Gram-Schmidt and the normalisation, all on the device: one
        // host round trip per iteration returns the column.  The second pass
        // runs only when the first removed more than half of |w|^2 (the test
        // and the skip happen on the device; a skipped pass adds zeros)
        double* dh1 = pr->d_h;
        double* dh2 = pr->d_h + 130;
        double* dn2 = pr->d_h + 260;
        double* dskip = pr->d_h + 390;
        if (krylov_dots(V, n, k + 1, pr->d_w, n, pr->d_partial, dh1, st, 1)) return fail(TS_ERR_CUDA, "dots");
        if (krylov_sub(pr->d_w, V, n, k + 1, dh1, n, st)) return fail(TS_ERR_CUDA, "sub");
        if (krylov_reorth_test(dh1, k + 1, dskip, st)) return fail(TS_ERR_CUDA, "reorth test");
        if (krylov_dots(V, n, k + 1, pr->d_w, n, pr->d_partial, dh2, st, 0, dskip)) return fail(TS_ERR_CUDA, "dots");
        if (krylov_sub(pr->d_w, V, n, k + 1, dh2, n, st, dskip)) return fail(TS_ERR_CUDA, "sub");
        if (krylov_dots(pr->d_w, n, 1, pr->d_w, n, pr->d_partial, dn2, st)) return fail(TS_ERR_CUDA, "norm");
        if (vec_normalise(V + (int64_t)(k + 1) * n, pr->d_w, dn2, n, st)) return fail(TS_ERR_CUDA, "normalise");
        double hh[3 * 130];
        TS_CUDA(cudaMemcpyAsync(hh, pr->d_h, 3 * 130 * sizeof(double), cudaMemcpyDeviceToHost, st));
        TS_CUDA(cudaStreamSynchronize(st));
        float ms_jvp = 0.f;
        cudaEventElapsedTime(&ms_jvp, pr->ev_a, pr->ev_b);
        rep->t_jvp += ms_jvp * 1e-3;
        double tk = now_s();
        rep->t_krylov += (tk - tj) - ms_jvp * 1e-3;
        double hcol[130];
        for (int j = 0; j <= k; ++j) hcol[j] = hh[j] + hh[130 + j];
        const double hn = std::sqrt(std::max(hh[260], 0.0));
        hcol[k + 1] = hn;
        // Givens rotations on the new Hessenberg column
        for (int j = 0; j < k; ++j) {
          double t = cs[j] * hcol[j] + sn[j] * hcol[j + 1];
          hcol[j + 1] = -sn[j] * hcol[j] + cs[j] * hcol[j + 1];
          hcol[j] = t;
        }
        double d = std::hypot(hcol[k], hcol[k + 1]);
        cs[k] = d > 0 ? hcol[k] / d : 1.0;
        sn[k] = d > 0 ? hcol[k + 1] / d : 0.0;
        hcol[k] = d;
        for (int j = 0; j <= k; ++j) H[(size_t)j * m + k] = hcol[j];
        g[k + 1] = -sn[k] * g[k];
        g[k] = cs[k] * g[k];
        k_used = k + 1;
        rep->t_krylov += now_s() - tk;
        if (std::fabs(g[k + 1]) <= o.eps_ls * bnorm || nmv >= o.max_matvec || hn == 0) break;
      }
      // back substitution and update d += V y
      for (int i = k_used - 1; i >= 0; --i) {
        double s = g[i];
        for (int j = i + 1; j < k_used; ++j) s -= H[(size_t)i * m + j] * yk[j];
        yk[i] = s / H[(size_t)i * m + i];
      }
      double tk = now_s();
      TS_CUDA(cudaMemcpyAsync(pr->d_h, yk.data(), k_used * sizeof(double), cudaMemcpyHostToDevice, st));
      if (krylov_combine(pr->d_w, V, n, k_used, pr->d_h, n, st)) return fail(TS_ERR_CUDA, "combine");
      const double* upd = pr->d_w;
      if (o.precond == 1 && vec_mul(pr->d_w, pr->d_D, pr->d_w, n, st)) return fail(TS_ERR_CUDA, "mul");
      if (o.precond == 2) {
        TS_TRY(block_apply_any(pr, pr->d_w, pr->d_t, st));
        upd = pr->d_t;
      } else if (o.precond == 3) {
        TS_TRY(sgs_apply_any(pr, pr->d_w, pr->d_t, st));
        upd = pr->d_t;
      }
      if (vec_axpy(pr->d_dy, upd, 1.0, n, st)) return fail(TS_ERR_CUDA, "axpy");
      rep->t_krylov += now_s() - tk;
      double est = std::fabs(g[k_used]);
      lin_res = est;
      if (est <= o.eps_ls * bnorm || nmv >= o.max_matvec) {
        done = true;
      } else {
        // restart: true linear residual b - J d with b = -r
        double tj = now_s();
        if (o.precision == 32) {
          if (vec_cast_d2f(pr->d_v32, pr->d_dy, n, st)) return fail(TS_ERR_CUDA, "cast");
          TS_TRY(ts_jvp(pr, pr->d_v32, pr->d_w32, 32, st));
          if (vec_cast_f2d(pr->d_w, pr->d_w32, n, st)) return fail(TS_ERR_CUDA, "cast");
        } else {
          TS_TRY(ts_jvp(pr, pr->d_dy, pr->d_w, 64, st));
        }
        ++nmv;
        rep->t_jvp += now_s() - tj;
        // d_w = J d + r  (= -(b - J d)), the scale at the loop head negates it
        if (vec_axpy(pr->d_w, pr->d_r, 1.0, n, st)) return fail(TS_ERR_CUDA, "axpy");
        TS_TRY(dnorm(pr, pr->d_w, n, st, &beta));
        lin_res = beta;
        if (beta <= o.eps_ls * bnorm) done = true;
      }
    }
    rep->matvecs += nmv;
    // a linear solve that stalled (restarted GMRES can stagnate once the mass
    // term has faded): shrink the next pseudo-time step
    if (rejecting && lin_res > 0.5 * bnorm) backoff *= 0.125;
    if (vec_axpy(y, pr->d_dy, 1.0, n, st)) return fail(TS_ERR_CUDA, "axpy");
  }
  pr->p.dt_pseudo = dt0;
  TS_CUDA(cudaStreamSynchronize(st));
  rep->steps = step;
  rep->r_ref = r_ref;
  rep->seconds = now_s() - t_start;
  if (status == TS_ERR_NOCONV) fail(TS_ERR_NOCONV, "ts_solve: step cap reached");
  return status;
}

}  // extern "C"
