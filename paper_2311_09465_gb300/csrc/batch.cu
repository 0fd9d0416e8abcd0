// Many instances solved in lockstep (no counterpart in the paper, which
// solves one problem at a time, section 2.5): every GMRES iteration applies
// the FP32 LIN_A tangent of all instances in one fused launch (a work list
// of element tiles, dispatched on each instance's N), runs FP64 classical
// Gram-Schmidt (two passes) as segmented reductions over the concatenated
// Krylov vectors, and normalises on the device.  The device work of an
// iteration is captured once per Krylov index as a CUDA graph and replayed
// across restarts and Newton steps: everything that changes between replays
// (the active instances, mass coefficients, preconditioner) lives in device
// tables.  One host round trip per iteration returns the Hessenberg columns
// of all instances for their Givens rotations.  The launch shape of the
// fused kernel is picked by timing a few candidates (autotune).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "abi_util.h"
#include "kernels.h"

namespace ts {
int problem_j32_inst(ts_problem* pr, J32Inst* I, cudaStream_t st);
int problem_j32_boundary(ts_problem* pr, const float* v, float* hv, cudaStream_t st);
int problem_precond(ts_problem* pr, const double* y, double* D, cudaStream_t st);
int64_t problem_field_len(const ts_problem* pr);
const ts_params* problem_params(const ts_problem* pr);

namespace {

constexpr int CHUNK = 16384;   // elements of a concatenated vector per reduction block
constexpr int BT = 256;
constexpr int MAXM = 128;

// active chunk table: lo, hi (global indices), owning instance
struct ChunkTab {
  const int64_t* lo;
  const int64_t* hi;
  const int* inst;
  const int* count;   // number of active chunks (device scalar)
};

__device__ __forceinline__ double bwarp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// partial[j * max_chunks + c] = sum over chunk c of basis_j . w, j < nvec
__global__ void __launch_bounds__(BT) seg_dots_kernel(ChunkTab ct, int max_chunks, const double* __restrict__ basis,
                                                      int64_t ld, int nvec, const double* __restrict__ w,
                                                      double* __restrict__ partial) {
  const int c = blockIdx.x;
  if (c >= *ct.count) return;
  __shared__ double red[BT / 32][4];
  const int64_t i0 = ct.lo[c], i1 = ct.hi[c];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j0 = 0; j0 < nvec; j0 += 4) {
    const int nj = nvec - j0 < 4 ? nvec - j0 : 4;
    double acc[4] = {0, 0, 0, 0};
    for (int64_t i = i0 + threadIdx.x; i < i1; i += BT) {
      const double wi = w[i];
#pragma unroll
      for (int jj = 0; jj < 4; ++jj)
        if (jj < nj) acc[jj] += basis[(int64_t)(j0 + jj) * ld + i] * wi;
    }
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const double s = bwarp_sum(acc[jj]);
      if (lane == 0) red[warp][jj] = s;
    }
    __syncthreads();
    if (threadIdx.x < nj) {
      double s = 0;
      for (int k = 0; k < BT / 32; ++k) s += red[k][threadIdx.x];
      partial[(int64_t)(j0 + threadIdx.x) * max_chunks + c] = s;
    }
    __syncthreads();
  }
}

// h[b * ldh + j] = sum of partials of instance b's chunks (in chunk order)
__global__ void seg_sum_kernel(const double* __restrict__ partial, int max_chunks, int nvec,
                               const int* __restrict__ first, const int* __restrict__ nchunk, int n_inst,
                               double* __restrict__ h, int ldh) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_inst * nvec) return;
  const int b = t / nvec, j = t - b * nvec;
  double s = 0;
  for (int c = first[b]; c < first[b] + nchunk[b]; ++c) s += partial[(int64_t)j * max_chunks + c];
  h[(int64_t)b * ldh + j] = s;
}

// w -= sum_j basis_j h[b][j] on the active chunks
__global__ void __launch_bounds__(BT) seg_sub_kernel(ChunkTab ct, double* __restrict__ w,
                                                     const double* __restrict__ basis, int64_t ld, int nvec,
                                                     const double* __restrict__ h, int ldh) {
  const int c = blockIdx.x;
  if (c >= *ct.count) return;
  __shared__ double hs[MAXM + 1];
  const int b = ct.inst[c];
  for (int j = threadIdx.x; j < nvec; j += BT) hs[j] = h[(int64_t)b * ldh + j];
  __syncthreads();
  for (int64_t i = ct.lo[c] + threadIdx.x; i < ct.hi[c]; i += BT) {
    double s = w[i];
    for (int j = 0; j < nvec; ++j) s -= basis[(int64_t)j * ld + i] * hs[j];
    w[i] = s;
  }
}

// out = w / sqrt(nrm2[b]) (zero when the norm vanishes)
__global__ void __launch_bounds__(BT) seg_normalise_kernel(ChunkTab ct, double* __restrict__ out,
                                                           const double* __restrict__ w,
                                                           const double* __restrict__ nrm2) {
  const int c = blockIdx.x;
  if (c >= *ct.count) return;
  const double n2 = nrm2[ct.inst[c]];
  const double s = n2 > 0 ? 1.0 / sqrt(n2) : 0.0;
  for (int64_t i = ct.lo[c] + threadIdx.x; i < ct.hi[c]; i += BT) out[i] = w[i] * s;
}

// out = fac[b] * in
__global__ void __launch_bounds__(BT) seg_scale_kernel(ChunkTab ct, double* __restrict__ out,
                                                       const double* __restrict__ in,
                                                       const double* __restrict__ fac) {
  const int c = blockIdx.x;
  if (c >= *ct.count) return;
  const double f = fac[ct.inst[c]];
  for (int64_t i = ct.lo[c] + threadIdx.x; i < ct.hi[c]; i += BT) out[i] = in[i] * f;
}

// v32 = (float)(D * x); w32 = 0
__global__ void __launch_bounds__(BT) seg_precond_cast_kernel(ChunkTab ct, float* __restrict__ v32,
                                                              const double* __restrict__ D,
                                                              const double* __restrict__ x,
                                                              float* __restrict__ w32) {
  const int c = blockIdx.x;
  if (c >= *ct.count) return;
  for (int64_t i = ct.lo[c] + threadIdx.x; i < ct.hi[c]; i += BT) {
    v32[i] = (float)(D[i] * x[i]);
    w32[i] = 0.f;
  }
}

// w = (double)w32 (+ r when add_r)
__global__ void __launch_bounds__(BT) seg_widen_kernel(ChunkTab ct, double* __restrict__ w,
                                                       const float* __restrict__ w32,
                                                       const double* __restrict__ r, int add_r) {
  const int c = blockIdx.x;
  if (c >= *ct.count) return;
  for (int64_t i = ct.lo[c] + threadIdx.x; i < ct.hi[c]; i += BT) w[i] = (double)w32[i] + (add_r ? r[i] : 0.0);
}

// dy += D * sum_j basis_j coef[b][j], j < coef[b][ldc - 1] (instance b's Krylov size:
// basis vectors beyond it were not written in this cycle and are never read)
__global__ void __launch_bounds__(BT) seg_combine_kernel(ChunkTab ct, double* __restrict__ dy,
                                                         const double* __restrict__ D,
                                                         const double* __restrict__ basis, int64_t ld,
                                                         const double* __restrict__ coef, int ldc) {
  const int c = blockIdx.x;
  if (c >= *ct.count) return;
  __shared__ double cs[MAXM + 1];
  const int b = ct.inst[c];
  const int nvec = (int)coef[(int64_t)b * ldc + ldc - 1];
  for (int j = threadIdx.x; j < nvec; j += BT) cs[j] = coef[(int64_t)b * ldc + j];
  __syncthreads();
  for (int64_t i = ct.lo[c] + threadIdx.x; i < ct.hi[c]; i += BT) {
    double s = 0;
    for (int j = 0; j < nvec; ++j) s += basis[(int64_t)j * ld + i] * cs[j];
    dy[i] += D[i] * s;
  }
}

__global__ void __launch_bounds__(BT) seg_cast_kernel(ChunkTab ct, float* __restrict__ v32,
                                                      const double* __restrict__ x, float* __restrict__ w32) {
  const int c = blockIdx.x;
  if (c >= *ct.count) return;
  for (int64_t i = ct.lo[c] + threadIdx.x; i < ct.hi[c]; i += BT) {
    v32[i] = (float)x[i];
    w32[i] = 0.f;
  }
}

__global__ void __launch_bounds__(BT) seg_fill_kernel(ChunkTab ct, double* __restrict__ x, double v) {
  const int c = blockIdx.x;
  if (c >= *ct.count) return;
  for (int64_t i = ct.lo[c] + threadIdx.x; i < ct.hi[c]; i += BT) x[i] = v;
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace
}  // namespace ts

using namespace ts;

struct ts_batch {
  std::vector<ts_problem*> probs;
  int n = 0;
  std::vector<int64_t> len, off;
  int64_t n_tot = 0;
  cudaStream_t st = nullptr;          // own stream (graphs cannot capture the legacy stream)
  cudaEvent_t ev = nullptr;
  // launch shape of the fused tangent kernel
  int warps = 4, blocks = 152 * 8;
  bool tuned = false;
  // instance table and tile prefix of the active set
  std::vector<J32Inst> inst;          // per instance, v/out into the concatenated FP32 vectors
  J32Inst* d_inst = nullptr;
  int64_t* d_tile_off = nullptr;
  int64_t* d_node_off = nullptr;      // node prefix of the fused table (node pre-pass)
  int64_t* d_counts = nullptr;        // {instances, tiles, nodes} of the fused table
  // chunk tables (all instances' chunks; the active ones first)
  int max_chunks = 0;
  int64_t *d_clo = nullptr, *d_chi = nullptr;
  int *d_cinst = nullptr, *d_ccount = nullptr, *d_first = nullptr, *d_nchunk = nullptr;
  // concatenated vectors
  int basis_m = 0;
  double *d_V = nullptr, *d_w = nullptr, *d_r = nullptr, *d_dy = nullptr, *d_D = nullptr;
  float *d_v32 = nullptr, *d_w32 = nullptr;
  double *d_partial = nullptr, *d_h1 = nullptr, *d_h2 = nullptr, *d_nrm = nullptr, *d_fac = nullptr,
         *d_coef = nullptr, *d_nrm_step = nullptr;
  // the active set the device tables currently describe
  std::vector<char> tab_active;
  bool tab_fused = false;
  // graphs per Krylov index
  std::vector<cudaGraphExec_t> graphs;
  std::vector<int> graph_nodes;
};

namespace {

ChunkTab tab(const ts_batch* B) { return ChunkTab{B->d_clo, B->d_chi, B->d_cinst, B->d_ccount}; }

// rebuild the device tables for the instances with active[b] != 0
int set_active(ts_batch* B, const std::vector<char>& active, bool fused_tiles) {
  if (active == B->tab_active && (B->tab_fused || !fused_tiles)) return 0;
  std::vector<int64_t> lo, hi;
  std::vector<int> ci, first(B->n, 0), nch(B->n, 0);
  std::vector<J32Inst> act;
  std::vector<int64_t> toff(1, 0), noff(1, 0);
  for (int b = 0; b < B->n; ++b) {
    if (!active[b]) continue;
    first[b] = (int)lo.size();
    for (int64_t s = 0; s < B->len[b]; s += CHUNK) {
      lo.push_back(B->off[b] + s);
      hi.push_back(B->off[b] + std::min<int64_t>(B->len[b], s + CHUNK));
      ci.push_back(b);
    }
    nch[b] = (int)lo.size() - first[b];
    if (fused_tiles) {
      act.push_back(B->inst[b]);
      toff.push_back(toff.back() + (B->inst[b].n_elem + 1) / 2);
      noff.push_back(noff.back() + B->inst[b].n_nodes);
    }
  }
  const int nc = (int)lo.size();
  TS_CUDA(cudaMemcpyAsync(B->d_clo, lo.data(), nc * sizeof(int64_t), cudaMemcpyHostToDevice, B->st));
  TS_CUDA(cudaMemcpyAsync(B->d_chi, hi.data(), nc * sizeof(int64_t), cudaMemcpyHostToDevice, B->st));
  TS_CUDA(cudaMemcpyAsync(B->d_cinst, ci.data(), nc * sizeof(int), cudaMemcpyHostToDevice, B->st));
  TS_CUDA(cudaMemcpyAsync(B->d_ccount, &nc, sizeof(int), cudaMemcpyHostToDevice, B->st));
  TS_CUDA(cudaMemcpyAsync(B->d_first, first.data(), B->n * sizeof(int), cudaMemcpyHostToDevice, B->st));
  TS_CUDA(cudaMemcpyAsync(B->d_nchunk, nch.data(), B->n * sizeof(int), cudaMemcpyHostToDevice, B->st));
  int64_t counts[3] = {(int64_t)act.size(), toff.back(), noff.back()};
  if (fused_tiles) {
    if (!act.empty()) {
      TS_CUDA(cudaMemcpyAsync(B->d_inst, act.data(), act.size() * sizeof(J32Inst), cudaMemcpyHostToDevice, B->st));
      TS_CUDA(cudaMemcpyAsync(B->d_node_off, noff.data(), noff.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                              B->st));
      TS_CUDA(cudaMemcpyAsync(B->d_tile_off, toff.data(), toff.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                              B->st));
    }
    TS_CUDA(cudaMemcpyAsync(B->d_counts, counts, sizeof(counts), cudaMemcpyHostToDevice, B->st));
  }
  // copies from pageable host memory are staged before cudaMemcpyAsync returns,
  // so the host vectors may go out of scope without a synchronisation
  B->tab_active = active;
  B->tab_fused = fused_tiles;
  return 0;
}

// hv = J v for every instance in the fused table (v32 -> w32), boundary terms included
int fused_tangent(ts_batch* B, const std::vector<char>& active) {
  if (launch_jvp32_batch(B->d_inst, B->d_tile_off, B->d_node_off, B->d_counts, B->warps, B->blocks, B->st))
    return fail(TS_ERR_CUDA, "batched tangent launch failed");
  for (int b = 0; b < B->n; ++b)
    if (active[b])
      TS_TRY(problem_j32_boundary(B->probs[b], B->d_v32 + B->off[b], B->d_w32 + B->off[b], B->st));
  return 0;
}

// segmented dots of nvec basis vectors with w, summed per instance into h [n][ldh]
int seg_dots(ts_batch* B, const double* basis, int nvec, const double* w, double* h, int ldh) {
  count_launches(2);
  seg_dots_kernel<<<B->max_chunks, BT, 0, B->st>>>(tab(B), B->max_chunks, basis, B->n_tot, nvec, w, B->d_partial);
  const int nt = B->n * nvec;
  seg_sum_kernel<<<(nt + 127) / 128, 128, 0, B->st>>>(B->d_partial, B->max_chunks, nvec, B->d_first, B->d_nchunk,
                                                       B->n, h, ldh);
  return cudaGetLastError() == cudaSuccess ? 0 : fail(TS_ERR_CUDA, "segmented dots");
}

// device work of Arnoldi step k: w = J D V_k, two CGS passes into h1/h2, V_{k+1} = w / |w|
int arnoldi_step(ts_batch* B, int k, const std::vector<char>& active) {
  const int ldh = B->basis_m;
  double* Vk = B->d_V + (int64_t)k * B->n_tot;
  count_launches(1);
  seg_precond_cast_kernel<<<B->max_chunks, BT, 0, B->st>>>(tab(B), B->d_v32, B->d_D, Vk, B->d_w32);
  TS_TRY(fused_tangent(B, active));
  count_launches(1);
  seg_widen_kernel<<<B->max_chunks, BT, 0, B->st>>>(tab(B), B->d_w, B->d_w32, nullptr, 0);
  for (int pass = 0; pass < 2; ++pass) {
    double* h = pass == 0 ? B->d_h1 : B->d_h2;
    TS_TRY(seg_dots(B, B->d_V, k + 1, B->d_w, h, ldh));
    count_launches(1);
    seg_sub_kernel<<<B->max_chunks, BT, 0, B->st>>>(tab(B), B->d_w, B->d_V, B->n_tot, k + 1, h, ldh);
  }
  TS_TRY(seg_dots(B, B->d_w, 1, B->d_w, B->d_nrm_step, 1));
  count_launches(1);
  seg_normalise_kernel<<<B->max_chunks, BT, 0, B->st>>>(tab(B), B->d_V + (int64_t)(k + 1) * B->n_tot, B->d_w,
                                                        B->d_nrm_step);
  return cudaGetLastError() == cudaSuccess ? 0 : fail(TS_ERR_CUDA, "arnoldi step");
}

// replay (capturing on first use) the graph of Arnoldi step k
int run_step_graph(ts_batch* B, int k, const std::vector<char>& all_active) {
  if ((int)B->graphs.size() <= k) {
    B->graphs.resize(k + 1, nullptr);
    B->graph_nodes.resize(k + 1, 0);
  }
  if (!B->graphs[k]) {
    const unsigned long long before = launches_total();
    TS_CUDA(cudaStreamBeginCapture(B->st, cudaStreamCaptureModeThreadLocal));
    int rc = arnoldi_step(B, k, all_active);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(B->st, &g);
    // kernels recorded during capture did not run: take them back off the counter
    count_launches(-(int)(launches_total() - before));
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return fail(TS_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(TS_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    B->graphs[k] = ex;
    B->graph_nodes[k] = (int)nn;
  }
  count_launches(B->graph_nodes[k]);
  TS_CUDA(cudaGraphLaunch(B->graphs[k], B->st));
  return 0;
}

void drop_graphs(ts_batch* B) {
  for (auto& g : B->graphs)
    if (g) cudaGraphExecDestroy(g);
  B->graphs.clear();
  B->graph_nodes.clear();
}

int ensure_basis(ts_batch* B, int m) {
  if (B->basis_m >= m + 1) return 0;
  drop_graphs(B);
  dfree(B->d_V);
  dfree(B->d_partial);
  dfree(B->d_h1);
  B->d_h2 = B->d_nrm_step = nullptr;
  dfree(B->d_coef);
  TS_TRY(dalloc(&B->d_V, (size_t)(m + 1) * B->n_tot));
  TS_TRY(dalloc(&B->d_partial, (size_t)(m + 1) * B->max_chunks));
  // h1 [n][m+1], h2 [n][m+1], squared norms [n] in one buffer (one copy back per step)
  TS_TRY(dalloc(&B->d_h1, (size_t)(2 * (m + 1) + 1) * B->n));
  B->d_h2 = B->d_h1 + (size_t)(m + 1) * B->n;
  B->d_nrm_step = B->d_h2 + (size_t)(m + 1) * B->n;
  TS_TRY(dalloc(&B->d_coef, (size_t)(m + 1) * B->n));
  B->basis_m = m + 1;
  return 0;
}

// instance operands (after each residual: mass coefficient, linearisation)
int refresh_inst(ts_batch* B, const std::vector<char>& active) {
  for (int b = 0; b < B->n; ++b) {
    if (!active[b]) continue;
    J32Inst I;
    TS_TRY(problem_j32_inst(B->probs[b], &I, B->st));
    I.v = B->d_v32 + B->off[b];
    I.out = B->d_w32 + B->off[b];
    B->inst[b] = I;
  }
  B->tab_active.clear();   // the fused table must be rewritten with the new operands
  return 0;
}

// time the fused tangent over a few launch shapes; keep the fastest
int autotune(ts_batch* B, const std::vector<char>& active) {
  const int cand_w[] = {2, 4};
  const int cand_b[] = {152 * 4, 152 * 8, 152 * 16, 152 * 32};
  cudaEvent_t e0, e1;
  TS_CUDA(cudaEventCreate(&e0));
  TS_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int bw = B->warps, bb = B->blocks;
  TS_CUDA(cudaMemsetAsync(B->d_v32, 0, B->n_tot * sizeof(float), B->st));
  for (int w : cand_w)
    for (int nb : cand_b) {
      B->warps = w;
      B->blocks = nb;
      TS_CUDA(cudaMemsetAsync(B->d_w32, 0, B->n_tot * sizeof(float), B->st));
      TS_TRY(fused_tangent(B, active));   // warm
      TS_CUDA(cudaEventRecord(e0, B->st));
      for (int r = 0; r < 2; ++r) TS_TRY(fused_tangent(B, active));
      TS_CUDA(cudaEventRecord(e1, B->st));
      TS_CUDA(cudaEventSynchronize(e1));
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        bw = w;
        bb = nb;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  B->warps = bw;
  B->blocks = bb;
  B->tuned = true;
  drop_graphs(B);
  return 0;
}

}  // namespace

namespace {

// instance norms of x over the active chunks into host nrm (sqrt taken)
int seg_norms(ts_batch* B, const double* x, std::vector<double>& nrm) {
  TS_TRY(seg_dots(B, x, 1, x, B->d_nrm, 1));
  nrm.assign(B->n, 0.0);
  TS_CUDA(cudaMemcpyAsync(nrm.data(), B->d_nrm, B->n * sizeof(double), cudaMemcpyDeviceToHost, B->st));
  TS_CUDA(cudaStreamSynchronize(B->st));
  for (double& v : nrm) v = std::sqrt(std::max(v, 0.0));
  return 0;
}

bool any(const std::vector<char>& f) {
  for (char c : f)
    if (c) return true;
  return false;
}

}  // namespace

extern "C" {

int ts_batch_create(ts_problem* const* probs, int n, ts_batch** out) {
  if (!out || !probs || n <= 0) return fail(TS_ERR_ARG, "ts_batch_create: bad argument");
  *out = nullptr;
  ts_batch* B = new ts_batch();
  B->n = n;
  int64_t off = 0;
  int chunks = 0;
  for (int b = 0; b < n; ++b) {
    if (!probs[b]) {
      delete B;
      return fail(TS_ERR_ARG, "ts_batch_create: NULL problem");
    }
    if (problem_params(probs[b])->N > J32_MAX_N) {
      delete B;
      return fail(TS_ERR_UNSUPPORTED, "ts_batch_create: N above the single-launch tangent kernel");
    }
    B->probs.push_back(probs[b]);
    const int64_t len = problem_field_len(probs[b]);
    B->len.push_back(len);
    B->off.push_back(off);
    off += (len + 31) / 32 * 32;   // 256-byte aligned segments
    chunks += (int)((len + CHUNK - 1) / CHUNK);
  }
  B->n_tot = off;
  B->max_chunks = chunks;
  B->inst.resize(n);
  int rc = 0;
  auto cuda_ok = [&](cudaError_t e) { return e == cudaSuccess; };
  if (!cuda_ok(cudaStreamCreateWithFlags(&B->st, cudaStreamNonBlocking)) ||
      !cuda_ok(cudaEventCreateWithFlags(&B->ev, cudaEventDisableTiming)) || j32_batch_configure())
    rc = fail(TS_ERR_CUDA, "ts_batch_create: stream set-up");
  if (!rc && ((rc = dalloc(&B->d_inst, n)) || (rc = dalloc(&B->d_tile_off, n + 1)) ||
              (rc = dalloc(&B->d_node_off, n + 1)) || (rc = dalloc(&B->d_counts, 3)) || (rc = dalloc(&B->d_clo, chunks)) ||
              (rc = dalloc(&B->d_chi, chunks)) || (rc = dalloc(&B->d_cinst, chunks)) ||
              (rc = dalloc(&B->d_ccount, 1)) || (rc = dalloc(&B->d_first, n)) || (rc = dalloc(&B->d_nchunk, n)) ||
              (rc = dalloc(&B->d_w, B->n_tot)) || (rc = dalloc(&B->d_r, B->n_tot)) ||
              (rc = dalloc(&B->d_dy, B->n_tot)) || (rc = dalloc(&B->d_D, B->n_tot)) ||
              (rc = dalloc(&B->d_v32, B->n_tot)) || (rc = dalloc(&B->d_w32, B->n_tot)) ||
              (rc = dalloc(&B->d_nrm, n)) || (rc = dalloc(&B->d_fac, n))))
    ;
  if (!rc && (cudaMemset(B->d_w, 0, B->n_tot * sizeof(double)) != cudaSuccess ||
              cudaMemset(B->d_v32, 0, B->n_tot * sizeof(float)) != cudaSuccess))
    rc = fail(TS_ERR_CUDA, "ts_batch_create: memset");
  if (rc) {
    ts_batch_free(B);
    return rc;
  }
  *out = B;
  return 0;
}

void ts_batch_free(ts_batch* B) {
  if (!B) return;
  if (B->st) cudaStreamSynchronize(B->st);
  drop_graphs(B);
  dfree(B->d_inst);
  dfree(B->d_tile_off);
  dfree(B->d_node_off);
  dfree(B->d_counts);
  dfree(B->d_clo);
  dfree(B->d_chi);
  dfree(B->d_cinst);
  dfree(B->d_ccount);
  dfree(B->d_first);
  dfree(B->d_nchunk);
  dfree(B->d_V);
  dfree(B->d_w);
  dfree(B->d_r);
  dfree(B->d_dy);
  dfree(B->d_D);
  dfree(B->d_v32);
  dfree(B->d_w32);
  dfree(B->d_partial);
  dfree(B->d_h1);
  dfree(B->d_nrm);
  dfree(B->d_fac);
  dfree(B->d_coef);
  if (B->ev) cudaEventDestroy(B->ev);
  if (B->st) cudaStreamDestroy(B->st);
  delete B;
}

int ts_batch_launch_shape(const ts_batch* B, int* warps_per_block, int* blocks) {
  if (!B) return fail(TS_ERR_ARG, "NULL batch");
  if (warps_per_block) *warps_per_block = B->warps;
  if (blocks) *blocks = B->blocks;
  return B->tuned ? 1 : 0;
}

int ts_batch_jvp(ts_batch* B, const float* const* v, float* const* hv, void* stream) {
  if (!B || !v || !hv) return fail(TS_ERR_ARG, "ts_batch_jvp: NULL argument");
  cudaStream_t cs = (cudaStream_t)stream;
  TS_CUDA(cudaEventRecord(B->ev, cs));
  TS_CUDA(cudaStreamWaitEvent(B->st, B->ev, 0));
  std::vector<char> all(B->n, 1);
  TS_TRY(refresh_inst(B, all));
  TS_TRY(set_active(B, all, true));
  for (int b = 0; b < B->n; ++b)
    TS_CUDA(cudaMemcpyAsync(B->d_v32 + B->off[b], v[b], B->len[b] * sizeof(float), cudaMemcpyDeviceToDevice, B->st));
  TS_CUDA(cudaMemsetAsync(B->d_w32, 0, B->n_tot * sizeof(float), B->st));
  TS_TRY(fused_tangent(B, all));
  for (int b = 0; b < B->n; ++b)
    TS_CUDA(cudaMemcpyAsync(hv[b], B->d_w32 + B->off[b], B->len[b] * sizeof(float), cudaMemcpyDeviceToDevice, B->st));
  TS_CUDA(cudaEventRecord(B->ev, B->st));
  TS_CUDA(cudaStreamWaitEvent(cs, B->ev, 0));
  return 0;
}

int ts_batch_solve(ts_batch* B, double* const* y, const ts_solve_opts* opts, ts_solve_report* reps, void* stream) {
  if (!B || !y || !opts || !reps) return fail(TS_ERR_ARG, "ts_batch_solve: NULL argument");
  ts_solve_opts o = *opts;
  if (o.precision != 32) return fail(TS_ERR_ARG, "ts_batch_solve: the batched solve is mixed precision (32)");
  if (o.tol <= 0) o.tol = 1e-8;
  if (o.max_steps <= 0) o.max_steps = 200;
  if (o.krylov <= 0) o.krylov = 100;
  if (o.eps_ls <= 0) o.eps_ls = 0.05;
  if (o.max_matvec <= 0) o.max_matvec = 10000;
  if (o.krylov > MAXM) return fail(TS_ERR_ARG, "ts_batch_solve: krylov must be <= 128");
  const int n = B->n, m = o.krylov;
  for (int b = 0; b < n; ++b)
    if (problem_params(B->probs[b])->jvp_variant != TS_JVP_LIN_A)
      return fail(TS_ERR_UNSUPPORTED, "ts_batch_solve: instances must use the LIN_A tangent");
  TS_TRY(ensure_basis(B, m));
  const int ldh = B->basis_m;
  cudaStream_t cs = (cudaStream_t)stream;
  cudaStream_t st = B->st;
  TS_CUDA(cudaEventRecord(B->ev, cs));
  TS_CUDA(cudaStreamWaitEvent(st, B->ev, 0));
  for (int b = 0; b < n; ++b) std::memset(&reps[b], 0, sizeof(ts_solve_report));
  const double t_start = now_s();
  std::vector<char> live(n, 1), all(n, 1);
  std::vector<double> r_ref(n, o.r_ref), r_first(n, -1.0), dt0(n), rn;
  std::vector<int> status(n, TS_ERR_NOCONV);
  for (int b = 0; b < n; ++b) dt0[b] = problem_params(B->probs[b])->dt_pseudo;
  std::vector<double> H((size_t)n * (m + 1) * m), csn((size_t)n * m), snn((size_t)n * m), g((size_t)n * (m + 1));
  std::vector<double> hbuf((size_t)(2 * ldh + 1) * n), coef((size_t)n * ldh);
  double t_res = 0, t_gm = 0;
  int rc = 0;
  for (int step = 0; step <= o.max_steps && any(live); ++step) {
    // residuals of the live instances, their norms
    double t0 = now_s();
    for (int b = 0; b < n && !rc; ++b)
      if (live[b]) rc = ts_residual(B->probs[b], y[b], B->d_r + B->off[b], 64, st);
    if (rc) break;
    if ((rc = set_active(B, live, false)) || (rc = seg_norms(B, B->d_r, rn))) break;
    t_res += now_s() - t0;
    std::vector<char> gm(n, 0);
    for (int b = 0; b < n; ++b) {
      if (!live[b]) continue;
      ts_solve_report& R = reps[b];
      if (!std::isfinite(rn[b])) {
        status[b] = TS_ERR_NAN;
        live[b] = 0;
        continue;
      }
      if (r_ref[b] <= 0) r_ref[b] = rn[b];
      const double rel = rn[b] / r_ref[b];
      if (R.hist_len < 512) R.hist[R.hist_len++] = rel;
      R.r_final = rel;
      R.steps = step;
      if (rel <= o.tol) {
        status[b] = 0;
        live[b] = 0;
        continue;
      }
      if (step == o.max_steps) {
        live[b] = 0;
        continue;
      }
      const ts_params* P = problem_params(B->probs[b]);
      if (o.ser > 0 && dt0[b] > 0 && std::isfinite(dt0[b])) {
        if (r_first[b] < 0) r_first[b] = o.r_ref > 0 ? o.r_ref : rn[b];
        double dt = dt0[b] * std::pow(r_first[b] / rn[b], o.ser);
        if (o.dt_max > 0 && dt > o.dt_max) dt = o.dt_max;
        ts_problem_set(B->probs[b], dt > 1e8 * dt0[b] ? INFINITY : dt, P->jvp_variant);
      }
      gm[b] = 1;
    }
    if (!any(gm)) break;
    t0 = now_s();
    // preconditioner and tangent operands of the instances in this Newton step
    for (int b = 0; b < n && !rc; ++b)
      if (gm[b] && o.precond) rc = problem_precond(B->probs[b], y[b], B->d_D + B->off[b], st);
    if (rc) break;
    if (!o.precond) {
      if ((rc = set_active(B, gm, false))) break;
      count_launches(1);
      seg_fill_kernel<<<B->max_chunks, BT, 0, st>>>(tab(B), B->d_D, 1.0);
    }
    // every instance needs FP32 operands before the first graph records its boundary terms
    if ((rc = refresh_inst(B, step == 0 ? all : gm))) break;
    if ((rc = set_active(B, gm, true))) break;
    if (!B->tuned && (rc = autotune(B, gm))) break;
    TS_CUDA(cudaMemsetAsync(B->d_dy, 0, B->n_tot * sizeof(double), st));
    TS_CUDA(cudaMemcpyAsync(B->d_w, B->d_r, B->n_tot * sizeof(double), cudaMemcpyDeviceToDevice, st));
    std::vector<double> beta(n), bnorm(n);
    std::vector<int> nmv(n, 0);
    for (int b = 0; b < n; ++b) beta[b] = bnorm[b] = gm[b] ? rn[b] : 0.0;
    std::vector<char> in_gm = gm;
    while (any(in_gm) && !rc) {
      // V_0 = -w / beta
      std::vector<double> fac(n, 0.0);
      for (int b = 0; b < n; ++b)
        if (in_gm[b]) fac[b] = -1.0 / beta[b];
      if ((rc = set_active(B, in_gm, true))) break;
      TS_CUDA(cudaMemcpyAsync(B->d_fac, fac.data(), n * sizeof(double), cudaMemcpyHostToDevice, st));
      count_launches(1);
      seg_scale_kernel<<<B->max_chunks, BT, 0, st>>>(tab(B), B->d_V, B->d_w, B->d_fac);
      for (int b = 0; b < n; ++b) {
        std::fill(g.begin() + (size_t)b * (m + 1), g.begin() + (size_t)(b + 1) * (m + 1), 0.0);
        g[(size_t)b * (m + 1)] = beta[b];
      }
      std::vector<int> k_used(n, 0);
      std::vector<char> cyc = in_gm;
      for (int k = 0; k < m && any(cyc); ++k) {
        if ((rc = set_active(B, cyc, true)) || (rc = run_step_graph(B, k, all))) break;
        TS_CUDA(cudaMemcpyAsync(hbuf.data(), B->d_h1, hbuf.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        TS_CUDA(cudaStreamSynchronize(st));
        const double* h1 = hbuf.data();
        const double* h2 = h1 + (size_t)n * ldh;
        const double* nr = h2 + (size_t)n * ldh;
        for (int b = 0; b < n; ++b) {
          if (!cyc[b]) continue;
          double hcol[MAXM + 2];
          for (int j = 0; j <= k; ++j) hcol[j] = h1[(size_t)b * ldh + j] + h2[(size_t)b * ldh + j];
          const double hn = std::sqrt(std::max(nr[b], 0.0));
          hcol[k + 1] = hn;
          double* cb = &csn[(size_t)b * m];
          double* sb = &snn[(size_t)b * m];
          double* gb = &g[(size_t)b * (m + 1)];
          for (int j = 0; j < k; ++j) {
            const double t = cb[j] * hcol[j] + sb[j] * hcol[j + 1];
            hcol[j + 1] = -sb[j] * hcol[j] + cb[j] * hcol[j + 1];
            hcol[j] = t;
          }
          const double d = std::hypot(hcol[k], hcol[k + 1]);
          cb[k] = d > 0 ? hcol[k] / d : 1.0;
          sb[k] = d > 0 ? hcol[k + 1] / d : 0.0;
          hcol[k] = d;
          for (int j = 0; j <= k; ++j) H[((size_t)b * (m + 1) + j) * m + k] = hcol[j];
          gb[k + 1] = -sb[k] * gb[k];
          gb[k] = cb[k] * gb[k];
          k_used[b] = k + 1;
          ++nmv[b];
          if (std::fabs(gb[k + 1]) <= o.eps_ls * bnorm[b] || nmv[b] >= o.max_matvec || hn == 0) cyc[b] = 0;
        }
      }
      if (rc) break;
      // least-squares solutions, dy += D V y for every instance of this cycle
      std::fill(coef.begin(), coef.end(), 0.0);
      std::vector<char> upd(n, 0);
      for (int b = 0; b < n; ++b) {
        const int ku = k_used[b];
        if (!in_gm[b] || ku == 0) continue;
        upd[b] = 1;
        double* yk = &coef[(size_t)b * ldh];
        const double* gb = &g[(size_t)b * (m + 1)];
        for (int i = ku - 1; i >= 0; --i) {
          double s = gb[i];
          for (int j = i + 1; j < ku; ++j) s -= H[((size_t)b * (m + 1) + i) * m + j] * yk[j];
          yk[i] = s / H[((size_t)b * (m + 1) + i) * m + i];
        }
        yk[ldh - 1] = ku;
      }
      if ((rc = set_active(B, upd, false))) break;
      TS_CUDA(cudaMemcpyAsync(B->d_coef, coef.data(), coef.size() * sizeof(double), cudaMemcpyHostToDevice, st));
      count_launches(1);
      seg_combine_kernel<<<B->max_chunks, BT, 0, st>>>(tab(B), B->d_dy, B->d_D, B->d_V, B->n_tot, B->d_coef, ldh);
      // instances whose linear solve is done leave; the rest restart from the true residual
      std::vector<char> rest(n, 0);
      for (int b = 0; b < n; ++b) {
        if (!in_gm[b]) continue;
        const double est = std::fabs(g[(size_t)b * (m + 1) + k_used[b]]);
        if (est <= o.eps_ls * bnorm[b] || nmv[b] >= o.max_matvec) in_gm[b] = 0;
        else rest[b] = 1;
      }
      if (!any(rest)) break;
      if ((rc = set_active(B, rest, true))) break;
      count_launches(1);
      seg_cast_kernel<<<B->max_chunks, BT, 0, st>>>(tab(B), B->d_v32, B->d_dy, B->d_w32);
      if ((rc = fused_tangent(B, rest))) break;
      count_launches(1);
      seg_widen_kernel<<<B->max_chunks, BT, 0, st>>>(tab(B), B->d_w, B->d_w32, B->d_r, 1);
      std::vector<double> nb;
      if ((rc = seg_norms(B, B->d_w, nb))) break;
      for (int b = 0; b < n; ++b) {
        if (!rest[b]) continue;
        ++nmv[b];
        beta[b] = nb[b];
        if (beta[b] <= o.eps_ls * bnorm[b]) in_gm[b] = 0;
      }
    }
    if (rc) break;
    // y += dy
    if ((rc = set_active(B, gm, false))) break;
    for (int b = 0; b < n; ++b)
      if (gm[b]) {
        if (vec_axpy(y[b], B->d_dy + B->off[b], 1.0, B->len[b], st)) {
          rc = fail(TS_ERR_CUDA, "axpy");
          break;
        }
        reps[b].matvecs += nmv[b];
      }
    t_gm += now_s() - t0;
  }
  cudaStreamSynchronize(st);
  for (int b = 0; b < n; ++b) {
    const ts_params* P = problem_params(B->probs[b]);
    ts_problem_set(B->probs[b], dt0[b], P->jvp_variant);
    reps[b].r_ref = r_ref[b];
    reps[b].seconds = now_s() - t_start;
    reps[b].t_residual = t_res;
    reps[b].t_jvp = t_gm;
  }
  TS_CUDA(cudaEventRecord(B->ev, st));
  TS_CUDA(cudaStreamWaitEvent(cs, B->ev, 0));
  if (rc) return rc;
  for (int b = 0; b < n; ++b)
    if (status[b] == TS_ERR_NAN) return fail(TS_ERR_NAN, "ts_batch_solve: non-finite residual norm");
  for (int b = 0; b < n; ++b)
    if (status[b] != 0) return fail(TS_ERR_NOCONV, "ts_batch_solve: step cap reached for some instances");
  return 0;
}

}  // extern "C"
