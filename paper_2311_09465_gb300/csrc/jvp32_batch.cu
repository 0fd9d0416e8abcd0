// Batched FP32 tangent products (LIN_A) of many instances: one node pre-pass
// over all instances' nodes, then one element launch over a work list of
// element tiles of all instances, dispatched per tile on the instance's N
// (see jvp32_batch_kernel in jvp32.cuh).
#define J32_NLIST 1, 2, 3, 4, 5, 7
#include "jvp32.cuh"

namespace ts {

int j32_upload_batch(const float* host_all) { return j32_upload_impl(host_all, dft_constant_offset); }

size_t j32_batch_warp_bytes() { return J32Layout<J32_MAX_N, MODE_JVP_LIN_A>::WARP * sizeof(float); }

// allows launches of up to 4 warps per block (call once, outside graph capture)
int j32_batch_configure() {
  auto kern = jvp32_batch_kernel<MODE_JVP_LIN_A, J32_MAX_N>;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(4 * j32_batch_warp_bytes())) == cudaSuccess ? 0 : -2;
}

int launch_jvp32_batch(const J32Inst* d_insts, const int64_t* d_tile_off, const int64_t* d_node_off,
                       const int64_t* d_counts, int warps_per_block, int blocks, cudaStream_t st) {
  if (warps_per_block < 1 || warps_per_block > 4 || blocks < 1) return -1;
  const size_t smem = (size_t)warps_per_block * j32_batch_warp_bytes();
  auto kern = jvp32_batch_kernel<MODE_JVP_LIN_A, J32_MAX_N>;
  count_launches(2);
  // node pre-pass of every instance (v sampled into each instance's vt), then the element pass
  node_samples_batch_kernel<<<152 * 8, 128, 0, st>>>(d_insts, d_node_off, d_counts);
  kern<<<blocks, warps_per_block * 32, smem, st>>>(d_insts, d_tile_off, d_counts);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace ts
