// FP32 single-launch tangent product (see jvp32.cuh) for N in {1, 2, 3}.
#define J32_NLIST 1, 2, 3
#include "jvp32.cuh"

namespace ts {

int j32_upload_n123(const float* host_all) { return j32_upload_impl(host_all, dft_constant_offset); }

template int launch_jvp32<1>(int, const J32Inst&, cudaStream_t, cudaEvent_t, cudaEvent_t);
template int launch_node_samples<1>(const float*, float*, int64_t, cudaStream_t);
template int launch_jvp32<2>(int, const J32Inst&, cudaStream_t, cudaEvent_t, cudaEvent_t);
template int launch_node_samples<2>(const float*, float*, int64_t, cudaStream_t);
template int launch_jvp32<3>(int, const J32Inst&, cudaStream_t, cudaEvent_t, cudaEvent_t);
template int launch_node_samples<3>(const float*, float*, int64_t, cudaStream_t);

}  // namespace ts
