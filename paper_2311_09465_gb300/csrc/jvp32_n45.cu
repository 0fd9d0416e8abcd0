// FP32 single-launch tangent product (see jvp32.cuh) for N in {4, 5}.
#define J32_NLIST 4, 5
#include "jvp32.cuh"

namespace ts {

int j32_upload_n45(const float* host_all) { return j32_upload_impl(host_all, dft_constant_offset); }

template int launch_jvp32<4>(int, const J32Inst&, cudaStream_t, cudaEvent_t, cudaEvent_t);
template int launch_node_samples<4>(const float*, float*, int64_t, cudaStream_t);
template int launch_jvp32<5>(int, const J32Inst&, cudaStream_t, cudaEvent_t, cudaEvent_t);
template int launch_node_samples<5>(const float*, float*, int64_t, cudaStream_t);

}  // namespace ts
