// ivs_hs_4.cu -- Hansen-Sengupta kernels for n = 14..16 (see ivs_hs.cuh).
#include "ivs_hs.cuh"

namespace ivs {

cudaError_t launch_hs_dim14(const SweepArgs &a, int num_sms, cudaStream_t st, int *kernels) { return launch_hs_n<14>(a, num_sms, st, kernels); }
cudaError_t launch_hs_dim15(const SweepArgs &a, int num_sms, cudaStream_t st, int *kernels) { return launch_hs_n<15>(a, num_sms, st, kernels); }
cudaError_t launch_hs_dim16(const SweepArgs &a, int num_sms, cudaStream_t st, int *kernels) { return launch_hs_n<16>(a, num_sms, st, kernels); }

}  // namespace ivs
