// ivs_hs_3.cu -- Hansen-Sengupta kernels for n = 11..13 (see ivs_hs.cuh).
#include "ivs_hs.cuh"

namespace ivs {

cudaError_t launch_hs_dim11(const SweepArgs &a, int num_sms, cudaStream_t st, int *kernels) { return launch_hs_n<11>(a, num_sms, st, kernels); }
cudaError_t launch_hs_dim12(const SweepArgs &a, int num_sms, cudaStream_t st, int *kernels) { return launch_hs_n<12>(a, num_sms, st, kernels); }
cudaError_t launch_hs_dim13(const SweepArgs &a, int num_sms, cudaStream_t st, int *kernels) { return launch_hs_n<13>(a, num_sms, st, kernels); }

}  // namespace ivs
