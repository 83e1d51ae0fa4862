// ivs_hs_2.cu -- Hansen-Sengupta kernels for n = 7..10 (see ivs_hs.cuh).
#include "ivs_hs.cuh"

namespace ivs {

cudaError_t launch_hs_dim7(const SweepArgs &a, int num_sms, cudaStream_t st, int *kernels) { return launch_hs_n<7>(a, num_sms, st, kernels); }
cudaError_t launch_hs_dim8(const SweepArgs &a, int num_sms, cudaStream_t st, int *kernels) { return launch_hs_n<8>(a, num_sms, st, kernels); }
cudaError_t launch_hs_dim9(const SweepArgs &a, int num_sms, cudaStream_t st, int *kernels) { return launch_hs_n<9>(a, num_sms, st, kernels); }
cudaError_t launch_hs_dim10(const SweepArgs &a, int num_sms, cudaStream_t st, int *kernels) { return launch_hs_n<10>(a, num_sms, st, kernels); }

}  // namespace ivs
