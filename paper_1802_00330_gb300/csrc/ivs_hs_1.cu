// ivs_hs_1.cu -- Hansen-Sengupta kernels for n = 1..6 (see ivs_hs.cuh).
#include "ivs_hs.cuh"

namespace ivs {

cudaError_t launch_hs_dim1(const SweepArgs &a, int num_sms, cudaStream_t st, int *kernels) { return launch_hs_n<1>(a, num_sms, st, kernels); }
cudaError_t launch_hs_dim2(const SweepArgs &a, int num_sms, cudaStream_t st, int *kernels) { return launch_hs_n<2>(a, num_sms, st, kernels); }
cudaError_t launch_hs_dim3(const SweepArgs &a, int num_sms, cudaStream_t st, int *kernels) { return launch_hs_n<3>(a, num_sms, st, kernels); }
cudaError_t launch_hs_dim4(const SweepArgs &a, int num_sms, cudaStream_t st, int *kernels) { return launch_hs_n<4>(a, num_sms, st, kernels); }
cudaError_t launch_hs_dim5(const SweepArgs &a, int num_sms, cudaStream_t st, int *kernels) { return launch_hs_n<5>(a, num_sms, st, kernels); }
cudaError_t launch_hs_dim6(const SweepArgs &a, int num_sms, cudaStream_t st, int *kernels) { return launch_hs_n<6>(a, num_sms, st, kernels); }

}  // namespace ivs
