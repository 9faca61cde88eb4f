// Forward kernels for gnomonic tiles (Sec. 3.2).
#include "ss_forward.cuh"
#include "ss_task.cuh"

namespace ss {

cudaError_t launch_dp_forward_gnomonic(const FwdArgs& a, int block, cudaStream_t s) {
    return dispatch<false, DpLaunch>(a, block, s);
}

cudaError_t launch_uniform_forward_gnomonic(const FwdArgs& a, int block, cudaStream_t s) {
    return dispatch<false, UniLaunch>(a, block, s);
}

}  // namespace ss
