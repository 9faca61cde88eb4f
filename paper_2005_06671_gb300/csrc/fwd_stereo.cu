// Forward kernels for polar stereographic tiles.
#include "ss_forward.cuh"
#include "ss_task.cuh"

namespace ss {

cudaError_t launch_dp_forward_stereo(const FwdArgs& a, int block, cudaStream_t s) {
    return dispatch<true, DpLaunch>(a, block, s);
}

cudaError_t launch_uniform_forward_stereo(const FwdArgs& a, int block, cudaStream_t s) {
    return dispatch<true, UniLaunch>(a, block, s);
}

}  // namespace ss
