// Launcher of the register-resident adjoint kernel (adjoint_reg.cuh), float: one warp (block) per wall.
#include "adjoint_reg.cuh"

namespace hygro {

cudaError_t launch_adjoint_reg_f32(const AdjDev<float> &d, cudaStream_t s)
{
    if (d.n_list <= 0) return cudaSuccess;
    adjoint_reg_kernel<float><<<d.n_list, 32, 0, s>>>(d);
    return cudaGetLastError();
}

}  // namespace hygro
