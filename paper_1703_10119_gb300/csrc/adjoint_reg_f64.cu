// Launcher of the register-resident adjoint kernel (adjoint_reg.cuh), double: one warp (block) per wall.
#include "adjoint_reg.cuh"

namespace hygro {

cudaError_t launch_adjoint_reg_f64(const AdjDev<double> &d, cudaStream_t s)
{
    if (d.n_list <= 0) return cudaSuccess;
    adjoint_reg_kernel<double><<<d.n_list, 32, 0, s>>>(d);
    return cudaGetLastError();
}

}  // namespace hygro
