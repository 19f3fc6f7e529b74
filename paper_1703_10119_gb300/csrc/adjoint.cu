// Launchers of the adjoint kernel (adjoint.cuh) in FP32 and FP64.
#include "adjoint.cuh"

namespace hygro {

template <typename real>
static cudaError_t launch_adjoint(const AdjDev<real> &d, int warps, cudaStream_t s)
{
    const size_t smem = (size_t)warps * adj_smem_per_warp<real>(d.Nmax);
    cudaError_t e = cudaFuncSetAttribute(adjoint_kernel<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int blocks = (d.n_list + warps - 1) / warps;
    adjoint_kernel<real><<<blocks, 32 * warps, smem, s>>>(d);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_f32(const AdjDev<float> &d, int warps, cudaStream_t s) { return launch_adjoint(d, warps, s); }
cudaError_t launch_adjoint_f64(const AdjDev<double> &d, int warps, cudaStream_t s) { return launch_adjoint(d, warps, s); }

}  // namespace hygro
