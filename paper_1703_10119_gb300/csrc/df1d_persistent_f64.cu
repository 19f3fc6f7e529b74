// FP64 instantiation of the persistent warp-per-wall DF kernel.
#include "df1d_persistent.cuh"

namespace hygro {

cudaError_t launch_persistent_f64(const DevCtx<double> &d, int64_t n0, int32_t n_steps, int32_t sample_every,
                                  double *samples, int grid, cudaStream_t s)
{
    df1d_persistent_kernel<double><<<grid, PersistCfg<double>::warps * 32, persistent_smem_bytes<double>(), s>>>(d, n0, n_steps, sample_every, samples);
    return cudaGetLastError();
}

cudaError_t occupancy_persistent_f64(int *blocks_per_sm)
{
    cudaError_t e = cudaFuncSetAttribute(df1d_persistent_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)persistent_smem_bytes<double>());
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, df1d_persistent_kernel<double>,
                                                         PersistCfg<double>::warps * 32, persistent_smem_bytes<double>());
}

}  // namespace hygro
