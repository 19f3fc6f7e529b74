// FP32 instantiation of the persistent warp-per-wall DF kernel.
#include "df1d_persistent.cuh"

namespace hygro {

cudaError_t launch_persistent_f32(const DevCtx<float> &d, int64_t n0, int32_t n_steps, int32_t sample_every,
                                  float *samples, int32_t *queue_counter, int grid, cudaStream_t s)
{
    df1d_persistent_kernel<float><<<grid, kWarpsPerBlock * 32, 0, s>>>(d, n0, n_steps, sample_every, samples,
                                                                       queue_counter);
    return cudaGetLastError();
}

cudaError_t occupancy_persistent_f32(int *blocks_per_sm)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, df1d_persistent_kernel<float>,
                                                         kWarpsPerBlock * 32, 0);
}

}  // namespace hygro
