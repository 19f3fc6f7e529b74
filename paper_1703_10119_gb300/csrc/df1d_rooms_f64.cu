// double instantiation of the room kernel.
#include "df1d_rooms.cuh"

namespace hygro {

cudaError_t launch_rooms_f64(const DevCtx<double> &d, int64_t n0, int32_t n_steps, int32_t sample_every,
                             double *samples, int n_rooms, int warps, cudaStream_t s)
{
    df1d_room_kernel<double><<<n_rooms, (warps + 1) * 32, 0, s>>>(d, n0, n_steps, sample_every, samples);
    return cudaGetLastError();
}

}  // namespace hygro
