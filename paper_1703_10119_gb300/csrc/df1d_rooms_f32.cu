// float instantiation of the room kernel.
#include "df1d_rooms.cuh"

namespace hygro {

cudaError_t launch_rooms_f32(const DevCtx<float> &d, int64_t n0, int32_t n_steps, int32_t sample_every,
                             float *samples, int n_rooms, int warps, cudaStream_t s)
{
    df1d_room_kernel<float><<<n_rooms, (warps + 1) * 32, 0, s>>>(d, n0, n_steps, sample_every, samples);
    return cudaGetLastError();
}

}  // namespace hygro
