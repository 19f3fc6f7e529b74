// double instantiation of the room kernel for blocks of linked room groups (up to kRoomBlockWarps warps).
#include "df1d_rooms.cuh"

namespace hygro {

cudaError_t launch_rooms_wide_f64(const DevCtx<double> &d, int64_t n0, int32_t n_steps, int32_t sample_every,
                                 double *samples, int n_groups, int warps, cudaStream_t s)
{
    if (warps > kRoomBlockWarps) return cudaErrorInvalidValue;
    df1d_room_kernel<double, kRoomBlockWarps><<<n_groups, warps * 32, 0, s>>>(d, n0, n_steps, sample_every, samples);
    return cudaGetLastError();
}

}  // namespace hygro
