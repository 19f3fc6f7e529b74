// double instantiation of the room kernel, blocks of up to HYGRO_MAX_ROOM_WALLS + 1 warps (one room); the
// blocks of linked room groups (up to kRoomBlockWarps warps) are in df1d_rooms_wide_f64.cu, compiled in
// parallel.
#include "df1d_rooms.cuh"

namespace hygro {

cudaError_t launch_rooms_wide_f64(const DevCtx<double> &d, int64_t n0, int32_t n_steps, int32_t sample_every,
                                 double *samples, int n_groups, int warps, cudaStream_t s);

cudaError_t launch_rooms_f64(const DevCtx<double> &d, int64_t n0, int32_t n_steps, int32_t sample_every,
                             double *samples, int n_groups, int warps, cudaStream_t s)
{
    if (warps > HYGRO_MAX_ROOM_WALLS + 1) return launch_rooms_wide_f64(d, n0, n_steps, sample_every, samples, n_groups, warps, s);
    df1d_room_kernel<double, HYGRO_MAX_ROOM_WALLS + 1><<<n_groups, warps * 32, 0, s>>>(d, n0, n_steps, sample_every, samples);
    return cudaGetLastError();
}

}  // namespace hygro
