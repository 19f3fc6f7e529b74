// Room kernel of the whole-building model: one block per room, one warp per wall facing the room, and
// one more warp (the last) for the room air. Each step every wall advances with the room air at level n
// on its room face, then the walls publish their level-n surface values, the block synchronises, the
// room warp advances the room air node in FP64 (paper Sec. 5.1-5.2), and the block synchronises again.
// The room warp computes the outdoor air and vapour production of 32 steps at a time, one step per
// lane, while the walls compute. Every thread passes exactly two block barriers per step (warps
// without a wall run an empty loop of the same barriers).
#pragma once

#include "df1d_persistent.cuh"

namespace hygro {

template <typename real>
__global__ void __launch_bounds__((HYGRO_MAX_ROOM_WALLS + 1) * 32, 1)
    df1d_room_kernel(const DevCtx<real> d, int64_t n0, int32_t n_steps, int32_t sample_every, real *samples)
{
    __shared__ RoomShared rs;
    __shared__ real s_tab[HYGRO_MAX_ROOM_WALLS][kMaxLayers * kLayerStride];
    const int r = blockIdx.x;
    const RoomInfo &ri = d.rooms[r];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        rs.Ta_p = d.room_state[(size_t)r * 4 + 0];
        rs.Ta_c = d.room_state[(size_t)r * 4 + 1];
        rs.Pa_p = d.room_state[(size_t)r * 4 + 2];
        rs.Pa_c = d.room_state[(size_t)r * 4 + 3];
    }
    __syncthreads();
    bool ran = false;
    const int room_warp = (int)(blockDim.x >> 5) - 1;
    if (wib == room_warp) {
        const RoomConst k = room_const(ri, d.faces, d.dt);
        for (int s = 0; s < n_steps; ++s) {
            if (s % kRoomAirChunk == 0) {
                room_air_chunk(rs, ri, k, n0 + s, d.t0, d.dt, d.Lv, lane);
                __syncwarp();
            }
            __syncthreads();   // the walls' level-n surface values are in rs
            if (lane == 0) room_update(rs, k, ri, s % kRoomAirChunk, d.dt, d.Lv);
            __syncthreads();
        }
        ran = true;
    } else if (wib < ri.n_walls) {
        const int w = ri.wall[wib];
        const WallInfo wi = d.walls[w];
        for (int i = lane; i < wi.n_layers * kLayerStride; i += 32)
            s_tab[wib][i] = d.layer_tab[(size_t)wi.layer_off * kLayerStride + i];
        __syncwarp();
        const real *tab = s_tab[wib];
        const int face = ri.face[wib];
        switch (wi.K) {
#define HYGRO_CASE(KK)                                                                                            \
    case KK:                                                                                                      \
        run_wall<real, KK, true, false, true>(d, wi, w, tab, n0, n_steps, sample_every, samples, nullptr, nullptr, \
                                              &rs, face);                                                         \
        ran = true;                                                                                               \
        break;
            HYGRO_CASE(1) HYGRO_CASE(2) HYGRO_CASE(3) HYGRO_CASE(4) HYGRO_CASE(5) HYGRO_CASE(6)
            HYGRO_CASE(7) HYGRO_CASE(8) HYGRO_CASE(9) HYGRO_CASE(10) HYGRO_CASE(11) HYGRO_CASE(12)
            HYGRO_CASE(13) HYGRO_CASE(14) HYGRO_CASE(15) HYGRO_CASE(16)
#undef HYGRO_CASE
            default: break;
        }
    }
    if (!ran)
        for (int s = 0; s < n_steps; ++s) {
            __syncthreads();
            __syncthreads();
        }
    __syncthreads();
    if (threadIdx.x == 0) {
        d.room_state[(size_t)r * 4 + 0] = rs.Ta_p;
        d.room_state[(size_t)r * 4 + 1] = rs.Ta_c;
        d.room_state[(size_t)r * 4 + 2] = rs.Pa_p;
        d.room_state[(size_t)r * 4 + 3] = rs.Pa_c;
    }
}

}  // namespace hygro
