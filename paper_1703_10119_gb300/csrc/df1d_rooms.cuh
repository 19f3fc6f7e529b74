// Room kernel of the whole-building model: one block per room (or per group of rooms linked by interzone
// airflow), one warp per wall facing a room, and one more warp per room for its air. The coupling is explicit (paper Sec. 5.2): step n of a wall
// takes the room air of level n, and the room's step takes the walls' level-n surface values, so both
// run at the same time. Step n: every wall advances with the room air of level n and publishes its
// level-n+1 surface values, while the room warp advances the room air node in FP64 (Sec. 5.1) from the
// level-n surface values; room air and surface values are double-buffered by level parity, and the
// block synchronises once per step. The room warp computes the outdoor air and vapour production of 32
// steps at a time, one step per lane. Every thread passes one block barrier before the first step and
// one per step (warps without a wall run an empty loop of the same barriers).
#pragma once

#include "df1d_persistent.cuh"

namespace hygro {

// One block per group of rooms (a room alone, or rooms linked by interzone airflow, which exchange their air
// of level n every step through the block's shared memory). NW: warps per block (HYGRO_MAX_ROOM_WALLS + 1
// for single rooms; kRoomBlockWarps for groups).
template <typename real, int NW>
__global__ void __launch_bounds__(NW * 32, 1)
    df1d_room_kernel(const DevCtx<real> d, int64_t n0, int32_t n_steps, int32_t sample_every, real *samples)
{
    __shared__ RoomShared rs[kMaxGroupZones];
    __shared__ real s_tab[NW][kMaxLayers * kLayerStride];
    const RoomGroup &grp = d.groups[blockIdx.x];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    if (threadIdx.x < grp.n_zones) {
        const int r = grp.zone[threadIdx.x];
        RoomShared &z = rs[threadIdx.x];
        z.Ta_p = d.room_state[(size_t)r * 4 + 0];
        z.Ta_c = d.room_state[(size_t)r * 4 + 1];
        z.Pa_p = d.room_state[(size_t)r * 4 + 2];
        z.Pa_c = d.room_state[(size_t)r * 4 + 3];
        z.airT[n0 & 1] = z.Ta_c;
        z.airP[n0 & 1] = z.Pa_c;
    }
    __syncthreads();
    // this warp's role: the air of zone (wib - air_warp0), or wall slot of a zone, or none
    int zone = -1, slot = -1;
    const bool air = wib >= grp.air_warp0 && wib < grp.air_warp0 + grp.n_zones;
    if (air) {
        zone = wib - grp.air_warp0;
    } else {
        for (int z = 0; z < grp.n_zones; ++z) {
            const int first = grp.wall_warp0[z];
            if (wib >= first && wib < first + d.rooms[grp.zone[z]].n_walls) {
                zone = z;
                slot = wib - first;
            }
        }
    }
    bool ran = false;
    if (air) {
        const RoomInfo &ri = d.rooms[grp.zone[zone]];
        RoomShared &z = rs[zone];
        const RoomConst k = room_const(ri, d.faces, d.dt);
        __syncthreads();   // the walls' level-n0 surface values are in rs
        for (int s = 0; s < n_steps; ++s) {
            if (s % kRoomAirChunk == 0) {
                room_air_chunk(z, ri, k, n0 + s, d.t0, d.dt, d.Lv, lane);
                __syncwarp();
            }
            const int b = (int)((n0 + s) & 1);
            if (lane == 0) {
                room_update(z, k, ri, s % kRoomAirChunk, b, d.dt, d.Lv, rs);
                z.airT[b ^ 1] = z.Ta_c;   // level n+1 for the walls' next step
                z.airP[b ^ 1] = z.Pa_c;
            }
            __syncthreads();
        }
        ran = true;
    } else if (slot >= 0) {
        const RoomInfo &ri = d.rooms[grp.zone[zone]];
        const int w = ri.wall[slot];
        const WallInfo wi = d.walls[w];
        for (int i = lane; i < wi.n_layers * kLayerStride; i += 32)
            s_tab[wib][i] = d.layer_tab[(size_t)wi.layer_off * kLayerStride + i];
        __syncwarp();
        const real *tab = s_tab[wib];
        const int face = ri.face[slot];
        // simple-heat walls with one layer per lane (FP32) take the simple variant, the others the general
        // one; a face exchanging long-wave radiation takes the general one (its conductance changes per step)
        const bool rad = ri.view > 0.0 && ri.emis[slot] > 0.0;
        const bool simple = kSimpleVariant<real> && wi.simple && wi.aligned && !rad;
        switch (wi.K * 2 + (simple ? 1 : 0)) {
#define HYGRO_CASE(KK)                                                                                             \
    case 2 * KK:                                                                                                   \
        if (rad)                                                                                                   \
            run_wall<real, KK, true, false, true, true>(d, wi, w, tab, n0, n_steps, sample_every, samples, nullptr, \
                                                        nullptr, &rs[zone], face, slot, &ri);                      \
        else                                                                                                       \
            run_wall<real, KK, true, false, true>(d, wi, w, tab, n0, n_steps, sample_every, samples, nullptr,       \
                                                  nullptr, &rs[zone], face, slot, &ri);                            \
        ran = true;                                                                                                \
        break;                                                                                                     \
    case 2 * KK + 1:                                                                                               \
        run_wall<real, KK, false, kSimpleVariant<real>, true>(d, wi, w, tab, n0, n_steps, sample_every, samples,   \
                                                              nullptr, nullptr, &rs[zone], face, slot, &ri);      \
        ran = true;                                                                                                \
        break;
            HYGRO_CASE(1) HYGRO_CASE(2) HYGRO_CASE(3) HYGRO_CASE(4) HYGRO_CASE(5) HYGRO_CASE(6)
            HYGRO_CASE(7) HYGRO_CASE(8) HYGRO_CASE(9) HYGRO_CASE(10) HYGRO_CASE(11) HYGRO_CASE(12)
            HYGRO_CASE(13) HYGRO_CASE(14) HYGRO_CASE(15) HYGRO_CASE(16)
#undef HYGRO_CASE
            default: break;
        }
    }
    if (!ran) {
        __syncthreads();
        for (int s = 0; s < n_steps; ++s) __syncthreads();
    }
    __syncthreads();
    if (threadIdx.x < grp.n_zones) {
        const int r = grp.zone[threadIdx.x];
        const RoomShared &z = rs[threadIdx.x];
        d.room_state[(size_t)r * 4 + 0] = z.Ta_p;
        d.room_state[(size_t)r * 4 + 1] = z.Ta_c;
        d.room_state[(size_t)r * 4 + 2] = z.Pa_p;
        d.room_state[(size_t)r * 4 + 3] = z.Pa_c;
    }
}

}  // namespace hygro
