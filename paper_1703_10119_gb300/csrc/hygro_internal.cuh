// Internal data layout of the hygro library (device side and launch helpers).
//
// A context stores every wall's two time levels (n and n-1) of T and Pv as
// deviations from a per-wall reference state (the initial state), in the
// working precision (float or double). Deviations keep the FP32 arithmetic
// on O(1..100) numbers instead of O(300..1000) ones: the coefficients are
// affine in Pv, so the reference only shifts their constant parts.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/hygro.h"

namespace hygro {

constexpr int kMaxLayers = HYGRO_MAX_LAYERS;
constexpr int kLayerStride = 12;   // reals per layer entry of a wall (9 used, padded)
constexpr int kMaxK = 16;          // nodes per lane of the persistent kernel
// Persistent kernel: one wall per warp; warps per block by precision. FP32 runs 16 warps (four per SM
// sub-partition, 128 registers): the variants with many nodes per lane spill a little, but the extra
// warps hide more latency than 12 warps at 168 registers (measured on the yearly batch). FP64 needs
// the 255-register budget of 8 warps.
template <typename real>
struct PersistCfg {
    static constexpr int warps = sizeof(real) == 4 ? 16 : 8;
};
// Dynamic shared memory of the persistent kernel per warp (in reals): layer table, then two per-slot
// tables of 32 lanes x kMaxK slots.
constexpr int kSmemRealsPerWarp = kMaxLayers * kLayerStride + 2 * kMaxK * 32;
template <typename real>
constexpr size_t persistent_smem_bytes()
{
    return (size_t)PersistCfg<real>::warps * kSmemRealsPerWarp * sizeof(real);
}
constexpr int kForcingBatch = 16;  // steps of ambient forcing computed per warp-wide batch

// Layer entry of one wall, in the wall's deviation variables (P' = Pv - P_ref):
//   [0] kMh_a, [1] kMh_b : kM  / (2 dx) = kMh_a + kMh_b P'
//   [2] kTh_a, [3] kTh_b : kTT / (2 dx)
//   [4] A_a,   [5] A_b   : dx cM  / (2 dt)
//   [6] B_a,   [7] B_b   : dx cTT / (2 dt)
//   [8] chi             : cTM / cM
enum { LT_KMA = 0, LT_KMB, LT_KTA, LT_KTB, LT_AA, LT_AB, LT_BA, LT_BB, LT_CHI };

struct WallInfo {
    int32_t N;            // nodes
    int32_t K;            // persistent kernel: nodes per lane
    int32_t Wl;           // persistent kernel: lanes holding nodes (lane Wl-1 always holds K)
    uint32_t short_mask;  // persistent kernel: bit i set when lane i holds K-1 nodes
    int32_t node_off;     // first node in the concatenated field arrays
    int32_t n_layers;
    int32_t layer_off;    // first layer entry of this wall
    int16_t aligned;      // 1 when every layer interface falls on a lane boundary
    int16_t simple;       // 1 when kTT, cTT do not depend on Pv and cTM = 0 in every layer, and nu = 1
    double nu;            // latent share of kM: kTM = nu Lv kM at the faces inside the wall
    double dx;            // node spacing (m)
    int32_t has_law;      // 1 when some layer takes a Table-1 coefficient law (plain kernel only)
    int32_t pad_;
};

struct FaceInfo {
    int32_t kind;       // HYGRO_BC_*
    int32_t room;
    int32_t noise_len;
    int32_t pad;
    int64_t noise_off;  // first (T, Pv) pair of this face's table in the context's noise array
    double hT, hM, q_inf, g_inf;     // exchange coefficients (0 for adiabatic faces)
    double T_mean_dev, T_amp;        // T_mean - T_ref
    double P_mean_dev, P_amp;        // P_mean - P_ref
    double period, phase_T, phase_P, noise_dt;
    double period_P;      // period of the Pv sinusoid (0: none)
    // fixed-point forms used by the FP32 kernels:
    uint64_t phT0, phP0;  // fraction of a period at step 0, scaled by 2^64 (sinusoid phase incl. phase_T/P)
    uint64_t pstep;       // fraction of the T period per step, scaled by 2^64
    uint64_t pstepP;      // fraction of the Pv period per step, scaled by 2^64
    int64_t npos0;        // noise table position at step 0, scaled by 2^40
    int64_t nstep;        // noise table positions per step, scaled by 2^40
    int64_t n_hi;         // first step whose position reaches the last table entry (held from there on)
};

constexpr int kMaxZoneLinks = 3;     // interzone links of one room
constexpr int kMaxGroupZones = 4;    // rooms of one block of the room kernel (rooms linked by airflow)
constexpr int kRoomBlockWarps = 16;  // warps of the room kernel's block for rooms linked by airflow

// A room and the walls facing it (room kernel: one warp per wall, one more for the room air).
struct RoomInfo {
    int32_t n_walls;
    int32_t wall[HYGRO_MAX_ROOM_WALLS];   // ascending wall indices
    int32_t face[HYGRO_MAX_ROOM_WALLS];   // which face of the wall is on the room
    double area[HYGRO_MAX_ROOM_WALLS];    // m^2
    double par[21];                       // hygro_room fields volume .. Pv_ref, the room scheme, then
                                          // period_P, g_pulse, pulse_on, pulse_off, pulse_period
    // long-wave exchange among the room's wall surfaces: view factor s (0: none) and each wall face's
    // emissivity
    double view;
    double emis[HYGRO_MAX_ROOM_WALLS];
    // interzone airflow: the linked rooms (their positions in the block's group) and the flows, kg/s
    int32_t n_links;
    int32_t link_slot[kMaxZoneLinks];
    double link_g[kMaxZoneLinks];
    double link_gw[kMaxZoneLinks];        // link_g / Pv_ref of the linked room (its humidity ratio w = Pv / Pv_ref)
};

// The rooms one block of the room kernel runs together (rooms linked by airflow share a block). Warps
// wall_warp0[z] .. wall_warp0[z] + n_walls - 1 advance room z's walls, warp air_warp0 + z its air.
struct RoomGroup {
    int32_t n_zones;
    int32_t zone[kMaxGroupZones];
    int32_t wall_warp0[kMaxGroupZones];
    int32_t air_warp0;
    int32_t n_warps;
};
enum { RP_VOL = 0, RP_ACH, RP_QGAIN, RP_GVAP, RP_TMEAN, RP_TAMP, RP_PMEAN, RP_PAMP, RP_PERIOD, RP_PHT, RP_PHP,
       RP_RHOA, RP_CPA, RP_CPV, RP_PVREF, RP_SCHEME, RP_PERIODP, RP_GPULSE, RP_PON, RP_POFF, RP_PPER };

template <typename real>
struct DevCtx {
    const WallInfo *walls;       // [W]
    const FaceInfo *faces;       // [W][2]
    const real *layer_tab;       // [sum layers][kLayerStride]
    const int32_t *layer_first;  // [sum layers]
    const float2 *noise;         // noise tables
    real *T[2];                  // level buffers: T[cur] level n, T[1-cur] level n-1
    real *P[2];
    int32_t cur;
    int32_t W;
    const real *Tref;            // [W]
    const real *Pref;            // [W]
    double *cumul;               // [W][2][2] running sums of dt * flux, FP64
    double *flast;               // [W][2][2] flux of the last step
    int32_t *nonfinite;          // set to 1 when a wall turns non-finite
    const int32_t *order;        // walls of the persistent blocks in rounds of round_size (-1: empty entry)
    const int32_t *block_off;    // [grid + 1] first entry of each persistent block's rounds in order
    int32_t round_size;          // walls per round (warp i of a block takes entry i of each of its rounds)
    unsigned long long *trace;   // optional [W][4]: SM id << 32 | block << 8 | warp, start ns, end ns, steps
    const RoomInfo *rooms;       // [n_rooms] (room kernel)
    const RoomGroup *groups;     // [n_groups] (room kernel: one block each)
    double *room_state;          // [n_rooms][4]: Ta(n-1), Ta(n), Pa(n-1), Pa(n)
    int32_t n_rooms;
    const int32_t *node_wall;    // [total nodes] (plain kernel)
    const int8_t *node_layer;    // [total nodes] (plain kernel)
    const int8_t *layer_law;     // [sum layers] HYGRO_LAW_* of each layer (plain kernel; walls with has_law)
    int32_t total_nodes;
    double dt, t0, Lv;
};

// Host helpers shared by the 1D and 2D entry points (hygro_api.cu).
// The entry points' plain cudaMemcpy / cudaMemset calls go to the legacy default stream. A non-blocking
// context stream (PyTorch's streams are) does not follow it, and a copy from pageable memory may return
// before its last transfer lands, so an entry point that enqueues kernels on such a stream first waits for
// the legacy stream. Returns at once for the legacy stream itself, for a blocking stream (which follows the
// legacy one), and while the stream is being captured into a graph.
cudaError_t after_host_copies(cudaStream_t stream);
// Validates one face description (kind, coefficients, noise table against the time step, and the
// table's values finite unless scan_noise is false, for a caller that checks them while copying);
// room faces only where allow_room. Returns HYGRO_OK, or an error status with the reason in *why.
hygro_status check_bc(const hygro_bc &b, bool allow_room, double t0, double dt, std::string *why,
                      bool scan_noise = true);
// Device form of one face in the deviation variables of its wall or section (reference T_ref, P_ref),
// with its noise table at noise_off of the context's noise array.
FaceInfo face_info(const hygro_bc &b, double T_ref, double P_ref, double t0, double dt, int64_t noise_off,
                   int64_t noise_len);

// Launchers (defined in the kernel translation units). All are stream-ordered.
cudaError_t launch_persistent_f32(const DevCtx<float> &d, int64_t n0, int32_t n_steps, int32_t sample_every,
                                  float *samples, int grid, cudaStream_t s);
cudaError_t launch_persistent_f64(const DevCtx<double> &d, int64_t n0, int32_t n_steps, int32_t sample_every,
                                  double *samples, int grid, cudaStream_t s);
cudaError_t occupancy_persistent_f32(int *blocks_per_sm);
cudaError_t occupancy_persistent_f64(int *blocks_per_sm);

// n_groups blocks of `warps` warps (<= HYGRO_MAX_ROOM_WALLS + 1: the single-room form; <= kRoomBlockWarps: the
// form for rooms linked by airflow).
cudaError_t launch_rooms_f32(const DevCtx<float> &d, int64_t n0, int32_t n_steps, int32_t sample_every,
                             float *samples, int n_groups, int warps, cudaStream_t s);
cudaError_t launch_rooms_f64(const DevCtx<double> &d, int64_t n0, int32_t n_steps, int32_t sample_every,
                             double *samples, int n_groups, int warps, cudaStream_t s);

template <typename real>
struct AdjDev;
cudaError_t launch_adjoint_f32(const AdjDev<float> &d, int warps, cudaStream_t s);
cudaError_t launch_adjoint_f64(const AdjDev<double> &d, int warps, cudaStream_t s);
cudaError_t launch_adjoint_reg_f32(const AdjDev<float> &d, cudaStream_t s);
cudaError_t launch_adjoint_reg_f64(const AdjDev<double> &d, cudaStream_t s);

cudaError_t launch_balance_f32(const DevCtx<float> &d, const float *Tp, const float *Pp, const float *Tn,
                               const float *Pn, int64_t n, double *bal, cudaStream_t s);
cudaError_t launch_balance_f64(const DevCtx<double> &d, const double *Tp, const double *Pp, const double *Tn,
                               const double *Pn, int64_t n, double *bal, cudaStream_t s);

cudaError_t launch_euler_start_f32(const DevCtx<float> &d, int Nmax, int64_t max_sub, int64_t *m_out, cudaStream_t s);
cudaError_t launch_euler_start_f64(const DevCtx<double> &d, int Nmax, int64_t max_sub, int64_t *m_out, cudaStream_t s);

cudaError_t launch_plain_step_f32(const DevCtx<float> &d, int64_t n, int32_t sample_idx, float *samples,
                                  cudaStream_t s);
cudaError_t launch_plain_step_f64(const DevCtx<double> &d, int64_t n, int32_t sample_idx, double *samples,
                                  cudaStream_t s);

}  // namespace hygro
