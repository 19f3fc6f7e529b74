// C-ABI of the hygro library: argument validation, device layout of a batch
// of walls, and the launches of the DF kernels (see include/hygro.h).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "hygro_internal.cuh"
#include "host_layout.h"
#include "host_noise.h"
#include "host_fault.h"
#include "host_forcing.h"
#include "adjoint_reg.cuh"

using namespace hygro;

static_assert(kLayoutMaxK == kMaxK, "lane layout and kernel disagree on the most nodes per lane");

namespace {

thread_local std::string g_create_error = "no error";

struct RawBc {
    hygro_bc bc;                 // noise pointer not kept
    int64_t noise_off = 0;       // first (T, Pv) pair of this wall's table in its face's region of the
                                 // context's noise array
    int64_t noise_len = 0;       // pairs (0: no table, or not an ambient face)
};

template <typename T>
cudaError_t dalloc(T **p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void **)p, count * sizeof(T));
}

bool is_device_ptr(const void *p)
{
    if (p == nullptr) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

bool finite_nonneg(double x) { return std::isfinite(x) && x >= 0.0; }

}  // namespace

namespace hygro {

cudaError_t after_host_copies(cudaStream_t stream)
{
    if (stream == nullptr) return cudaSuccess;
    // first the capture status: the one query made while a graph may be being captured
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess) {
        (void)cudaGetLastError();   // leave no error behind for the launchers' cudaGetLastError
        cs = cudaStreamCaptureStatusNone;
    }
    if (cs != cudaStreamCaptureStatusNone) return cudaSuccess;
    unsigned int flags = 0;
    if (cudaStreamGetFlags(stream, &flags) != cudaSuccess) {
        (void)cudaGetLastError();
        flags = cudaStreamNonBlocking;
    }
    if (!(flags & cudaStreamNonBlocking)) return cudaSuccess;
    return cudaStreamSynchronize(cudaStreamLegacy);
}

hygro_status check_bc(const hygro_bc &b, bool allow_room, double t0, double dt, std::string *why, bool scan_noise)
{
    if (b.kind == HYGRO_BC_ROOM && !allow_room) {
        *why = "room faces are not accepted here";
        return HYGRO_E_INVALID;
    }
    if (b.kind == HYGRO_BC_ROOM && b.room < 0) {
        *why = "room index must be >= 0";
        return HYGRO_E_INVALID;
    }
    if (b.kind != HYGRO_BC_AMBIENT && b.kind != HYGRO_BC_ADIABATIC && b.kind != HYGRO_BC_ROOM) {
        *why = "unknown kind " + std::to_string(b.kind);
        return HYGRO_E_INVALID;
    }
    if (b.kind == HYGRO_BC_ADIABATIC) return HYGRO_OK;
    if (!finite_nonneg(b.hT) || !finite_nonneg(b.hM)) {
        *why = "hT and hM must be finite and >= 0";
        return HYGRO_E_INVALID;
    }
    const double v[] = {b.q_inf, b.g_inf, b.T_mean, b.T_amp, b.P_mean, b.P_amp, b.phase_T, b.phase_P};
    for (double x : v)
        if (!std::isfinite(x)) {
            *why = "non-finite value";
            return HYGRO_E_INVALID;
        }
    if (!finite_nonneg(b.period) || !finite_nonneg(b.period_P)) {
        *why = "period and period_P must be >= 0";
        return HYGRO_E_INVALID;
    }
    if (b.noise_len < 0) {
        *why = "noise_len < 0";
        return HYGRO_E_INVALID;
    }
    if (b.noise_len > 0) {
        if (b.noise == nullptr) {
            *why = "noise is NULL";
            return HYGRO_E_INVALID;
        }
        if (!(std::isfinite(b.noise_dt) && b.noise_dt > 0)) {
            *why = "noise_dt must be > 0";
            return HYGRO_E_INVALID;
        }
        if (b.noise_len > (1 << 22) || std::fabs(t0 / b.noise_dt) > 4.0e6 || dt / b.noise_dt > 4.0e6) {
            *why = "noise table too long for its time step";
            return HYGRO_E_UNSUPPORTED;
        }
        // branch-free scan, which the compiler vectorises: a float is finite unless its exponent bits
        // are all ones
        const int64_t n = scan_noise ? 2 * (int64_t)b.noise_len : 0;
        uint32_t bad = 0;
        for (int64_t k = 0; k < n; ++k) {
            uint32_t u;
            memcpy(&u, b.noise + k, sizeof u);
            bad |= (uint32_t)((u & 0x7f800000u) == 0x7f800000u);
        }
        if (bad) {
            *why = "non-finite noise";
            return HYGRO_E_INVALID;
        }
    }
    return HYGRO_OK;
}

FaceInfo face_info(const hygro_bc &b, double T_ref, double P_ref, double t0, double dt, int64_t noise_off,
                   int64_t noise_len)
{
    FaceInfo o;
    memset(&o, 0, sizeof o);
    o.kind = b.kind;
    o.room = b.room;
    if (b.kind == HYGRO_BC_ADIABATIC) return o;
    o.hT = b.hT;
    o.hM = b.hM;
    o.q_inf = b.q_inf;
    o.g_inf = b.g_inf;
    o.T_mean_dev = b.T_mean - T_ref;
    o.T_amp = b.T_amp;
    o.P_mean_dev = b.P_mean - P_ref;
    o.P_amp = b.P_amp;
    o.period = b.period > 0 ? b.period : 0.0;
    const double pP = b.period_P > 0 ? b.period_P : b.period;
    o.period_P = pP > 0 ? pP : 0.0;
    o.phase_T = b.phase_T;
    o.phase_P = b.phase_P;
    o.noise_dt = b.noise_dt;
    const double two_pi = 6.283185307179586476925286766559;
    if (o.period > 0) {
        o.phT0 = turns_fixed(t0 / o.period + b.phase_T / two_pi);
        o.pstep = turns_fixed(dt / o.period);
    }
    if (o.period_P > 0) {
        o.phP0 = turns_fixed(t0 / o.period_P + b.phase_P / two_pi);
        o.pstepP = turns_fixed(dt / o.period_P);
    }
    if (noise_len > 0) {
        o.noise_len = (int32_t)noise_len;
        o.noise_off = noise_off;
        const NoiseFixed nf = noise_fixed(t0, dt, b.noise_dt, noise_len);   // host_forcing.h
        o.npos0 = nf.npos0;
        o.nstep = nf.nstep;
        o.n_hi = nf.n_hi;
    } else {
        o.n_hi = INT64_MAX;
    }
    return o;
}

}  // namespace hygro

struct hygro_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int precision = HYGRO_FP32;
    int kernel = HYGRO_KERNEL_PERSISTENT;
    int W = 0;
    int64_t total_nodes = 0;
    double dt = 0, t0 = 0, Lv = 0, Psat = 0;
    std::vector<int32_t> N;
    std::vector<double> L;
    std::vector<WallInfo> walls;
    std::vector<double> Tref, Pref;
    std::vector<int32_t> n_layers, layer_first;
    std::vector<hygro_layer> layers;
    std::vector<RawBc> bc[2];
    bool have_materials = false, have_bc[2] = {false, false};
    int64_t step = 0;
    int cur = 0;
    int grid_persistent = 1;
    int round_size = 1;
    CostModel cost = default_cost_model();   // step-time model of the wall schedule (hygro_autotune refits it)
    size_t real_size = 4;
    std::string err = "no error";

    // device
    void *dT[2] = {nullptr, nullptr}, *dP[2] = {nullptr, nullptr};
    WallInfo *d_walls = nullptr;
    FaceInfo *d_faces = nullptr;
    void *d_layer_tab = nullptr;
    int32_t *d_layer_first = nullptr;
    float2 *d_noise = nullptr;         // noise tables: face 0's region, then face 1's
    size_t noise_reg[2] = {0, 0};      // pairs reserved for each face's region
    size_t noise_used[2] = {0, 0};     // pairs in use
    // noise upload pipeline: two host chunks (pinned when the allocation succeeds), their copy events,
    // and a device staging area that receives a face's tables before they are known to be finite
    float *h_stage[2] = {nullptr, nullptr};
    bool stage_pinned = false;
    size_t stage_pairs = 0;            // pairs per host chunk
    cudaEvent_t stage_ev[2] = {nullptr, nullptr};
    float2 *d_stage = nullptr;
    unsigned long long *d_bad = nullptr;   // first non-finite pair of a directly copied noise upload
    size_t stage_cap = 0;              // pairs
    void *d_Tref = nullptr, *d_Pref = nullptr;
    double *d_cumul = nullptr, *d_flast = nullptr;
    int32_t *d_nonfinite = nullptr;
    int32_t *d_order = nullptr;
    int32_t *d_block_off = nullptr;
    unsigned long long *d_trace = nullptr;   // wall trace of the persistent kernel (HYGRO_TRACE)
    // rooms (whole-building model)
    std::vector<hygro_room> rooms;
    std::vector<double> wall_area;
    bool have_rooms = false;
    RoomInfo *d_rooms = nullptr;
    size_t rooms_cap = 0;
    std::vector<double> face_emis;   // [W][2] emissivity of room faces (hygro_set_radiation; empty: none)
    std::vector<double> room_view;   // [n_rooms] view factor s of each room
    std::vector<int32_t> link_zone;  // [n_links][2] (hygro_set_interzone)
    std::vector<double> link_flow;   // [n_links] kg/s
    RoomGroup *d_groups = nullptr;   // room kernel blocks: rooms alone or linked by airflow
    int n_groups = 0;
    double *d_room_state = nullptr;
    bool any_room_walls = false;   // some wall has a face on a room (those walls run in the room kernel)
    int room_warps = 1;            // warps of the room kernel's blocks (most walls of one room)
    int room_scheme = HYGRO_ROOM_DF;
    int n_free = 0;                // walls of the persistent kernel
    std::string room_issue;        // room configuration problem reported by hygro_run
    std::string trace_path;
    int32_t *d_node_wall = nullptr;
    int8_t *d_node_layer = nullptr;
    std::vector<int32_t> law;      // coefficient law of each layer (HYGRO_LAW_*)
    bool any_law = false;          // some layer takes a Table-1 law
    int8_t *d_layer_law = nullptr; // [sum layers]
    void *d_samples = nullptr;
    size_t samples_cap = 0;
};

namespace {

hygro_status fail(hygro_ctx *c, hygro_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c)
        c->err = buf;
    else
        g_create_error = buf;
    return st;
}

#define CUDA_TRY(ctx, call)                                                                              \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess) return fail(ctx, HYGRO_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// Host-side fault injection (host_fault.h): HYGRO_FAULT=<entry point>:<n> fails the n-th call of that entry
// point with HYGRO_E_CUDA before it changes anything.
bool fault_hit(const char *call)
{
    static FaultInjector inj(parse_fault(getenv("HYGRO_FAULT")));
    return inj.hit(call);
}

#define FAULT_POINT(ctx, name)                                                                     \
    do {                                                                                           \
        if (fault_hit(name)) return fail(ctx, HYGRO_E_CUDA, "%s: injected fault (HYGRO_FAULT)", name); \
    } while (0)

cudaError_t after_host_copies(const hygro_ctx *c) { return hygro::after_host_copies(c->stream); }

void free_all(hygro_ctx *c)
{
    void *ptrs[] = {c->dT[0], c->dT[1], c->dP[0], c->dP[1], c->d_walls, c->d_faces, c->d_layer_tab,
                    c->d_layer_first, c->d_noise, c->d_Tref, c->d_Pref, c->d_cumul, c->d_flast,
                    c->d_nonfinite, c->d_order, c->d_block_off, c->d_trace, c->d_rooms, c->d_room_state, c->d_node_wall, c->d_node_layer, c->d_samples, c->d_layer_law, c->d_groups};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (c->d_stage) cudaFree(c->d_stage);
    if (c->d_bad) cudaFree(c->d_bad);
    for (int i = 0; i < 2; ++i) {
        if (c->h_stage[i]) {
            if (c->stage_pinned)
                cudaFreeHost(c->h_stage[i]);
            else
                free(c->h_stage[i]);
        }
        if (c->stage_ev[i]) cudaEventDestroy(c->stage_ev[i]);
    }
}

template <typename real>
DevCtx<real> make_dev(const hygro_ctx *c)
{
    DevCtx<real> d;
    d.walls = c->d_walls;
    d.faces = c->d_faces;
    d.layer_tab = (const real *)c->d_layer_tab;
    d.layer_first = c->d_layer_first;
    d.noise = c->d_noise;
    d.T[0] = (real *)c->dT[0];
    d.T[1] = (real *)c->dT[1];
    d.P[0] = (real *)c->dP[0];
    d.P[1] = (real *)c->dP[1];
    d.cur = c->cur;
    d.W = c->W;
    d.Tref = (const real *)c->d_Tref;
    d.Pref = (const real *)c->d_Pref;
    d.cumul = c->d_cumul;
    d.flast = c->d_flast;
    d.nonfinite = c->d_nonfinite;
    d.order = c->d_order;
    d.block_off = c->d_block_off;
    d.round_size = c->round_size;
    d.trace = c->d_trace;
    d.rooms = c->d_rooms;
    d.groups = c->d_groups;
    d.room_state = c->d_room_state;
    d.n_rooms = (int32_t)c->rooms.size();
    d.node_wall = c->d_node_wall;
    d.node_layer = c->d_node_layer;
    d.layer_law = c->d_layer_law;
    d.total_nodes = (int32_t)c->total_nodes;
    d.dt = c->dt;
    d.t0 = c->t0;
    d.Lv = c->Lv;
    return d;
}

// Device copy of one real-typed host vector of doubles.
hygro_status upload_reals(hygro_ctx *c, void *dst, const std::vector<double> &src)
{
    if (c->precision == HYGRO_FP64) {
        CUDA_TRY(c, cudaMemcpy(dst, src.data(), src.size() * sizeof(double), cudaMemcpyHostToDevice));
    } else {
        std::vector<float> f(src.size());
        for (size_t i = 0; i < src.size(); ++i) f[i] = (float)src[i];
        CUDA_TRY(c, cudaMemcpy(dst, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
    return HYGRO_OK;
}

hygro_status download_reals(hygro_ctx *c, const void *src, std::vector<double> &dst)
{
    if (c->precision == HYGRO_FP64) {
        CUDA_TRY(c, cudaMemcpy(dst.data(), src, dst.size() * sizeof(double), cudaMemcpyDeviceToHost));
    } else {
        std::vector<float> f(dst.size());
        CUDA_TRY(c, cudaMemcpy(f.data(), src, f.size() * sizeof(float), cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < f.size(); ++i) dst[i] = (double)f[i];
    }
    return HYGRO_OK;
}

// Face descriptors in the deviation variables of each wall; needs the
// materials (for T_ref, P_ref) and both faces. The noise tables are already
// on the device (upload_noise); only their offsets enter the descriptors.
hygro_status upload_faces(hygro_ctx *c)
{
    if (!(c->have_materials && c->have_bc[0] && c->have_bc[1])) return HYGRO_OK;
    const int W = c->W;
    std::vector<FaceInfo> fi((size_t)W * 2);
    for (int w = 0; w < W; ++w)
        for (int f = 0; f < 2; ++f) {
            const RawBc &r = c->bc[f][w];
            const int64_t base = f == 0 ? 0 : (int64_t)c->noise_reg[0];
            fi[(size_t)w * 2 + f] =
                face_info(r.bc, c->Tref[w], c->Pref[w], c->t0, c->dt, base + r.noise_off, r.noise_len);
        }
    CUDA_TRY(c, cudaMemcpy(c->d_faces, fi.data(), fi.size() * sizeof(FaceInfo), cudaMemcpyHostToDevice));
    return HYGRO_OK;
}

constexpr size_t kStagePairs = size_t(1) << 23;   // (T, Pv) pairs per host chunk of the noise upload (64 MB)

// First (T, Pv) pair of tab[0 .. n) with a non-finite value into *bad (which starts at ~0).
__global__ void first_nonfinite_kernel(const float2 *tab, int64_t n, unsigned long long *bad)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = tab[i];
        if (!isfinite(v.x) || !isfinite(v.y)) atomicMin(bad, (unsigned long long)i);
    }
}

// True when p lies in page-locked host memory, device memory or managed memory: memory the DMA engines
// read directly (pageable memory goes through the driver's own staging).
bool dma_direct(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Uploads the noise tables of one face (hygro_bc array, validated except for the table values) and
// records each wall's offset and length in v. Host threads gather the per-wall tables into two host
// chunks (pinned when possible), checking each value as they copy, while the previous chunk's copy to
// the device runs; the chunks land in a device staging area, which reaches the face's region of the
// context's noise array only when every value was finite, so a refused call leaves the face as it was.
// Tables in page-locked (or device) memory skip the host gather: each run of tables adjacent in memory
// goes to the staging area in one copy, and a device kernel looks for non-finite values there.
// The array grows when the region is too small (the other face's tables move with a device copy).
hygro_status upload_noise(hygro_ctx *c, int face, const hygro_bc *bc, std::vector<RawBc> &v)
{
    const int W = c->W;
    std::vector<int> wid;
    std::vector<const float *> src;
    std::vector<int64_t> start, len;
    int64_t total = 0;
    for (int w = 0; w < W; ++w) {
        const bool has = bc[w].kind == HYGRO_BC_AMBIENT && bc[w].noise_len > 0;
        v[w].noise_off = total;
        v[w].noise_len = has ? bc[w].noise_len : 0;
        if (!has) continue;
        wid.push_back(w);
        src.push_back(bc[w].noise);
        start.push_back(total);
        len.push_back(bc[w].noise_len);
        total += bc[w].noise_len;
    }
    if (total > 0) {
        if ((size_t)total > c->stage_cap) {
            if (c->d_stage) cudaFree(c->d_stage);
            c->d_stage = nullptr;
            c->stage_cap = 0;
            CUDA_TRY(c, dalloc(&c->d_stage, (size_t)total));
            c->stage_cap = (size_t)total;
        }
        // runs of tables adjacent in memory; the direct path when each run starts in DMA-readable memory
        std::vector<size_t> run0;
        for (size_t k = 0; k < src.size(); ++k)
            if (k == 0 || src[k] != src[k - 1] + 2 * len[k - 1]) run0.push_back(k);
        bool direct = true;
        for (size_t r = 0; r < run0.size() && direct; ++r) direct = dma_direct(src[run0[r]]);
        const size_t want = direct ? 0 : std::min(kStagePairs, (size_t)total);
        if (want > c->stage_pairs) {   // host chunks sized to the need, up to kStagePairs
            for (int i = 0; i < 2; ++i) {
                if (c->h_stage[i]) {
                    if (c->stage_pinned)
                        cudaFreeHost(c->h_stage[i]);
                    else
                        free(c->h_stage[i]);
                }
                c->h_stage[i] = nullptr;
            }
            c->stage_pairs = 0;
            const size_t bytes = want * 2 * sizeof(float);
            c->stage_pinned = cudaHostAlloc((void **)&c->h_stage[0], bytes, cudaHostAllocDefault) == cudaSuccess &&
                              cudaHostAlloc((void **)&c->h_stage[1], bytes, cudaHostAllocDefault) == cudaSuccess;
            if (!c->stage_pinned) {   // pageable chunks: the same pipeline, with synchronous copies
                for (int i = 0; i < 2; ++i) {
                    if (c->h_stage[i]) cudaFreeHost(c->h_stage[i]);
                    c->h_stage[i] = (float *)malloc(bytes);
                }
                if (!c->h_stage[0] || !c->h_stage[1]) return fail(c, HYGRO_E_NOMEM, "noise upload buffers");
            }
            c->stage_pairs = want;
        }
        for (int i = 0; i < 2; ++i)
            if (c->stage_ev[i] == nullptr)
                CUDA_TRY(c, cudaEventCreateWithFlags(&c->stage_ev[i], cudaEventDisableTiming));
        const int threads = (int)std::min(8u, std::max(1u, std::thread::hardware_concurrency()));
        int64_t bad = -1;
        if (direct) {
            if (c->d_bad == nullptr) CUDA_TRY(c, dalloc(&c->d_bad, 1));
            CUDA_TRY(c, cudaMemsetAsync(c->d_bad, 0xff, sizeof(unsigned long long), c->stream));
            for (size_t r = 0; r < run0.size(); ++r) {
                const size_t k0 = run0[r], k1 = r + 1 < run0.size() ? run0[r + 1] : src.size();
                const int64_t pairs = start[k1 - 1] + len[k1 - 1] - start[k0];
                CUDA_TRY(c, cudaMemcpyAsync(c->d_stage + start[k0], src[k0], (size_t)pairs * sizeof(float2),
                                            cudaMemcpyDefault, c->stream));
            }
            first_nonfinite_kernel<<<4 * 152, 256, 0, c->stream>>>(c->d_stage, total, c->d_bad);
            CUDA_TRY(c, cudaGetLastError());
            unsigned long long first = 0;
            CUDA_TRY(c, cudaMemcpyAsync(&first, c->d_bad, sizeof first, cudaMemcpyDeviceToHost, c->stream));
            CUDA_TRY(c, cudaStreamSynchronize(c->stream));
            if (first != ~0ull) bad = (int64_t)first;
        }
        int chunk = 0;
        for (int64_t p0 = direct ? total : 0; p0 < total; p0 += (int64_t)c->stage_pairs, ++chunk) {
            const int64_t p1 = std::min(total, p0 + (int64_t)c->stage_pairs);
            const int slot = chunk & 1;
            if (chunk >= 2) CUDA_TRY(c, cudaEventSynchronize(c->stage_ev[slot]));
            bad = gather_tables(src, start, len, p0, p1, c->h_stage[slot], threads);
            if (bad >= 0) break;
            CUDA_TRY(c, cudaMemcpyAsync(c->d_stage + p0, c->h_stage[slot], (size_t)(p1 - p0) * sizeof(float2),
                                        cudaMemcpyHostToDevice, c->stream));
            CUDA_TRY(c, cudaEventRecord(c->stage_ev[slot], c->stream));
        }
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        if (bad >= 0) {
            const size_t k = (size_t)(std::upper_bound(start.begin(), start.end(), bad) - start.begin()) - 1;
            return fail(c, HYGRO_E_INVALID, "wall %d face %d: non-finite noise", wid[k], face);
        }
    }
    const int other = 1 - face;
    if ((size_t)total > c->noise_reg[face] || c->d_noise == nullptr) {
        size_t reg[2];
        reg[face] = (size_t)total;
        reg[other] = c->noise_reg[other];
        float2 *fresh = nullptr;
        CUDA_TRY(c, dalloc(&fresh, reg[0] + reg[1]));
        const size_t old_base = other == 0 ? 0 : c->noise_reg[0];
        const size_t new_base = other == 0 ? 0 : reg[0];
        if (c->noise_used[other] > 0) {
            const cudaError_t e = cudaMemcpy(fresh + new_base, c->d_noise + old_base,
                                             c->noise_used[other] * sizeof(float2), cudaMemcpyDeviceToDevice);
            if (e != cudaSuccess) {
                cudaFree(fresh);
                return fail(c, HYGRO_E_CUDA, "noise table copy: %s", cudaGetErrorString(e));
            }
        }
        if (c->d_noise) cudaFree(c->d_noise);
        c->d_noise = fresh;
        c->noise_reg[0] = reg[0];
        c->noise_reg[1] = reg[1];
    }
    if (total > 0) {
        float2 *dst = c->d_noise + (face == 0 ? 0 : c->noise_reg[0]);
        CUDA_TRY(c, cudaMemcpyAsync(dst, c->d_stage, (size_t)total * sizeof(float2), cudaMemcpyDeviceToDevice,
                                    c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    }
    c->noise_used[face] = (size_t)total;
    return HYGRO_OK;
}

hygro_status check_nonfinite(hygro_ctx *c)
{
    int32_t flag = 0;
    CUDA_TRY(c, cudaMemcpyAsync(&flag, c->d_nonfinite, sizeof flag, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (flag) {
        CUDA_TRY(c, cudaMemsetAsync(c->d_nonfinite, 0, sizeof(int32_t), c->stream));
        return fail(c, HYGRO_E_NONFINITE, "a wall produced a non-finite value");
    }
    return HYGRO_OK;
}

const uint64_t kStateMagic = 0x6879677273746174ull;  // "hygrstat"

// Lane layout of one wall for the persistent kernel (host_layout.h).
void wall_layout(int N, const int32_t *first, int nl, WallInfo &wi)
{
    const LaneLayout o = hygro::wall_layout(N, first, nl);
    wi.K = o.K;
    wi.Wl = o.Wl;
    wi.short_mask = o.short_mask;
    wi.aligned = o.aligned;
}


// Work partition of hygro_run. Walls with no face on a room go to the persistent kernel: sorted by
// nodes per lane and code variant, cut into rounds, rounds dealt to blocks by LPT. Walls facing a
// room are grouped by room for the room kernel. Problems of the room configuration are kept and
// reported by hygro_run (rooms and boundaries may be set in either order).
hygro_status build_schedule(hygro_ctx *c)
{
    if (!c->have_materials) return HYGRO_OK;
    const int W = c->W;
    std::vector<char> in_room(W, 0);
    c->room_issue.clear();
    const int NR = (int)c->rooms.size();
    std::vector<std::vector<std::pair<int, int>>> members(NR);
    char msg[256];
    for (int w = 0; w < W; ++w) {
        int nf = 0;
        for (int f = 0; f < 2; ++f) {
            if (!c->have_bc[f] || c->bc[f][w].bc.kind != HYGRO_BC_ROOM) continue;
            ++nf;
            const int r = c->bc[f][w].bc.room;
            if (r < 0 || r >= NR) {
                if (c->room_issue.empty()) {
                    snprintf(msg, sizeof msg, "wall %d face %d: room %d is not defined (hygro_set_rooms)", w, f, r);
                    c->room_issue = msg;
                }
                continue;
            }
            members[r].push_back({w, f});
        }
        if (nf > 0) in_room[w] = 1;
        if (nf > 1 && c->room_issue.empty()) {
            snprintf(msg, sizeof msg, "wall %d has both faces on rooms; a wall may face one room", w);
            c->room_issue = msg;
        }
    }
    c->any_room_walls = false;
    c->room_warps = 1;
    for (int w = 0; w < W; ++w)
        if (in_room[w]) c->any_room_walls = true;
    if (NR > 0) {
        // rooms linked by interzone airflow share a block: the groups are the link graph's components
        std::vector<int> root(NR);
        for (int r = 0; r < NR; ++r) root[r] = r;
        auto find = [&](int r) {
            while (root[r] != r) r = root[r] = root[root[r]];
            return r;
        };
        const int NL = (int)c->link_flow.size();
        for (int l = 0; l < NL; ++l) root[find(c->link_zone[2 * l])] = find(c->link_zone[2 * l + 1]);
        std::vector<std::vector<int>> comp(NR);
        for (int r = 0; r < NR; ++r) comp[find(r)].push_back(r);
        std::vector<int> slot_of(NR, 0);
        std::vector<RoomGroup> groups;
        for (int r = 0; r < NR; ++r) {
            if (comp[r].empty()) continue;
            RoomGroup g;
            memset(&g, 0, sizeof g);
            const int nz = (int)comp[r].size();
            int warps = 0;
            for (int z = 0; z < nz && z < kMaxGroupZones; ++z) {
                g.zone[z] = comp[r][z];
                slot_of[comp[r][z]] = z;
                g.wall_warp0[z] = warps;
                warps += (int)members[comp[r][z]].size();
            }
            g.n_zones = std::min(nz, kMaxGroupZones);
            g.air_warp0 = warps;
            g.n_warps = warps + g.n_zones;
            const int cap = nz > 1 ? kRoomBlockWarps : HYGRO_MAX_ROOM_WALLS + 1;
            if ((nz > kMaxGroupZones || g.n_warps > cap) && c->room_issue.empty()) {
                snprintf(msg, sizeof msg,
                         "rooms linked by airflow with room %d: %d rooms and %d walls; a linked group holds at most %d "
                         "rooms and %d walls plus one air warp per room",
                         comp[r][0], nz, warps, kMaxGroupZones, kRoomBlockWarps);
                c->room_issue = msg;
            }
            c->room_warps = std::max(c->room_warps, g.n_warps);
            groups.push_back(g);
        }
        c->n_groups = (int)groups.size();
        if (c->d_groups) cudaFree(c->d_groups);
        c->d_groups = nullptr;
        CUDA_TRY(c, dalloc(&c->d_groups, groups.size()));
        CUDA_TRY(c, cudaMemcpy(c->d_groups, groups.data(), groups.size() * sizeof(RoomGroup), cudaMemcpyHostToDevice));
        std::vector<RoomInfo> ri(NR);
        for (int r = 0; r < NR; ++r) {
            RoomInfo &o = ri[r];
            memset(&o, 0, sizeof o);
            if ((int)members[r].size() > HYGRO_MAX_ROOM_WALLS) {
                if (c->room_issue.empty()) {
                    snprintf(msg, sizeof msg, "room %d has %zu walls; at most %d", r, members[r].size(),
                             HYGRO_MAX_ROOM_WALLS);
                    c->room_issue = msg;
                }
                continue;
            }
            o.n_walls = (int32_t)members[r].size();
            for (int i = 0; i < o.n_walls; ++i) {
                o.wall[i] = members[r][i].first;
                o.face[i] = members[r][i].second;
                o.area[i] = c->wall_area[members[r][i].first];
            }
            const hygro_room &q = c->rooms[r];
            const double pv[15] = {q.volume, q.ach, q.Q_gain, q.g_vap, q.T_out_mean, q.T_out_amp, q.P_out_mean,
                                   q.P_out_amp, q.period, q.phase_T, q.phase_P, q.rho_a, q.cp_a, q.cp_v, q.Pv_ref};
            for (int k = 0; k < 15; ++k) o.par[k] = pv[k];
            o.par[RP_PERIODP] = q.period_P > 0 ? q.period_P : q.period;
            o.par[RP_GPULSE] = q.g_pulse;
            o.par[RP_PON] = q.pulse_on;
            o.par[RP_POFF] = q.pulse_off;
            o.par[RP_PPER] = q.pulse_period;
            o.par[RP_SCHEME] = (double)c->room_scheme;
            // long-wave exchange among the room's faces
            o.view = c->room_view.empty() ? 0.0 : c->room_view[r];
            for (int i = 0; i < o.n_walls; ++i)
                o.emis[i] = c->face_emis.empty() ? 0.0 : c->face_emis[(size_t)o.wall[i] * 2 + o.face[i]];
            // interzone links to rooms of the same group
            o.n_links = 0;
            for (int l = 0; l < NL; ++l)
                for (int e = 0; e < 2; ++e) {
                    if (c->link_zone[2 * l + e] != r) continue;
                    const int other = c->link_zone[2 * l + 1 - e];
                    if (o.n_links >= kMaxZoneLinks) {
                        if (c->room_issue.empty()) {
                            snprintf(msg, sizeof msg, "room %d has more than %d interzone links", r, kMaxZoneLinks);
                            c->room_issue = msg;
                        }
                        continue;
                    }
                    o.link_slot[o.n_links] = slot_of[other];
                    o.link_g[o.n_links] = c->link_flow[l];
                    o.link_gw[o.n_links] = c->link_flow[l] / c->rooms[other].Pv_ref;
                    ++o.n_links;
                }
        }
        CUDA_TRY(c, cudaMemcpy(c->d_rooms, ri.data(), ri.size() * sizeof(RoomInfo), cudaMemcpyHostToDevice));
    }
    {
        // Persistent blocks: rounds of same-size walls dealt to blocks by estimated cost (host_layout.h)
        std::vector<SchedWall> sw;
        for (int w = 0; w < W; ++w) {
            if (in_room[w]) continue;
            const WallInfo &x = c->walls[w];
            const bool simple = x.simple && c->precision == HYGRO_FP32;
            sw.push_back({w, x.K, x.aligned ? (simple ? 0 : 1) : (simple ? 3 : 2), x.N});
        }
        const int Wf = (int)sw.size();
        c->n_free = Wf;
        const int G = c->grid_persistent;
        const int wpb = c->precision == HYGRO_FP64 ? PersistCfg<double>::warps : PersistCfg<float>::warps;
        const int R = std::max(1, std::min(wpb, Wf / G));
        c->round_size = R;
        std::vector<int32_t> order, boff;
        lpt_rounds(std::move(sw), G, R, order, boff, nullptr, c->cost);
        if (!order.empty())
            CUDA_TRY(c, cudaMemcpy(c->d_order, order.data(), order.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
        CUDA_TRY(c, cudaMemcpy(c->d_block_off, boff.data(), boff.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    }
    return HYGRO_OK;
}

// Checks that the rooms of a context can run (hygro_run, hygro_run_noalloc), and that walls with a Table-1
// coefficient law run on the plain kernel (the only one that evaluates those laws).
hygro_status rooms_ready(hygro_ctx *c)
{
    if (c->any_law && c->kernel != HYGRO_KERNEL_PLAIN)
        return fail(c, HYGRO_E_UNSUPPORTED, "walls with a Table-1 coefficient law run on the plain kernel only");
    if (!c->room_issue.empty()) return fail(c, HYGRO_E_STATE, "%s", c->room_issue.c_str());
    if (c->any_room_walls && c->kernel != HYGRO_KERNEL_PERSISTENT)
        return fail(c, HYGRO_E_UNSUPPORTED, "rooms need the persistent kernel");
    return HYGRO_OK;
}

// Enqueues n_steps steps of every wall (and room) on the context's stream; samples go to dsamp.
hygro_status launch_steps(hygro_ctx *c, int64_t n_steps, int se, void *dsamp)
{
    CUDA_TRY(c, after_host_copies(c));
    if (c->kernel == HYGRO_KERNEL_PERSISTENT) {
        // chunks of whole sampling periods below 2^30 steps
        int64_t chunk = int64_t(1) << 30;
        if (se > 0) chunk -= chunk % se;
        int64_t done = 0;
        const int NR = (int)c->rooms.size();
        while (done < n_steps) {
            const int64_t len = std::min(chunk, n_steps - done);
            const size_t soff = se > 0 ? (size_t)(done / se) * c->W * 4 : 0;
            if (c->precision == HYGRO_FP64) {
                double *sp = dsamp ? (double *)dsamp + soff : nullptr;
                if (c->n_free > 0)
                    CUDA_TRY(c, launch_persistent_f64(make_dev<double>(c), c->step + done, (int32_t)len, se, sp,
                                                      c->grid_persistent, c->stream));
                if (c->any_room_walls)
                    CUDA_TRY(c, launch_rooms_f64(make_dev<double>(c), c->step + done, (int32_t)len, se, sp,
                                                 c->n_groups, c->room_warps, c->stream));
            } else {
                float *sp = dsamp ? (float *)dsamp + soff : nullptr;
                if (c->n_free > 0)
                    CUDA_TRY(c, launch_persistent_f32(make_dev<float>(c), c->step + done, (int32_t)len, se, sp,
                                                      c->grid_persistent, c->stream));
                if (c->any_room_walls)
                    CUDA_TRY(c, launch_rooms_f32(make_dev<float>(c), c->step + done, (int32_t)len, se, sp,
                                                 c->n_groups, c->room_warps, c->stream));
            }
            done += len;
        }
    } else {
        for (int64_t s = 0; s < n_steps; ++s) {
            const int32_t sidx = (se > 0 && (s + 1) % se == 0) ? (int32_t)((s + 1) / se - 1) : -1;
            if (c->precision == HYGRO_FP64)
                CUDA_TRY(c, launch_plain_step_f64(make_dev<double>(c), c->step + s, sidx, (double *)dsamp, c->stream));
            else
                CUDA_TRY(c, launch_plain_step_f32(make_dev<float>(c), c->step + s, sidx, (float *)dsamp, c->stream));
            c->cur = 1 - c->cur;
        }
    }
    return HYGRO_OK;
}

// State image of hygro_get_state / hygro_set_state (no fault point: internal callers use these too).
hygro_status get_state_impl(hygro_ctx *c, void *buf, size_t *bytes);
hygro_status set_state_impl(hygro_ctx *c, const void *buf, size_t bytes);
}  // namespace

extern "C" {

hygro_status hygro_create(const hygro_desc *desc, hygro_ctx **out)
{
    if (out == nullptr) return fail(nullptr, HYGRO_E_INVALID, "out is NULL");
    *out = nullptr;
    FAULT_POINT(nullptr, "hygro_create");
    if (desc == nullptr) return fail(nullptr, HYGRO_E_INVALID, "desc is NULL");
    if (desc->n_walls < 1) return fail(nullptr, HYGRO_E_INVALID, "n_walls must be >= 1");
    if (desc->n_nodes == nullptr || desc->thickness == nullptr)
        return fail(nullptr, HYGRO_E_INVALID, "n_nodes and thickness are required");
    if (!(std::isfinite(desc->dt) && desc->dt > 0)) return fail(nullptr, HYGRO_E_INVALID, "dt must be > 0");
    if (!std::isfinite(desc->t0)) return fail(nullptr, HYGRO_E_INVALID, "t0 must be finite");
    if (!(std::isfinite(desc->Psat) && desc->Psat > 0)) return fail(nullptr, HYGRO_E_INVALID, "Psat must be > 0");
    if (!std::isfinite(desc->Lv)) return fail(nullptr, HYGRO_E_INVALID, "Lv must be finite");
    if (desc->precision != HYGRO_FP32 && desc->precision != HYGRO_FP64)
        return fail(nullptr, HYGRO_E_INVALID, "precision must be HYGRO_FP32 or HYGRO_FP64");
    if (desc->kernel != HYGRO_KERNEL_PERSISTENT && desc->kernel != HYGRO_KERNEL_PLAIN)
        return fail(nullptr, HYGRO_E_INVALID, "unknown kernel %d", desc->kernel);
    int64_t total = 0;
    for (int w = 0; w < desc->n_walls; ++w) {
        if (desc->n_nodes[w] < 3) return fail(nullptr, HYGRO_E_INVALID, "wall %d: n_nodes must be >= 3", w);
        if (!(std::isfinite(desc->thickness[w]) && desc->thickness[w] > 0))
            return fail(nullptr, HYGRO_E_INVALID, "wall %d: thickness must be > 0", w);
        if (desc->kernel == HYGRO_KERNEL_PERSISTENT && desc->n_nodes[w] > HYGRO_PERSISTENT_MAX_NODES)
            return fail(nullptr, HYGRO_E_UNSUPPORTED, "wall %d: %d nodes exceed the persistent kernel's %d", w,
                        desc->n_nodes[w], HYGRO_PERSISTENT_MAX_NODES);
        total += desc->n_nodes[w];
    }
    if (total > (int64_t)INT32_MAX / 2) return fail(nullptr, HYGRO_E_UNSUPPORTED, "too many nodes in total");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(nullptr, HYGRO_E_CUDA, "no CUDA device available");
    }
    if (desc->device < 0 || desc->device >= ndev) return fail(nullptr, HYGRO_E_INVALID, "bad device %d", desc->device);

    hygro_ctx *c = new (std::nothrow) hygro_ctx();
    if (c == nullptr) return fail(nullptr, HYGRO_E_NOMEM, "host allocation failed");
    c->device = desc->device;
    c->stream = (cudaStream_t)desc->stream;
    c->precision = desc->precision;
    c->kernel = desc->kernel;
    c->W = desc->n_walls;
    c->dt = desc->dt;
    c->t0 = desc->t0;
    c->Lv = desc->Lv;
    c->Psat = desc->Psat;
    c->real_size = desc->precision == HYGRO_FP64 ? 8 : 4;
    c->N.assign(desc->n_nodes, desc->n_nodes + desc->n_walls);
    c->L.assign(desc->thickness, desc->thickness + desc->n_walls);
    c->total_nodes = total;
    c->walls.resize(c->W);
    int64_t off = 0;
    for (int w = 0; w < c->W; ++w) {
        WallInfo &wi = c->walls[w];
        memset(&wi, 0, sizeof wi);
        wi.N = c->N[w];
        wi.nu = 1.0;
        const int32_t zero = 0;
        wall_layout(wi.N, &zero, 1, wi);
        wi.node_off = (int32_t)off;
        off += wi.N;
    }
    auto bail = [&](hygro_status s) {
        g_create_error = c->err;
        free_all(c);
        delete c;
        return s;
    };
#define CREATE_TRY(call)                                                                          \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            fail(c, e_ == cudaErrorMemoryAllocation ? HYGRO_E_NOMEM : HYGRO_E_CUDA, "%s: %s", #call, \
                 cudaGetErrorString(e_));                                                         \
            return bail(e_ == cudaErrorMemoryAllocation ? HYGRO_E_NOMEM : HYGRO_E_CUDA);          \
        }                                                                                         \
    } while (0)
    CREATE_TRY(cudaSetDevice(c->device));
    const size_t rs = c->real_size;
    for (int i = 0; i < 2; ++i) {
        CREATE_TRY(cudaMalloc(&c->dT[i], (size_t)total * rs));
        CREATE_TRY(cudaMalloc(&c->dP[i], (size_t)total * rs));
        CREATE_TRY(cudaMemset(c->dT[i], 0, (size_t)total * rs));
        CREATE_TRY(cudaMemset(c->dP[i], 0, (size_t)total * rs));
    }
    CREATE_TRY(dalloc(&c->d_walls, c->W));
    CREATE_TRY(dalloc(&c->d_faces, (size_t)c->W * 2));
    CREATE_TRY(cudaMalloc(&c->d_Tref, (size_t)c->W * rs));
    CREATE_TRY(cudaMalloc(&c->d_Pref, (size_t)c->W * rs));
    CREATE_TRY(dalloc(&c->d_cumul, (size_t)c->W * 4));
    CREATE_TRY(dalloc(&c->d_flast, (size_t)c->W * 4));
    CREATE_TRY(cudaMemset(c->d_cumul, 0, (size_t)c->W * 4 * sizeof(double)));
    CREATE_TRY(cudaMemset(c->d_flast, 0, (size_t)c->W * 4 * sizeof(double)));
    CREATE_TRY(dalloc(&c->d_nonfinite, 1));
    CREATE_TRY(cudaMemset(c->d_nonfinite, 0, sizeof(int32_t)));
    CREATE_TRY(dalloc(&c->d_order, (size_t)c->W + PersistCfg<float>::warps + PersistCfg<double>::warps));
    CREATE_TRY(dalloc(&c->d_node_wall, (size_t)total));
    CREATE_TRY(dalloc(&c->d_node_layer, (size_t)total));
    CREATE_TRY(cudaMemset(c->d_node_layer, 0, (size_t)total));
    {
        std::vector<int32_t> nw((size_t)total);
        for (int w = 0; w < c->W; ++w)
            for (int j = 0; j < c->N[w]; ++j) nw[(size_t)c->walls[w].node_off + j] = w;
        CREATE_TRY(cudaMemcpy(c->d_node_wall, nw.data(), nw.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    }
    {
        int sms = 0, per_sm = 0;
        CREATE_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
        CREATE_TRY(c->precision == HYGRO_FP64 ? occupancy_persistent_f64(&per_sm) : occupancy_persistent_f32(&per_sm));
        if (per_sm < 1) per_sm = 1;
        // one persistent block per SM slot, but never more blocks than walls (few walls spread over SMs)
        c->grid_persistent = std::max(1, std::min(c->W, sms * per_sm));
        CREATE_TRY(dalloc(&c->d_block_off, (size_t)c->grid_persistent + 1));
    }
    if (const char *tp = getenv("HYGRO_TRACE")) {
        // diagnostic: per-wall SM, block, warp and start / end times of every persistent launch,
        // appended to the named file after each hygro_run
        c->trace_path = tp;
        CREATE_TRY(dalloc(&c->d_trace, (size_t)c->W * 4));
        CREATE_TRY(cudaMemset(c->d_trace, 0, (size_t)c->W * 4 * sizeof(unsigned long long)));
    }
#undef CREATE_TRY
    *out = c;
    return HYGRO_OK;
}

hygro_status hygro_set_materials(hygro_ctx *c, const int32_t *n_layers, const int32_t *layer_first,
                                 const hygro_layer *layers, const double *T_init, const double *P_init)
{
    if (c == nullptr) return fail(nullptr, HYGRO_E_INVALID, "ctx is NULL");
    FAULT_POINT(c, "hygro_set_materials");
    if (!n_layers || !layer_first || !layers || !T_init || !P_init)
        return fail(c, HYGRO_E_INVALID, "n_layers, layer_first, layers, T_init and P_init are required");
    const int W = c->W;
    size_t total_layers = 0;
    for (int w = 0; w < W; ++w) {
        const int nl = n_layers[w];
        if (nl < 1 || nl > HYGRO_MAX_LAYERS)
            return fail(c, HYGRO_E_INVALID, "wall %d: n_layers must be in 1..%d", w, HYGRO_MAX_LAYERS);
        const int32_t *lf = layer_first + total_layers;
        if (lf[0] != 0) return fail(c, HYGRO_E_INVALID, "wall %d: the first layer must start at node 0", w);
        for (int l = 1; l < nl; ++l)
            if (lf[l] <= lf[l - 1] || lf[l] >= c->N[w])
                return fail(c, HYGRO_E_INVALID, "wall %d: layer_first must increase and stay below N", w);
        for (int l = 0; l < nl; ++l) {
            const hygro_layer &y = layers[total_layers + l];
            if (!(y.kM0 > 0 && y.cM0 > 0 && y.kTT0 > 0 && y.cTT0 > 0) || !std::isfinite(y.kM0) ||
                !std::isfinite(y.cM0) || !std::isfinite(y.kTT0) || !std::isfinite(y.cTT0) || !std::isfinite(y.a) ||
                !std::isfinite(y.b) || !std::isfinite(y.aT) || !std::isfinite(y.bT) || !std::isfinite(y.chi))
                return fail(c, HYGRO_E_INVALID, "wall %d layer %d: coefficients must be finite, kM0, cM0, kTT0, cTT0 > 0",
                            w, l);
        }
        if (!std::isfinite(T_init[w]) || !std::isfinite(P_init[w]))
            return fail(c, HYGRO_E_INVALID, "wall %d: initial state must be finite", w);
        total_layers += nl;
    }
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, HYGRO_E_CUDA, "cudaSetDevice failed");
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->n_layers.assign(n_layers, n_layers + W);
    c->layer_first.assign(layer_first, layer_first + total_layers);
    c->layers.assign(layers, layers + total_layers);
    c->Tref.assign(T_init, T_init + W);
    c->Pref.assign(P_init, P_init + W);

    std::vector<double> tab(total_layers * kLayerStride, 0.0);
    std::vector<int8_t> node_layer((size_t)c->total_nodes, 0);
    size_t lo = 0;
    for (int w = 0; w < W; ++w) {
        WallInfo &wi = c->walls[w];
        wi.n_layers = n_layers[w];
        wi.layer_off = (int32_t)lo;
        wall_layout(wi.N, layer_first + lo, wi.n_layers, wi);
        wi.simple = wi.nu == 1.0 ? 1 : 0;
        for (int l = 0; l < wi.n_layers; ++l) {
            const hygro_layer &y = layers[lo + l];
            if (y.aT != 0.0 || y.bT != 0.0 || y.chi != 0.0) wi.simple = 0;
        }
        const double dx = c->L[w] / (double)(c->N[w] - 1);
        wi.dx = dx;
        wi.has_law = 0;
        const double Ps = c->Psat, Pr = c->Pref[w], dt = c->dt;
        for (int l = 0; l < wi.n_layers; ++l) {
            const hygro_layer &y = layers[lo + l];
            double *t = &tab[(lo + l) * kLayerStride];
            t[LT_KMA] = y.kM0 * (1.0 + y.a * Pr / Ps) / (2.0 * dx);
            t[LT_KMB] = y.kM0 * y.a / Ps / (2.0 * dx);
            t[LT_KTA] = y.kTT0 * (1.0 + y.aT * Pr / Ps) / (2.0 * dx);
            t[LT_KTB] = y.kTT0 * y.aT / Ps / (2.0 * dx);
            t[LT_AA] = dx * y.cM0 * (1.0 + y.b * Pr / Ps) / (2.0 * dt);
            t[LT_AB] = dx * y.cM0 * y.b / Ps / (2.0 * dt);
            t[LT_BA] = dx * y.cTT0 * (1.0 + y.bT * Pr / Ps) / (2.0 * dt);
            t[LT_BB] = dx * y.cTT0 * y.bT / Ps / (2.0 * dt);
            t[LT_CHI] = y.chi;
            const int j0 = layer_first[lo + l];
            const int j1 = l + 1 < wi.n_layers ? layer_first[lo + l + 1] : c->N[w];
            for (int j = j0; j < j1; ++j) node_layer[(size_t)wi.node_off + j] = (int8_t)l;
        }
        lo += wi.n_layers;
    }
    if (c->d_layer_tab) cudaFree(c->d_layer_tab);
    if (c->d_layer_first) cudaFree(c->d_layer_first);
    c->d_layer_tab = nullptr;
    c->d_layer_first = nullptr;
    CUDA_TRY(c, cudaMalloc(&c->d_layer_tab, std::max<size_t>(1, tab.size()) * c->real_size));
    CUDA_TRY(c, dalloc(&c->d_layer_first, total_layers));
    hygro_status st = upload_reals(c, c->d_layer_tab, tab);
    if (st != HYGRO_OK) return st;
    CUDA_TRY(c, cudaMemcpy(c->d_layer_first, layer_first, total_layers * sizeof(int32_t), cudaMemcpyHostToDevice));
    // every layer back to its affine laws
    c->law.assign(total_layers, HYGRO_LAW_AFFINE);
    c->any_law = false;
    if (c->d_layer_law) cudaFree(c->d_layer_law);
    c->d_layer_law = nullptr;
    CUDA_TRY(c, cudaMalloc(&c->d_layer_law, std::max<size_t>(1, total_layers)));
    CUDA_TRY(c, cudaMemset(c->d_layer_law, 0, std::max<size_t>(1, total_layers)));
    CUDA_TRY(c, cudaMemcpy(c->d_node_layer, node_layer.data(), node_layer.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(c, cudaMemcpy(c->d_walls, c->walls.data(), c->walls.size() * sizeof(WallInfo), cudaMemcpyHostToDevice));

    if ((st = upload_reals(c, c->d_Tref, c->Tref)) != HYGRO_OK) return st;
    if ((st = upload_reals(c, c->d_Pref, c->Pref)) != HYGRO_OK) return st;
    // uniform initial state: zero deviation at both levels, step 0, no accumulated flux
    for (int i = 0; i < 2; ++i) {
        CUDA_TRY(c, cudaMemset(c->dT[i], 0, (size_t)c->total_nodes * c->real_size));
        CUDA_TRY(c, cudaMemset(c->dP[i], 0, (size_t)c->total_nodes * c->real_size));
    }
    CUDA_TRY(c, cudaMemset(c->d_cumul, 0, (size_t)W * 4 * sizeof(double)));
    CUDA_TRY(c, cudaMemset(c->d_flast, 0, (size_t)W * 4 * sizeof(double)));
    c->step = 0;
    c->cur = 0;
    c->have_materials = true;
    hygro_status sst = build_schedule(c);
    if (sst != HYGRO_OK) return sst;
    return upload_faces(c);
}

hygro_status hygro_set_bc(hygro_ctx *c, int32_t face, const hygro_bc *bc)
{
    if (c == nullptr) return fail(nullptr, HYGRO_E_INVALID, "ctx is NULL");
    FAULT_POINT(c, "hygro_set_bc");
    if (face != 0 && face != 1) return fail(c, HYGRO_E_INVALID, "face must be 0 or 1");
    if (bc == nullptr) return fail(c, HYGRO_E_INVALID, "bc is NULL");
    for (int w = 0; w < c->W; ++w) {
        std::string why;
        // the table values are checked by upload_noise as they are copied
        const hygro_status st = check_bc(bc[w], true, c->t0, c->dt, &why, false);
        if (st != HYGRO_OK) return fail(c, st, "wall %d face %d: %s", w, face, why.c_str());
    }
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, HYGRO_E_CUDA, "cudaSetDevice failed");
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    std::vector<RawBc> v(c->W);
    for (int w = 0; w < c->W; ++w) {
        v[w].bc = bc[w];
        v[w].bc.noise = nullptr;
    }
    {
        const hygro_status nst = upload_noise(c, face, bc, v);
        if (nst != HYGRO_OK) return nst;
    }
    c->bc[face].swap(v);
    c->have_bc[face] = true;
    hygro_status sst = build_schedule(c);
    if (sst != HYGRO_OK) return sst;
    return upload_faces(c);
}

hygro_status hygro_set_rooms(hygro_ctx *c, int32_t n_rooms, const hygro_room *rooms, const double *wall_area)
{
    if (c == nullptr) return fail(nullptr, HYGRO_E_INVALID, "ctx is NULL");
    FAULT_POINT(c, "hygro_set_rooms");
    if (n_rooms < 0) return fail(c, HYGRO_E_INVALID, "n_rooms must be >= 0");
    if (n_rooms > 0 && (rooms == nullptr || wall_area == nullptr))
        return fail(c, HYGRO_E_INVALID, "rooms and wall_area are required");
    for (int r = 0; r < n_rooms; ++r) {
        const hygro_room &q = rooms[r];
        const double v[] = {q.volume, q.ach, q.Q_gain, q.g_vap, q.T_out_mean, q.T_out_amp, q.P_out_mean, q.P_out_amp,
                            q.period, q.phase_T, q.phase_P, q.rho_a, q.cp_a, q.cp_v, q.Pv_ref, q.Ta0, q.Pa0,
                            q.period_P, q.g_pulse, q.pulse_on, q.pulse_off, q.pulse_period};
        for (double x : v)
            if (!std::isfinite(x)) return fail(c, HYGRO_E_INVALID, "room %d: non-finite value", r);
        if (!(q.volume > 0 && q.rho_a > 0 && q.cp_a > 0 && q.Pv_ref > 0 && q.ach >= 0 && q.period >= 0 &&
              q.period_P >= 0 && q.pulse_period >= 0))
            return fail(c, HYGRO_E_INVALID,
                        "room %d: volume, rho_a, cp_a, Pv_ref must be > 0, ach, period, period_P, pulse_period >= 0", r);
    }
    if (n_rooms > 0)
        for (int w = 0; w < c->W; ++w)
            if (!finite_nonneg(wall_area[w])) return fail(c, HYGRO_E_INVALID, "wall %d: area must be >= 0", w);
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, HYGRO_E_CUDA, "cudaSetDevice failed");
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if ((size_t)n_rooms > c->rooms_cap) {
        if (c->d_rooms) cudaFree(c->d_rooms);
        if (c->d_room_state) cudaFree(c->d_room_state);
        c->d_rooms = nullptr;
        c->d_room_state = nullptr;
        c->rooms_cap = 0;
        CUDA_TRY(c, dalloc(&c->d_rooms, (size_t)n_rooms));
        CUDA_TRY(c, dalloc(&c->d_room_state, (size_t)n_rooms * 4));
        c->rooms_cap = (size_t)n_rooms;
    }
    c->rooms.assign(rooms, rooms + n_rooms);
    c->face_emis.clear();
    c->room_view.clear();
    c->link_zone.clear();
    c->link_flow.clear();
    if (n_rooms > 0)
        c->wall_area.assign(wall_area, wall_area + c->W);
    else
        c->wall_area.clear();
    std::vector<double> st((size_t)n_rooms * 4);
    for (int r = 0; r < n_rooms; ++r) {
        st[r * 4 + 0] = st[r * 4 + 1] = rooms[r].Ta0;
        st[r * 4 + 2] = st[r * 4 + 3] = rooms[r].Pa0;
    }
    if (n_rooms > 0)
        CUDA_TRY(c, cudaMemcpy(c->d_room_state, st.data(), st.size() * sizeof(double), cudaMemcpyHostToDevice));
    c->have_rooms = true;
    return build_schedule(c);
}

hygro_status hygro_set_radiation(hygro_ctx *c, const double *emissivity, const double *view)
{
    if (c == nullptr) return fail(nullptr, HYGRO_E_INVALID, "ctx is NULL");
    FAULT_POINT(c, "hygro_set_radiation");
    if (!c->have_rooms || c->rooms.empty()) return fail(c, HYGRO_E_STATE, "hygro_set_rooms must come first");
    if (emissivity == nullptr || view == nullptr) return fail(c, HYGRO_E_INVALID, "emissivity and view are required");
    for (int i = 0; i < 2 * c->W; ++i)
        if (!(emissivity[i] >= 0.0 && emissivity[i] <= 1.0))
            return fail(c, HYGRO_E_INVALID, "wall %d face %d: emissivity must be in [0, 1]", i / 2, i % 2);
    for (size_t r = 0; r < c->rooms.size(); ++r)
        if (!(view[r] >= 0.0 && view[r] <= 1.0)) return fail(c, HYGRO_E_INVALID, "room %zu: view factor must be in [0, 1]", r);
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, HYGRO_E_CUDA, "cudaSetDevice failed");
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->face_emis.assign(emissivity, emissivity + 2 * c->W);
    c->room_view.assign(view, view + c->rooms.size());
    return build_schedule(c);
}

hygro_status hygro_set_interzone(hygro_ctx *c, int32_t n_links, const int32_t *zones, const double *flow)
{
    if (c == nullptr) return fail(nullptr, HYGRO_E_INVALID, "ctx is NULL");
    FAULT_POINT(c, "hygro_set_interzone");
    if (!c->have_rooms || c->rooms.empty()) return fail(c, HYGRO_E_STATE, "hygro_set_rooms must come first");
    if (n_links < 0 || (n_links > 0 && (zones == nullptr || flow == nullptr)))
        return fail(c, HYGRO_E_INVALID, "n_links must be >= 0, zones and flow given");
    const int NR = (int)c->rooms.size();
    for (int l = 0; l < n_links; ++l) {
        const int a = zones[2 * l], b = zones[2 * l + 1];
        if (a < 0 || a >= NR || b < 0 || b >= NR || a == b)
            return fail(c, HYGRO_E_INVALID, "link %d: rooms must be two different rooms in 0..%d", l, NR - 1);
        if (!(flow[l] >= 0.0) || !std::isfinite(flow[l]))
            return fail(c, HYGRO_E_INVALID, "link %d: flow must be finite and >= 0", l);
    }
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, HYGRO_E_CUDA, "cudaSetDevice failed");
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->link_zone.assign(zones, zones + 2 * n_links);
    c->link_flow.assign(flow, flow + n_links);
    return build_schedule(c);
}

hygro_status hygro_set_vapour_fraction(hygro_ctx *c, const double *nu)
{
    if (c == nullptr) return fail(nullptr, HYGRO_E_INVALID, "ctx is NULL");
    FAULT_POINT(c, "hygro_set_vapour_fraction");
    if (nu == nullptr) return fail(c, HYGRO_E_INVALID, "nu is NULL");
    for (int w = 0; w < c->W; ++w)
        if (!finite_nonneg(nu[w])) return fail(c, HYGRO_E_INVALID, "wall %d: nu must be finite and >= 0", w);
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, HYGRO_E_CUDA, "cudaSetDevice failed");
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    size_t lo = 0;
    for (int w = 0; w < c->W; ++w) {
        WallInfo &wi = c->walls[w];
        wi.nu = nu[w];
        // the simple-heat code variant assumes nu = 1
        if (c->have_materials) {
            wi.simple = wi.nu == 1.0 ? 1 : 0;
            for (int l = 0; l < c->n_layers[w]; ++l) {
                const hygro_layer &y = c->layers[lo + l];
                if (y.aT != 0.0 || y.bT != 0.0 || y.chi != 0.0) wi.simple = 0;
            }
            lo += c->n_layers[w];
        }
    }
    CUDA_TRY(c, cudaMemcpy(c->d_walls, c->walls.data(), c->walls.size() * sizeof(WallInfo), cudaMemcpyHostToDevice));
    if (c->have_materials) {
        const hygro_status st = build_schedule(c);
        if (st != HYGRO_OK) return st;
    }
    return HYGRO_OK;
}

hygro_status hygro_set_layer_law(hygro_ctx *c, const int32_t *law)
{
    if (c == nullptr) return fail(nullptr, HYGRO_E_INVALID, "ctx is NULL");
    FAULT_POINT(c, "hygro_set_layer_law");
    if (law == nullptr) return fail(c, HYGRO_E_INVALID, "law is NULL");
    if (!c->have_materials) return fail(c, HYGRO_E_STATE, "hygro_set_materials must come first");
    const size_t nl = c->law.size();
    for (size_t l = 0; l < nl; ++l)
        if (law[l] < HYGRO_LAW_AFFINE || law[l] > HYGRO_LAW_TABLE1_C)
            return fail(c, HYGRO_E_INVALID, "layer %zu: unknown coefficient law %d", l, law[l]);
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, HYGRO_E_CUDA, "cudaSetDevice failed");
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    std::vector<int8_t> l8(std::max<size_t>(1, nl), 0);
    bool any = false;
    for (int w = 0; w < c->W; ++w) {
        WallInfo &wi = c->walls[w];
        wi.has_law = 0;
        for (int l = 0; l < wi.n_layers; ++l) {
            const int32_t v = law[wi.layer_off + l];
            l8[wi.layer_off + l] = (int8_t)v;
            if (v != HYGRO_LAW_AFFINE) wi.has_law = 1;
        }
        any = any || wi.has_law;
    }
    CUDA_TRY(c, cudaMemcpy(c->d_layer_law, l8.data(), l8.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(c, cudaMemcpy(c->d_walls, c->walls.data(), c->walls.size() * sizeof(WallInfo), cudaMemcpyHostToDevice));
    c->law.assign(law, law + nl);
    c->any_law = any;
    return HYGRO_OK;
}

hygro_status hygro_set_option(hygro_ctx *c, int32_t option, int64_t value)
{
    if (c == nullptr) return fail(nullptr, HYGRO_E_INVALID, "ctx is NULL");
    FAULT_POINT(c, "hygro_set_option");
    if (option == HYGRO_OPT_ROOM_SCHEME) {
        if (value != HYGRO_ROOM_DF && value != HYGRO_ROOM_EULER)
            return fail(c, HYGRO_E_INVALID, "room scheme must be HYGRO_ROOM_DF or HYGRO_ROOM_EULER");
        if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, HYGRO_E_CUDA, "cudaSetDevice failed");
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        c->room_scheme = (int)value;
        return build_schedule(c);   // rebuilds the device room descriptors
    }
    return fail(c, HYGRO_E_INVALID, "unknown option %d", option);
}

hygro_status hygro_get_rooms(hygro_ctx *c, int32_t level, double *Ta, double *Pa)
{
    if (c == nullptr) return fail(nullptr, HYGRO_E_INVALID, "ctx is NULL");
    FAULT_POINT(c, "hygro_get_rooms");
    if (level != 0 && level != 1) return fail(c, HYGRO_E_INVALID, "level must be 0 (n) or 1 (n-1)");
    const int NR = (int)c->rooms.size();
    if (NR == 0) return HYGRO_OK;
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, HYGRO_E_CUDA, "cudaSetDevice failed");
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    std::vector<double> st((size_t)NR * 4), a(NR), b(NR);
    CUDA_TRY(c, cudaMemcpy(st.data(), c->d_room_state, st.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (int r = 0; r < NR; ++r) {
        a[r] = st[r * 4 + (level == 0 ? 1 : 0)];
        b[r] = st[r * 4 + (level == 0 ? 3 : 2)];
    }
    if (Ta) CUDA_TRY(c, cudaMemcpy(Ta, a.data(), NR * sizeof(double), cudaMemcpyDefault));
    if (Pa) CUDA_TRY(c, cudaMemcpy(Pa, b.data(), NR * sizeof(double), cudaMemcpyDefault));
    return HYGRO_OK;
}

hygro_status hygro_run(hygro_ctx *c, int64_t n_steps, int32_t sample_every, void *samples, size_t samples_bytes)
{
    if (c == nullptr) return fail(nullptr, HYGRO_E_INVALID, "ctx is NULL");
    FAULT_POINT(c, "hygro_run");
    if (n_steps < 0) return fail(c, HYGRO_E_INVALID, "n_steps must be >= 0");
    if (samples != nullptr && sample_every < 1) return fail(c, HYGRO_E_INVALID, "sample_every must be >= 1");
    if (!(c->have_materials && c->have_bc[0] && c->have_bc[1]))
        return fail(c, HYGRO_E_STATE, "hygro_set_materials and hygro_set_bc (both faces) must come first");
    {
        const hygro_status rst = rooms_ready(c);
        if (rst != HYGRO_OK) return rst;
    }
    const int64_t n_samples = samples ? n_steps / sample_every : 0;
    const size_t need = (size_t)n_samples * c->W * 4 * c->real_size;
    if (samples != nullptr && samples_bytes < need)
        return fail(c, HYGRO_E_INVALID, "samples_bytes %zu < %zu needed", samples_bytes, need);
    if (n_steps == 0) return HYGRO_OK;
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, HYGRO_E_CUDA, "cudaSetDevice failed");

    const bool host_samples = samples != nullptr && n_samples > 0 && !is_device_ptr(samples);
    void *dsamp = samples;
    if (host_samples) {
        if (need > c->samples_cap) {
            if (c->d_samples) cudaFree(c->d_samples);
            c->d_samples = nullptr;
            c->samples_cap = 0;
            CUDA_TRY(c, cudaMalloc(&c->d_samples, need));
            c->samples_cap = need;
        }
        dsamp = c->d_samples;
    }
    if (n_samples == 0) dsamp = nullptr;
    const int se = samples ? sample_every : 0;

    {
        const hygro_status lst = launch_steps(c, n_steps, se, dsamp);
        if (lst != HYGRO_OK) return lst;
    }
    c->step += n_steps;
    if (c->d_trace != nullptr && c->kernel == HYGRO_KERNEL_PERSISTENT) {
        std::vector<unsigned long long> tr((size_t)c->W * 4);
        CUDA_TRY(c, cudaMemcpyAsync(tr.data(), c->d_trace, tr.size() * sizeof(unsigned long long),
                                    cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        if (FILE *f = fopen(c->trace_path.c_str(), "a")) {
            for (int w = 0; w < c->W; ++w) {
                const unsigned long long *t = &tr[(size_t)w * 4];
                fprintf(f, "%d %d %d %d %llu %llu %llu %d %d %d\n", w, (int)(t[0] >> 32), (int)((t[0] >> 8) & 0xFFFFFF),
                        (int)(t[0] & 0xFF), t[1], t[2], t[3], c->walls[w].K, c->walls[w].N,
                        c->walls[w].aligned ? (c->walls[w].simple ? 0 : 1) : (c->walls[w].simple ? 3 : 2));
            }
            fclose(f);
        }
    }
    if (host_samples) {
        CUDA_TRY(c, cudaMemcpyAsync(samples, dsamp, need, cudaMemcpyDeviceToHost, c->stream));
        return check_nonfinite(c);
    }
    return HYGRO_OK;
}

hygro_status hygro_start_euler(hygro_ctx *c)
{
    if (c == nullptr) return fail(nullptr, HYGRO_E_INVALID, "ctx is NULL");
    FAULT_POINT(c, "hygro_start_euler");
    if (!(c->have_materials && c->have_bc[0] && c->have_bc[1]))
        return fail(c, HYGRO_E_STATE, "hygro_set_materials and hygro_set_bc (both faces) must come first");
    if (c->step != 0) return fail(c, HYGRO_E_STATE, "the Euler start applies at step 0 (the context is at %lld)",
                                  (long long)c->step);
    if (c->any_law) return fail(c, HYGRO_E_UNSUPPORTED, "the Euler start covers the affine coefficient laws only");
    for (int w = 0; w < c->W; ++w)
        for (int f = 0; f < 2; ++f)
            if (c->bc[f][w].bc.kind == HYGRO_BC_ROOM)
                return fail(c, HYGRO_E_UNSUPPORTED, "wall %d has a room face: the Euler start covers walls without rooms",
                            w);
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, HYGRO_E_CUDA, "cudaSetDevice failed");
    int Nmax = 0;
    for (int w = 0; w < c->W; ++w) Nmax = std::max(Nmax, c->N[w]);
    const int64_t max_sub = (int64_t)1 << 24;
    const size_t nb = (size_t)c->total_nodes * c->real_size;
    int64_t *dm = nullptr;
    void *s1T = nullptr, *s1P = nullptr;
    std::vector<double> cum_save((size_t)c->W * 4), fl_save((size_t)c->W * 4);
    cudaError_t e = cudaMalloc(&dm, (size_t)c->W * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMalloc(&s1T, nb);
    if (e == cudaSuccess) e = cudaMalloc(&s1P, nb);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = cudaMemcpy(cum_save.data(), c->d_cumul, cum_save.size() * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(fl_save.data(), c->d_flast, fl_save.size() * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) {
        // level 1 goes to scratch buffers; the stored levels change only if every wall is accepted
        const int prv = 1 - c->cur;
        if (c->precision == HYGRO_FP64) {
            DevCtx<double> d = make_dev<double>(c);
            d.T[prv] = (double *)s1T;
            d.P[prv] = (double *)s1P;
            e = launch_euler_start_f64(d, Nmax, max_sub, dm, c->stream);
        } else {
            DevCtx<float> d = make_dev<float>(c);
            d.T[prv] = (float *)s1T;
            d.P[prv] = (float *)s1P;
            e = launch_euler_start_f32(d, Nmax, max_sub, dm, c->stream);
        }
    }
    std::vector<int64_t> m((size_t)c->W, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m.data(), dm, m.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    bool refused = false;
    int bad_wall = -1;
    if (e == cudaSuccess)
        for (int w = 0; w < c->W && !refused; ++w)
            if (m[w] == 0) {
                refused = true;
                bad_wall = w;
            }
    if (e == cudaSuccess && !refused) {
        const int prv = 1 - c->cur;
        e = cudaMemcpy(c->dT[prv], s1T, nb, cudaMemcpyDeviceToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(c->dP[prv], s1P, nb, cudaMemcpyDeviceToDevice);
    }
    if (e == cudaSuccess && refused) {
        e = cudaMemcpy(c->d_cumul, cum_save.data(), cum_save.size() * sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(c->d_flast, fl_save.data(), fl_save.size() * sizeof(double), cudaMemcpyHostToDevice);
    }
    cudaFree(dm);
    cudaFree(s1T);
    cudaFree(s1P);
    if (e != cudaSuccess) return fail(c, HYGRO_E_CUDA, "Euler start: %s", cudaGetErrorString(e));
    if (refused)
        return fail(c, HYGRO_E_UNSUPPORTED, "wall %d needs more than %lld Euler substeps", bad_wall, (long long)max_sub);
    c->cur = 1 - c->cur;
    c->step = 1;
    return check_nonfinite(c);
}

hygro_status hygro_sync(hygro_ctx *c)
{
    if (c == nullptr) return fail(nullptr, HYGRO_E_INVALID, "ctx is NULL");
    FAULT_POINT(c, "hygro_sync");
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, HYGRO_E_CUDA, "cudaSetDevice failed");
    return check_nonfinite(c);
}

hygro_status hygro_fluxes(hygro_ctx *c, double *flux, double *cumulative)
{
    if (c == nullptr) return fail(nullptr, HYGRO_E_INVALID, "ctx is NULL");
    FAULT_POINT(c, "hygro_fluxes");
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, HYGRO_E_CUDA, "cudaSetDevice failed");
    const size_t bytes = (size_t)c->W * 4 * sizeof(double);
    if (flux) CUDA_TRY(c, cudaMemcpyAsync(flux, c->d_flast, bytes, cudaMemcpyDefault, c->stream));
    if (cumulative) CUDA_TRY(c, cudaMemcpyAsync(cumulative, c->d_cumul, bytes, cudaMemcpyDefault, c->stream));
    return check_nonfinite(c);
}

hygro_status hygro_balance(hygro_ctx *c, double *bal)
{
    if (c == nullptr) return fail(nullptr, HYGRO_E_INVALID, "ctx is NULL");
    FAULT_POINT(c, "hygro_balance");
    if (bal == nullptr) return fail(c, HYGRO_E_INVALID, "bal is NULL");
    if (!(c->have_materials && c->have_bc[0] && c->have_bc[1]))
        return fail(c, HYGRO_E_STATE, "hygro_set_materials and hygro_set_bc (both faces) must come first");
    for (int w = 0; w < c->W; ++w)
        for (int f = 0; f < 2; ++f)
            if (c->bc[f][w].bc.kind == HYGRO_BC_ROOM)
                return fail(c, HYGRO_E_UNSUPPORTED, "wall %d has a room face: the balance covers walls without rooms", w);
    if (c->any_law) return fail(c, HYGRO_E_UNSUPPORTED, "the balance covers the affine coefficient laws only");
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, HYGRO_E_CUDA, "cudaSetDevice failed");
    const size_t nb = (size_t)c->total_nodes * c->real_size;
    void *sT = nullptr, *sP = nullptr, *sc = nullptr, *sf = nullptr, *db = nullptr;
    hygro_status st = HYGRO_OK;
    auto release = [&]() {
        void *ps[] = {sT, sP, sc, sf, db};
        for (void *q : ps)
            if (q) cudaFree(q);
    };
#define BAL_TRY(call)                                                                                   \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess) {                                                                        \
            st = fail(c, e_ == cudaErrorMemoryAllocation ? HYGRO_E_NOMEM : HYGRO_E_CUDA, "%s: %s", #call, \
                      cudaGetErrorString(e_));                                                          \
            release();                                                                                  \
            return st;                                                                                  \
        }                                                                                               \
    } while (0)
    BAL_TRY(cudaMalloc(&sT, nb));
    BAL_TRY(cudaMalloc(&sP, nb));
    BAL_TRY(cudaMalloc(&sc, (size_t)c->W * 4 * sizeof(double)));
    BAL_TRY(cudaMalloc(&sf, (size_t)c->W * 4 * sizeof(double)));
    BAL_TRY(cudaMalloc(&db, (size_t)c->W * 8 * sizeof(double)));
    BAL_TRY(after_host_copies(c));
    BAL_TRY(cudaMemsetAsync(db, 0, (size_t)c->W * 8 * sizeof(double), c->stream));
    BAL_TRY(cudaMemsetAsync(sc, 0, (size_t)c->W * 4 * sizeof(double), c->stream));
    // pass 1: the step n -> n+1 into scratch copies of level n-1 (the plain kernel writes in place)
    const int prv = 1 - c->cur;
    BAL_TRY(cudaMemcpyAsync(sT, c->dT[prv], nb, cudaMemcpyDeviceToDevice, c->stream));
    BAL_TRY(cudaMemcpyAsync(sP, c->dP[prv], nb, cudaMemcpyDeviceToDevice, c->stream));
    cudaError_t e;
    if (c->precision == HYGRO_FP64) {
        DevCtx<double> d = make_dev<double>(c);
        DevCtx<double> ds = d;
        ds.T[prv] = (double *)sT;
        ds.P[prv] = (double *)sP;
        ds.cumul = (double *)sc;
        ds.flast = (double *)sf;
        e = launch_plain_step_f64(ds, c->step, -1, nullptr, c->stream);
        if (e == cudaSuccess)
            e = launch_balance_f64(d, (const double *)c->dT[prv], (const double *)c->dP[prv], (const double *)sT,
                                   (const double *)sP, c->step, (double *)db, c->stream);
    } else {
        DevCtx<float> d = make_dev<float>(c);
        DevCtx<float> ds = d;
        ds.T[prv] = (float *)sT;
        ds.P[prv] = (float *)sP;
        ds.cumul = (double *)sc;
        ds.flast = (double *)sf;
        e = launch_plain_step_f32(ds, c->step, -1, nullptr, c->stream);
        if (e == cudaSuccess)
            e = launch_balance_f32(d, (const float *)c->dT[prv], (const float *)c->dP[prv], (const float *)sT,
                                   (const float *)sP, c->step, (double *)db, c->stream);
    }
    BAL_TRY(e);
    BAL_TRY(cudaMemcpyAsync(bal, db, (size_t)c->W * 8 * sizeof(double), cudaMemcpyDefault, c->stream));
    BAL_TRY(cudaStreamSynchronize(c->stream));
#undef BAL_TRY
    release();
    return check_nonfinite(c);
}

hygro_status hygro_get_fields(hygro_ctx *c, int32_t level, double *T, double *P)
{
    if (c == nullptr) return fail(nullptr, HYGRO_E_INVALID, "ctx is NULL");
    FAULT_POINT(c, "hygro_get_fields");
    if (level != 0 && level != 1) return fail(c, HYGRO_E_INVALID, "level must be 0 (n) or 1 (n-1)");
    if (!c->have_materials) return fail(c, HYGRO_E_STATE, "hygro_set_materials must come first");
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, HYGRO_E_CUDA, "cudaSetDevice failed");
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    const int buf = level == 0 ? c->cur : 1 - c->cur;
    std::vector<double> v((size_t)c->total_nodes);
    for (int f = 0; f < 2; ++f) {
        double *dst = f == 0 ? T : P;
        if (dst == nullptr) continue;
        hygro_status st = download_reals(c, f == 0 ? c->dT[buf] : c->dP[buf], v);
        if (st != HYGRO_OK) return st;
        const std::vector<double> &ref = f == 0 ? c->Tref : c->Pref;
        for (int w = 0; w < c->W; ++w)
            for (int j = 0; j < c->N[w]; ++j) v[(size_t)c->walls[w].node_off + j] += ref[w];
        CUDA_TRY(c, cudaMemcpy(dst, v.data(), v.size() * sizeof(double), cudaMemcpyDefault));
    }
    return check_nonfinite(c);
}

hygro_status hygro_set_fields(hygro_ctx *c, int32_t level, const double *T, const double *P)
{
    if (c == nullptr) return fail(nullptr, HYGRO_E_INVALID, "ctx is NULL");
    FAULT_POINT(c, "hygro_set_fields");
    if (level != 0 && level != 1) return fail(c, HYGRO_E_INVALID, "level must be 0 (n) or 1 (n-1)");
    if (!c->have_materials) return fail(c, HYGRO_E_STATE, "hygro_set_materials must come first");
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, HYGRO_E_CUDA, "cudaSetDevice failed");
    std::vector<double> v[2];
    for (int f = 0; f < 2; ++f) {
        const double *src = f == 0 ? T : P;
        if (src == nullptr) continue;
        v[f].resize((size_t)c->total_nodes);
        CUDA_TRY(c, cudaMemcpy(v[f].data(), src, v[f].size() * sizeof(double), cudaMemcpyDefault));
        for (double x : v[f])
            if (!std::isfinite(x)) return fail(c, HYGRO_E_INVALID, "non-finite field value");
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    const int buf = level == 0 ? c->cur : 1 - c->cur;
    for (int f = 0; f < 2; ++f) {
        if (v[f].empty()) continue;
        const std::vector<double> &ref = f == 0 ? c->Tref : c->Pref;
        for (int w = 0; w < c->W; ++w)
            for (int j = 0; j < c->N[w]; ++j) v[f][(size_t)c->walls[w].node_off + j] -= ref[w];
        hygro_status st = upload_reals(c, f == 0 ? c->dT[buf] : c->dP[buf], v[f]);
        if (st != HYGRO_OK) return st;
    }
    return HYGRO_OK;
}

hygro_status hygro_get_step(const hygro_ctx *c, int64_t *step)
{
    if (c == nullptr || step == nullptr) return fail(nullptr, HYGRO_E_INVALID, "ctx or step is NULL");
    *step = c->step;
    return HYGRO_OK;
}

// State image: magic, precision, walls, nodes, step | T[n], T[n-1], P[n], P[n-1] (working precision) | cumul,
// flast (FP64).
hygro_status hygro_get_state(hygro_ctx *c, void *buf, size_t *bytes)
{
    if (c == nullptr || bytes == nullptr) return fail(c, HYGRO_E_INVALID, "ctx or bytes is NULL");
    FAULT_POINT(c, "hygro_get_state");
    return get_state_impl(c, buf, bytes);
}

hygro_status hygro_set_state(hygro_ctx *c, const void *buf, size_t bytes)
{
    if (c == nullptr || buf == nullptr) return fail(c, HYGRO_E_INVALID, "ctx or buf is NULL");
    FAULT_POINT(c, "hygro_set_state");
    return set_state_impl(c, buf, bytes);
}

}  // extern "C"

namespace {

hygro_status get_state_impl(hygro_ctx *c, void *buf, size_t *bytes)
{
    const size_t nf = (size_t)c->total_nodes * c->real_size;
    const size_t nroom = c->rooms.size() * 4 * sizeof(double);
    const size_t need = 5 * sizeof(int64_t) + 4 * nf + 2 * (size_t)c->W * 4 * sizeof(double) + nroom;
    if (buf == nullptr) {
        *bytes = need;
        return HYGRO_OK;
    }
    if (*bytes < need) return fail(c, HYGRO_E_INVALID, "state buffer too small (%zu < %zu)", *bytes, need);
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, HYGRO_E_CUDA, "cudaSetDevice failed");
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    char *p = (char *)buf;
    const int64_t hdr[5] = {(int64_t)kStateMagic, c->precision, c->W, c->total_nodes, c->step};
    memcpy(p, hdr, sizeof hdr);
    p += sizeof hdr;
    void *src[4] = {c->dT[c->cur], c->dT[1 - c->cur], c->dP[c->cur], c->dP[1 - c->cur]};
    for (void *s : src) {
        CUDA_TRY(c, cudaMemcpy(p, s, nf, cudaMemcpyDeviceToHost));
        p += nf;
    }
    CUDA_TRY(c, cudaMemcpy(p, c->d_cumul, (size_t)c->W * 4 * sizeof(double), cudaMemcpyDeviceToHost));
    p += (size_t)c->W * 4 * sizeof(double);
    CUDA_TRY(c, cudaMemcpy(p, c->d_flast, (size_t)c->W * 4 * sizeof(double), cudaMemcpyDeviceToHost));
    p += (size_t)c->W * 4 * sizeof(double);
    if (nroom) CUDA_TRY(c, cudaMemcpy(p, c->d_room_state, nroom, cudaMemcpyDeviceToHost));
    *bytes = need;
    return HYGRO_OK;
}

hygro_status set_state_impl(hygro_ctx *c, const void *buf, size_t bytes)
{
    const size_t nf = (size_t)c->total_nodes * c->real_size;
    const size_t nroom = c->rooms.size() * 4 * sizeof(double);
    const size_t need = 5 * sizeof(int64_t) + 4 * nf + 2 * (size_t)c->W * 4 * sizeof(double) + nroom;
    if (bytes < need) return fail(c, HYGRO_E_INVALID, "state image too small");
    int64_t hdr[5];
    memcpy(hdr, buf, sizeof hdr);
    if (hdr[0] != (int64_t)kStateMagic || hdr[1] != c->precision || hdr[2] != c->W || hdr[3] != c->total_nodes)
        return fail(c, HYGRO_E_INVALID, "state image does not match this context");
    if (!c->have_materials) return fail(c, HYGRO_E_STATE, "hygro_set_materials must come first");
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, HYGRO_E_CUDA, "cudaSetDevice failed");
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    const char *p = (const char *)buf + sizeof hdr;
    c->cur = 0;
    void *dst[4] = {c->dT[0], c->dT[1], c->dP[0], c->dP[1]};
    for (void *d : dst) {
        CUDA_TRY(c, cudaMemcpy(d, p, nf, cudaMemcpyHostToDevice));
        p += nf;
    }
    CUDA_TRY(c, cudaMemcpy(c->d_cumul, p, (size_t)c->W * 4 * sizeof(double), cudaMemcpyHostToDevice));
    p += (size_t)c->W * 4 * sizeof(double);
    CUDA_TRY(c, cudaMemcpy(c->d_flast, p, (size_t)c->W * 4 * sizeof(double), cudaMemcpyHostToDevice));
    p += (size_t)c->W * 4 * sizeof(double);
    if (nroom) CUDA_TRY(c, cudaMemcpy(c->d_room_state, p, nroom, cudaMemcpyHostToDevice));
    c->step = hdr[4];
    return HYGRO_OK;
}

// The persistent kernel's n_steps from the current state, timed with CUDA events on the context's stream.
hygro_status timed_probe(hygro_ctx *c, int64_t n_steps, float *ms)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CUDA_TRY(c, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(c, HYGRO_E_CUDA, "cudaEventCreate failed");
    }
    hygro_status st = HYGRO_OK;
    if (cudaEventRecord(e0, c->stream) != cudaSuccess) st = fail(c, HYGRO_E_CUDA, "cudaEventRecord failed");
    if (st == HYGRO_OK) st = launch_steps(c, n_steps, 0, nullptr);
    if (st == HYGRO_OK && (cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                           cudaEventElapsedTime(ms, e0, e1) != cudaSuccess))
        st = fail(c, HYGRO_E_CUDA, "timing the probe failed");
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

}  // namespace

extern "C" {

hygro_status hygro_autotune(hygro_ctx *c, int32_t probe_steps, double *model, double *ms)
{
    if (c == nullptr) return fail(nullptr, HYGRO_E_INVALID, "ctx is NULL");
    FAULT_POINT(c, "hygro_autotune");
    if (probe_steps < 16 || probe_steps > (1 << 20)) return fail(c, HYGRO_E_INVALID, "probe_steps must be in 16..2^20");
    if (!(c->have_materials && c->have_bc[0] && c->have_bc[1]))
        return fail(c, HYGRO_E_STATE, "hygro_set_materials and hygro_set_bc (both faces) must come first");
    if (c->kernel != HYGRO_KERNEL_PERSISTENT || c->any_room_walls || c->n_free == 0 || c->any_law)
        return fail(c, HYGRO_E_UNSUPPORTED, "the autotuner schedules walls of the persistent kernel without rooms");
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, HYGRO_E_CUDA, "cudaSetDevice failed");
    size_t bytes = 0;
    hygro_status st = get_state_impl(c, nullptr, &bytes);
    if (st != HYGRO_OK) return st;
    std::vector<char> saved(bytes);
    st = get_state_impl(c, saved.data(), &bytes);
    if (st != HYGRO_OK) return st;
    const CostModel old_model = c->cost;
    // 1. a traced probe: every wall's start and end time on the GPU clock
    unsigned long long *own_trace = nullptr;
    if (c->d_trace == nullptr) {
        CUDA_TRY(c, cudaMalloc(&own_trace, (size_t)c->W * 4 * sizeof(unsigned long long)));
        c->d_trace = own_trace;
    }
    auto finish = [&](hygro_status s) {
        if (own_trace) {
            cudaFree(own_trace);
            c->d_trace = nullptr;
        }
        const hygro_status r = set_state_impl(c, saved.data(), saved.size());
        return s != HYGRO_OK ? s : r;
    };
    st = launch_steps(c, probe_steps, 0, nullptr);
    std::vector<unsigned long long> tr((size_t)c->W * 4);
    if (st == HYGRO_OK && (cudaMemcpyAsync(tr.data(), c->d_trace, tr.size() * sizeof(unsigned long long),
                                           cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
                           cudaStreamSynchronize(c->stream) != cudaSuccess))
        st = fail(c, HYGRO_E_CUDA, "reading the probe's wall trace failed");
    if (own_trace) {
        cudaFree(own_trace);
        own_trace = nullptr;
        c->d_trace = nullptr;
    }
    if (st != HYGRO_OK) return finish(st);
    // 2. fit the per-variant step time a + b K to the walls' measured ns per step
    std::vector<SchedWall> sw;
    std::vector<double> ns;
    for (int w = 0; w < c->W; ++w) {
        const WallInfo &x = c->walls[w];
        const bool simple = x.simple && c->precision == HYGRO_FP32;
        sw.push_back({w, x.K, x.aligned ? (simple ? 0 : 1) : (simple ? 3 : 2), x.N});
        const unsigned long long *t = &tr[(size_t)w * 4];
        ns.push_back(t[2] > t[1] && t[3] > 0 ? (double)(t[2] - t[1]) / (double)t[3] : -1.0);
    }
    CostModel fitted;
    fit_cost_model(sw, ns, old_model, fitted);
    // 3. the probe again with the current schedule and with the refitted one; keep the faster
    float ms_old = 0.0f, ms_new = 0.0f;
    st = set_state_impl(c, saved.data(), saved.size());
    if (st == HYGRO_OK) st = timed_probe(c, probe_steps, &ms_old);
    if (st == HYGRO_OK) {
        c->cost = fitted;
        st = build_schedule(c);
    }
    if (st == HYGRO_OK) st = set_state_impl(c, saved.data(), saved.size());
    if (st == HYGRO_OK) st = timed_probe(c, probe_steps, &ms_new);
    if (st != HYGRO_OK || ms_new > ms_old) {
        c->cost = old_model;
        const hygro_status rs = build_schedule(c);
        if (st == HYGRO_OK) st = rs;
    }
    if (model) {
        for (int v = 0; v < 4; ++v) {
            model[v] = fitted.a[v];
            model[4 + v] = fitted.b[v];
        }
    }
    if (ms) {
        ms[0] = ms_old;
        ms[1] = ms_new;
    }
    return finish(st);
}

}  // extern "C"

// ---- hygro_run_noalloc: the same run with no device allocation ----------------------------------
//
// hygro_run stages samples bound for host memory in a device buffer that it allocates (and grows)
// on demand. This entry point stages them instead in the fixed array below, which is part of the
// library image: every GPU that loads the library holds it in its global memory until the process
// exits. Host code must not use the array's name as a device address (it names a host-side stand-in);
// the device address is looked up once per device with that device current and then reused.

static __device__ __align__(256) unsigned char g_noalloc_scratch[HYGRO_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mutex;
void *g_noalloc_ptr[kNoallocMaxDevices] = {};
}  // namespace

extern "C" {

hygro_status hygro_run_noalloc(hygro_ctx *c, int64_t n_steps, int32_t sample_every, void *samples,
                               size_t samples_bytes)
{
    if (c == nullptr) return fail(nullptr, HYGRO_E_INVALID, "ctx is NULL");
    FAULT_POINT(c, "hygro_run_noalloc");
    if (n_steps < 0) return fail(c, HYGRO_E_INVALID, "n_steps must be >= 0");
    if (samples != nullptr && sample_every < 1) return fail(c, HYGRO_E_INVALID, "sample_every must be >= 1");
    if (!(c->have_materials && c->have_bc[0] && c->have_bc[1]))
        return fail(c, HYGRO_E_STATE, "hygro_set_materials and hygro_set_bc (both faces) must come first");
    {
        const hygro_status rst = rooms_ready(c);
        if (rst != HYGRO_OK) return rst;
    }
    const int64_t n_samples = samples ? n_steps / sample_every : 0;
    const size_t need = (size_t)n_samples * c->W * 4 * c->real_size;
    if (samples != nullptr && samples_bytes < need)
        return fail(c, HYGRO_E_INVALID, "samples_bytes %zu < %zu needed", samples_bytes, need);
    if (c->device < 0 || c->device >= kNoallocMaxDevices)
        return fail(c, HYGRO_E_UNSUPPORTED, "device %d is beyond the no-allocation entry point's table", c->device);
    const bool host_samples = samples != nullptr && n_samples > 0 && !is_device_ptr(samples);
    if (host_samples && need > (size_t)HYGRO_NOALLOC_SCRATCH_BYTES)
        return fail(c, HYGRO_E_UNSUPPORTED,
                    "samples need %zu bytes of staging; hygro_run_noalloc holds %zu (use hygro_run, or fewer "
                    "samples per call)",
                    need, (size_t)HYGRO_NOALLOC_SCRATCH_BYTES);
    if (n_steps == 0) return HYGRO_OK;
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, HYGRO_E_CUDA, "cudaSetDevice failed");

    void *dsamp = samples;
    if (host_samples) {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (g_noalloc_ptr[c->device] == nullptr) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || p == nullptr)
                return fail(c, HYGRO_E_CUDA, "cudaGetSymbolAddress of the staging array: %s", cudaGetErrorString(e));
            g_noalloc_ptr[c->device] = p;
        }
        dsamp = g_noalloc_ptr[c->device];
    }
    if (n_samples == 0) dsamp = nullptr;
    const int se = samples ? sample_every : 0;

    // the staged samples are written in full by the kernels (both faces of every wall for every
    // sample), so nothing in the array has to be cleared first
    {
        const hygro_status lst = launch_steps(c, n_steps, se, dsamp);
        if (lst != HYGRO_OK) return lst;
    }
    c->step += n_steps;
    if (host_samples) {
        CUDA_TRY(c, cudaMemcpyAsync(samples, dsamp, need, cudaMemcpyDeviceToHost, c->stream));
        return check_nonfinite(c);
    }
    return HYGRO_OK;
}

hygro_status hygro_loss_grad(hygro_ctx *c, int64_t n_steps, int32_t sample_every, const float *obs, double wT,
                             double wP, int32_t checkpoint_every, double *loss, double *grad)
{
    if (c == nullptr) return fail(nullptr, HYGRO_E_INVALID, "ctx is NULL");
    FAULT_POINT(c, "hygro_loss_grad");
    if (n_steps < 1) return fail(c, HYGRO_E_INVALID, "n_steps must be >= 1");
    if (sample_every < 1) return fail(c, HYGRO_E_INVALID, "sample_every must be >= 1");
    if (loss == nullptr) return fail(c, HYGRO_E_INVALID, "loss is NULL");
    if (!std::isfinite(wT) || !std::isfinite(wP)) return fail(c, HYGRO_E_INVALID, "weights must be finite");
    if (checkpoint_every < 0) return fail(c, HYGRO_E_INVALID, "checkpoint_every must be >= 0");
    const int64_t K = n_steps / sample_every;
    if (K > 0 && obs == nullptr) return fail(c, HYGRO_E_INVALID, "obs is NULL");
    if (!(c->have_materials && c->have_bc[0] && c->have_bc[1]))
        return fail(c, HYGRO_E_STATE, "hygro_set_materials and hygro_set_bc (both faces) must come first");
    for (int w = 0; w < c->W; ++w) {
        for (int f = 0; f < 2; ++f)
            if (c->bc[f][w].bc.kind == HYGRO_BC_ROOM)
                return fail(c, HYGRO_E_UNSUPPORTED, "wall %d has a room face: the adjoint runs walls without rooms", w);
        if (c->any_law) return fail(c, HYGRO_E_UNSUPPORTED, "the adjoint differentiates the affine coefficient laws only");
        if (c->walls[w].nu != 1.0)
            return fail(c, HYGRO_E_UNSUPPORTED, "wall %d: the adjoint takes kTM = Lv kM (vapour fraction 1)", w);
    }
    int64_t C = checkpoint_every > 0 ? checkpoint_every : (int64_t)std::ceil(std::sqrt((double)n_steps));
    if (C > n_steps) C = n_steps;
    if (C > (1 << 20)) return fail(c, HYGRO_E_UNSUPPORTED, "checkpoint stride too long");
    const int64_t n_seg = (n_steps + C - 1) / C;
    if (n_seg > INT32_MAX) return fail(c, HYGRO_E_UNSUPPORTED, "too many checkpoints");
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, HYGRO_E_CUDA, "cudaSetDevice failed");
    const int W = c->W;
    const size_t rs = c->real_size;
    const bool f64 = c->precision == HYGRO_FP64;
    const int maxk = f64 ? adj_reg_max_k<double>() : adj_reg_max_k<float>();
    // lane layout: contiguous runs of nodes, one layer per lane (the smallest run length that fits 32
    // lanes). Runs up to maxk nodes take the register kernel, longer ones the shared-memory kernel.
    std::vector<AdjWall> aw(W);
    std::vector<int32_t> reg_list, sm_list;
    size_t lo = 0;
    int Nmax_sm = 0;
    for (int w = 0; w < W; ++w) {
        AdjWall &a = aw[w];
        memset(&a, 0, sizeof a);
        a.N = c->N[w];
        a.node_off = c->walls[w].node_off;
        a.layer_off = (int32_t)lo;
        a.n_layers = c->n_layers[w];
        a.dx = c->L[w] / (double)(a.N - 1);
        std::vector<int> cnt(a.n_layers);
        for (int l = 0; l < a.n_layers; ++l) {
            const int j0 = c->layer_first[lo + l];
            const int j1 = l + 1 < a.n_layers ? c->layer_first[lo + l + 1] : a.N;
            cnt[l] = j1 - j0;
        }
        int K = 1;
        for (;; ++K) {
            int lanes = 0;
            for (int l = 0; l < a.n_layers; ++l) lanes += (cnt[l] + K - 1) / K;
            if (lanes <= 32) break;
        }
        int lane = 0, node = 0;
        for (int l = 0; l < a.n_layers; ++l) {
            const int m = (cnt[l] + K - 1) / K;
            for (int i = 0; i < m; ++i) {
                const int take = cnt[l] / m + (i < cnt[l] % m ? 1 : 0);
                a.start[lane] = (int16_t)node;
                a.layer[lane] = (int8_t)l;
                node += take;
                ++lane;
            }
        }
        for (; lane < 32; ++lane) {
            a.start[lane] = (int16_t)a.N;
            a.layer[lane] = -1;
        }
        a.start[32] = (int16_t)a.N;
        a.kt = K <= maxk ? adj_reg_slots(K) : 0;
        a.dense = 1;
        for (int l = 0; l < 32; ++l) {
            const int nl = a.start[l + 1] - a.start[l];
            if (nl > 0 && nl < a.kt - 1) a.dense = 0;
        }
        if (a.kt > 0) {
            reg_list.push_back(w);
        } else {
            sm_list.push_back(w);
            Nmax_sm = std::max(Nmax_sm, a.N);
        }
        lo += c->n_layers[w];
    }
    // checkpoint and segment storage of each wall: node-major (Nmax_sm nodes) for the shared-memory
    // kernel, slot-major (kt x 32 slots) for the register kernel
    size_t ck_total = 0, seg_total = 0;
    for (int w = 0; w < W; ++w) {
        AdjWall &a = aw[w];
        const size_t ns = a.kt > 0 ? (size_t)a.kt * 32 : (size_t)Nmax_sm;
        a.ck_off = (int64_t)ck_total;
        a.seg_off = (int64_t)seg_total;
        ck_total += (size_t)n_seg * 4 * ns;
        seg_total += (size_t)(C + 2) * 2 * ns;
    }
    // heavier walls first (more slots per lane), so the block scheduler starts them early
    std::stable_sort(reg_list.begin(), reg_list.end(), [&](int x, int y) { return aw[x].kt > aw[y].kt; });
    int warps = 0;
    if (!sm_list.empty()) {
        const size_t per_warp = f64 ? adj_smem_per_warp<double>(Nmax_sm) : adj_smem_per_warp<float>(Nmax_sm);
        int optin = 0;
        CUDA_TRY(c, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
        warps = (int)std::min<size_t>((size_t)kAdjWarps, (size_t)optin / per_warp);
        if (warps < 1)
            return fail(c, HYGRO_E_UNSUPPORTED, "walls of %d nodes need more shared memory than a block has", Nmax_sm);
    }
    const size_t total_layers = lo;
    // physical laws of every layer, in the working precision
    std::vector<double> phys(total_layers * 9);
    for (size_t l = 0; l < total_layers; ++l) {
        const hygro_layer &y = c->layers[l];
        const double v[9] = {y.kM0, y.a, y.cM0, y.b, y.kTT0, y.aT, y.cTT0, y.bT, y.chi};
        for (int k = 0; k < 9; ++k) phys[l * 9 + k] = v[k];
    }
    void *d_aw = nullptr, *d_phys = nullptr, *d_obs = nullptr, *d_ck = nullptr, *d_sg = nullptr, *d_list = nullptr;
    double *d_loss = nullptr, *d_grad = nullptr;
    hygro_status st = HYGRO_OK;
    auto release = [&]() {
        void *ps[] = {d_aw, d_phys, d_obs, d_ck, d_sg, d_list, d_loss, d_grad};
        for (void *q : ps)
            if (q) cudaFree(q);
    };
#define ADJ_TRY(call)                                                                                   \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess) {                                                                        \
            st = fail(c, e_ == cudaErrorMemoryAllocation ? HYGRO_E_NOMEM : HYGRO_E_CUDA, "%s: %s", #call, \
                      cudaGetErrorString(e_));                                                          \
            release();                                                                                  \
            return st;                                                                                  \
        }                                                                                               \
    } while (0)
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    ADJ_TRY(cudaMalloc(&d_aw, W * sizeof(AdjWall)));
    ADJ_TRY(cudaMemcpy(d_aw, aw.data(), W * sizeof(AdjWall), cudaMemcpyHostToDevice));
    std::vector<int32_t> lists(reg_list);
    lists.insert(lists.end(), sm_list.begin(), sm_list.end());
    ADJ_TRY(cudaMalloc(&d_list, lists.size() * sizeof(int32_t)));
    ADJ_TRY(cudaMemcpy(d_list, lists.data(), lists.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    ADJ_TRY(cudaMalloc(&d_phys, std::max<size_t>(1, phys.size()) * rs));
    if ((st = upload_reals(c, d_phys, phys)) != HYGRO_OK) {
        release();
        return st;
    }
    const size_t obs_n = (size_t)K * W * 4;
    if (K > 0) {
        if (is_device_ptr(obs)) {
            d_obs = nullptr;
        } else {
            ADJ_TRY(cudaMalloc(&d_obs, obs_n * sizeof(float)));
            ADJ_TRY(cudaMemcpy(d_obs, obs, obs_n * sizeof(float), cudaMemcpyHostToDevice));
        }
    }
    ADJ_TRY(cudaMalloc(&d_ck, std::max<size_t>(1, ck_total) * rs));
    ADJ_TRY(cudaMalloc(&d_sg, std::max<size_t>(1, seg_total) * rs));
    ADJ_TRY(cudaMalloc(&d_loss, W * sizeof(double)));
    ADJ_TRY(cudaMalloc(&d_grad, std::max<size_t>(1, total_layers * 9) * sizeof(double)));
    ADJ_TRY(cudaMemsetAsync(d_grad, 0, std::max<size_t>(1, total_layers * 9) * sizeof(double), c->stream));
    auto fill = [&](auto &d) {
        using real = typename std::remove_pointer<decltype(d.ckpt)>::type;
        d.walls = (const AdjWall *)d_aw;
        d.W = W;
        d.Nmax = Nmax_sm;
        d.faces = c->d_faces;
        d.layer_tab = (const real *)c->d_layer_tab;
        d.phys = (const real *)d_phys;
        d.Pref = (const real *)c->d_Pref;
        d.Tref = (const real *)c->d_Tref;
        d.noise = c->d_noise;
        d.obs = K > 0 ? (d_obs ? (const float *)d_obs : obs) : nullptr;
        d.wT = wT;
        d.wP = wP;
        d.se = sample_every;
        d.K = (int32_t)K;
        d.n_steps = n_steps;
        d.C = (int32_t)C;
        d.n_seg = (int32_t)n_seg;
        d.ckpt = (real *)d_ck;
        d.seg = (real *)d_sg;
        d.loss = d_loss;
        d.grad = d_grad;
        d.nonfinite = c->d_nonfinite;
        d.dt = c->dt;
        d.t0 = c->t0;
        d.Lv = c->Lv;
        d.Psat = c->Psat;
    };
    ADJ_TRY(after_host_copies(c));
    cudaError_t le = cudaSuccess;
    if (f64) {
        AdjDev<double> d;
        fill(d);
        d.list = (const int32_t *)d_list;
        d.n_list = (int32_t)reg_list.size();
        le = launch_adjoint_reg_f64(d, c->stream);
        d.list = (const int32_t *)d_list + reg_list.size();
        d.n_list = (int32_t)sm_list.size();
        if (le == cudaSuccess && d.n_list > 0) le = launch_adjoint_f64(d, warps, c->stream);
    } else {
        AdjDev<float> d;
        fill(d);
        d.list = (const int32_t *)d_list;
        d.n_list = (int32_t)reg_list.size();
        le = launch_adjoint_reg_f32(d, c->stream);
        d.list = (const int32_t *)d_list + reg_list.size();
        d.n_list = (int32_t)sm_list.size();
        if (le == cudaSuccess && d.n_list > 0) le = launch_adjoint_f32(d, warps, c->stream);
    }
    ADJ_TRY(le);
    std::vector<double> lw(W);
    ADJ_TRY(cudaMemcpyAsync(lw.data(), d_loss, W * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (grad) ADJ_TRY(cudaMemcpyAsync(grad, d_grad, total_layers * 9 * sizeof(double), cudaMemcpyDefault, c->stream));
    ADJ_TRY(cudaStreamSynchronize(c->stream));
#undef ADJ_TRY
    release();
    double L = 0.0;
    for (double x : lw) L += x;
    *loss = L;
    return check_nonfinite(c);
}

const char *hygro_last_error(const hygro_ctx *c) { return c ? c->err.c_str() : g_create_error.c_str(); }

void hygro_destroy(hygro_ctx *c)
{
    if (c == nullptr) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
}

}  // extern "C"
