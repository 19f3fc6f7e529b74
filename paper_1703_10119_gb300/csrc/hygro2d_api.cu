// C-ABI of the 2D sections (include/hygro2d.h): validation, device layout, tensor maps, and the
// launches of the temporally blocked DF kernel (df2d.cuh).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "../../include/hygro2d.h"
#include "df2d.cuh"

using namespace hygro;

namespace {

// Tile shapes (a 4-node halo, so up to 4 fused steps): FP32 64 x 64 cores in 72 x 72 boxes, 4 runs of
// rows per column, two CTAs per SM; FP64 32 x 32 cores in 40 x 40 boxes, 4 runs, two CTAs per SM.
// Each CTA holds both levels of its box as (T, Pv) pairs and the node flags in shared memory.
constexpr int kTX32 = 64, kTY32 = 64, kH32 = 4, kSeg32 = 4, kMinB32 = 2;
constexpr int kTX64 = 32, kTY64 = 32, kH64 = 4, kSeg64 = 4, kMinB64 = 2;
using Cfg32 = Tile2D<float, kTX32, kTY32, kH32, kSeg32>;
using Cfg64 = Tile2D<double, kTX64, kTY64, kH64, kSeg64>;

thread_local std::string g_create_error2d = "no error";

struct RawBc2 {
    hygro_bc bc;
    std::vector<float> noise;
};

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

}  // namespace

struct hygro2d_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int precision = HYGRO_FP32;
    int G = 0, nx = 0, ny = 0, pitch = 0;
    double h = 0, dt = 0, t0 = 0, Lv = 0, Psat = 0;
    int k = 1;             // steps per launch
    int halo = 1;          // halo depth of the tile shape (most steps per launch)
    size_t rs = 4;         // bytes per real
    int n_regions = 0;
    std::vector<double> Tref, Pref;
    std::vector<RawBc2> bc[4];
    bool have_materials = false, have_bc[4] = {false, false, false, false};
    int64_t step = 0;
    int set = 0;           // buffer set holding the newest levels
    std::string err = "no error";
    // device: F[s][0], F[s][1] = (T, Pv) pairs of level n and n-1 of buffer set s
    void *F[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    CUtensorMap maps[2][2];
    CUtensorMap flag_map;
    uint8_t *d_flags8 = nullptr;   // node flags: region | neighbour-in-another-region bits
    void *d_tab = nullptr;
    FaceInfo *d_faces = nullptr;
    float2 *d_noise = nullptr;
    size_t noise_cap = 0;
    int32_t *d_flags = nullptr;   // [0] wait gave up, [1] non-finite
    // CUDA graphs of graph_launches launches (an even count: the buffer sets are back where they were),
    // one per buffer set at the interval's start, replayed for the whole intervals of a run; the launches
    // read their first step from d_step, which the graph's last node advances
    int graph_launches = 64;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    int64_t *d_step = nullptr;
    size_t cells() const { return (size_t)G * ny * pitch; }
};

namespace {

hygro_status fail(hygro2d_ctx *c, hygro_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c)
        c->err = buf;
    else
        g_create_error2d = buf;
    return st;
}

#define CUDA_TRY2(ctx, call)                                                                             \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess)                                                                           \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? HYGRO_E_NOMEM : HYGRO_E_CUDA, "%s: %s", #call, \
                        cudaGetErrorString(e_));                                                         \
    } while (0)

void drop_graphs(hygro2d_ctx *c)
{
    for (int s = 0; s < 2; ++s)
        if (c->gexec[s]) {
            cudaGraphExecDestroy(c->gexec[s]);
            c->gexec[s] = nullptr;
        }
}

void free_all(hygro2d_ctx *c)
{
    drop_graphs(c);
    for (int s = 0; s < 2; ++s)
        for (int l = 0; l < 2; ++l)
            if (c->F[s][l]) cudaFree(c->F[s][l]);
    void *p[] = {c->d_flags8, c->d_tab, c->d_faces, c->d_noise, c->d_flags, c->d_step};
    for (void *q : p)
        if (q) cudaFree(q);
}

hygro_status encode_maps(hygro2d_ctx *c)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (enc == nullptr) return fail(c, HYGRO_E_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const bool f64 = c->precision == HYGRO_FP64;
    const cuuint32_t BX = f64 ? Cfg64::BX : Cfg32::BX, BY = f64 ? Cfg64::BY : Cfg32::BY;
    const cuuint64_t P = (cuuint64_t)c->pitch, NY = (cuuint64_t)c->ny;
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    for (int s = 0; s < 2; ++s)
        for (int l = 0; l < 2; ++l) {
            CUresult r;
            if (f64) {
                // (T, Pv) doubles as a 4D tensor (component, x, y, grid): 16-byte rows of the innermost dimension
                const cuuint64_t dims[4] = {2, (cuuint64_t)c->nx, NY, (cuuint64_t)c->G};
                const cuuint64_t strides[3] = {16, P * 16, P * NY * 16};
                const cuuint32_t box[4] = {2, BX, BY, 1};
                r = enc(&c->maps[s][l], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, c->F[s][l], dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            } else {
                // (T, Pv) floats as one 8-byte element per node
                const cuuint64_t dims[3] = {(cuuint64_t)c->nx, NY, (cuuint64_t)c->G};
                const cuuint64_t strides[2] = {P * 8, P * NY * 8};
                const cuuint32_t box[3] = {BX, BY, 1};
                r = enc(&c->maps[s][l], CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, c->F[s][l], dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            }
            if (r != CUDA_SUCCESS) return fail(c, HYGRO_E_CUDA, "cuTensorMapEncodeTiled (levels) failed (%d)", (int)r);
        }
    const cuuint64_t dims[3] = {(cuuint64_t)c->nx, NY, (cuuint64_t)c->G};
    const cuuint64_t strides[2] = {P, P * NY};
    const cuuint32_t box[3] = {(cuuint32_t)(f64 ? Cfg64::FBX : Cfg32::FBX), BY, 1};
    const CUresult r = enc(&c->flag_map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, c->d_flags8, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(c, HYGRO_E_CUDA, "cuTensorMapEncodeTiled (flags) failed (%d)", (int)r);
    return HYGRO_OK;
}

__global__ void step_set_kernel(int64_t *p, int64_t v) { *p = v; }
__global__ void step_add_kernel(int64_t *p, int64_t v) { *p += v; }

// Kernel arguments of a launch that reads buffer set `set` (levels n, n-1) and writes the other one.
Dev2D dev_args(const hygro2d_ctx *c, int set, const int64_t *step_dev)
{
    Dev2D d;
    d.G = c->G;
    d.nx = c->nx;
    d.ny = c->ny;
    d.pitch = c->pitch;
    d.n_regions = c->n_regions;
    d.region_tab = c->d_tab;
    d.faces = c->d_faces;
    d.noise = c->d_noise;
    d.out_new = c->F[1 - set][0];
    d.out_old = c->F[1 - set][1];
    d.err = c->d_flags;
    d.nonfinite = c->d_flags + 1;
    d.step_dev = step_dev;
    d.dt = c->dt;
    d.t0 = c->t0;
    d.Lv = c->Lv;
    return d;
}

template <typename real, int TX, int TY, int H, int SEG, int MINB>
cudaError_t launch2d(const hygro2d_ctx *c, int64_t n0, int n_sub)
{
    using L = Tile2D<real, TX, TY, H, SEG>;
    const Dev2D d = dev_args(c, c->set, nullptr);
    const int tiles = ((c->nx + TX - 1) / TX) * ((c->ny + TY - 1) / TY);
    const CUtensorMap *m = c->maps[c->set];
    df2d_kernel<real, TX, TY, H, SEG, MINB><<<(unsigned)((int64_t)tiles * c->G), L::NT, L::BYTES, c->stream>>>(
        m[0], m[1], c->flag_map, d, n0, n_sub);
    return cudaGetLastError();
}

// The graph of one interval starting on buffer set `set0`: graph_launches launches of k steps each, launch i
// on set set0 ^ (i & 1) with its first step *d_step + i k, then d_step advanced by the interval's steps.
template <typename real, int TX, int TY, int H, int SEG, int MINB>
cudaError_t build_graph(hygro2d_ctx *c, int set0, cudaGraphExec_t *out)
{
    using L = Tile2D<real, TX, TY, H, SEG>;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return e;
    const int tiles = ((c->nx + TX - 1) / TX) * ((c->ny + TY - 1) / TY);
    cudaGraphNode_t prev = nullptr;
    for (int i = 0; i < c->graph_launches && e == cudaSuccess; ++i) {
        const int set = set0 ^ (i & 1);
        Dev2D d = dev_args(c, set, c->d_step);
        CUtensorMap m0 = c->maps[set][0], m1 = c->maps[set][1], mf = c->flag_map;
        int64_t n0 = (int64_t)i * c->k;
        int32_t n_sub = c->k;
        void *args[] = {&m0, &m1, &mf, &d, &n0, &n_sub};
        cudaKernelNodeParams p = {};
        p.func = (void *)df2d_kernel<real, TX, TY, H, SEG, MINB>;
        p.gridDim = dim3((unsigned)((int64_t)tiles * c->G));
        p.blockDim = dim3(L::NT);
        p.sharedMemBytes = L::BYTES;
        p.kernelParams = args;
        cudaGraphNode_t node;
        e = cudaGraphAddKernelNode(&node, g, prev ? &prev : nullptr, prev ? 1 : 0, &p);
        prev = node;
    }
    if (e == cudaSuccess) {
        int64_t *ptr = c->d_step;
        int64_t inc = (int64_t)c->graph_launches * c->k;
        void *args[] = {&ptr, &inc};
        cudaKernelNodeParams p = {};
        p.func = (void *)step_add_kernel;
        p.gridDim = dim3(1);
        p.blockDim = dim3(1);
        p.kernelParams = args;
        cudaGraphNode_t node;
        e = cudaGraphAddKernelNode(&node, g, prev ? &prev : nullptr, prev ? 1 : 0, &p);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    return e;
}

// Launches of n_steps from the current state: whole graph intervals replayed from the interval's graph,
// the rest as single launches.
hygro_status run2d(hygro2d_ctx *c, int64_t n_steps, bool use_graph)
{
    const bool f64 = c->precision == HYGRO_FP64;
    int64_t done = 0;
    const int64_t unit = (int64_t)c->graph_launches * c->k;
    if (use_graph && c->graph_launches > 0 && n_steps >= unit) {
        const int64_t reps = n_steps / unit;
        if (c->gexec[c->set] == nullptr) {
            const cudaError_t e = f64 ? build_graph<double, kTX64, kTY64, kH64, kSeg64, kMinB64>(c, c->set, &c->gexec[c->set])
                                      : build_graph<float, kTX32, kTY32, kH32, kSeg32, kMinB32>(c, c->set, &c->gexec[c->set]);
            if (e != cudaSuccess) {
                c->gexec[c->set] = nullptr;
                return fail(c, HYGRO_E_CUDA, "building the 2D run's CUDA graph: %s", cudaGetErrorString(e));
            }
        }
        step_set_kernel<<<1, 1, 0, c->stream>>>(c->d_step, c->step);
        CUDA_TRY2(c, cudaGetLastError());
        for (int64_t r = 0; r < reps; ++r) CUDA_TRY2(c, cudaGraphLaunch(c->gexec[c->set], c->stream));
        c->step += reps * unit;   // an even launch count leaves the buffer sets where they were
        done = reps * unit;
    }
    while (done < n_steps) {
        const int sub = (int)std::min<int64_t>(c->k, n_steps - done);
        const cudaError_t e = f64 ? launch2d<double, kTX64, kTY64, kH64, kSeg64, kMinB64>(c, c->step, sub)
                                  : launch2d<float, kTX32, kTY32, kH32, kSeg32, kMinB32>(c, c->step, sub);
        if (e != cudaSuccess) return fail(c, HYGRO_E_CUDA, "2D DF launch: %s", cudaGetErrorString(e));
        c->set = 1 - c->set;
        c->step += sub;
        done += sub;
    }
    return HYGRO_OK;
}

// Opt the kernel of the context's precision into its dynamic shared memory (on the current device).
cudaError_t prepare_kernel(int precision)
{
    if (precision == HYGRO_FP64)
        return cudaFuncSetAttribute(df2d_kernel<double, kTX64, kTY64, kH64, kSeg64, kMinB64>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg64::BYTES);
    return cudaFuncSetAttribute(df2d_kernel<float, kTX32, kTY32, kH32, kSeg32, kMinB32>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg32::BYTES);
}

hygro_status upload_faces2d(hygro2d_ctx *c)
{
    drop_graphs(c);   // the graphs hold the face and noise-table addresses
    if (!(c->have_materials && c->have_bc[0] && c->have_bc[1] && c->have_bc[2] && c->have_bc[3])) return HYGRO_OK;
    std::vector<FaceInfo> fi((size_t)c->G * 4);
    size_t total = 0;
    for (int f = 0; f < 4; ++f)
        for (int g = 0; g < c->G; ++g) total += c->bc[f][g].noise.size() / 2;
    std::vector<float2> noise(std::max<size_t>(1, total));
    size_t off = 0;
    for (int g = 0; g < c->G; ++g)
        for (int f = 0; f < 4; ++f) {
            const RawBc2 &r = c->bc[f][g];
            const int64_t nl = (int64_t)r.noise.size() / 2;
            fi[(size_t)g * 4 + f] = face_info(r.bc, c->Tref[g], c->Pref[g], c->t0, c->dt, (int64_t)off, nl);
            for (int64_t q = 0; q < nl; ++q) noise[off + q] = make_float2(r.noise[2 * q], r.noise[2 * q + 1]);
            off += (size_t)nl;
        }
    if (noise.size() > c->noise_cap) {
        if (c->d_noise) cudaFree(c->d_noise);
        c->d_noise = nullptr;
        c->noise_cap = 0;
        CUDA_TRY2(c, cudaMalloc(&c->d_noise, noise.size() * sizeof(float2)));
        c->noise_cap = noise.size();
    }
    CUDA_TRY2(c, cudaMemcpy(c->d_noise, noise.data(), noise.size() * sizeof(float2), cudaMemcpyHostToDevice));
    CUDA_TRY2(c, cudaMemcpy(c->d_faces, fi.data(), fi.size() * sizeof(FaceInfo), cudaMemcpyHostToDevice));
    return HYGRO_OK;
}

// Device level (pairs) <-> absolute FP64 [G][ny][nx] host arrays of T and P (either may be skipped).
hygro_status download_level(hygro2d_ctx *c, const void *src, std::vector<double> *T, std::vector<double> *P)
{
    const size_t n = c->cells();
    std::vector<double> v(2 * n);
    if (c->precision == HYGRO_FP64) {
        CUDA_TRY2(c, cudaMemcpy(v.data(), src, 2 * n * 8, cudaMemcpyDeviceToHost));
    } else {
        std::vector<float> f(2 * n);
        CUDA_TRY2(c, cudaMemcpy(f.data(), src, 2 * n * 4, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < 2 * n; ++i) v[i] = (double)f[i];
    }
    const size_t m = (size_t)c->G * c->ny * c->nx;
    if (T) T->resize(m);
    if (P) P->resize(m);
    for (int g = 0; g < c->G; ++g)
        for (int j = 0; j < c->ny; ++j)
            for (int i = 0; i < c->nx; ++i) {
                const size_t a = ((size_t)g * c->ny + j) * c->nx + i, b = ((size_t)g * c->ny + j) * c->pitch + i;
                if (T) (*T)[a] = v[2 * b] + c->Tref[g];
                if (P) (*P)[a] = v[2 * b + 1] + c->Pref[g];
            }
    return HYGRO_OK;
}

// Overwrite the T and / or P components of one device level (absent components keep their values).
hygro_status upload_level(hygro2d_ctx *c, void *dst, const std::vector<double> *T, const std::vector<double> *P)
{
    const size_t n = c->cells();
    std::vector<double> v(2 * n, 0.0);
    if (!(T && P)) {
        // read-modify-write: keep the component not given
        if (c->precision == HYGRO_FP64) {
            CUDA_TRY2(c, cudaMemcpy(v.data(), dst, 2 * n * 8, cudaMemcpyDeviceToHost));
        } else {
            std::vector<float> f(2 * n);
            CUDA_TRY2(c, cudaMemcpy(f.data(), dst, 2 * n * 4, cudaMemcpyDeviceToHost));
            for (size_t i = 0; i < 2 * n; ++i) v[i] = (double)f[i];
        }
    }
    for (int g = 0; g < c->G; ++g)
        for (int j = 0; j < c->ny; ++j)
            for (int i = 0; i < c->nx; ++i) {
                const size_t a = ((size_t)g * c->ny + j) * c->nx + i, b = ((size_t)g * c->ny + j) * c->pitch + i;
                if (T) v[2 * b] = (*T)[a] - c->Tref[g];
                if (P) v[2 * b + 1] = (*P)[a] - c->Pref[g];
            }
    if (c->precision == HYGRO_FP64) {
        CUDA_TRY2(c, cudaMemcpy(dst, v.data(), 2 * n * 8, cudaMemcpyHostToDevice));
    } else {
        std::vector<float> f(v.begin(), v.end());
        CUDA_TRY2(c, cudaMemcpy(dst, f.data(), 2 * n * 4, cudaMemcpyHostToDevice));
    }
    return HYGRO_OK;
}

}  // namespace

extern "C" {

hygro_status hygro2d_create(const hygro2d_desc *desc, hygro2d_ctx **out)
{
    if (out == nullptr) return fail(nullptr, HYGRO_E_INVALID, "out is NULL");
    *out = nullptr;
    if (desc == nullptr) return fail(nullptr, HYGRO_E_INVALID, "desc is NULL");
    if (desc->n_grids < 1) return fail(nullptr, HYGRO_E_INVALID, "n_grids must be >= 1");
    if (desc->nx < 2 || desc->ny < 2) return fail(nullptr, HYGRO_E_INVALID, "nx and ny must be >= 2");
    if (!(std::isfinite(desc->h) && desc->h > 0)) return fail(nullptr, HYGRO_E_INVALID, "h must be > 0");
    if (!(std::isfinite(desc->dt) && desc->dt > 0)) return fail(nullptr, HYGRO_E_INVALID, "dt must be > 0");
    if (!std::isfinite(desc->t0)) return fail(nullptr, HYGRO_E_INVALID, "t0 must be finite");
    if (!(std::isfinite(desc->Psat) && desc->Psat > 0)) return fail(nullptr, HYGRO_E_INVALID, "Psat must be > 0");
    if (!std::isfinite(desc->Lv)) return fail(nullptr, HYGRO_E_INVALID, "Lv must be finite");
    if (desc->precision != HYGRO_FP32 && desc->precision != HYGRO_FP64)
        return fail(nullptr, HYGRO_E_INVALID, "precision must be HYGRO_FP32 or HYGRO_FP64");
    const int halo = desc->precision == HYGRO_FP64 ? kH64 : kH32;
    if (desc->steps_per_launch < 0 || desc->steps_per_launch > halo)
        return fail(nullptr, HYGRO_E_INVALID, "steps_per_launch must be in 0..%d", halo);
    const int64_t pitch = ((int64_t)desc->nx + 31) / 32 * 32;
    const int64_t cells = pitch * desc->ny * (int64_t)desc->n_grids;
    if (desc->nx > (1 << 24) || desc->ny > (1 << 24) || cells > ((int64_t)1 << 31))
        return fail(nullptr, HYGRO_E_UNSUPPORTED, "sections too large for 32-bit node indices");
    const int tiles = desc->precision == HYGRO_FP64
                          ? ((desc->nx + kTX64 - 1) / kTX64) * ((desc->ny + kTY64 - 1) / kTY64)
                          : ((desc->nx + kTX32 - 1) / kTX32) * ((desc->ny + kTY32 - 1) / kTY32);
    if ((int64_t)tiles * desc->n_grids > INT32_MAX) return fail(nullptr, HYGRO_E_UNSUPPORTED, "too many tiles");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(nullptr, HYGRO_E_CUDA, "no CUDA device available");
    }
    if (desc->device < 0 || desc->device >= ndev) return fail(nullptr, HYGRO_E_INVALID, "bad device %d", desc->device);
    int smem_optin = 0;
    if (cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, desc->device) != cudaSuccess)
        return fail(nullptr, HYGRO_E_CUDA, "cudaDeviceGetAttribute failed");
    const size_t need_smem = desc->precision == HYGRO_FP64 ? Cfg64::BYTES : Cfg32::BYTES;
    if ((size_t)smem_optin < need_smem)
        return fail(nullptr, HYGRO_E_UNSUPPORTED, "device offers %d bytes of shared memory per block, the tile needs %zu",
                    smem_optin, need_smem);

    hygro2d_ctx *c = new (std::nothrow) hygro2d_ctx();
    if (c == nullptr) return fail(nullptr, HYGRO_E_NOMEM, "host allocation failed");
    c->device = desc->device;
    c->stream = (cudaStream_t)desc->stream;
    c->precision = desc->precision;
    c->G = desc->n_grids;
    c->nx = desc->nx;
    c->ny = desc->ny;
    c->pitch = (int)pitch;
    c->h = desc->h;
    c->dt = desc->dt;
    c->t0 = desc->t0;
    c->Lv = desc->Lv;
    c->Psat = desc->Psat;
    c->halo = halo;
    c->k = desc->steps_per_launch == 0 ? halo : desc->steps_per_launch;
    c->rs = desc->precision == HYGRO_FP64 ? 8 : 4;
    auto bail = [&](hygro_status s) {
        g_create_error2d = c->err;
        free_all(c);
        delete c;
        return s;
    };
    hygro_status st;
#define CREATE2D_TRY(call)                               \
    do {                                                 \
        if ((st = (call)) != HYGRO_OK) return bail(st);  \
    } while (0)
    auto cu = [&](cudaError_t e, const char *what) {
        if (e == cudaSuccess) return HYGRO_OK;
        return fail(c, e == cudaErrorMemoryAllocation ? HYGRO_E_NOMEM : HYGRO_E_CUDA, "%s: %s", what,
                    cudaGetErrorString(e));
    };
    CREATE2D_TRY(cu(cudaSetDevice(c->device), "cudaSetDevice"));
    CREATE2D_TRY(cu(prepare_kernel(c->precision), "cudaFuncSetAttribute(df2d_kernel)"));
    const size_t bytes = c->cells() * 2 * c->rs;
    for (int s = 0; s < 2; ++s)
        for (int l = 0; l < 2; ++l) {
            CREATE2D_TRY(cu(cudaMalloc(&c->F[s][l], bytes), "cudaMalloc(levels)"));
            CREATE2D_TRY(cu(cudaMemset(c->F[s][l], 0, bytes), "cudaMemset(levels)"));
        }
    CREATE2D_TRY(cu(cudaMalloc(&c->d_flags8, c->cells()), "cudaMalloc(node flags)"));
    CREATE2D_TRY(cu(cudaMemset(c->d_flags8, 0, c->cells()), "cudaMemset(node flags)"));
    CREATE2D_TRY(cu(cudaMalloc(&c->d_faces, (size_t)c->G * 4 * sizeof(FaceInfo)), "cudaMalloc(faces)"));
    CREATE2D_TRY(cu(cudaMalloc(&c->d_flags, 2 * sizeof(int32_t)), "cudaMalloc(flags)"));
    CREATE2D_TRY(cu(cudaMemset(c->d_flags, 0, 2 * sizeof(int32_t)), "cudaMemset(flags)"));
    CREATE2D_TRY(cu(cudaMalloc(&c->d_step, sizeof(int64_t)), "cudaMalloc(step counter)"));
    CREATE2D_TRY(encode_maps(c));
#undef CREATE2D_TRY
    *out = c;
    return HYGRO_OK;
}

hygro_status hygro2d_set_materials(hygro2d_ctx *c, int32_t n_regions, const uint8_t *region, const hygro_layer *layers,
                                   const double *T_init, const double *P_init)
{
    if (c == nullptr) return fail(nullptr, HYGRO_E_INVALID, "ctx is NULL");
    if (!region || !layers || !T_init || !P_init)
        return fail(c, HYGRO_E_INVALID, "region, layers, T_init and P_init are required");
    if (n_regions < 1 || n_regions > HYGRO2D_MAX_REGIONS)
        return fail(c, HYGRO_E_INVALID, "n_regions must be in 1..%d", HYGRO2D_MAX_REGIONS);
    const size_t n = (size_t)c->G * c->ny * c->nx;
    for (size_t i = 0; i < n; ++i)
        if (region[i] >= n_regions) return fail(c, HYGRO_E_INVALID, "node %zu: region %d >= n_regions", i, region[i]);
    for (int g = 0; g < c->G; ++g) {
        for (int r = 0; r < n_regions; ++r) {
            const hygro_layer &y = layers[(size_t)g * n_regions + r];
            if (!(y.kM0 > 0 && y.cM0 > 0 && y.kTT0 > 0 && y.cTT0 > 0) || !std::isfinite(y.kM0) ||
                !std::isfinite(y.cM0) || !std::isfinite(y.kTT0) || !std::isfinite(y.cTT0) || !std::isfinite(y.a) ||
                !std::isfinite(y.b) || !std::isfinite(y.aT) || !std::isfinite(y.bT) || !std::isfinite(y.chi))
                return fail(c, HYGRO_E_INVALID,
                            "grid %d region %d: coefficients must be finite, kM0, cM0, kTT0, cTT0 > 0", g, r);
        }
        if (!std::isfinite(T_init[g]) || !std::isfinite(P_init[g]))
            return fail(c, HYGRO_E_INVALID, "grid %d: initial state must be finite", g);
    }
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, HYGRO_E_CUDA, "cudaSetDevice failed");
    CUDA_TRY2(c, cudaStreamSynchronize(c->stream));
    c->n_regions = n_regions;
    c->Tref.assign(T_init, T_init + c->G);
    c->Pref.assign(P_init, P_init + c->G);
    // region constants in the deviation variables of each grid (P' = Pv - P_ref):
    // kh = k / (2h) for both conductivities, storage h c / (2 dt)
    std::vector<double> tab((size_t)c->G * n_regions * kLayerStride, 0.0);
    const double h = c->h, dt = c->dt, Ps = c->Psat;
    for (int g = 0; g < c->G; ++g) {
        const double Pr = c->Pref[g];
        for (int r = 0; r < n_regions; ++r) {
            const hygro_layer &y = layers[(size_t)g * n_regions + r];
            double *t = &tab[((size_t)g * n_regions + r) * kLayerStride];
            t[LT_KMA] = y.kM0 * (1.0 + y.a * Pr / Ps) / (2.0 * h);
            t[LT_KMB] = y.kM0 * y.a / Ps / (2.0 * h);
            t[LT_KTA] = y.kTT0 * (1.0 + y.aT * Pr / Ps) / (2.0 * h);
            t[LT_KTB] = y.kTT0 * y.aT / Ps / (2.0 * h);
            t[LT_AA] = h * y.cM0 * (1.0 + y.b * Pr / Ps) / (2.0 * dt);
            t[LT_AB] = h * y.cM0 * y.b / Ps / (2.0 * dt);
            t[LT_BA] = h * y.cTT0 * (1.0 + y.bT * Pr / Ps) / (2.0 * dt);
            t[LT_BB] = h * y.cTT0 * y.bT / Ps / (2.0 * dt);
            t[LT_CHI] = y.chi;
        }
    }
    drop_graphs(c);   // the graphs hold the region table's address
    if (c->d_tab) cudaFree(c->d_tab);
    c->d_tab = nullptr;
    CUDA_TRY2(c, cudaMalloc(&c->d_tab, tab.size() * c->rs));
    if (c->precision == HYGRO_FP64) {
        CUDA_TRY2(c, cudaMemcpy(c->d_tab, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice));
    } else {
        std::vector<float> f(tab.begin(), tab.end());
        CUDA_TRY2(c, cudaMemcpy(c->d_tab, f.data(), f.size() * 4, cudaMemcpyHostToDevice));
    }
    // node flags: region, the section-edge bit, and one bit per neighbour that lies in another region
    std::vector<uint8_t> fl(c->cells(), 0);
    for (int g = 0; g < c->G; ++g)
        for (int j = 0; j < c->ny; ++j)
            for (int i = 0; i < c->nx; ++i) {
                const uint8_t *rg = region + (size_t)g * c->ny * c->nx;
                const int r = rg[(size_t)j * c->nx + i];
                uint32_t f = (uint32_t)r;
                if (i == 0 || i == c->nx - 1 || j == 0 || j == c->ny - 1) f |= kEdge2D;
                if (i > 0 && rg[(size_t)j * c->nx + i - 1] != r) f |= kDiffL;
                if (i < c->nx - 1 && rg[(size_t)j * c->nx + i + 1] != r) f |= kDiffR;
                if (j > 0 && rg[(size_t)(j - 1) * c->nx + i] != r) f |= kDiffU;
                if (j < c->ny - 1 && rg[(size_t)(j + 1) * c->nx + i] != r) f |= kDiffD;
                fl[((size_t)g * c->ny + j) * c->pitch + i] = (uint8_t)f;
            }
    CUDA_TRY2(c, cudaMemcpy(c->d_flags8, fl.data(), fl.size(), cudaMemcpyHostToDevice));
    // uniform initial state: zero deviation at both levels of the current set
    for (int l = 0; l < 2; ++l) CUDA_TRY2(c, cudaMemset(c->F[c->set][l], 0, c->cells() * 2 * c->rs));
    CUDA_TRY2(c, cudaMemset(c->d_flags, 0, 2 * sizeof(int32_t)));
    c->step = 0;
    c->have_materials = true;
    return upload_faces2d(c);
}

hygro_status hygro2d_set_bc(hygro2d_ctx *c, int32_t face, const hygro_bc *bc)
{
    if (c == nullptr) return fail(nullptr, HYGRO_E_INVALID, "ctx is NULL");
    if (face < 0 || face > 3) return fail(c, HYGRO_E_INVALID, "face must be in 0..3");
    if (bc == nullptr) return fail(c, HYGRO_E_INVALID, "bc is NULL");
    for (int g = 0; g < c->G; ++g) {
        std::string why;
        const hygro_status st = check_bc(bc[g], false, c->t0, c->dt, &why);
        if (st != HYGRO_OK) return fail(c, st, "grid %d face %d: %s", g, face, why.c_str());
    }
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, HYGRO_E_CUDA, "cudaSetDevice failed");
    CUDA_TRY2(c, cudaStreamSynchronize(c->stream));
    std::vector<RawBc2> v(c->G);
    for (int g = 0; g < c->G; ++g) {
        v[g].bc = bc[g];
        v[g].bc.noise = nullptr;
        if (bc[g].kind == HYGRO_BC_AMBIENT && bc[g].noise_len > 0)
            v[g].noise.assign(bc[g].noise, bc[g].noise + 2 * (size_t)bc[g].noise_len);
    }
    c->bc[face].swap(v);
    c->have_bc[face] = true;
    return upload_faces2d(c);
}

hygro_status hygro2d_run(hygro2d_ctx *c, int64_t n_steps)
{
    if (c == nullptr) return fail(nullptr, HYGRO_E_INVALID, "ctx is NULL");
    if (n_steps < 0) return fail(c, HYGRO_E_INVALID, "n_steps must be >= 0");
    if (!(c->have_materials && c->have_bc[0] && c->have_bc[1] && c->have_bc[2] && c->have_bc[3]))
        return fail(c, HYGRO_E_STATE, "hygro2d_set_materials and hygro2d_set_bc (all four faces) must come first");
    if (n_steps == 0) return HYGRO_OK;
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, HYGRO_E_CUDA, "cudaSetDevice failed");
    CUDA_TRY2(c, after_host_copies(c->stream));
    return run2d(c, n_steps, true);
}

hygro_status hygro2d_set_option(hygro2d_ctx *c, int32_t option, int64_t value)
{
    if (c == nullptr) return fail(nullptr, HYGRO_E_INVALID, "ctx is NULL");
    if (option == HYGRO2D_OPT_STEPS_PER_LAUNCH) {
        if (value < 1 || value > c->halo) return fail(c, HYGRO_E_INVALID, "steps per launch must be in 1..%d", c->halo);
        if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, HYGRO_E_CUDA, "cudaSetDevice failed");
        CUDA_TRY2(c, cudaStreamSynchronize(c->stream));
        drop_graphs(c);
        c->k = (int)value;
        return HYGRO_OK;
    }
    if (option == HYGRO2D_OPT_GRAPH_LAUNCHES) {
        if (value < 0 || value > 4096 || (value & 1))
            return fail(c, HYGRO_E_INVALID, "launches per graph must be 0 or an even count up to 4096");
        if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, HYGRO_E_CUDA, "cudaSetDevice failed");
        CUDA_TRY2(c, cudaStreamSynchronize(c->stream));
        drop_graphs(c);
        c->graph_launches = (int)value;
        return HYGRO_OK;
    }
    return fail(c, HYGRO_E_INVALID, "unknown option %d", option);
}

hygro_status hygro2d_get_option(const hygro2d_ctx *c, int32_t option, int64_t *value)
{
    if (c == nullptr || value == nullptr) return HYGRO_E_INVALID;
    if (option == HYGRO2D_OPT_STEPS_PER_LAUNCH) {
        *value = c->k;
        return HYGRO_OK;
    }
    if (option == HYGRO2D_OPT_GRAPH_LAUNCHES) {
        *value = c->graph_launches;
        return HYGRO_OK;
    }
    return HYGRO_E_INVALID;
}

hygro_status hygro2d_autotune(hygro2d_ctx *c, int32_t probe_steps, int32_t *k_best, double *ms_per_step)
{
    if (c == nullptr) return fail(nullptr, HYGRO_E_INVALID, "ctx is NULL");
    if (probe_steps < 1 || probe_steps > 100000) return fail(c, HYGRO_E_INVALID, "probe_steps must be in 1..100000");
    if (!(c->have_materials && c->have_bc[0] && c->have_bc[1] && c->have_bc[2] && c->have_bc[3]))
        return fail(c, HYGRO_E_STATE, "hygro2d_set_materials and hygro2d_set_bc (all four faces) must come first");
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, HYGRO_E_CUDA, "cudaSetDevice failed");
    CUDA_TRY2(c, after_host_copies(c->stream));
    CUDA_TRY2(c, cudaStreamSynchronize(c->stream));
    const size_t bytes = c->cells() * 2 * c->rs;
    void *save[2] = {nullptr, nullptr};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const int set0 = c->set, k0 = c->k;
    const int64_t step0 = c->step;
    hygro_status st = HYGRO_OK;
    auto cu = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess && st == HYGRO_OK)
            st = fail(c, e == cudaErrorMemoryAllocation ? HYGRO_E_NOMEM : HYGRO_E_CUDA, "autotune, %s: %s", what,
                      cudaGetErrorString(e));
        return st == HYGRO_OK;
    };
    auto restore = [&]() {
        for (int l = 0; l < 2; ++l)
            cu(cudaMemcpyAsync(c->F[set0][l], save[l], bytes, cudaMemcpyDeviceToDevice, c->stream), "restore");
        c->set = set0;
        c->step = step0;
    };
    bool ok = cu(cudaMalloc(&save[0], bytes), "cudaMalloc") && cu(cudaMalloc(&save[1], bytes), "cudaMalloc") &&
              cu(cudaEventCreate(&e0), "event") && cu(cudaEventCreate(&e1), "event");
    for (int l = 0; l < 2 && ok; ++l)
        ok = cu(cudaMemcpyAsync(save[l], c->F[set0][l], bytes, cudaMemcpyDeviceToDevice, c->stream), "save");
    double best_ms = 0.0;
    int best = k0;
    for (int k = 1; k <= c->halo && ok; ++k) {
        c->k = k;
        restore();   // a warm-up launch from the saved state, then the timed probe from it again
        hygro_status rs = st == HYGRO_OK ? run2d(c, std::min<int64_t>(k, probe_steps), false) : st;
        if (rs == HYGRO_OK) restore();
        float ms = 0.0f;
        if (rs == HYGRO_OK && st == HYGRO_OK && cu(cudaEventRecord(e0, c->stream), "event")) rs = run2d(c, probe_steps, false);
        ok = rs == HYGRO_OK && st == HYGRO_OK && cu(cudaEventRecord(e1, c->stream), "event") &&
             cu(cudaEventSynchronize(e1), "event") && cu(cudaEventElapsedTime(&ms, e0, e1), "event");
        if (rs != HYGRO_OK && st == HYGRO_OK) st = rs;
        if (!ok) break;
        const double per = (double)ms / probe_steps;
        if (ms_per_step) ms_per_step[k - 1] = per;
        if (k == 1 || per < best_ms) {
            best_ms = per;
            best = k;
        }
    }
    if (save[0] && save[1]) restore();
    cudaStreamSynchronize(c->stream);
    c->k = ok ? best : k0;
    drop_graphs(c);
    for (void *p : save)
        if (p) cudaFree(p);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (!ok) return st != HYGRO_OK ? st : fail(c, HYGRO_E_CUDA, "autotune failed");
    if (k_best) *k_best = best;
    return HYGRO_OK;
}

hygro_status hygro2d_sync(hygro2d_ctx *c)
{
    if (c == nullptr) return fail(nullptr, HYGRO_E_INVALID, "ctx is NULL");
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, HYGRO_E_CUDA, "cudaSetDevice failed");
    int32_t fl[2] = {0, 0};
    CUDA_TRY2(c, cudaMemcpyAsync(fl, c->d_flags, sizeof fl, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY2(c, cudaStreamSynchronize(c->stream));
    if (fl[0] || fl[1]) CUDA_TRY2(c, cudaMemsetAsync(c->d_flags, 0, sizeof fl, c->stream));
    if (fl[0]) return fail(c, HYGRO_E_TIMEOUT, "a tile's bounded wait for its TMA loads gave up");
    if (fl[1]) return fail(c, HYGRO_E_NONFINITE, "a section produced a NaN or infinity");
    return HYGRO_OK;
}

hygro_status hygro2d_get_fields(hygro2d_ctx *c, int32_t level, double *T, double *P)
{
    if (c == nullptr) return fail(nullptr, HYGRO_E_INVALID, "ctx is NULL");
    if (level != 0 && level != 1) return fail(c, HYGRO_E_INVALID, "level must be 0 (n) or 1 (n-1)");
    if (!c->have_materials) return fail(c, HYGRO_E_STATE, "hygro2d_set_materials must come first");
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, HYGRO_E_CUDA, "cudaSetDevice failed");
    CUDA_TRY2(c, cudaStreamSynchronize(c->stream));
    std::vector<double> vT, vP;
    {
        const hygro_status st = download_level(c, c->F[c->set][level], T ? &vT : nullptr, P ? &vP : nullptr);
        if (st != HYGRO_OK) return st;
    }
    if (T) CUDA_TRY2(c, cudaMemcpy(T, vT.data(), vT.size() * sizeof(double), cudaMemcpyDefault));
    if (P) CUDA_TRY2(c, cudaMemcpy(P, vP.data(), vP.size() * sizeof(double), cudaMemcpyDefault));
    return hygro2d_sync(c);
}

hygro_status hygro2d_set_fields(hygro2d_ctx *c, int32_t level, const double *T, const double *P)
{
    if (c == nullptr) return fail(nullptr, HYGRO_E_INVALID, "ctx is NULL");
    if (level != 0 && level != 1) return fail(c, HYGRO_E_INVALID, "level must be 0 (n) or 1 (n-1)");
    if (!c->have_materials) return fail(c, HYGRO_E_STATE, "hygro2d_set_materials must come first");
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, HYGRO_E_CUDA, "cudaSetDevice failed");
    const size_t n = (size_t)c->G * c->ny * c->nx;
    std::vector<double> v[2];
    for (int f = 0; f < 2; ++f) {
        const double *src = f == 0 ? T : P;
        if (src == nullptr) continue;
        v[f].resize(n);
        CUDA_TRY2(c, cudaMemcpy(v[f].data(), src, n * sizeof(double), cudaMemcpyDefault));
        for (double x : v[f])
            if (!std::isfinite(x)) return fail(c, HYGRO_E_INVALID, "non-finite field value");
    }
    if (T == nullptr && P == nullptr) return HYGRO_OK;
    CUDA_TRY2(c, cudaStreamSynchronize(c->stream));
    return upload_level(c, c->F[c->set][level], T ? &v[0] : nullptr, P ? &v[1] : nullptr);
}

hygro_status hygro2d_get_step(const hygro2d_ctx *c, int64_t *step)
{
    if (c == nullptr || step == nullptr) return fail(nullptr, HYGRO_E_INVALID, "ctx or step is NULL");
    *step = c->step;
    return HYGRO_OK;
}

const char *hygro2d_last_error(const hygro2d_ctx *c) { return c ? c->err.c_str() : g_create_error2d.c_str(); }

void hygro2d_destroy(hygro2d_ctx *c)
{
    if (c == nullptr) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
}

}  // extern "C"
