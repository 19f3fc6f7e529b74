// DF update of 2D wall sections on uniform grids (dx = dy = h), temporal blocking in shared memory.
//
// One CTA owns a TX x TY tile of one section. It loads the tile plus a halo of H nodes of the two
// stored levels of T and Pv with TMA (cp.async.bulk.tensor, zero fill outside the section), advances
// up to H steps in shared memory -- the valid region shrinks by one node per step -- and writes the
// tile core of the two newest levels to the other buffer set. Per node the balance is the 1D one of
// the DF scheme ([eq:DF_NL], Pv first, then T with Pv^{n+1}) with four faces: the control area is
// wx wy h^2 (half weights on the section edges), a face has the length of its perpendicular weight,
// and a Robin face of the section ([eq:HAM_BC]) enters with that length on an edge node.
#pragma once

#include <cuda.h>

#include "df1d_common.cuh"

namespace hygro {

constexpr int kMaxRegions2D = 8;
constexpr uint8_t kOutside2D = 255;   // region code of box cells outside the section

struct Dev2D {
    int32_t G, nx, ny, pitch;   // row pitch of every field and of the region map, in elements
    int32_t n_regions;
    const uint8_t *region;      // [G][ny][pitch]
    const void *region_tab;     // [G][n_regions][kLayerStride] reals (kh = k / (2h), storage h c / (2 dt))
    const FaceInfo *faces;      // [G][4]
    const float2 *noise;
    void *outT[2], *outP[2];    // output set: [0] level n, [1] level n-1 (after this launch)
    int32_t *err;               // 1: a bounded wait gave up
    int32_t *nonfinite;         // 1: some node went non-finite
    double dt, t0, Lv;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_try_wait_parity(uint32_t bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

template <typename real, int TX, int TY, int H, int NT>
struct Tile2D {
    static constexpr int BX = TX + 2 * H;
    static constexpr int BY = TY + 2 * H;
    static constexpr int CELLS = BX * BY;
    static constexpr int THREADS = NT;
    static_assert((CELLS * sizeof(real)) % 128 == 0, "field arrays must keep 128-byte alignment for TMA");
    static_assert((BX * sizeof(real)) % 16 == 0, "TMA box rows must be a multiple of 16 bytes");
    static_assert((H * sizeof(real)) % 16 == 0, "the halo keeps the tile's x start on a 16-byte boundary");
    static_assert((TX * sizeof(real)) % 16 == 0, "tile starts on a 16-byte boundary");
    // dynamic shared memory layout (bytes): T(cur), T(prev), P(cur), P(prev), khM, khT, region, tail
    static constexpr size_t FIELD = (size_t)CELLS * sizeof(real);
    static constexpr size_t OFF_KHM = 4 * FIELD;
    static constexpr size_t OFF_KHT = 5 * FIELD;
    static constexpr size_t OFF_REG = 6 * FIELD;
    static constexpr size_t OFF_TAIL = OFF_REG + ((CELLS + 127) / 128) * 128;
    static constexpr size_t OFF_AIR = OFF_TAIL + 64;
    static constexpr size_t OFF_TAB = OFF_TAIL + 128;
    static constexpr size_t BYTES = OFF_TAB + kMaxRegions2D * kLayerStride * sizeof(real);
};

template <typename real, int TX, int TY, int H, int NT>
__global__ void __launch_bounds__(NT, 1)
    df2d_kernel(const __grid_constant__ CUtensorMap mTc, const __grid_constant__ CUtensorMap mTp,
                const __grid_constant__ CUtensorMap mPc, const __grid_constant__ CUtensorMap mPp, const Dev2D d,
                int64_t n0, int32_t n_sub)
{
    using L = Tile2D<real, TX, TY, H, NT>;
    constexpr int BX = L::BX, BY = L::BY;
    extern __shared__ __align__(128) unsigned char smem[];
    // level arrays: slot 0 holds level n at the start, slot 1 level n-1; they swap roles every step
    real *const sT0 = reinterpret_cast<real *>(smem), *const sT1 = reinterpret_cast<real *>(smem + L::FIELD);
    real *const sP0 = reinterpret_cast<real *>(smem + 2 * L::FIELD);
    real *const sP1 = reinterpret_cast<real *>(smem + 3 * L::FIELD);
    real *khM = reinterpret_cast<real *>(smem + L::OFF_KHM);
    real *khT = reinterpret_cast<real *>(smem + L::OFF_KHT);
    uint8_t *reg = smem + L::OFF_REG;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + L::OFF_TAIL);
    real *air = reinterpret_cast<real *>(smem + L::OFF_AIR);   // [4 faces][2]: T_inf', Pv_inf'
    real *rtab = reinterpret_cast<real *>(smem + L::OFF_TAB);  // region constants of this grid

    const int tid = threadIdx.x;
    const int tiles_x = (d.nx + TX - 1) / TX, tiles_y = (d.ny + TY - 1) / TY;
    const int g = blockIdx.x / (tiles_x * tiles_y);
    const int trem = blockIdx.x % (tiles_x * tiles_y);
    const int x0 = (trem % tiles_x) * TX - H;    // section coordinates of box cell (0, 0)
    const int y0 = (trem / tiles_x) * TY - H;
    const uint32_t bar = smem_u32(mbar);

    // 1. the four levels by TMA (one thread), the region map and the constants by plain loads
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"((uint32_t)(4 * L::FIELD))
                     : "memory");
        const CUtensorMap *maps[4] = {&mTc, &mTp, &mPc, &mPp};
        const uint32_t dst[4] = {smem_u32(sT0), smem_u32(sT1), smem_u32(sP0), smem_u32(sP1)};
#pragma unroll
        for (int f = 0; f < 4; ++f)
            asm volatile(
                "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
                "[%5];" ::"r"(dst[f]),
                "l"(maps[f]), "r"(x0), "r"(y0), "r"(g), "r"(bar)
                : "memory");
    }
    const uint8_t *greg = d.region + (size_t)g * d.ny * d.pitch;
    for (int c = tid; c < BX * BY; c += NT) {
        const int gx = x0 + c % BX, gy = y0 + c / BX;
        reg[c] = (gx >= 0 && gx < d.nx && gy >= 0 && gy < d.ny) ? greg[(size_t)gy * d.pitch + gx] : kOutside2D;
    }
    const real *gtab = reinterpret_cast<const real *>(d.region_tab) + (size_t)g * d.n_regions * kLayerStride;
    for (int i = tid; i < d.n_regions * kLayerStride; i += NT) rtab[i] = gtab[i];
    {
        // bounded wait for the copies (phase 0). If any thread gave up, the whole CTA flags it, waits
        // (bounded again) for the copies still in flight and leaves without touching the output.
        bool done = false;
        for (long it = 0; it < (1L << 24) && !done; ++it) done = mbar_try_wait_parity(bar, 0);
        if (__syncthreads_or(!done)) {
            if (tid == 0) atomicExch(d.err, 1);
            for (long it = 0; it < (1L << 26) && !done; ++it) done = mbar_try_wait_parity(bar, 0);
            return;
        }
    }

    const FaceInfo *fc = d.faces + (size_t)g * 4;
    const real Lv = (real)d.Lv, half = real(0.5);
    int cur = 0;
    for (int s = 1; s <= n_sub; ++s) {
        // ambient air of the four faces at t^n, and the half-conductances of the cells still valid
        if (tid < 4) {
            real aT = real(0), aP = real(0);
            if (fc[tid].kind == HYGRO_BC_AMBIENT) ambient_at(fc[tid], d.noise, n0 + s - 1, d.t0, d.dt, aT, aP);
            air[tid * 2] = aT;
            air[tid * 2 + 1] = aP;
        }
        const real *Tc = cur ? sT1 : sT0, *Pc = cur ? sP1 : sP0;
        real *Tp = cur ? sT0 : sT1, *Pp = cur ? sP0 : sP1;
        {
            const int lo = s - 1, w = BX - 2 * lo, n = w * (BY - 2 * lo);
            for (int i = tid; i < n; i += NT) {
                const int c = (lo + i / w) * BX + lo + i % w;
                const int r = reg[c];
                if (r == kOutside2D) continue;
                const real *q = rtab + r * kLayerStride;
                khM[c] = fma(q[LT_KMB], Pc[c], q[LT_KMA]);
                khT[c] = fma(q[LT_KTB], Pc[c], q[LT_KTA]);
            }
        }
        __syncthreads();
        // update the cells at distance >= s from the box edge (all their neighbours are valid)
        const int w = BX - 2 * s, n = w * (BY - 2 * s);
        for (int i = tid; i < n; i += NT) {
            const int by = s + i / w, bx = s + i % w;
            const int c = by * BX + bx;
            const int r = reg[c];
            if (r == kOutside2D) continue;
            const int gx = x0 + bx, gy = y0 + by;
            const real wx = (gx == 0 || gx == d.nx - 1) ? half : real(1);
            const real wy = (gy == 0 || gy == d.ny - 1) ? half : real(1);
            const real *q = rtab + r * kLayerStride;
            const real Pk = Pc[c], pp = Pp[c], tp = Tp[c];
            const real A = wx * wy * fma(q[LT_AB], Pk, q[LT_AA]);
            const real B = wx * wy * fma(q[LT_BB], Pk, q[LT_BA]);
            const real kMc = khM[c], kTc = khT[c];
            real numP = real(0), S = real(0), numT = real(0), ST = real(0), gsrc = real(0);
            const int nbs[4] = {c - 1, c + 1, c - BX, c + BX};
            const bool inside[4] = {gx > 0, gx < d.nx - 1, gy > 0, gy < d.ny - 1};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (!inside[k]) continue;
                const int e = nbs[k];
                const real wp = k < 2 ? wy : wx;
                real FM, FT;
                if (reg[e] == r) {
                    FM = kMc + khM[e];
                    FT = kTc + khT[e];
                } else {
                    FM = face_harmonic(kMc, khM[e]);
                    FT = face_harmonic(kTc, khT[e]);
                }
                FM *= wp;
                FT *= wp;
                numP = fma(FM, Pc[e] - pp, numP);
                S += FM;
                numT = fma(FT, Tc[e] - tp, numT);
                ST += FT;
            }
            // Robin faces of the section on this node (face 0: x = 0, 1: x = Lx, 2: y = 0, 3: y = Ly)
            const bool on[4] = {gx == 0, gx == d.nx - 1, gy == 0, gy == d.ny - 1};
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                if (!on[f] || fc[f].kind != HYGRO_BC_AMBIENT) continue;
                const real wp = f < 2 ? wy : wx;
                const real hM = wp * (real)fc[f].hM, hT = wp * (real)fc[f].hT;
                numP = fma(hM, air[f * 2 + 1] - pp, numP);
                S += hM;
                gsrc += wp * (real)fc[f].g_inf;
                numT = fma(hT, air[f * 2] - tp, numT + wp * (real)fc[f].q_inf);
                ST += hT;
            }
            const real dP = fast_div(numP + gsrc, fma(half, S, A));
            const real X = fma(-S, half * dP, numP);   // latent cross flux with the time-averaged Pv
            numT = fma(Lv, X, numT);
            numT = fma(-q[LT_CHI] * A, dP, numT);
            const real dT = fast_div(numT, fma(half, ST, B));
            Pp[c] = pp + dP;
            Tp[c] = tp + dT;
        }
        __syncthreads();
        cur = 1 - cur;
    }

    // 2. the tile core of the two newest levels to the output set
    bool bad = false;
    for (int c = tid; c < TX * TY; c += NT) {
        const int bx = H + c % TX, by = H + c / TX;
        const int gx = x0 + bx, gy = y0 + by;
        if (gx >= d.nx || gy >= d.ny) continue;
        const size_t o = ((size_t)g * d.ny + gy) * d.pitch + gx;
        const int b = by * BX + bx;
        const real t0v = (cur ? sT1 : sT0)[b], t1v = (cur ? sT0 : sT1)[b];
        const real p0v = (cur ? sP1 : sP0)[b], p1v = (cur ? sP0 : sP1)[b];
        bad |= !isfinite(t0v) || !isfinite(p0v);
        reinterpret_cast<real *>(d.outT[0])[o] = t0v;
        reinterpret_cast<real *>(d.outT[1])[o] = t1v;
        reinterpret_cast<real *>(d.outP[0])[o] = p0v;
        reinterpret_cast<real *>(d.outP[1])[o] = p1v;
    }
    if (bad) atomicExch(d.nonfinite, 1);
}

}  // namespace hygro
