// DF update of 2D wall sections on uniform grids (dx = dy = h), temporal blocking in shared memory.
//
// One CTA owns a TX x TY tile of one section. It loads the tile plus a halo of H nodes of the two
// stored levels -- each node's (T, Pv) pair, interleaved -- and the node flags with TMA
// (cp.async.bulk.tensor, zero fill outside the section), advances up to H steps in shared memory (the
// valid region shrinks by one node per step), and writes the tile core of the two newest levels to the
// other buffer set. A thread owns one column of the box and sweeps a run of its rows, keeping the
// (T, Pv) values and half-conductances of the cells above, at and below the current one in registers;
// the left and right neighbours come from shared memory. Per node the balance is the 1D one of the DF
// scheme ([eq:DF_NL], Pv first, then T with Pv^{n+1}) with four faces: the control area is wx wy h^2
// (half weights on the section edges), a face has the length of its perpendicular weight, and a Robin
// face of the section ([eq:HAM_BC]) enters an edge node with that length.
#pragma once

#include <cuda.h>

#include "df1d_common.cuh"

namespace hygro {

constexpr int kMaxRegions2D = 8;
// Node flags byte: region in bits 0-2; bit 3 set on the section's edge nodes (half weights, Robin faces);
// bit 4 / 5 / 6 / 7 set when the neighbour at x-1 / x+1 / y-1 / y+1 lies in another region (its face
// takes the harmonic mean).
constexpr uint32_t kRegionMask2D = 7u;
constexpr uint32_t kEdge2D = 1u << 3;
constexpr uint32_t kDiffL = 1u << 4, kDiffR = 1u << 5, kDiffU = 1u << 6, kDiffD = 1u << 7;
constexpr uint32_t kDiffAny2D = kDiffL | kDiffR | kDiffU | kDiffD;

template <typename real>
struct PairOf;
template <>
struct PairOf<float> {
    using type = float2;
};
template <>
struct PairOf<double> {
    using type = double2;
};

struct Dev2D {
    int32_t G, nx, ny, pitch;   // row pitch of the level arrays and of the flags, in nodes
    int32_t n_regions;
    const void *region_tab;     // [G][n_regions][kLayerStride] reals (kh = k / (2h), storage h c / (2 dt))
    const FaceInfo *faces;      // [G][4]
    const float2 *noise;
    void *out_new, *out_old;    // output set: (T, Pv) pairs of level n and n-1 after this launch
    int32_t *err;               // 1: a bounded wait gave up
    int32_t *nonfinite;         // 1: some node went non-finite
    const int64_t *step_dev;    // if set, the launch's first step is *step_dev + n0 (launches replayed from a
                                // CUDA graph read the step from the device)
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

// Shapes and shared-memory layout of one tile. SEG threads share a column of the box, each sweeping
// the same number of rows at every step (the last run of rows reads PAD rows past the box, which are
// allocated but never stored), so every warp takes the same trip count.
template <typename real, int TX, int TY, int H, int SEG>
struct Tile2D {
    using pair = typename PairOf<real>::type;
    static constexpr int BX = TX + 2 * H;
    static constexpr int BY = TY + 2 * H;
    static constexpr int NT = BX * SEG;
    static constexpr int PAD = SEG;                   // rows past the box read by the last run (with prefetch)
    static constexpr int ROWS = BY + PAD;
    // the flags box starts on a 16-byte boundary of the row: FOFF bytes left of box column 0
    static constexpr int FOFF = (16 - H % 16) % 16;
    static constexpr int FBX = (FOFF + BX + 15) / 16 * 16;
    static_assert(TX % 16 == 0, "tile columns start on 16-byte boundaries of the flags rows");
    static_assert(NT % 32 == 0, "whole warps");
    static_assert((H * sizeof(pair)) % 16 == 0, "the box's x start stays on a 16-byte boundary");
    static constexpr size_t LEVEL = ((size_t)BX * ROWS * sizeof(pair) + 127) / 128 * 128;
    static constexpr size_t OFF_FLAGS = 2 * LEVEL;
    static constexpr size_t FLAGS = (size_t)FBX * ROWS;
    static constexpr size_t OFF_AIR = OFF_FLAGS + (FLAGS + 127) / 128 * 128;   // [H steps][4 faces][2]
    static constexpr size_t OFF_FACE = OFF_AIR + (size_t)H * 8 * sizeof(real); // [4 faces][4]: hM, hT, g, q
    static constexpr size_t OFF_TAB = OFF_FACE + 16 * sizeof(real);
    static constexpr size_t OFF_BAR = OFF_TAB + (size_t)kMaxRegions2D * kLayerStride * sizeof(real);
    static constexpr size_t BYTES = OFF_BAR + 16;
    // bytes the TMA copies deliver: two boxes of pairs and one box of flags
    static constexpr uint32_t TX_BYTES = (uint32_t)(2 * (size_t)BX * BY * sizeof(pair) + (size_t)FBX * BY);
};

// Constants of one region in pair form: (kTT, kM) / (2h) = ka + kb Pv', (cTT, cM) storage = sa + sb Pv'.
template <typename real>
struct RegionC {
    uint32_t r;
    P2<real> ka, kb, sa, sb;
    real chi;
};

template <typename real>
__device__ __forceinline__ void fetch_region(RegionC<real> &c, uint32_t r, const real *tab)
{
    const real *q = tab + r * kLayerStride;
    c.r = r;
    c.ka = p2_make(q[LT_KTA], q[LT_KMA]);
    c.kb = p2_make(q[LT_KTB], q[LT_KMB]);
    c.sa = p2_make(q[LT_BA], q[LT_AA]);
    c.sb = p2_make(q[LT_BB], q[LT_AB]);
    c.chi = q[LT_CHI];
}

// (kTT, kM) / (2h) of a node with vapour-pressure deviation P, from the cached constants when the node
// lies in their region (same), else from its region's row of the table.
template <typename real>
__device__ __forceinline__ P2<real> half_k(const RegionC<real> &c, bool same, uint32_t fl, real P, const real *tab)
{
    if (same) return p2_fma(c.kb, p2_make(P, P), c.ka);
    const real *q = tab + (fl & kRegionMask2D) * kLayerStride;
    return p2_make(fma(q[LT_KTB], P, q[LT_KTA]), fma(q[LT_KMB], P, q[LT_KMA]));
}

template <typename real, int TX, int TY, int H, int SEG, int MINB>
__global__ void __launch_bounds__(Tile2D<real, TX, TY, H, SEG>::NT, MINB)
    df2d_kernel(const __grid_constant__ CUtensorMap mCur, const __grid_constant__ CUtensorMap mPrev,
                const __grid_constant__ CUtensorMap mFlags, const Dev2D d, int64_t n0, int32_t n_sub)
{
    if (d.step_dev != nullptr) n0 += *d.step_dev;
    using L = Tile2D<real, TX, TY, H, SEG>;
    using pair = typename L::pair;
    constexpr int BX = L::BX, BY = L::BY, NT = L::NT;
    constexpr bool kPairMap4D = sizeof(real) == 8;   // FP64 pairs: 4D map over (component, x, y, grid)
    extern __shared__ __align__(128) unsigned char smem[];
    // slot 0 holds level n at the start, slot 1 level n-1; they swap roles every step
    pair *const slot0 = reinterpret_cast<pair *>(smem);
    pair *const slot1 = reinterpret_cast<pair *>(smem + L::LEVEL);
    const uint8_t *flags = smem + L::OFF_FLAGS;
    real *air = reinterpret_cast<real *>(smem + L::OFF_AIR);
    real *fconst = reinterpret_cast<real *>(smem + L::OFF_FACE);
    real *tab = reinterpret_cast<real *>(smem + L::OFF_TAB);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + L::OFF_BAR);

    const int tid = threadIdx.x;
    const int tiles_x = (d.nx + TX - 1) / TX, tiles_y = (d.ny + TY - 1) / TY;
    const int g = blockIdx.x / (tiles_x * tiles_y);
    const int trem = blockIdx.x % (tiles_x * tiles_y);
    const int x0 = (trem % tiles_x) * TX - H;    // section coordinates of box cell (0, 0)
    const int y0 = (trem / tiles_x) * TY - H;
    const uint32_t bar = smem_u32(mbar);

    // 1. both levels and the flags by TMA (one thread); the face data and region constants by plain loads
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(L::TX_BYTES) : "memory");
        if constexpr (kPairMap4D) {
            asm volatile(
                "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
                "%4, %5}], [%6];" ::"r"(smem_u32(slot0)),
                "l"(&mCur), "r"(0), "r"(x0), "r"(y0), "r"(g), "r"(bar)
                : "memory");
            asm volatile(
                "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
                "%4, %5}], [%6];" ::"r"(smem_u32(slot1)),
                "l"(&mPrev), "r"(0), "r"(x0), "r"(y0), "r"(g), "r"(bar)
                : "memory");
        } else {
            asm volatile(
                "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
                "%4}], [%5];" ::"r"(smem_u32(slot0)),
                "l"(&mCur), "r"(x0), "r"(y0), "r"(g), "r"(bar)
                : "memory");
            asm volatile(
                "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
                "%4}], [%5];" ::"r"(smem_u32(slot1)),
                "l"(&mPrev), "r"(x0), "r"(y0), "r"(g), "r"(bar)
                : "memory");
        }
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
            "[%5];" ::"r"(smem_u32(flags)),
            "l"(&mFlags), "r"(x0 - L::FOFF), "r"(y0), "r"(g), "r"(bar)
            : "memory");
    }
    const FaceInfo *fc = d.faces + (size_t)g * 4;
    if (tid < 4 * n_sub) {
        // ambient air of face f at t^{n0+s}, for every step s of this launch
        const int s = tid >> 2, f = tid & 3;
        real aT = real(0), aP = real(0);
        if (fc[f].kind == HYGRO_BC_AMBIENT) ambient_at(fc[f], d.noise, n0 + s, d.t0, d.dt, aT, aP);
        air[s * 8 + f * 2] = aT;
        air[s * 8 + f * 2 + 1] = aP;
    }
    if (tid >= NT - 4) {
        const int f = tid - (NT - 4);
        const bool amb = fc[f].kind == HYGRO_BC_AMBIENT;
        fconst[f * 4 + 0] = amb ? (real)fc[f].hM : real(0);
        fconst[f * 4 + 1] = amb ? (real)fc[f].hT : real(0);
        fconst[f * 4 + 2] = amb ? (real)fc[f].g_inf : real(0);
        fconst[f * 4 + 3] = amb ? (real)fc[f].q_inf : real(0);
    }
    const real *gtab = reinterpret_cast<const real *>(d.region_tab) + (size_t)g * d.n_regions * kLayerStride;
    for (int i = tid; i < d.n_regions * kLayerStride; i += NT) tab[i] = gtab[i];
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

    // 2. n_sub DF steps in shared memory. Thread (x, seg) sweeps a run of rows of box column x; every
    // thread takes the same number of rows, and threads outside the section or the step's valid band
    // compute without storing. Every node goes through the same arithmetic: arithmetic face means with
    // the node's own region constants, then (only on the few nodes that need it) the harmonic means of
    // faces to another region, and the half weights and Robin terms of section edges.
    const int x = tid % BX, seg = tid / BX;
    const int gx = x0 + x;
    const real Lv = (real)d.Lv, half = real(0.5), one = real(1), zero = real(0);
    const real wx = (gx == 0 || gx == d.nx - 1) ? half : one;
    const real mL = gx > 0 ? one : zero, mR = gx < d.nx - 1 ? one : zero;   // x-faces present
    // Robin face of this column on x = 0 (face 0) or x = Lx (face 1); other columns take zeros
    const int fcol = gx == 0 ? 0 : (gx == d.nx - 1 ? 1 : -1);
    const real rx = fcol >= 0 ? one : zero;
    const real *qx = fconst + (fcol > 0 ? 4 : 0);
    const real fxM = rx * qx[0], fxT = rx * qx[1], fxG = rx * qx[2], fxQ = rx * qx[3];
    const bool col_in = gx >= 0 && gx < d.nx;
    // rows of the section inside the box
    const int ylo = max(0, -y0), yhi = min(BY, d.ny - y0);
    // a launch of fewer than H steps only updates the cells its tile core depends on
    const int margin = H - n_sub;
    for (int s = 1; s <= n_sub; ++s) {
        const pair *cur = (s & 1) ? slot0 : slot1;
        pair *prv = (s & 1) ? slot1 : slot0;
        const int lo = margin + s;   // cells at distance >= lo from the box edge are updated
        const int len = (BY - 2 * lo + SEG - 1) / SEG;
        const int yfirst = lo + seg * len;
        const int rlo = max(lo, ylo), rhi = min(BY - lo, yhi);   // rows stored at this step
        const bool col_ok = col_in && x >= lo && x < BX - lo;
        // run indices i whose row is stored: i - ilo in [0, nst)
        const int ilo = rlo - yfirst;
        const unsigned nst = col_ok && rhi > rlo ? (unsigned)(rhi - rlo) : 0u;
        const real aTx = air[(s - 1) * 8 + (fcol > 0 ? 2 : 0)], aPx = air[(s - 1) * 8 + (fcol > 0 ? 3 : 1)];
        // prime the window: the cell above the first row and the first row (half-conductances
        // with each cell's own region), then the neighbours of the first row
        RegionC<real> cc;
        uint32_t fcen = flags[yfirst * L::FBX + x + L::FOFF];
        fetch_region(cc, fcen & kRegionMask2D, tab);
        P2<real> pu = p2_load(cur + (yfirst - 1) * BX + x), pc = p2_load(cur + yfirst * BX + x);
        P2<real> ku;
        {
            const uint32_t fu = flags[(yfirst - 1) * L::FBX + x + L::FOFF];
            ku = half_k(cc, (fu & kRegionMask2D) == cc.r, fu, p2_p(pu), tab);
        }
        P2<real> kc = p2_fma(cc.kb, p2_make(p2_p(pc), p2_p(pc)), cc.ka);
        int c = yfirst * BX + x;
        P2<real> pd = p2_load(cur + c + BX), pl = p2_load(cur + c - 1), pr = p2_load(cur + c + 1);
        P2<real> pv = p2_load(prv + c);
        uint32_t fd = flags[(yfirst + 1) * L::FBX + x + L::FOFF];
#pragma unroll 2
        for (int i = 0; i < len; ++i, c += BX) {
            const int y = yfirst + i;
            // the next row's neighbours, read before this row's result is stored
            const P2<real> pdn = p2_load(cur + c + 2 * BX), pln = p2_load(cur + c + BX - 1);
            const P2<real> prn = p2_load(cur + c + BX + 1), pvn = p2_load(prv + c + BX);
            const uint32_t fdn = flags[(y + 2) * L::FBX + x + L::FOFF];
            const real Pk = p2_p(pc);
            // half-conductances of the neighbours with the node's region constants
            P2<real> kd = p2_fma(cc.kb, p2_make(p2_p(pd), p2_p(pd)), cc.ka);
            const P2<real> kl = p2_fma(cc.kb, p2_make(p2_p(pl), p2_p(pl)), cc.ka);
            const P2<real> kr = p2_fma(cc.kb, p2_make(p2_p(pr), p2_p(pr)), cc.ka);
            P2<real> Fl = p2_add(kc, kl), Fr = p2_add(kc, kr), Fu = p2_add(kc, ku), Fd = p2_add(kc, kd);
            P2<real> st = p2_fma(cc.sb, p2_make(Pk, Pk), cc.sa);   // (B, A) storage terms
            // rare nodes (faces to another region, section edges) in one test
            const bool edge = fcen & kEdge2D;
            bool edge_y = false;
            int gy = 0;
            real wy = one;
            if (fcen & (kDiffAny2D | kEdge2D)) {
                if (fcen & kDiffAny2D) {
                    // faces to another region: that region's constants, harmonic mean
                    if (fcen & kDiffL) {
                        const P2<real> k = half_k(cc, false, flags[y * L::FBX + x - 1 + L::FOFF], p2_p(pl), tab);
                        Fl = p2_make(face_harmonic(p2_t(kc), p2_t(k)), face_harmonic(p2_p(kc), p2_p(k)));
                    }
                    if (fcen & kDiffR) {
                        const P2<real> k = half_k(cc, false, flags[y * L::FBX + x + 1 + L::FOFF], p2_p(pr), tab);
                        Fr = p2_make(face_harmonic(p2_t(kc), p2_t(k)), face_harmonic(p2_p(kc), p2_p(k)));
                    }
                    if (fcen & kDiffU) Fu = p2_make(face_harmonic(p2_t(kc), p2_t(ku)), face_harmonic(p2_p(kc), p2_p(ku)));
                    if (fcen & kDiffD) {
                        kd = half_k(cc, false, fd, p2_p(pd), tab);
                        Fd = p2_make(face_harmonic(p2_t(kc), p2_t(kd)), face_harmonic(p2_p(kc), p2_p(kd)));
                    }
                }
                if (edge) {
                    // section edges: half control areas and face lengths, absent faces weighted 0
                    gy = y0 + y;
                    edge_y = gy == 0 || gy == d.ny - 1;
                    wy = edge_y ? half : one;
                    const real wl = wy * mL, wr = wy * mR, wu = gy > 0 ? wx : zero, wd = gy < d.ny - 1 ? wx : zero;
                    Fl = p2_mul(Fl, p2_make(wl, wl));
                    Fr = p2_mul(Fr, p2_make(wr, wr));
                    Fu = p2_mul(Fu, p2_make(wu, wu));
                    Fd = p2_mul(Fd, p2_make(wd, wd));
                    const real wxy = wx * wy;
                    st = p2_mul(p2_make(wxy, wxy), st);
                }
            }
            P2<real> num = p2_mul(Fl, p2_sub(pl, pv));
            num = p2_fma(Fr, p2_sub(pr, pv), num);
            num = p2_fma(Fu, p2_sub(pu, pv), num);
            num = p2_fma(Fd, p2_sub(pd, pv), num);
            const P2<real> S2 = p2_add(p2_add(p2_add(Fl, Fr), Fu), Fd);
            real numP = p2_p(num), S = p2_p(S2), numT = p2_t(num), ST = p2_t(S2), gsrc = zero;
            if (edge) {
                // Robin faces (0: x = 0, 1: x = Lx as zeros on the other columns; 2: y = 0, 3: y = Ly)
                const real tp = p2_t(pv), pp = p2_p(pv);
                {
                    const real hM = wy * fxM, hT = wy * fxT;
                    numP = fma(hM, aPx - pp, numP);
                    S += hM;
                    gsrc = wy * fxG;
                    numT = fma(hT, aTx - tp, numT + wy * fxQ);
                    ST += hT;
                }
                if (edge_y) {
                    const int f = gy == 0 ? 2 : 3;
                    const real *q = fconst + f * 4;
                    const real hM = wx * q[0], hT = wx * q[1];
                    numP = fma(hM, air[(s - 1) * 8 + f * 2 + 1] - pp, numP);
                    S += hM;
                    gsrc += wx * q[2];
                    numT = fma(hT, air[(s - 1) * 8 + f * 2] - tp, numT + wx * q[3]);
                    ST += hT;
                }
            }
            const real A = p2_p(st);
            const real dP = fast_div(numP + gsrc, fma(half, S, A));
            const real X = fma(-S, half * dP, numP);   // latent cross flux with the time-averaged Pv
            numT = fma(Lv, X, numT);
            numT = fma(-cc.chi * A, dP, numT);
            const real dT = fast_div(numT, fma(half, ST, p2_t(st)));
            if ((unsigned)(i - ilo) < nst) p2_store(prv + c, p2_add(pv, p2_make(dT, dP)));
            // roll the window down one row; a cell below in another region than the node was
            // evaluated with the node's constants, so a change of region recomputes it
            pu = pc;
            ku = kc;
            pc = pd;
            kc = kd;
            fcen = fd;
            if ((fd & kRegionMask2D) != cc.r) {
                fetch_region(cc, fd & kRegionMask2D, tab);
                kc = p2_fma(cc.kb, p2_make(p2_p(pd), p2_p(pd)), cc.ka);
            }
            pd = pdn;
            pl = pln;
            pr = prn;
            pv = pvn;
            fd = fdn;
        }
        __syncthreads();
    }

    // 3. the tile core of the two newest levels to the output set
    const pair *newest = (n_sub & 1) ? slot1 : slot0;
    const pair *older = (n_sub & 1) ? slot0 : slot1;
    pair *on = reinterpret_cast<pair *>(d.out_new), *oo = reinterpret_cast<pair *>(d.out_old);
    bool bad = false;
    for (int c = tid; c < TX * TY; c += NT) {
        const int bx = H + c % TX, by = H + c / TX;
        const int ex = x0 + bx, ey = y0 + by;
        if (ex >= d.nx || ey >= d.ny) continue;
        const size_t o = ((size_t)g * d.ny + ey) * d.pitch + ex;
        const int b = by * BX + bx;
        const pair v = newest[b];
        bad |= !isfinite(v.x) || !isfinite(v.y);
        on[o] = v;
        oo[o] = older[b];
    }
    if (bad) atomicExch(d.nonfinite, 1);
}

}  // namespace hygro
