// fdtd_kernels.cu -- sm_103a kernels of the Yee + UPML leapfrog step.
//
// One step (Model section: H at half steps from E, then E from H and J) is
// four launches over a Plan (one board or a batch of boards):
//   k_slab_h     H^{n+1/2} (and B~) on UPML/boundary slab nodes   (Eqs. 1-5)
//   k_interior   fused H^{n+1/2} and E^{n+1} on the interior box (plain Yee,
//                uint8 coefficient ids; halo H recomputed or read from slabs)
//   k_slab_e     E^{n+1} (and D~) on slab nodes, PEC/PMC outer walls
//   k_post       current sources (Eq. 8) and probe samples of E^{n+1}
// and, once per chunk, k_dft folds the new probe samples into the FP64
// running DFT (Results section: spectrum of the ground-plane E_z) with warp
// shuffles.  Fields are ping-ponged, so no launch reads what it writes except
// the per-node UPML auxiliaries, which only their own thread touches.
//
// All curl and update arithmetic goes through curl2()/the update helpers with
// explicit round-to-nearest intrinsics, so a value recomputed as a halo is
// bit-identical to the one its owner stores.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fdtd_internal.h"

namespace fdtd {



// ------------------------------------------------------------------ storage
template <typename T>
struct Io;
template <>
struct Io<float> {
    static __device__ __forceinline__ float ld(const float *p) { return __ldg(p); }
    static __device__ __forceinline__ float ldw(const float *p) { return *p; }
    static __device__ __forceinline__ void st(float *p, float v) { *p = v; }
};
template <>
struct Io<__half> {
    static __device__ __forceinline__ float ld(const __half *p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ float ldw(const __half *p) { return __half2float(*p); }
    static __device__ __forceinline__ void st(__half *p, float v) { *p = __float2half_rn(v); }
};
template <>
struct Io<__nv_bfloat16> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
    static __device__ __forceinline__ float ldw(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
};

// ------------------------------------------------------------------ arithmetic
// Sa (a1 - a0) - Sb (b1 - b0): one component of S * curl.
__device__ __forceinline__ float curl2(float a1, float a0, float b1, float b0, float Sa, float Sb)
{
    return __fmaf_rn(-Sb, __fsub_rn(b1, b0), __fmul_rn(Sa, __fsub_rn(a1, a0)));
}

__device__ __forceinline__ int find_board(const long long *prefix, int nb, long long item)
{
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(prefix + mid) <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ bool board_active(const Board *B)
{
    return *((volatile long long *)B->step) < *((volatile long long *)B->stop);
}

// ------------------------------------------------------------------ fused region
// H~^{n+1/2} components at node q straight from global memory (input parity);
// used once per z-segment for the plane below the segment.
template <typename T>
struct Fields {
    const T *__restrict__ ex, *__restrict__ ey, *__restrict__ ez;
    const T *__restrict__ hx, *__restrict__ hy, *__restrict__ hz;
    T *__restrict__ oex, *__restrict__ oey, *__restrict__ oez;
    T *__restrict__ ohx, *__restrict__ ohy, *__restrict__ ohz;
    __device__ __forceinline__ Fields(const Board *B, int par)
    {
        ex = (const T *)B->f[par][0]; ey = (const T *)B->f[par][1]; ez = (const T *)B->f[par][2];
        hx = (const T *)B->f[par][3]; hy = (const T *)B->f[par][4]; hz = (const T *)B->f[par][5];
        oex = (T *)B->f[par ^ 1][0]; oey = (T *)B->f[par ^ 1][1]; oez = (T *)B->f[par ^ 1][2];
        ohx = (T *)B->f[par ^ 1][3]; ohy = (T *)B->f[par ^ 1][4]; ohz = (T *)B->f[par ^ 1][5];
    }
};

__device__ __forceinline__ int cid_at(const Board *B, long long idx)
{
    return B->id16 ? (int)__ldg((const uint16_t *)B->cid + idx) : (int)__ldg((const uint8_t *)B->cid + idx);
}

// Gedney two-step update of one H~ component (B~ recurrence along w+1, H~
// recurrence along w+2, B~->H~ along w).  scurl = S * (curl E)_w.  Bo/Bn are
// the old/new auxiliaries (no auxiliary: pass aux == false).
__device__ __forceinline__ float upml_h2(float h, float scurl, const Coef &a, const Coef &bb, const Coef &c, bool aux,
                                         float Bo, float &Bn)
{
    if (aux) {
        Bn = __fmaf_rn(-a.g, scurl, __fmul_rn(a.b1, Bo));
        return __fmaf_rn(bb.g, __fmaf_rn(c.ap, Bn, -__fmul_rn(c.am, Bo)), __fmul_rn(bb.b1, h));
    }
    return __fmaf_rn(-bb.g, scurl, __fmul_rn(bb.b1, h));
}

// Same for E (D~ along w+1, E along w+2, D~->E along w); ce = 1/eps_r.
__device__ __forceinline__ float upml_e2(float e, float scurl, float ce, const Coef &a, const Coef &bb, const Coef &c,
                                         bool aux, float Do, float &Dn)
{
    if (aux) {
        Dn = __fmaf_rn(a.g, scurl, __fmul_rn(a.b1, Do));
        return __fmaf_rn(__fmul_rn(ce, bb.g), __fmaf_rn(c.ap, Dn, -__fmul_rn(c.am, Do)), __fmul_rn(bb.b1, e));
    }
    return __fmaf_rn(__fmul_rn(ce, bb.g), scurl, __fmul_rn(bb.b1, e));
}

__device__ __constant__ Coef kOne = {1.0f, 1.0f, 1.0f, 1.0f};

// z-UPML plane kinds of the fused region: 0 none, 1 lower box, 2 upper box.
__device__ __forceinline__ int zbox_of(const Board *B, int k) { return k < B->iz0 ? 1 : (k >= B->iz1 ? 2 : 0); }

__device__ __forceinline__ long long zaux_index(const Board *B, int box, int i, int j, int k)
{
    const int k0 = box == 1 ? 1 : B->iz1;
    return ((long long)(k - k0) * (B->iy1 - B->iy0) + (j - B->iy0)) * (long long)B->zpitch + (i - B->ix0);
}

// New H~x, H~y, H~z at a fused-region node from already-fetched operands.
// In z-UPML planes only sigma_z is non-zero: H~x has no auxiliary, H~y and
// H~z carry B~y, B~z.
struct ZCoef {
    Coef zi, zh;   // z factors at the node's integer and half positions
};

__device__ __forceinline__ float fused_hx(float h, float sc, int zb, const ZCoef &z)
{
    float dummy;
    if (!zb) return __fsub_rn(h, sc);
    return upml_h2(h, sc, kOne, z.zh, kOne, false, 0.f, dummy);
}
__device__ __forceinline__ float fused_hy(float h, float sc, int zb, const ZCoef &z, float Bo, float &Bn)
{
    if (!zb) return __fsub_rn(h, sc);
    return upml_h2(h, sc, z.zh, kOne, kOne, true, Bo, Bn);
}
__device__ __forceinline__ float fused_hz(float h, float sc, int zb, const ZCoef &z, float Bo, float &Bn)
{
    if (!zb) return __fsub_rn(h, sc);
    return upml_h2(h, sc, kOne, kOne, z.zi, true, Bo, Bn);
}

// ------------------------------------------------------------------ TMA + mbarrier
__device__ __forceinline__ uint32_t s_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t n)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_addr(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_addr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *b, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(s_addr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait on a phase: gives up after ~2^21 polls (each poll itself
// suspends for a hardware-defined slice) and reports it in *status.
__device__ __forceinline__ void mbar_wait(uint64_t *b, uint32_t parity, int *status, int *abort_flag)
{
    if (*(volatile int *)abort_flag) return;
    for (uint32_t it = 0; it < (1u << 21); ++it)
        if (mbar_try(b, parity)) return;
    atomicOr(status, 2);
    *(volatile int *)abort_flag = 1;
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            s_addr(dst)),
        "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(s_addr(bar))
        : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

template <typename T>
__device__ __forceinline__ float cvt(T v);
template <>
__device__ __forceinline__ float cvt<float>(float v) { return v; }
template <>
__device__ __forceinline__ float cvt<__half>(__half v) { return __half2float(v); }
template <>
__device__ __forceinline__ float cvt<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

// Shared-memory stage of one plane for a tile of W warps x 31 columns by TY
// rows.  Boxes start at x rounded down to the 16-byte TMA boundary:
//   E  3 x (TY+2) x EW   nodes i0-1 .. i0+31W, rows j0-1 .. j0+TY
//   H  3 x (TY+1) x HW   nodes i0-1 .. i0+31W-1, rows j0-1 .. j0+TY-1
//   id TY x C8W bytes (or TY x C16W uint16), rows j0 .. j0+TY-1
// Every box starts 128-byte aligned.
template <typename T, int TY, int W>
struct Stage {
    static constexpr int al(int x) { return (x + 127) & ~127; }
    static constexpr int TX = 31 * W;
    static constexpr int ES = (int)sizeof(T);
    static constexpr int EW = box_e(TX), HW = box_h(TX), C8W = box_c8(TX), C16W = box_c16(TX);
    static constexpr int E_COMP = (TY + 2) * EW, H_COMP = (TY + 1) * HW;
    static constexpr int E_CS = al(E_COMP * ES) / ES, H_CS = al(H_COMP * ES) / ES;
    static constexpr int E_BYTES = 3 * E_COMP * ES;
    static constexpr int H_BYTES = 3 * H_COMP * ES;
    static constexpr int C8_BYTES = TY * C8W, C16_BYTES = TY * C16W * 2;
    static constexpr int E_OFF = 0;
    static constexpr int H_OFF = 3 * E_CS * ES;
    static constexpr int C_OFF = H_OFF + 3 * H_CS * ES;
    static constexpr int ITEM_OFF = C_OFF + al(C8_BYTES > C16_BYTES ? C8_BYTES : C16_BYTES);   // item id of the plane
    static constexpr int BYTES = ITEM_OFF + 128;
};

template <typename T, int TY, int W, int NS>
struct FusedLayout {
    using St = Stage<T, TY, W>;
    static constexpr int BAR_OFF = NS * St::BYTES;
    static constexpr int BYTES = BAR_OFF + 2 * NS * 8 + 16;
};

__device__ __forceinline__ void mbar_arrive(uint64_t *b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_addr(b)) : "memory");
}

// Work item -> tile; identical in the producer and the consumer warps.
struct Tile {
    const Board *B;
    int ok;
    int i0, j0, kb, ke, kstart, par;
};

template <int TY, int W>
__device__ __forceinline__ Tile decode_tile(const Plan &plan, long long item)
{
    Tile t;
    const int b = find_board(plan.int_prefix, plan.nb, item);
    t.B = plan.boards[b];
    t.ok = board_active(t.B);
    const long long step = *((volatile long long *)t.B->step);
    t.par = (int)(step & 1);
    const long long local = item - __ldg(plan.int_prefix + b);
    const int ntx = (t.B->ix1 - t.B->ix0 + 31 * W - 1) / (31 * W), nty = (t.B->iy1 - t.B->iy0 + TY - 1) / TY;
    const int tx = (int)(local % ntx);
    const long long rest = local / ntx;
    const int ty = (int)(rest % nty), tz = (int)(rest / nty);
    t.i0 = t.B->ix0 + tx * 31 * W;
    t.j0 = t.B->iy0 + ty * TY;
    t.kb = 1 + tz * plan.zseg;
    t.ke = min(t.kb + plan.zseg, t.B->nz);
    t.kstart = t.kb >= 2 ? t.kb - 1 : t.kb;
    return t;
}

// Fused H+E kernel over the fused region, fed by TMA, warp-specialised.
// Warps 0..W-1 compute; warp W (one lane) is the producer, streaming planes
// kstart..ke of the tile into an NS-stage ring (E^n with a one-node halo,
// H~^{n-1/2} with the low halo row and column, coefficient ids), each stage
// with a "full" mbarrier (TMA bytes) and an "empty" one (one arrival per
// compute warp).  Compute warp w owns a strip of 31 columns: lane l sits on
// column i0-1+31w+l, lane 0 being the strip's low-x halo.  Per plane k a lane
// marches the tile's rows in y: it forms H~^{n+1/2}(k) at its column for the
// halo row j0-1 and then row by row, so H(j-1) is already in registers, takes
// H(i-1) from the lane to its left with a shuffle, and updates E^{n+1}(k).
// H~ of halo nodes outside the fused region is read from the slab kernel's
// output instead.  The plane below the segment is run once for the tile's
// H~x, H~y there; the plane above is read for E only.  In z-UPML planes
// (sigma_z only) H~y, H~z carry B~y, B~z and E_y, E_z carry D~y, D~z.
template <typename T, int TY, int W, int NS>
__global__ void __launch_bounds__(32 * W + 32, W == 4 ? 2 : 4) k_fused(Plan plan)
{
    using St = Stage<T, TY, W>;
    using L = FusedLayout<T, TY, W, NS>;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + L::BAR_OFF);
    uint64_t *empty = full + NS;
    int *abort_flag = reinterpret_cast<int *>(empty + NS);
    const int lx = threadIdx.x, wy = threadIdx.y;

    if (wy == 0 && lx == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], W);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();

    if (wy == W) {
        // ------------------------------------------------------------ producer
        // Items are taken from a global counter; the first plane of an item
        // carries the item id to the compute warps, an id of -1 ends the work.
        if (lx != 0) return;
        uint32_t eph = 0;
        long long q = 0;
        int s = 0;
        auto acquire = [&]() {
            if (q >= NS) {
                mbar_wait(&empty[s], (eph >> s) & 1u, plan.boards[0]->status, abort_flag);
                eph ^= 1u << s;
            }
        };
        for (;;) {
            const long long item = atomicAdd(plan.work, 1);
            if (item >= plan.n_int) break;
            const Tile t = decode_tile<TY, W>(plan, item);
            const Board *B = t.B;
            const CUtensorMap *tm = B->tm;
            const int id16 = B->id16;
            const int xe0 = (t.i0 - 1) & ~7;
            const int xc0 = id16 ? (t.i0 & ~7) : (t.i0 & ~15);
            const int last = t.ok ? t.ke : t.kstart;    // inactive board: one empty plane
            for (int p = t.kstart; p <= last; ++p, ++q, s = (s + 1 == NS ? 0 : s + 1)) {
                acquire();
                unsigned char *st = smem + s * St::BYTES;
                *reinterpret_cast<volatile long long *>(st + St::ITEM_OFF) = (p == t.kstart) ? item : -2;
                if (!t.ok) {
                    mbar_expect_tx(&full[s], 0);
                    continue;
                }
                const bool e_only = (p == t.ke);
                uint32_t bytes = St::E_BYTES;
                if (!e_only) bytes += St::H_BYTES + (id16 ? St::C16_BYTES : St::C8_BYTES);
                mbar_expect_tx(&full[s], bytes);
                for (int c = 0; c < 3; ++c)
                    tma_load_3d(st + St::E_OFF + c * St::E_CS * St::ES, tm + tm_e(t.par, c), xe0, t.j0 - 1, p, &full[s]);
                if (!e_only) {
                    for (int c = 0; c < 3; ++c)
                        tma_load_3d(st + St::H_OFF + c * St::H_CS * St::ES, tm + tm_h(t.par, c), xe0, t.j0 - 1, p,
                                    &full[s]);
                    tma_load_3d(st + St::C_OFF, tm + kTmCid, xc0, t.j0, p, &full[s]);
                }
            }
        }
        acquire();
        *reinterpret_cast<volatile long long *>(smem + s * St::BYTES + St::ITEM_OFF) = -1;
        mbar_expect_tx(&full[s], 0);
        return;
    }

    // ---------------------------------------------------------------- compute warps
    uint32_t fph = 0;
    int sq = 0;
    for (;;) {
        mbar_wait(&full[sq], (fph >> sq) & 1u, plan.boards[0]->status, abort_flag);
        const long long item = *reinterpret_cast<volatile long long *>(smem + sq * St::BYTES + St::ITEM_OFF);
        if (item < 0) break;   // -1: no more work (the stage is left full)
        const Tile t = decode_tile<TY, W>(plan, item);
        if (!t.ok) {           // one empty plane was sent for an inactive board
            fph ^= 1u << sq;
            __syncwarp();
            if (lx == 0) mbar_arrive(&empty[sq]);
            sq = sq + 1 == NS ? 0 : sq + 1;
            continue;
        }
        const Board *__restrict__ B = t.B;
        const int par = t.par, i0 = t.i0, j0 = t.j0, kb = t.kb, ke = t.ke, kstart = t.kstart;
        const int ix0 = B->ix0, ix1 = B->ix1, iy0 = B->iy0, iy1 = B->iy1, iz0 = B->iz0, iz1 = B->iz1;
        const int X = B->pitch;
        const long long P = B->plane, NN = B->nodes;
        const float Sx = B->S[0], Sy = B->S[1], Sz = B->S[2];
        const int id16 = B->id16;
        const float4 *__restrict__ ctab = B->ctab;
        int *const status = B->status;
        const int c = i0 - 1 + 31 * wy + lx;                  // this lane's column
        const bool own_col = (lx > 0) && (c < ix1);
        const bool col_slab = (c < ix0);                      // only lane 0 of warp 0 can be outside
        const bool row_slab = (j0 - 1 < iy0);
        const int ecol = ((i0 - 1) & 7) + 31 * wy + lx;       // column in the E/H boxes
        const int ccol = (i0 - (id16 ? (i0 & ~7) : (i0 & ~15))) - 1 + 31 * wy + lx;   // in the id box
        // global element (c, j0-1, kstart) in the output parity, advanced by P per plane
        T *gp = (T *)B->f[par ^ 1][0] + ((long long)kstart * P + (long long)(j0 - 1) * X + c);
        const int zrow = B->zpitch;
        const long long zplane = (long long)(iy1 - iy0) * zrow;
        const long long zcol = (long long)(j0 - 1 - iy0) * zrow + (c - ix0);   // aux of (c, j0-1)
        int s0 = sq, s1 = sq + 1 == NS ? 0 : sq + 1;
        // z-UPML auxiliaries of this lane's column, fetched one plane ahead:
        // B~y, B~z for box rows 0..TY (halo row and the tile rows), D~y, D~z
        // for the tile rows
        struct Aux {
            float by[TY + 1], bz[TY + 1], dy[TY], dz[TY];
        };
        auto fetch_aux = [&](int k, Aux &a) {
            const int zb = k < iz0 ? 1 : (k >= iz1 ? 2 : 0);
            if (!zb) return;
            const long long base = (long long)(k - (zb == 1 ? 1 : iz1)) * zplane + zcol;
            const float *by = B->zB[zb - 1][0][par], *bz = B->zB[zb - 1][1][par];
            const float *dy = B->zD[zb - 1][0], *dz = B->zD[zb - 1][1];
            const bool cin = !col_slab && c < ix1;
#pragma unroll
            for (int rr = 0; rr <= TY; ++rr) {
                const int j = j0 - 1 + rr;
                if (cin && j >= iy0 && j < iy1) {
                    const long long x = base + (long long)rr * zrow;
                    a.by[rr] = __ldg(by + x);
                    a.bz[rr] = __ldg(bz + x);
                    if (rr > 0 && lx > 0) { a.dy[rr - 1] = dy[x]; a.dz[rr - 1] = dz[x]; }
                }
            }
        };
        Aux ax, axn;
        fetch_aux(kstart, ax);

        float hk1x[TY], hk1y[TY];   // H~x, H~y of the previous plane, per row
#pragma unroll
        for (int r = 0; r < TY; ++r) { hk1x[r] = 0.f; hk1y[r] = 0.f; }
        if (kstart == kb) {        // plane kb-1 is an outer z plane: read its H~
#pragma unroll
            for (int r = 0; r < TY; ++r)
                if (own_col && j0 + r < iy1) {
                    const T *g = gp - P + (long long)(r + 1) * X;
                    hk1x[r] = Io<T>::ld(g + 3 * NN);
                    hk1y[r] = Io<T>::ld(g + 4 * NN);
                }
        }
        fph ^= 1u << s0;     // the item's first plane was waited for above
        (void)status;
        for (int k = kstart; k < ke; ++k, gp += P) {
            if (k + 1 < ke) fetch_aux(k + 1, axn);
            mbar_wait(&full[s1], (fph >> s1) & 1u, status, abort_flag);
            fph ^= 1u << s1;
            const unsigned char *st0 = smem + s0 * St::BYTES, *st1 = smem + s1 * St::BYTES;
            const T *E0 = reinterpret_cast<const T *>(st0 + St::E_OFF) + ecol;
            const T *E1 = reinterpret_cast<const T *>(st1 + St::E_OFF) + ecol;
            const T *H0 = reinterpret_cast<const T *>(st0 + St::H_OFF) + ecol;
            const unsigned char *C0 = st0 + St::C_OFF;
            constexpr int EW = St::EW, HW = St::HW, ECS = St::E_CS, HCS = St::H_CS;
            const int zb = k < iz0 ? 1 : (k >= iz1 ? 2 : 0);
            ZCoef z;
            float *zdy = nullptr, *zdz = nullptr, *nzby = nullptr, *nzbz = nullptr;
            long long za = 0;
            if (zb) {
                z.zi = B->cw[2][0][k];
                z.zh = B->cw[2][1][k];
                za = (long long)(k - (zb == 1 ? 1 : iz1)) * zplane + zcol;
                nzby = B->zB[zb - 1][0][par ^ 1]; nzbz = B->zB[zb - 1][1][par ^ 1];
                zdy = B->zD[zb - 1][0]; zdz = B->zD[zb - 1][1];
            }
            const bool full_plane = k >= kb;
            // H~^{n+1/2}(k) at (c, j0-1+rr) from box row rr; Bo/Bn: B~y, B~z
            auto hnode = [&](int rr, bool in_f, float &hx, float &hy, float &hz, float &nby, float &nbz) {
                const float ezr = cvt<T>(E0[2 * ECS + rr * EW]), ezu = cvt<T>(E0[2 * ECS + (rr + 1) * EW]);
                const float eyr = cvt<T>(E0[ECS + rr * EW]), eyk = cvt<T>(E1[ECS + rr * EW]);
                const float exr = cvt<T>(E0[rr * EW]), exk = cvt<T>(E1[rr * EW]), exu = cvt<T>(E0[(rr + 1) * EW]);
                const float ezx = cvt<T>(E0[2 * ECS + rr * EW + 1]), eyx = cvt<T>(E0[ECS + rr * EW + 1]);
                const float scx = curl2(ezu, ezr, eyk, eyr, Sy, Sz);
                const float scy = curl2(exk, exr, ezx, ezr, Sz, Sx);
                const float scz = curl2(eyx, eyr, exu, exr, Sx, Sy);
                const float Boy = (zb && in_f) ? ax.by[rr] : 0.f;
                const float Boz = (zb && in_f) ? ax.bz[rr] : 0.f;
                hx = fused_hx(cvt<T>(H0[rr * HW]), scx, zb, z);
                hy = fused_hy(cvt<T>(H0[HCS + rr * HW]), scy, zb, z, Boy, nby);
                hz = fused_hz(cvt<T>(H0[2 * HCS + rr * HW]), scz, zb, z, Boz, nbz);
            };

            float4 ce[TY];   // coefficient rows of the lane's nodes, fetched first
#pragma unroll
            for (int r = 0; r < TY; ++r) {
                ce[r] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (full_plane && own_col && j0 + r < iy1) {
                    const int id = id16 ? (int)reinterpret_cast<const uint16_t *>(C0)[r * St::C16W + ccol]
                                        : (int)C0[r * St::C8W + ccol];
                    ce[r] = __ldg(ctab + id);
                }
            }
            float px = 0.f, py = 0.f, pz = 0.f;   // H~ at (c, j-1)
            if (full_plane) {
                float d0, d1;
                if (row_slab || col_slab) {
                    const T *g = gp;
                    px = Io<T>::ld(g + 3 * NN); py = Io<T>::ld(g + 4 * NN); pz = Io<T>::ld(g + 5 * NN);
                } else {
                    hnode(0, true, px, py, pz, d0, d1);
                }
            }
#pragma unroll
            for (int r = 0; r < TY; ++r) {
                const int j = j0 + r;
                float hx, hy, hz, nby = 0.f, nbz = 0.f;
                if (col_slab) {
                    const T *g = gp + (long long)(r + 1) * X;
                    hx = Io<T>::ld(g + 3 * NN); hy = Io<T>::ld(g + 4 * NN); hz = Io<T>::ld(g + 5 * NN);
                } else {
                    hnode(r + 1, j < iy1, hx, hy, hz, nby, nbz);
                }
                const float hyl = __shfl_up_sync(0xffffffffu, hy, 1);   // H~ at (c-1, j)
                const float hzl = __shfl_up_sync(0xffffffffu, hz, 1);
                if (full_plane && own_col && j < iy1) {
                    const int rr = r + 1;
                    const float4 cr = ce[r];
                    const float scx = curl2(hz, pz, hy, hk1y[r], Sy, Sz);
                    const float scy = curl2(hx, hk1x[r], hz, hzl, Sz, Sx);
                    const float scz = curl2(hy, hyl, hx, px, Sx, Sy);
                    const float exo = cvt<T>(E0[rr * EW]), eyo = cvt<T>(E0[ECS + rr * EW]), ezo = cvt<T>(E0[2 * ECS + rr * EW]);
                    float exv, eyv, ezv;
                    T *o = gp + (long long)rr * X;
                    if (!zb) {
                        exv = __fmaf_rn(cr.x, scx, exo);
                        eyv = __fmaf_rn(cr.y, scy, eyo);
                        ezv = __fmaf_rn(cr.z, scz, ezo);
                    } else {
                        const long long a = za + (long long)rr * zrow;
                        float nd, ndy, ndz;
                        exv = upml_e2(exo, scx, cr.x, kOne, z.zi, kOne, false, 0.f, nd);
                        eyv = upml_e2(eyo, scy, cr.y, z.zi, kOne, kOne, true, ax.dy[r], ndy);
                        ezv = upml_e2(ezo, scz, cr.z, kOne, kOne, z.zh, true, ax.dz[r], ndz);
                        zdy[a] = ndy;
                        zdz[a] = ndz;
                        nzby[a] = nby;
                        nzbz[a] = nbz;
                    }
                    Io<T>::st(o + 3 * NN, hx);
                    Io<T>::st(o + 4 * NN, hy);
                    Io<T>::st(o + 5 * NN, hz);
                    Io<T>::st(o, exv);
                    Io<T>::st(o + NN, eyv);
                    Io<T>::st(o + 2 * NN, ezv);
                }
                hk1x[r] = hx;
                hk1y[r] = hy;
                px = hx; py = hy; pz = hz;
            }
            (void)py;
            ax = axn;
            __syncwarp();
            if (lx == 0) mbar_arrive(&empty[s0]);
            s0 = s1;
            s1 = s1 + 1 == NS ? 0 : s1 + 1;
        }
        __syncwarp();
        if (lx == 0) mbar_arrive(&empty[s0]);   // the E-only plane above the segment
        sq = s1;
    }
}

// ------------------------------------------------------------------ slabs
struct SlabPos {
    const Slab *sl;
    long long t;          // slab-local index (aux index)
    int i, j, k;
};

__device__ __forceinline__ bool slab_locate(const Plan &plan, long long blk, const Board *&B, SlabPos &sp)
{
    const int b = find_board(plan.slab_prefix, plan.nb, blk);
    B = plan.boards[b];
    if (!board_active(B)) return false;
    const int lb = (int)(blk - __ldg(plan.slab_prefix + b));
    int s = 0;
    while (s + 1 < B->n_slab && B->slab[s + 1].block0 <= lb) ++s;
    const Slab *sl = &B->slab[s];
    const long long t = (long long)(lb - sl->block0) * kSlabThreads + threadIdx.x;
    if (t >= sl->n) return false;
    sp.sl = sl;
    sp.t = t;
    sp.i = sl->i0 + (int)(t % sl->ni);
    const long long r = t / sl->ni;
    sp.j = sl->j0 + (int)(r % sl->nj);
    sp.k = sl->k0 + (int)(r / sl->nj);
    return true;
}

// Gedney two-step update of one H~ component (B~ recurrence along w+1, H~
// recurrence along w+2, B~->H~ along w).  scurl = S * (curl E)_w.
__device__ __forceinline__ float upml_h(float h, float scurl, const Coef &a, const Coef &bb, const Coef &c,
                                        float *aux, long long t)
{
    if (aux) {
        const float Bo = aux[t];
        const float Bn = __fmaf_rn(-a.g, scurl, __fmul_rn(a.b1, Bo));
        aux[t] = Bn;
        return __fmaf_rn(bb.g, __fmaf_rn(c.ap, Bn, -__fmul_rn(c.am, Bo)), __fmul_rn(bb.b1, h));
    }
    return __fmaf_rn(-bb.g, scurl, __fmul_rn(bb.b1, h));
}

// Same for E (D~ recurrence along w+1, E recurrence along w+2, D~->E along
// w); ce = 1/eps_r of the edge (0 on PEC).
__device__ __forceinline__ float upml_e(float e, float scurl, float ce, const Coef &a, const Coef &bb,
                                        const Coef &c, float *aux, long long t)
{
    if (aux) {
        const float Do = aux[t];
        const float Dn = __fmaf_rn(a.g, scurl, __fmul_rn(a.b1, Do));
        aux[t] = Dn;
        return __fmaf_rn(__fmul_rn(ce, bb.g), __fmaf_rn(c.ap, Dn, -__fmul_rn(c.am, Do)), __fmul_rn(bb.b1, e));
    }
    return __fmaf_rn(__fmul_rn(ce, bb.g), scurl, __fmul_rn(bb.b1, e));
}

template <typename T>
__global__ void __launch_bounds__(kSlabThreads) k_slab_h(Plan plan)
{
    for (long long blk = blockIdx.x; blk < plan.n_slab; blk += gridDim.x) {
        const Board *B;
        SlabPos sp;
        if (!slab_locate(plan, blk, B, sp)) continue;
        const long long step = *((volatile long long *)B->step);
        const Fields<T> F(B, (int)(step & 1));
        const int i = sp.i, j = sp.j, k = sp.k;
        const int X = B->pitch;
        const long long P = B->plane;
        const long long idx = (long long)k * P + (long long)j * X + i;
        const float Sx = B->S[0], Sy = B->S[1], Sz = B->S[2];
        const Slab &sl = *sp.sl;
        if (j < B->ny && k < B->nz) {   // H_x(i, j+1/2, k+1/2)
            const float sc = curl2(Io<T>::ld(F.ez + idx + X), Io<T>::ld(F.ez + idx),
                                   Io<T>::ld(F.ey + idx + P), Io<T>::ld(F.ey + idx), Sy, Sz);
            const float h = upml_h(Io<T>::ld(F.hx + idx), sc, B->cw[1][1][j], B->cw[2][1][k], B->cw[0][0][i],
                                   sl.aux[3], sp.t);
            Io<T>::st(F.ohx + idx, h);
        }
        if (i < B->nx && k < B->nz) {   // H_y(i+1/2, j, k+1/2)
            const float sc = curl2(Io<T>::ld(F.ex + idx + P), Io<T>::ld(F.ex + idx),
                                   Io<T>::ld(F.ez + idx + 1), Io<T>::ld(F.ez + idx), Sz, Sx);
            const float h = upml_h(Io<T>::ld(F.hy + idx), sc, B->cw[2][1][k], B->cw[0][1][i], B->cw[1][0][j],
                                   sl.aux[4], sp.t);
            Io<T>::st(F.ohy + idx, h);
        }
        if (i < B->nx && j < B->ny) {   // H_z(i+1/2, j+1/2, k)
            const float sc = curl2(Io<T>::ld(F.ey + idx + 1), Io<T>::ld(F.ey + idx),
                                   Io<T>::ld(F.ex + idx + X), Io<T>::ld(F.ex + idx), Sx, Sy);
            const float h = upml_h(Io<T>::ld(F.hz + idx), sc, B->cw[0][1][i], B->cw[1][1][j], B->cw[2][0][k],
                                   sl.aux[5], sp.t);
            Io<T>::st(F.ohz + idx, h);
        }
    }
}

// H~^{n+1/2} at `in` or, when `outside` the grid, its image across the wall:
// PMC mirrors tangential H with a sign change, PEC gives 0.
template <typename T>
__device__ __forceinline__ float hwall(const T *h, bool outside, int wall, long long in, long long mirror)
{
    if (!outside) return Io<T>::ld(h + in);
    return wall == 1 ? -Io<T>::ld(h + mirror) : 0.0f;
}

template <typename T>
__global__ void __launch_bounds__(kSlabThreads) k_slab_e(Plan plan)
{
    for (long long blk = blockIdx.x; blk < plan.n_slab; blk += gridDim.x) {
        const Board *B;
        SlabPos sp;
        if (!slab_locate(plan, blk, B, sp)) continue;
        const long long step = *((volatile long long *)B->step);
        const Fields<T> F(B, (int)(step & 1));
        const int i = sp.i, j = sp.j, k = sp.k;
        const int nx = B->nx, ny = B->ny, nz = B->nz;
        const int X = B->pitch;
        const long long P = B->plane;
        const long long idx = (long long)k * P + (long long)j * X + i;
        const float Sx = B->S[0], Sy = B->S[1], Sz = B->S[2];
        const Slab &sl = *sp.sl;
        const float4 ce = __ldg(B->ctab + cid_at(B, idx));
        const int *w = B->wall;
        if (i < nx) {   // E_x(i+1/2, j, k)
            const float hz1 = hwall(F.ohz, j == ny, w[3], idx, idx - X);
            const float hz0 = hwall(F.ohz, j == 0, w[2], idx - X, idx);
            const float hy1 = hwall(F.ohy, k == nz, w[5], idx, idx - P);
            const float hy0 = hwall(F.ohy, k == 0, w[4], idx - P, idx);
            const float sc = curl2(hz1, hz0, hy1, hy0, Sy, Sz);
            const float e = upml_e(Io<T>::ld(F.ex + idx), sc, ce.x, B->cw[1][0][j], B->cw[2][0][k], B->cw[0][1][i],
                                   sl.aux[0], sp.t);
            Io<T>::st(F.oex + idx, e);
        }
        if (j < ny) {   // E_y(i, j+1/2, k)
            const float hx1 = hwall(F.ohx, k == nz, w[5], idx, idx - P);
            const float hx0 = hwall(F.ohx, k == 0, w[4], idx - P, idx);
            const float hz1 = hwall(F.ohz, i == nx, w[1], idx, idx - 1);
            const float hz0 = hwall(F.ohz, i == 0, w[0], idx - 1, idx);
            const float sc = curl2(hx1, hx0, hz1, hz0, Sz, Sx);
            const float e = upml_e(Io<T>::ld(F.ey + idx), sc, ce.y, B->cw[2][0][k], B->cw[0][0][i], B->cw[1][1][j],
                                   sl.aux[1], sp.t);
            Io<T>::st(F.oey + idx, e);
        }
        if (k < nz) {   // E_z(i, j, k+1/2)
            const float hy1 = hwall(F.ohy, i == nx, w[1], idx, idx - 1);
            const float hy0 = hwall(F.ohy, i == 0, w[0], idx - 1, idx);
            const float hx1 = hwall(F.ohx, j == ny, w[3], idx, idx - X);
            const float hx0 = hwall(F.ohx, j == 0, w[2], idx - X, idx);
            const float sc = curl2(hy1, hy0, hx1, hx0, Sx, Sy);
            const float e = upml_e(Io<T>::ld(F.ez + idx), sc, ce.z, B->cw[0][0][i], B->cw[1][0][j], B->cw[2][1][k],
                                   sl.aux[2], sp.t);
            Io<T>::st(F.oez + idx, e);
        }
    }
}

// ------------------------------------------------------------------ sources, probes
template <typename T>
__global__ void k_post(Plan plan)
{
    const int b = blockIdx.x;
    if (b >= plan.nb) return;
    Board *B = plan.boards[b];
    if (!board_active(B)) return;
    const long long step = *((volatile long long *)B->step);
    const int out = (int)(step & 1) ^ 1;
    if (threadIdx.x == 0) {
        const double t = ((double)step + 0.5) * B->dt;
        for (int s = 0; s < B->n_src; ++s) {
            const Source &S = B->src[s];
            const double u = (t - S.t0) / S.tau;
            const double J = S.J0 * u * exp(-u * u);
            T *e = (T *)B->f[out][S.comp] + S.node;
            Io<T>::st(e, __fsub_rn(Io<T>::ldw(e), (float)(S.coef * J)));
        }
    }
    __syncthreads();
    const bool rec = step < (long long)B->n_total;
    for (int p = threadIdx.x; p < B->n_probe; p += blockDim.x) {
        const Probe &Q = B->probe[p];
        const float v = Io<T>::ldw((const T *)B->f[out][Q.comp] + Q.node) * B->scale;
        if (rec) B->trace[(long long)p * B->n_total + step] = v;
        if (!isfinite(v)) atomicOr(B->status, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) *((volatile long long *)B->step) = step + 1;
}

// ------------------------------------------------------------------ running DFT
// One warp per (board, bin q, group of kDftProbeGroup probes): lanes stride
// the new samples, each forms exp(-j 2 pi ((q n) mod N) / N) in FP64, and the
// partial sums meet by warp shuffles.
__global__ void __launch_bounds__(256) k_dft(Plan plan)
{
    const int lane = threadIdx.x & 31;
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < plan.n_dft; w += nwarps) {
        const int b = find_board(plan.dft_prefix, plan.nb, w);
        const Board *B = plan.boards[b];
        const long long local = w - __ldg(plan.dft_prefix + b);
        const int groups = (B->n_probe + kDftProbeGroup - 1) / kDftProbeGroup;
        const int q = (int)(local / groups);
        const int g = (int)(local % groups);
        const long long N = B->n_total;
        const long long n0 = *((volatile long long *)B->dft_done);
        const long long n1 = min(*((volatile long long *)B->step), N);
        if (n1 <= n0) continue;
        double re[kDftProbeGroup], im[kDftProbeGroup];
#pragma unroll
        for (int u = 0; u < kDftProbeGroup; ++u) re[u] = im[u] = 0.0;
        for (long long n = n0 + lane; n < n1; n += 32) {
            const long long r = ((long long)q * n) % N;
            double s, c;
            sincospi(-2.0 * (double)r / (double)N, &s, &c);
#pragma unroll
            for (int u = 0; u < kDftProbeGroup; ++u) {
                const int p = g * kDftProbeGroup + u;
                if (p < B->n_probe) {
                    const double x = (double)B->trace[(long long)p * N + n];
                    re[u] = fma(x, c, re[u]);
                    im[u] = fma(x, s, im[u]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kDftProbeGroup; ++u) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                re[u] += __shfl_down_sync(0xffffffffu, re[u], off);
                im[u] += __shfl_down_sync(0xffffffffu, im[u], off);
            }
        }
        if (lane == 0) {
            for (int u = 0; u < kDftProbeGroup; ++u) {
                const int p = g * kDftProbeGroup + u;
                if (p < B->n_probe) {
                    double *d = B->dft + ((long long)p * B->n_bins + q) * 2;
                    d[0] += B->dt * re[u];
                    d[1] += B->dt * im[u];
                }
            }
        }
    }
}

__global__ void k_dft_commit(Plan plan)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= plan.nb) return;
    Board *B = plan.boards[b];
    const long long s = *((volatile long long *)B->step);
    *B->dft_done = s < (long long)B->n_total ? s : (long long)B->n_total;
}

__global__ void k_set_i64(long long *p, long long v) { *p = v; }

// ------------------------------------------------------------------ diagnostics
// Discrete energy of the last step (FP64) and max |sum_w S_w dH~_w| over cells
// outside the UPML; one partial pair per block, reduced by k_energy_final.
template <typename T>
__global__ void __launch_bounds__(256) k_energy(const Board *B, double *partials)
{
    const long long step = *((volatile long long *)B->step);
    const int pin = (int)((step - 1) & 1), pout = (int)(step & 1);
    const int nx = B->nx, ny = B->ny, nz = B->nz, X = B->pitch;
    const long long P = B->plane;
    const long long total = (long long)(nx + 1) * (ny + 1) * (nz + 1);
    const T *E[3] = {(const T *)B->f[pin][0], (const T *)B->f[pin][1], (const T *)B->f[pin][2]};
    const T *H0[3] = {(const T *)B->f[pin][3], (const T *)B->f[pin][4], (const T *)B->f[pin][5]};
    const T *H1[3] = {(const T *)B->f[pout][3], (const T *)B->f[pout][4], (const T *)B->f[pout][5]};
    // cells outside the UPML: [d_lo, n - d_hi) per axis
    const int cx0 = B->depth[0], cx1 = nx - B->depth[1];
    const int cy0 = B->depth[2], cy1 = ny - B->depth[3];
    const int cz0 = B->depth[4], cz1 = nz - B->depth[5];
    double wsum = 0.0, dmax = 0.0;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % (nx + 1));
        const long long r = t / (nx + 1);
        const int j = (int)(r % (ny + 1));
        const int k = (int)(r / (ny + 1));
        const long long idx = (long long)k * P + (long long)j * X + i;
        const float4 ce = B->ctab[cid_at(B, idx)];
        const double hx = (i == 0 || i == nx) ? 0.5 : 1.0;
        const double hy = (j == 0 || j == ny) ? 0.5 : 1.0;
        const double hz = (k == 0 || k == nz) ? 0.5 : 1.0;
        if (i < nx && ce.x != 0.0f) { const double e = Io<T>::ldw(E[0] + idx); wsum += hy * hz * e * e / ce.x; }
        if (j < ny && ce.y != 0.0f) { const double e = Io<T>::ldw(E[1] + idx); wsum += hx * hz * e * e / ce.y; }
        if (k < nz && ce.z != 0.0f) { const double e = Io<T>::ldw(E[2] + idx); wsum += hx * hy * e * e / ce.z; }
        if (j < ny && k < nz) wsum += hx * (double)Io<T>::ldw(H0[0] + idx) * Io<T>::ldw(H1[0] + idx);
        if (i < nx && k < nz) wsum += hy * (double)Io<T>::ldw(H0[1] + idx) * Io<T>::ldw(H1[1] + idx);
        if (i < nx && j < ny) wsum += hz * (double)Io<T>::ldw(H0[2] + idx) * Io<T>::ldw(H1[2] + idx);
        if (i >= cx0 && i < cx1 && j >= cy0 && j < cy1 && k >= cz0 && k < cz1) {
            const double dv = (double)B->S[0] * ((double)Io<T>::ldw(H1[0] + idx + 1) - Io<T>::ldw(H1[0] + idx))
                            + (double)B->S[1] * ((double)Io<T>::ldw(H1[1] + idx + X) - Io<T>::ldw(H1[1] + idx))
                            + (double)B->S[2] * ((double)Io<T>::ldw(H1[2] + idx + P) - Io<T>::ldw(H1[2] + idx));
            dmax = fmax(dmax, fabs(dv));
        }
    }
    __shared__ double sw[256], sd[256];
    sw[threadIdx.x] = wsum;
    sd[threadIdx.x] = dmax;
    __syncthreads();
    for (int off = blockDim.x >> 1; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) {
            sw[threadIdx.x] += sw[threadIdx.x + off];
            sd[threadIdx.x] = fmax(sd[threadIdx.x], sd[threadIdx.x + off]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = sw[0];
        partials[2 * blockIdx.x + 1] = sd[0];
    }
}

__global__ void k_energy_final(const double *partials, int n, double *out2)
{
    __shared__ double sw[256], sd[256];
    double a = 0.0, m = 0.0;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        a += partials[2 * t];
        m = fmax(m, partials[2 * t + 1]);
    }
    sw[threadIdx.x] = a;
    sd[threadIdx.x] = m;
    __syncthreads();
    for (int off = blockDim.x >> 1; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) {
            sw[threadIdx.x] += sw[threadIdx.x + off];
            sd[threadIdx.x] = fmax(sd[threadIdx.x], sd[threadIdx.x + off]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out2[0] = sw[0];
        out2[1] = sd[0];
    }
}

// ------------------------------------------------------------------ launchers
// Fused-kernel configurations: W compute warps x 31 columns by TY rows.
template <int TY, int W>
struct FusedTune {
    static constexpr int NS = 4;
};

template <typename T, int TY, int W>
struct FusedCfg {
    static constexpr int NS = FusedTune<TY, W>::NS;
    using L = FusedLayout<T, TY, W, NS>;
    static dim3 block() { return dim3(32, W + 1); }
    static int grid()
    {
        static int g = 0;
        if (!g) {
            int dev = 0, sms = 0, per = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fused<T, TY, W, NS>, 32 * (W + 1), L::BYTES);
            g = (sms > 0 ? sms : 152) * (per > 0 ? per : 1);
        }
        return g;
    }
    static cudaError_t set_limit()
    {
        return cudaFuncSetAttribute(k_fused<T, TY, W, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, L::BYTES);
    }
    static void launch(const Plan &plan, cudaStream_t st)
    {
        const int g = (int)(plan.n_int < grid() ? plan.n_int : grid());
        cudaMemsetAsync(plan.work, 0, sizeof(int), st);
        k_fused<T, TY, W, NS><<<g, block(), L::BYTES, st>>>(plan);
    }
};

// Supported fused tiles (tile_x columns x tile_y rows): 62x4, 62x8, 124x4, 124x8.
template <typename T>
static void launch_fused(const Plan &plan, cudaStream_t st)
{
    const int key = plan.tile_x * 16 + plan.tile_y;
    switch (key) {
    case 62 * 16 + 4: FusedCfg<T, 4, 2>::launch(plan, st); break;
    case 62 * 16 + 8: FusedCfg<T, 8, 2>::launch(plan, st); break;
    case 124 * 16 + 8: FusedCfg<T, 8, 4>::launch(plan, st); break;
    default: FusedCfg<T, 4, 4>::launch(plan, st); break;
    }
}

template <typename T>
static cudaError_t phase_t(const Plan &plan, int phase, int grid_cap, cudaStream_t st)
{
    switch (phase) {
    case kPhaseSlabH:
        if (plan.n_slab > 0)
            k_slab_h<T><<<(int)(plan.n_slab < grid_cap ? plan.n_slab : grid_cap), kSlabThreads, 0, st>>>(plan);
        break;
    case kPhaseInterior:
        if (plan.n_int > 0) launch_fused<T>(plan, st);
        break;
    case kPhaseSlabE:
        if (plan.n_slab > 0)
            k_slab_e<T><<<(int)(plan.n_slab < grid_cap ? plan.n_slab : grid_cap), kSlabThreads, 0, st>>>(plan);
        break;
    default:
        k_post<T><<<plan.nb, 128, 0, st>>>(plan);
        break;
    }
    return cudaGetLastError();
}

cudaError_t launch_phase(const Plan &plan, int prec, int phase, int grid_cap, cudaStream_t st)
{
    switch (prec) {
    case kFP16: return phase_t<__half>(plan, phase, grid_cap, st);
    case kBF16: return phase_t<__nv_bfloat16>(plan, phase, grid_cap, st);
    default: return phase_t<float>(plan, phase, grid_cap, st);
    }
}

cudaError_t launch_step(const Plan &plan, int prec, int grid_cap, cudaStream_t st)
{
    for (int ph = 0; ph < kNumPhases; ++ph) {
        cudaError_t e = launch_phase(plan, prec, ph, grid_cap, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

bool fused_tile_supported(int tx, int ty) { return (tx == 62 || tx == 124) && (ty == 4 || ty == 8); }

template <typename T>
static cudaError_t limits_t()
{
    cudaError_t e[4] = {FusedCfg<T, 4, 2>::set_limit(), FusedCfg<T, 8, 2>::set_limit(), FusedCfg<T, 4, 4>::set_limit(),
                        FusedCfg<T, 8, 4>::set_limit()};
    for (cudaError_t x : e)
        if (x != cudaSuccess) return x;
    return cudaSuccess;
}

cudaError_t fused_set_smem_limits()
{
    cudaError_t a = limits_t<float>(), b = limits_t<__half>(), c = limits_t<__nv_bfloat16>();
    return a != cudaSuccess ? a : (b != cudaSuccess ? b : c);
}

cudaError_t launch_dft(const Plan &plan, int grid_cap, cudaStream_t st)
{
    if (plan.n_dft > 0) {
        long long blocks = (plan.n_dft + 7) / 8;
        if (blocks > grid_cap) blocks = grid_cap;
        k_dft<<<(int)blocks, 256, 0, st>>>(plan);
    }
    k_dft_commit<<<(plan.nb + 127) / 128, 128, 0, st>>>(plan);
    return cudaGetLastError();
}

cudaError_t launch_set_i64(long long *p, long long v, cudaStream_t st)
{
    k_set_i64<<<1, 1, 0, st>>>(p, v);
    return cudaGetLastError();
}

int energy_partials(const Board &b)
{
    const long long total = (long long)(b.nx + 1) * (b.ny + 1) * (b.nz + 1);
    long long blocks = (total + 255) / 256;
    return (int)(blocks < 1024 ? blocks : 1024);
}

cudaError_t launch_energy(const Board *b_dev, const Board &b_host, double *partials, int n_part, double *out2,
                          cudaStream_t st)
{
    switch (b_host.prec) {
    case kFP16: k_energy<__half><<<n_part, 256, 0, st>>>(b_dev, partials); break;
    case kBF16: k_energy<__nv_bfloat16><<<n_part, 256, 0, st>>>(b_dev, partials); break;
    default: k_energy<float><<<n_part, 256, 0, st>>>(b_dev, partials); break;
    }
    k_energy_final<<<1, 256, 0, st>>>(partials, n_part, out2);
    return cudaGetLastError();
}

}  // namespace fdtd
