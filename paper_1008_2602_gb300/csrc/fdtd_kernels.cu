// fdtd_kernels.cu -- sm_103a kernels of the Yee + UPML leapfrog step.
//
// One step (Model section: H at half steps from E, then E from H and J) is
// five launches over a Plan (one board or a batch of boards):
//   k_slab_h        H^{n+1/2} (and B~) on the x/y UPML slabs and the outer
//                   z planes                                        (Eqs. 1-5)
//   k_fused<..,1>   fused H^{n+1/2} and E^{n+1} on the interior columns'
//                   z-UPML planes (sigma_z only; B~z, D~z staged by TMA)
//   k_fused<..,0>   fused H^{n+1/2} and E^{n+1} on the interior columns'
//                   remaining planes (plain Yee, coefficient ids, TMA-fed)
//   k_slab_e        E^{n+1} (and D~) on the slab nodes, PEC/PMC outer walls
//   k_post          current sources (Eq. 8), resistive voltage sources
//                   (Results section) and probe samples of E^{n+1}
// and, once per chunk, k_dft folds the new probe samples into the FP64
// running DFT (Results section: spectrum of the ground-plane E_z) with warp
// shuffles.  Each step reads one field set and writes another (set_of), so no
// launch reads what it writes except the per-node UPML auxiliaries, which
// only their own thread touches.  With time blocking (depth 2) a pair of
// steps replaces the two interior launches by one two-step pass (k_pair) and
// lets the slab kernels finish the interior region's outer layer.
//
// All curl and update arithmetic goes through curl2()/the update helpers (or
// their paired FFMA2 forms) with explicit round-to-nearest intrinsics, so a
// value recomputed as a halo is bit-identical to the one its owner stores.
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

// The step counters as seen by the field kernels: written only by other
// launches (k_post, the host's stop updates), so within one launch they are
// read-only and every warp may read them through the cached read-only path
// (a per-warp L2 read of one shared line would serialise on that line).
__device__ __forceinline__ long long step_ro(const Board *B) { return __ldg(B->step); }
__device__ __forceinline__ bool active_ro(const Board *B) { return __ldg(B->step) < __ldg(B->stop); }

// Eq. 8 pulse of a source at the half step n + 1/2: J for a current source,
// Vs for a voltage source.
__device__ __forceinline__ double src_pulse(const Source &S, long long step, double dt)
{
    const double t = ((double)step + 0.5) * dt;
    const double u = (t - S.t0) / S.tau;
    return S.J0 * u * exp(-u * u);
}

// A source applied to the plainly updated edge value ep (as stored), given the
// edge's previous value en (as stored); returns the new value before storage
// rounding.  Current source: E -= coef J.  Resistive voltage source: the lumped
// current (l E^{n+1/2} + Vs) / Rs in Ampere's law turns the plain update
// E_p = E^n + ce S curl into E^{n+1} = (E_p - beta E^n - gam Vs) / (1 + beta).
__device__ __forceinline__ float src_apply(const Source &S, double w, float ep, float en)
{
    if (S.kind == kSrcCurrent) return __fsub_rn(ep, (float)(S.coef * w));
    return (float)(((double)ep - S.beta * (double)en - S.gam * w) / (1.0 + S.beta));
}

// Whether node (i, j, k) lies in the interior region I = [ix0,ix1) x [iy0,iy1) x [iz0,iz1).
__device__ __forceinline__ bool in_interior(const Board *B, int i, int j, int k)
{
    return i >= B->ix0 && i < B->ix1 && j >= B->iy0 && j < B->iy1 && k >= B->iz0 && k < B->iz1;
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
    Fields() = default;
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
    // no auxiliary: c is trivial and at most one of a, bb is graded, so the
    // products below are exact
    return __fmaf_rn(-__fmul_rn(a.g, bb.g), scurl, __fmul_rn(__fmul_rn(a.b1, bb.b1), h));
}

// Same for E (D~ along w+1, E along w+2, D~->E along w); ce = 1/eps_r.
__device__ __forceinline__ float upml_e2(float e, float scurl, float ce, const Coef &a, const Coef &bb, const Coef &c,
                                         bool aux, float Do, float &Dn)
{
    if (aux) {
        Dn = __fmaf_rn(a.g, scurl, __fmul_rn(a.b1, Do));
        return __fmaf_rn(__fmul_rn(ce, bb.g), __fmaf_rn(c.ap, Dn, -__fmul_rn(c.am, Do)), __fmul_rn(bb.b1, e));
    }
    // no auxiliary (see upml_h2)
    return __fmaf_rn(__fmul_rn(ce, __fmul_rn(a.g, bb.g)), scurl, __fmul_rn(__fmul_rn(a.b1, bb.b1), e));
}

__device__ __constant__ Coef kOne = {1.0f, 1.0f, 1.0f, 1.0f};

// z-UPML plane kinds of the fused region: 0 none, 1 lower box, 2 upper box.
__device__ __forceinline__ int zbox_of(const Board *B, int k) { return k < B->iz0 ? 1 : (k >= B->iz1 ? 2 : 0); }

__device__ __forceinline__ long long zaux_index(const Board *B, int box, int i, int j, int k)
{
    const int k0 = box == 1 ? B->zlo : B->iz1;
    return ((long long)(k - k0) * (B->iy1 - B->iy0) + (j - B->iy0)) * (long long)B->zpitch + (i - B->ix0);
}

// New H~x, H~y, H~z at a fused-region node from already-fetched operands.
// In z-UPML planes only sigma_z is non-zero: H~x and H~y update in the lossy
// form (no auxiliary), H~z carries B~z.
struct ZCoef {
    Coef zi, zh;   // z factors at the node's integer and half positions
};

__device__ __forceinline__ float fused_hx(float h, float sc, int zb, const ZCoef &z)
{
    float dummy;
    if (!zb) return __fsub_rn(h, sc);
    return upml_h2(h, sc, kOne, z.zh, kOne, false, 0.f, dummy);
}
__device__ __forceinline__ float fused_hy(float h, float sc, int zb, const ZCoef &z)
{
    float dummy;
    if (!zb) return __fsub_rn(h, sc);
    return upml_h2(h, sc, z.zh, kOne, kOne, false, 0.f, dummy);
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
__device__ __forceinline__ void mbar_wait(uint64_t *b, uint32_t parity, int *status, int *abort_flag,
                                          uint32_t max_polls = 1u << 21)
{
    if (*(volatile int *)abort_flag) return;
    for (uint32_t it = 0; it < max_polls; ++it)
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

// Two adjacent elements of one row (8-byte aligned for FP32, 4-byte for the
// 16-bit storage types), converted to/from FP32.
template <typename T>
struct Pair;
template <>
struct Pair<float> {
    static __device__ __forceinline__ float2 lds(const float *p) { return *reinterpret_cast<const float2 *>(p); }
    static __device__ __forceinline__ float2 ldg(const float *p) { return __ldg(reinterpret_cast<const float2 *>(p)); }
    static __device__ __forceinline__ void st(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }
};
template <>
struct Pair<__half> {
    static __device__ __forceinline__ float2 lds(const __half *p)
    {
        return __half22float2(*reinterpret_cast<const __half2 *>(p));
    }
    static __device__ __forceinline__ float2 ldg(const __half *p)
    {
        return __half22float2(__ldg(reinterpret_cast<const __half2 *>(p)));
    }
    static __device__ __forceinline__ void st(__half *p, float2 v) { *reinterpret_cast<__half2 *>(p) = __float22half2_rn(v); }
};

// Stores of the fused kernel.  Written as global-space stores without a
// compiler memory barrier, so the compiler knows they cannot alias the
// shared-memory stages and may hoist the next row's shared loads above them.
// (No value this kernel stores is read back by it.)
__device__ __forceinline__ size_t gaddr(const void *p) { return __cvta_generic_to_global(p); }
__device__ __forceinline__ void stg1(float *p, float v)
{
    asm volatile("st.global.f32 [%0], %1;" ::"l"(gaddr(p)), "f"(v));
}
__device__ __forceinline__ void stg1(__half *p, float v)
{
    const __half h = __float2half_rn(v);
    asm volatile("st.global.b16 [%0], %1;" ::"l"(gaddr(p)), "h"(*reinterpret_cast<const unsigned short *>(&h)));
}
__device__ __forceinline__ void stg2(float *p, float2 v)
{
    asm volatile("st.global.v2.f32 [%0], {%1, %2};" ::"l"(gaddr(p)), "f"(v.x), "f"(v.y));
}
__device__ __forceinline__ void stg2(__half *p, float2 v)
{
    const __half2 h = __float22half2_rn(v);
    asm volatile("st.global.b32 [%0], %1;" ::"l"(gaddr(p)), "r"(*reinterpret_cast<const unsigned int *>(&h)));
}

// Paired forms of curl2 and of h - s.  Per element they round exactly like
// the scalar forms: a - b == fma(b, -1, a) (the product is exact), and
// fma(-Sb, d, x) is the same single rounding either way.
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 curl2v(float2 a1, float2 a0, float2 b1, float2 b0, float2 Sa, float2 nSb)
{
    return __ffma2_rn(nSb, sub2(b1, b0), __fmul2_rn(Sa, sub2(a1, a0)));
}

// Columns owned by one compute warp: lane l holds the pair g + 2l, g + 2l + 1
// with g the even column at or just below the strip's low-x halo.  A tile of
// TY rows may be split into R row groups, one compute warp each, sharing the
// tile's stage (each group recomputes H~ on the row above it).
constexpr int kWarpCols = 62;

// Shared-memory stage of one plane for a tile of W warps x 62 columns by TY
// rows.  Boxes start at x rounded down to the 16-byte TMA boundary:
//   E  3 x (TY+2) x EW   rows j0-1 .. j0+TY
//   H  3 x (TY+1) x HW   rows j0-1 .. j0+TY-1
//   id TY x C8W bytes (or TY x C16W uint16), rows j0 .. j0+TY-1
//   z-UPML kernel only: B~z (TY+1) x AW and D~z TY x AW floats
// Every box starts 128-byte aligned.
template <typename T, int TY, int W, bool ZP>
struct Stage {
    static constexpr int al(int x) { return (x + 127) & ~127; }
    static constexpr int TX = kWarpCols * W;
    static constexpr int ES = (int)sizeof(T);
    static constexpr int EW = box_e(TX), HW = box_h(TX), C8W = box_c8(TX), C16W = box_c16(TX), AW = box_a(TX);
    static constexpr int E_COMP = (TY + 2) * EW, H_COMP = (TY + 1) * HW;
    static constexpr int E_CS = al(E_COMP * ES) / ES, H_CS = al(H_COMP * ES) / ES;
    static constexpr int E_BYTES = 3 * E_COMP * ES;
    static constexpr int H_BYTES = 3 * H_COMP * ES;
    static constexpr int C8_BYTES = TY * C8W, C16_BYTES = TY * C16W * 2;
    static constexpr int B_COMP = (TY + 1) * AW, D_COMP = TY * AW;
    static constexpr int B_CS = al(B_COMP * 4) / 4, D_CS = al(D_COMP * 4) / 4;
    static constexpr int A_BYTES = (B_COMP + D_COMP) * 4;
    static constexpr int E_OFF = 0;
    static constexpr int H_OFF = 3 * E_CS * ES;
    static constexpr int C_OFF = H_OFF + 3 * H_CS * ES;
    static constexpr int ITEM_OFF = (C_OFF + (C8_BYTES > C16_BYTES ? C8_BYTES : C16_BYTES) + 7) & ~7;   // item id
    static constexpr int A_OFF = al(ITEM_OFF + 8);
    static constexpr int BYTES = A_OFF + (ZP ? (B_CS + D_CS) * 4 : 0);
};

template <typename T, int TY, int W, int NS, bool ZP, int R>
struct FusedLayout {
    using St = Stage<T, TY, W, ZP>;
    static constexpr int BAR_OFF = NS * St::BYTES;
    static constexpr int BYTES = BAR_OFF + 2 * NS * 8 + 16;
    // blocks per SM that shared memory allows (227 KB usable per SM, 1 KB
    // reserved per block); the register budget keeps them resident but never
    // drops below a per-thread floor that the warp's row count sets: 176 for
    // 8 rows, 168 (z-UPML) or 128 for 4 rows, 136 (z-UPML) or 96 for 2 rows
    static constexpr int REG_FLOOR = TY / R >= 8 ? 176 : (TY / R >= 4 ? (ZP ? 168 : 128) : (ZP ? 136 : 96));
    static constexpr int PER_SM = 232448 / (BYTES + 1024);
    static constexpr int REG_SM = 65536 / (REG_FLOOR * (32 * W * R + 32));
    static constexpr int CAP = PER_SM < REG_SM ? PER_SM : REG_SM;
    static constexpr int MINB = CAP < 1 ? 1 : (CAP > 8 ? 8 : CAP);
};

__device__ __forceinline__ void mbar_arrive(uint64_t *b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_addr(b)) : "memory");
}

// Work item -> tile; identical in the producer and the consumer warps.
struct Tile {
    const Board *B;
    int ok;
    int i0, j0, kb, ke, kstart, par;   // par: step parity (B~z ping-pong)
    int in, out;                        // field sets read and written
};

// Items of one board: x tiles fastest, then y tiles within a band of rows,
// then z segments, then bands.  In the interior launch a band holds about as
// many tiles as the launch has resident blocks, so the next z segment of a
// tile starts about when the previous one ends, and the planes the two
// segments both stage (the segment's E-only plane above, the next one's
// recomputed plane below) are read while still in L2 (measured: interior
// launch 0.384 -> 0.374 ms on the 880x680x100 board, 2 bands of 41 tile rows;
// bands of 1.5, 0.5 or 0.25 waves were slower).  The z-UPML launch, whose layers split
// into a long and a short segment, keeps one band (x, then y, then z; banding
// it cost 2 %).  The interior kernel (ZP false) covers planes
// [iz0, iz1); the z-UPML kernel
// covers [zlo, iz0) and [max(iz1, iz0), nz).  kstart is the plane below the
// segment when the tile recomputes its H~ there, else kb (that plane's H~ is
// then read from the output: an outer plane, or a z-UPML plane written by the
// z-UPML launch, which runs first).
template <int TY, int W, bool ZP>
__device__ __forceinline__ Tile decode_tile(const Plan &plan, long long item)
{
    Tile t;
    const long long *prefix = ZP ? plan.zp_prefix : plan.int_prefix;
    const int b = find_board(prefix, plan.nb, item);
    t.B = plan.boards[b];
    // a board whose tensor maps were encoded for another tile is skipped (its
    // boxes would not fit this kernel's stages); the producer flags it
    t.ok = active_ro(t.B) && t.B->tm_tx == kWarpCols * W && t.B->tm_ty == TY;
    const long long step = step_ro(t.B);
    t.par = (int)(step & 1);
    const int depth = t.B->tdepth;
    t.in = set_of(depth, step);
    t.out = set_of(depth, step + 1);
    const long long local = item - __ldg(prefix + b);
    constexpr int TX = kWarpCols * W;
    const int ntx = (t.B->ix1 - t.B->ix0 + TX - 1) / TX, nty = (t.B->iy1 - t.B->iy0 + TY - 1) / TY;
    const int zs = plan.zseg, iz0 = t.B->iz0, iz1 = t.B->iz1;
    int nseg;
    if (!ZP) nseg = (iz1 - iz0 + zs - 1) / zs;
    else nseg = (iz0 - t.B->zlo + zs - 1) / zs + (t.B->nz - max(iz1, iz0) + zs - 1) / zs;
    // bands of about one wave of tiles, of equal height
    const int wave_rows = max(1, plan.slots / ntx), nband = (nty + wave_rows - 1) / wave_rows;
    const int band = ZP ? nty : (nty + nband - 1) / nband;
    const long long per_band = (long long)ntx * band * nseg;
    const int bi = (int)(local / per_band);
    const long long within = local - bi * per_band;
    const int rows = min(band, nty - bi * band);
    const long long layer = (long long)ntx * rows;
    const int tz = (int)(within / layer);
    const int rem = (int)(within - tz * layer);
    const int ty = bi * band + rem / ntx, tx = rem % ntx;
    t.i0 = t.B->ix0 + tx * TX;
    t.j0 = t.B->iy0 + ty * TY;
    if (!ZP) {
        t.kb = iz0 + tz * zs;
        t.ke = min(t.kb + zs, iz1);
        t.kstart = t.kb - 1 >= iz0 ? t.kb - 1 : t.kb;
    } else {
        // planes [zlo, iz0) and [max(iz1, iz0), nz); a segment starting at
        // plane 0 (zlo = 0) has no plane below, one starting at plane 1
        // (zlo = 1) reads the slab's wall plane below
        const int zlo = t.B->zlo;
        const int nlo = (iz0 - zlo + zs - 1) / zs;
        if (tz < nlo) {
            t.kb = zlo + tz * zs;
            t.ke = min(t.kb + zs, iz0);
        } else {
            t.kb = max(iz1, iz0) + (tz - nlo) * zs;
            t.ke = min(t.kb + zs, t.B->nz);
        }
        t.kstart = t.kb > zlo ? t.kb - 1 : t.kb;
    }
    return t;
}

// Fused H+E kernel over the fused region, fed by TMA, warp-specialised.
// Warps 0..W-1 compute; warp W (one lane) is the producer, streaming planes
// kstart..ke of the tile into an NS-stage ring (E^n with a one-node halo,
// H~^{n-1/2} with the low halo row and column, coefficient ids, and in the
// z-UPML kernel the B~z/D~z auxiliaries of z-UPML planes), each stage with a
// "full" mbarrier (TMA bytes) and an "empty" one (one arrival per compute
// warp).  Compute warp (w, row group) owns 62 columns [i0 + 62w, i0 + 62w + 62)
// of its rows; lane l
// holds the column pair (g + 2l, g + 2l + 1), g = (i0 + 62w - 1) & ~1, so
// one lane's loads and stores are 8 bytes and its arithmetic is paired FP32
// (FFMA2/FMUL2).  Per plane k a lane marches the tile's rows in y: it forms
// H~^{n+1/2}(k) at its two columns for the halo row j0-1 and then row by
// row, so H(j-1) is already in registers; H(i-1) of its first column comes
// from the lane to its left with a shuffle; then it updates E^{n+1}(k).  H~
// of halo nodes outside the fused region is read from the slab kernel's
// output instead.  The plane below the segment is run once for the tile's
// H~x, H~y there (or read, see decode_tile); the plane above is read for E
// only.  In z-UPML planes (sigma_z only) H~z carries B~z and E_z carries
// D~z, while H~x, H~y, E_x, E_y update in the lossy form; those planes use
// the scalar update helpers per element, every other plane the paired form.
template <typename T, int TY, int W, int NS, bool ZP, int R>
__global__ void __launch_bounds__(32 * W * R + 32, (FusedLayout<T, TY, W, NS, ZP, R>::MINB)) k_fused(Plan plan)
{
    using St = Stage<T, TY, W, ZP>;
    using L = FusedLayout<T, TY, W, NS, ZP, R>;
    constexpr int TYW = TY / R;   // rows of one compute warp
    static_assert(TY % R == 0, "row groups must split the tile evenly");
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + L::BAR_OFF);
    uint64_t *empty = full + NS;
    int *abort_flag = reinterpret_cast<int *>(empty + NS);
    const int lx = threadIdx.x, wy = threadIdx.y;

    if (wy == 0 && lx == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], W * R);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();

    if (wy == W * R) {
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
        const long long n_items = ZP ? plan.n_zp : plan.n_int;
        for (;;) {
            const long long item = atomicAdd(plan.work + (ZP ? 1 : 0), 1);
            if (item >= n_items) break;
            const Tile t = decode_tile<TY, W, ZP>(plan, item);
            const Board *B = t.B;
            if (!t.ok && (B->tm_tx != kWarpCols * W || B->tm_ty != TY)) atomicOr(B->status, 4);
            const CUtensorMap *tm = B->tm;
            const int id16 = B->id16;
            const int xe0 = (t.i0 - 1) & ~7;
            const int xc0 = id16 ? (t.i0 & ~7) : (t.i0 & ~15);
            const int xa0 = ((((t.i0 - 1) & ~1) - B->ix0)) & ~3;   // aux boxes: x relative to ix0
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
                const int zb = ZP && !e_only ? (p < B->iz0 ? 1 : (p >= B->iz1 ? 2 : 0)) : 0;
                uint32_t bytes = St::E_BYTES;
                if (!e_only) bytes += St::H_BYTES + (id16 ? St::C16_BYTES : St::C8_BYTES);
                if (zb) bytes += St::A_BYTES;
                mbar_expect_tx(&full[s], bytes);
                for (int c = 0; c < 3; ++c)
                    tma_load_3d(st + St::E_OFF + c * St::E_CS * St::ES, tm + tm_e(t.in, c), xe0, t.j0 - 1, p, &full[s]);
                if (!e_only) {
                    for (int c = 0; c < 3; ++c)
                        tma_load_3d(st + St::H_OFF + c * St::H_CS * St::ES, tm + tm_h(t.in, c), xe0, t.j0 - 1, p,
                                    &full[s]);
                    tma_load_3d(st + St::C_OFF, tm + kTmCid, xc0, t.j0, p, &full[s]);
                }
                if (zb) {
                    const int bx = zb - 1, kz = p - (zb == 1 ? B->zlo : B->iz1);
                    unsigned char *a = st + St::A_OFF;
                    tma_load_3d(a, tm + tm_zb(bx, t.par), xa0, t.j0 - 1 - B->iy0, kz, &full[s]);
                    tma_load_3d(a + St::B_CS * 4, tm + tm_zd(bx), xa0, t.j0 - B->iy0, kz, &full[s]);
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
        const Tile t = decode_tile<TY, W, ZP>(plan, item);
        if (!t.ok) {           // one empty plane was sent for an inactive board
            fph ^= 1u << sq;
            __syncwarp();
            if (lx == 0) mbar_arrive(&empty[sq]);
            sq = sq + 1 == NS ? 0 : sq + 1;
            continue;
        }
        const Board *__restrict__ B = t.B;
        const int par = t.par, i0 = t.i0, j0 = t.j0, kb = t.kb, ke = t.ke, kstart = t.kstart, oset = t.out;
        const int ix0 = B->ix0, ix1 = B->ix1, iy0 = B->iy0, iy1 = B->iy1, iz0 = B->iz0, iz1 = B->iz1;
        const int X = B->pitch;
        const long long P = B->plane, NN = B->nodes;
        const float2 Sx2 = make_float2(B->S[0], B->S[0]), Sy2 = make_float2(B->S[1], B->S[1]);
        const float2 Sz2 = make_float2(B->S[2], B->S[2]);
        const float2 nSx2 = make_float2(-B->S[0], -B->S[0]), nSy2 = make_float2(-B->S[1], -B->S[1]);
        const float2 nSz2 = make_float2(-B->S[2], -B->S[2]);
        const int id16 = B->id16;
        const float4 *__restrict__ ctab = B->ctab;
        int *const status = B->status;
        const int wx = wy % W, R0 = (wy / W) * TYW;        // column strip; first tile row of the warp
        const int jb = j0 + R0;                            // first grid row the warp owns
        const int wlo = i0 + kWarpCols * wx;               // first column the warp owns
        const int whi = min(wlo + kWarpCols, ix1);
        const int g = (wlo - 1) & ~1;
        const int ca = g + 2 * lx, cb = ca + 1;            // this lane's columns
        const bool own_a = ca >= wlo && ca < whi, own_b = cb >= wlo && cb < whi;
        const bool slab_a = ca < ix0, slab_b = cb < ix0;  // halo column outside the fused region
        const int ecol = (g - ((i0 - 1) & ~7)) + 2 * lx;   // column of ca in the E/H boxes (even)
        const int xc0 = id16 ? (i0 & ~7) : (i0 & ~15);
        const int ida = max(ca - xc0, 0), idb = cb - xc0;  // columns in the id box (clamped into it)
        const bool row_slab = (jb - 1 < iy0);
        // element (ca, jb-1, kstart) of component 0 in the output set, advanced by P per plane
        T *gp = (T *)B->f[oset][0] + ((long long)kstart * P + (long long)(jb - 1) * X + ca);
        const int zrow = B->zpitch;
        const long long zplane = (long long)(iy1 - iy0) * zrow;
        const long long zcol = (long long)(jb - iy0) * zrow + (ca - ix0);   // aux index of (ca, jb) in a plane
        const int acol = (ca - ix0) - ((((i0 - 1) & ~1) - ix0) & ~3);       // column of ca in the aux boxes
        int s0 = sq, s1 = sq + 1 == NS ? 0 : sq + 1;

        float2 hk1x[TYW], hk1y[TYW];   // H~x, H~y of the previous plane, per row
#pragma unroll
        for (int r = 0; r < TYW; ++r) { hk1x[r] = make_float2(0.f, 0.f); hk1y[r] = make_float2(0.f, 0.f); }
        if (kstart == kb && kb > 0) {   // plane kb-1 is not recomputed: read its H~ (none below plane 0)
#pragma unroll
            for (int r = 0; r < TYW; ++r)
                if (jb + r < iy1) {
                    const T *gq = gp - P + (long long)(r + 1) * X;
                    if (own_a) { hk1x[r].x = Io<T>::ld(gq + 3 * NN); hk1y[r].x = Io<T>::ld(gq + 4 * NN); }
                    if (own_b) { hk1x[r].y = Io<T>::ld(gq + 3 * NN + 1); hk1y[r].y = Io<T>::ld(gq + 4 * NN + 1); }
                }
        }
        fph ^= 1u << s0;     // the item's first plane was waited for above
        for (int k = kstart; k < ke; ++k, gp += P) {
            mbar_wait(&full[s1], (fph >> s1) & 1u, status, abort_flag);
            fph ^= 1u << s1;
            const unsigned char *st0 = smem + s0 * St::BYTES, *st1 = smem + s1 * St::BYTES;
            // the warp's rows: box rows from R0 on (E, H and B~ boxes start one row above the tile)
            const T *E0 = reinterpret_cast<const T *>(st0 + St::E_OFF) + ecol + R0 * St::EW;
            const T *E1 = reinterpret_cast<const T *>(st1 + St::E_OFF) + ecol + R0 * St::EW;
            const T *H0 = reinterpret_cast<const T *>(st0 + St::H_OFF) + ecol + R0 * St::HW;
            const unsigned char *C0 = st0 + St::C_OFF + R0 * (id16 ? 2 * St::C16W : St::C8W);
            const float *A0 = reinterpret_cast<const float *>(st0 + St::A_OFF) + acol + R0 * St::AW;
            constexpr int EW = St::EW, HW = St::HW, ECS = St::E_CS, HCS = St::H_CS;
            constexpr int AW = St::AW, BCS = St::B_CS;
            const int zb = ZP ? (k < iz0 ? 1 : (k >= iz1 ? 2 : 0)) : 0;
            ZCoef z;
            float *zdz = nullptr, *nzbz = nullptr;
            long long za = 0;
            if (ZP && zb) {
                z.zi = B->cw[2][0][k];
                z.zh = B->cw[2][1][k];
                za = (long long)(k - (zb == 1 ? B->zlo : iz1)) * zplane + zcol;
                nzbz = B->zB[zb - 1][par ^ 1];
                zdz = B->zD[zb - 1];
            }
            const bool full_plane = k >= kb;
            // coefficient rows of the lane's two nodes (ids clamped into the box,
            // so every lookup is a valid row)
            float4 cea[TYW], ceb[TYW];
#pragma unroll
            for (int r = 0; r < TYW; ++r) {
                const int ia = id16 ? (int)reinterpret_cast<const uint16_t *>(C0)[r * St::C16W + ida]
                                    : (int)C0[r * St::C8W + ida];
                const int ib = id16 ? (int)reinterpret_cast<const uint16_t *>(C0)[r * St::C16W + idb]
                                    : (int)C0[r * St::C8W + idb];
                cea[r] = __ldg(ctab + ia);
                ceb[r] = __ldg(ctab + ib);
            }
            // E^n at box row rr (own node), and H~^{n+1/2}(k) there from the staged planes
            auto hrow = [&](int rr, bool in_f, float2 &ex, float2 &ey, float2 &ez, float2 &hx, float2 &hy, float2 &hz,
                            float2 &nbz) {
                ez = Pair<T>::lds(E0 + 2 * ECS + rr * EW);
                ey = Pair<T>::lds(E0 + ECS + rr * EW);
                ex = Pair<T>::lds(E0 + rr * EW);
                const float2 ezu = Pair<T>::lds(E0 + 2 * ECS + (rr + 1) * EW);
                const float2 exu = Pair<T>::lds(E0 + (rr + 1) * EW);
                const float2 eyk = Pair<T>::lds(E1 + ECS + rr * EW), exk = Pair<T>::lds(E1 + rr * EW);
                const float ez2 = cvt<T>(E0[2 * ECS + rr * EW + 2]), ey2 = cvt<T>(E0[ECS + rr * EW + 2]);
                const float2 ezx = make_float2(ez.y, ez2), eyx = make_float2(ey.y, ey2);   // E at (c+1)
                const float2 scx = curl2v(ezu, ez, eyk, ey, Sy2, nSz2);
                const float2 scy = curl2v(exk, ex, ezx, ez, Sz2, nSx2);
                const float2 scz = curl2v(eyx, ey, exu, ex, Sx2, nSy2);
                const float2 ohx = Pair<T>::lds(H0 + rr * HW), ohy = Pair<T>::lds(H0 + HCS + rr * HW);
                const float2 ohz = Pair<T>::lds(H0 + 2 * HCS + rr * HW);
                if (!ZP || !zb) {
                    hx = sub2(ohx, scx);
                    hy = sub2(ohy, scy);
                    hz = sub2(ohz, scz);
                } else {
                    // B~z of the node: box row rr; zero outside the fused rows
                    float2 boz = make_float2(A0[rr * AW], A0[rr * AW + 1]);
                    if (!in_f) boz = make_float2(0.f, 0.f);
                    hx.x = fused_hx(ohx.x, scx.x, zb, z);
                    hx.y = fused_hx(ohx.y, scx.y, zb, z);
                    hy.x = fused_hy(ohy.x, scy.x, zb, z);
                    hy.y = fused_hy(ohy.y, scy.y, zb, z);
                    hz.x = fused_hz(ohz.x, scz.x, zb, z, boz.x, nbz.x);
                    hz.y = fused_hz(ohz.y, scz.y, zb, z, boz.y, nbz.y);
                }
            };
            // halo elements outside the fused region come from the slab output
            auto slab_fix = [&](int rr, float2 &hx, float2 &hy, float2 &hz) {
                if (jb - 1 + rr >= iy1) return;
                const T *gq = gp + (long long)rr * X;
                if (slab_a) { hx.x = Io<T>::ld(gq + 3 * NN); hy.x = Io<T>::ld(gq + 4 * NN); hz.x = Io<T>::ld(gq + 5 * NN); }
                if (slab_b) {
                    hx.y = Io<T>::ld(gq + 3 * NN + 1); hy.y = Io<T>::ld(gq + 4 * NN + 1); hz.y = Io<T>::ld(gq + 5 * NN + 1);
                }
            };

            float2 px = make_float2(0.f, 0.f), pz = px;   // H~x, H~z at (., j-1)
            if (full_plane) {
                if (row_slab) {   // row jb-1 lies in the low-y slab: read its H~ (own columns)
                    if (own_a && own_b) {
                        px = Pair<T>::ldg(gp + 3 * NN);
                        pz = Pair<T>::ldg(gp + 5 * NN);
                    } else if (own_a) {
                        px.x = Io<T>::ld(gp + 3 * NN);
                        pz.x = Io<T>::ld(gp + 5 * NN);
                    } else if (own_b) {
                        px.y = Io<T>::ld(gp + 3 * NN + 1);
                        pz.y = Io<T>::ld(gp + 5 * NN + 1);
                    }
                } else {
                    float2 ex, ey, ez, hy, d0;
                    hrow(0, true, ex, ey, ez, px, hy, pz, d0);
                    slab_fix(0, px, hy, pz);
                }
            }
#pragma unroll
            for (int r = 0; r < TYW; ++r) {
                const int j = jb + r, rr = r + 1;
                float2 ex, ey, ez, hx, hy, hz, nbz = make_float2(0.f, 0.f);
                hrow(rr, j < iy1, ex, ey, ez, hx, hy, hz, nbz);
                slab_fix(rr, hx, hy, hz);
                const float hyl = __shfl_up_sync(0xffffffffu, hy.y, 1);   // H~ at (ca-1, j)
                const float hzl = __shfl_up_sync(0xffffffffu, hz.y, 1);
                if (full_plane && j < iy1) {
                    const float2 hym = make_float2(hyl, hy.x), hzm = make_float2(hzl, hz.x);   // H~ at (c-1, j)
                    const float2 scx = curl2v(hz, pz, hy, hk1y[r], Sy2, nSz2);
                    const float2 scy = curl2v(hx, hk1x[r], hz, hzm, Sz2, nSx2);
                    const float2 scz = curl2v(hy, hym, hx, px, Sx2, nSy2);
                    float2 exv, eyv, ezv;
                    T *o = gp + (long long)rr * X;
                    if (!ZP || !zb) {
                        exv = make_float2(__fmaf_rn(cea[r].x, scx.x, ex.x), __fmaf_rn(ceb[r].x, scx.y, ex.y));
                        eyv = make_float2(__fmaf_rn(cea[r].y, scy.x, ey.x), __fmaf_rn(ceb[r].y, scy.y, ey.y));
                        ezv = make_float2(__fmaf_rn(cea[r].z, scz.x, ez.x), __fmaf_rn(ceb[r].z, scz.y, ez.y));
                    } else {
                        const long long a = za + (long long)r * zrow;
                        const float *dzo = A0 + BCS + r * AW;   // D~z of the node (box row r)
                        float nd;
                        float2 ndz;
                        exv.x = upml_e2(ex.x, scx.x, cea[r].x, kOne, z.zi, kOne, false, 0.f, nd);
                        exv.y = upml_e2(ex.y, scx.y, ceb[r].x, kOne, z.zi, kOne, false, 0.f, nd);
                        eyv.x = upml_e2(ey.x, scy.x, cea[r].y, z.zi, kOne, kOne, false, 0.f, nd);
                        eyv.y = upml_e2(ey.y, scy.y, ceb[r].y, z.zi, kOne, kOne, false, 0.f, nd);
                        ezv.x = upml_e2(ez.x, scz.x, cea[r].z, kOne, kOne, z.zh, true, dzo[0], ndz.x);
                        ezv.y = upml_e2(ez.y, scz.y, ceb[r].z, kOne, kOne, z.zh, true, dzo[1], ndz.y);
                        if (own_a) { stg1(zdz + a, ndz.x); stg1(nzbz + a, nbz.x); }
                        if (own_b) { stg1(zdz + a + 1, ndz.y); stg1(nzbz + a + 1, nbz.y); }
                    }
                    if (own_a && own_b) {
                        stg2(o + 3 * NN, hx); stg2(o + 4 * NN, hy); stg2(o + 5 * NN, hz);
                        stg2(o, exv); stg2(o + NN, eyv); stg2(o + 2 * NN, ezv);
                    } else if (own_a) {
                        stg1(o + 3 * NN, hx.x); stg1(o + 4 * NN, hy.x); stg1(o + 5 * NN, hz.x);
                        stg1(o, exv.x); stg1(o + NN, eyv.x); stg1(o + 2 * NN, ezv.x);
                    } else if (own_b) {
                        stg1(o + 3 * NN + 1, hx.y); stg1(o + 4 * NN + 1, hy.y); stg1(o + 5 * NN + 1, hz.y);
                        stg1(o + 1, exv.y); stg1(o + NN + 1, eyv.y); stg1(o + 2 * NN + 1, ezv.y);
                    }
                }
                hk1x[r] = hx;
                hk1y[r] = hy;
                px = hx;
                pz = hz;
            }
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

// ------------------------------------------------------------------ two-step pass
// Time blocking of the interior region I = [ix0,ix1) x [iy0,iy1) x [iz0,iz1)
// (Model section: the leapfrog H^{n+1/2} from E^n, E^{n+1} from H^{n+1/2};
// two of its steps per sweep over I).  With field sets A = set_of(2, n)
// (n even), M = 2 and A' = set_of(2, n + 2), a pair of steps runs:
//   k_slab_h, z-UPML launch      step n:   A -> M
//   k_pair                       steps n, n+1 of I from A (and M, below):
//                                  state n+2 of I minus its one-node outer
//                                  layer (the band) -> A'; the state n+1 of
//                                  the band and of probe and source edges -> M
//   k_slab_e, k_post             step n:   A, M -> M (k_post skips the
//                                  sources inside I, which the pass applied)
//   k_slab_h + band H boxes, z-UPML launch   step n+1: M -> A'
//   k_slab_e + band E boxes, k_post          step n+1: M, A' -> A'
// The pass reads from M only what the step-n launches before it wrote:
// H~^{n+1/2} of slab nodes next to I, of the z-UPML plane below I, and
// E^{n+1} of the z-UPML plane above I.  Values of the band that need the
// slab kernels' state n+1 (E^{n+2} on all six faces of I but the top, H~^{n+3/2}
// on its high x and y faces) are left to the band boxes.
//
// A work item is a tile of kPairCols x kPairRows owned nodes and a z segment
// [kb, ke).  A block has a producer warp streaming planes into a ring of
// input stages (E^n with two halo rows below and above, H~^{n-1/2} with two
// below and one above, ids), five step-1 warps and four step-2 warps.  Lane l
// holds the column pair g + 2l, g + 2l + 1 with g = i0 - 2 (i0 even).  Step-1
// warp w forms H~^{n+1/2} and E^{n+1} on grid rows j0-1+2w, j0+2w (and H~ on
// the row above) of plane k into a ring of shared-memory slots, with every
// value rounded to the storage type, so the slots hold what a one-step
// launch would have stored.  Step-2 warp v forms H~^{n+3/2} and E^{n+2} on
// rows j0+2v, j0+2v+1 of plane k-1 from the slots of planes k-1 and k.  The
// arithmetic is the one-step kernel's, element by element, so with FP32
// storage both depths give the same bits.  (With 16-bit storage the band's
// E, which the slab kernels finish, is formed from the stored H~ where the
// one-step kernel uses the unrounded value.)
template <typename T>
struct PairStage {   // one input plane
    static constexpr int al(int x) { return (x + 127) & ~127; }
    static constexpr int TY = kPairRows, ES = (int)sizeof(T), EW = kPairEW;
    static constexpr int E_COMP = (TY + 4) * EW, H_COMP = (TY + 3) * EW, M_COMP = (TY + 2) * EW;
    static constexpr int E_CS = al(E_COMP * ES) / ES, H_CS = al(H_COMP * ES) / ES;
    static constexpr int E_BYTES = 3 * E_COMP * ES, H_BYTES = 3 * H_COMP * ES, M_BYTES = 3 * M_COMP * ES;
    static constexpr int C8_BYTES = (TY + 2) * kPairC8W, C16_BYTES = (TY + 2) * kPairC16W * 2;
    static constexpr int E_OFF = 0, H_OFF = 3 * E_CS * ES, C_OFF = H_OFF + 3 * H_CS * ES;
    static constexpr int ITEM_OFF = (C_OFF + (C8_BYTES > C16_BYTES ? C8_BYTES : C16_BYTES) + 7) & ~7;
    static constexpr int BYTES = al(ITEM_OFF + 8);
    static_assert(M_COMP <= H_CS, "the E^{n+1} box of the plane above I fits the H~ area");
};
template <typename T>
struct PairSlot {    // the step-1 results of one plane: E^{n+1}, H~^{n+1/2} on rows j0-1 .. j0+8, ids of rows j0 .. j0+7
    static constexpr int al(int x) { return (x + 127) & ~127; }
    static constexpr int TY = kPairRows, ES = (int)sizeof(T), OW = 64;
    static constexpr int COMP = (TY + 2) * OW;
    static constexpr int CS = al(COMP * ES) / ES;
    static constexpr int E_OFF = 0, H_OFF = 3 * CS * ES, ID_OFF = 6 * CS * ES;
    static constexpr int ITEM_OFF = ID_OFF + TY * OW * 2;
    static constexpr int BYTES = al(ITEM_OFF + 8);
};
constexpr int kPairW1 = 5, kPairW2 = 4;   // step-1, step-2 warps; one producer warp follows
template <typename T>
struct PairLayout {
    static constexpr int NS = 3, NO = 3;
    static constexpr int SLOT_OFF = NS * PairStage<T>::BYTES;
    static constexpr int BAR_OFF = SLOT_OFF + NO * PairSlot<T>::BYTES;
    static constexpr int BYTES = BAR_OFF + 2 * (NS + NO) * 8 + 16;
    static constexpr int THREADS = 32 * (kPairW1 + kPairW2 + 1);
    static_assert(2 * (BYTES + 1024) <= 232448, "two blocks per SM");
};

template <typename T>
__device__ __forceinline__ float rnd(float v);
template <>
__device__ __forceinline__ float rnd<float>(float v) { return v; }
template <>
__device__ __forceinline__ float rnd<__half>(float v) { return __half2float(__float2half_rn(v)); }
template <typename T>
__device__ __forceinline__ float2 rnd2(float2 v) { return make_float2(rnd<T>(v.x), rnd<T>(v.y)); }

struct PairTile {
    const Board *B;
    bool ok, bot, top;
    int i0, j0, kb, ke;
    int in, out;
    long long step;
};

// Items: x tiles fastest, then tile rows within a band of about one wave,
// then z segments, then bands (as the one-step interior launch).
__device__ __forceinline__ PairTile decode_pair(const Plan &plan, long long item)
{
    PairTile t;
    const Board *B = plan.boards[0];
    t.B = B;
    t.step = step_ro(B);
    t.ok = active_ro(B) && B->pair_ok && B->tdepth == 2 && !(t.step & 1);
    t.in = set_of(2, t.step);
    t.out = set_of(2, t.step + 2);
    const PairConst &pc = plan.pc;
    const int ntx = (pc.ix1 - pc.ix0 + kPairCols - 1) / kPairCols;
    const int nty = (pc.iy1 - pc.iy0 + kPairRows - 1) / kPairRows;
    const int zs = plan.pair_zseg, iz0 = pc.iz0, iz1 = pc.iz1;
    const int nseg = (iz1 - iz0 + zs - 1) / zs;
    const int wave_rows = max(1, plan.slots / ntx), nband = (nty + wave_rows - 1) / wave_rows;
    const int band = (nty + nband - 1) / nband;
    const long long per_band = (long long)ntx * band * nseg;
    const int bi = (int)(item / per_band);
    const long long within = item - bi * per_band;
    const int rows = min(band, nty - bi * band);
    const long long layer = (long long)ntx * rows;
    const int tz = (int)(within / layer);
    const int rem = (int)(within - tz * layer);
    t.i0 = pc.ix0 + (rem % ntx) * kPairCols;
    t.j0 = pc.iy0 + (bi * band + rem / ntx) * kPairRows;
    t.kb = iz0 + tz * zs;
    t.ke = min(t.kb + zs, iz1);
    t.bot = t.kb == iz0;
    t.top = t.ke == iz1;
    return t;
}

template <typename T>
__global__ void __launch_bounds__(PairLayout<T>::THREADS, 2) k_pair(Plan plan)
{
    using St = PairStage<T>;
    using Sl = PairSlot<T>;
    using L = PairLayout<T>;
    constexpr int NS = L::NS, NO = L::NO, TY = kPairRows, EW = St::EW, OW = Sl::OW;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + L::BAR_OFF);
    uint64_t *empty = full + NS;
    uint64_t *ofull = empty + NS;
    uint64_t *oempty = ofull + NO;
    int *abort_flag = reinterpret_cast<int *>(oempty + NO);
    const int lx = threadIdx.x, wy = threadIdx.y;
    int *const status0 = plan.boards[0]->status;

    if (wy == 0 && lx == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kPairW1);
        }
        for (int o = 0; o < NO; ++o) {
            mbar_init(&ofull[o], kPairW1);
            mbar_init(&oempty[o], kPairW2);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();

    if (wy == kPairW1 + kPairW2) {
        // ------------------------------------------------------------ producer
        // planes ps .. pe of an item: ps = kb - 2 (kb at the bottom of I), pe =
        // ke + 1 (E^n only), or at the top of I pe = ke = iz1 with E^n and
        // the E^{n+1} that the z-UPML launch of step n wrote into M
        if (lx != 0) return;
        uint32_t eph = 0;
        long long q = 0;
        int s = 0;
        auto acquire = [&]() {
            if (q >= NS) {
                mbar_wait(&empty[s], (eph >> s) & 1u, status0, abort_flag);
                eph ^= 1u << s;
            }
        };
        for (;;) {
            const long long item = atomicAdd(plan.work + 2, 1);
            if (item >= plan.n_pair) break;
            const PairTile t = decode_pair(plan, item);
            if (!t.ok) continue;   // nothing is sent for an item that does not run
            const Board *B = t.B;
            const CUtensorMap *tm = B->tm;
            const int id16 = B->id16;
            const int g = t.i0 - 2;
            const int xe0 = g & ~(16 / St::ES - 1);
            const int xc0 = id16 ? (g & ~7) : (g & ~15);
            const int ps = t.bot ? t.kb : t.kb - 2, pe = t.top ? t.ke : t.ke + 1;
            for (int p = ps; p <= pe; ++p, ++q, s = (s + 1 == NS ? 0 : s + 1)) {
                acquire();
                unsigned char *st = smem + s * St::BYTES;
                *reinterpret_cast<volatile long long *>(st + St::ITEM_OFF) = (p == ps) ? item : -2;
                const bool last = p == pe;
                uint32_t bytes = St::E_BYTES;
                if (last && t.top) bytes += St::M_BYTES;
                else if (!last) bytes += St::H_BYTES + (id16 ? St::C16_BYTES : St::C8_BYTES);
                mbar_expect_tx(&full[s], bytes);
                for (int c = 0; c < 3; ++c)
                    tma_load_3d(st + St::E_OFF + c * St::E_CS * St::ES, tm + tp_e(t.in, c), xe0, t.j0 - 2, p, &full[s]);
                if (last && t.top) {
                    for (int c = 0; c < 3; ++c)
                        tma_load_3d(st + St::H_OFF + c * St::H_CS * St::ES, tm + tp_t(c), xe0, t.j0 - 1, p, &full[s]);
                } else if (!last) {
                    for (int c = 0; c < 3; ++c)
                        tma_load_3d(st + St::H_OFF + c * St::H_CS * St::ES, tm + tp_h(t.in, c), xe0, t.j0 - 2, p,
                                    &full[s]);
                    tma_load_3d(st + St::C_OFF, tm + kTpCid, xc0, t.j0 - 1, p, &full[s]);
                }
            }
        }
        acquire();
        *reinterpret_cast<volatile long long *>(smem + s * St::BYTES + St::ITEM_OFF) = -1;
        mbar_expect_tx(&full[s], 0);
        return;
    }

    const bool step1 = wy < kPairW1;
    const int w = step1 ? wy : wy - kPairW1;
    if (step1) {
        // ------------------------------------------------------------ step 1
        uint32_t fph = 0, oeph = 0;
        int sq = 0, so = 0;
        long long nslot = 0;
        auto slot_acquire = [&]() {
            if (nslot >= NO) {
                mbar_wait(&oempty[so], (oeph >> so) & 1u, status0, abort_flag);
                oeph ^= 1u << so;
            }
        };
        auto slot_publish = [&]() {
            __syncwarp();
            if (lx == 0) mbar_arrive(&ofull[so]);
            so = so + 1 == NO ? 0 : so + 1;
            ++nslot;
        };
        for (;;) {
            mbar_wait(&full[sq], (fph >> sq) & 1u, status0, abort_flag);
            const long long item = *reinterpret_cast<volatile long long *>(smem + sq * St::BYTES + St::ITEM_OFF);
            if (item < 0) {   // no more work: pass the end mark to the step-2 warps
                slot_acquire();
                if (w == 0 && lx == 0)
                    *reinterpret_cast<volatile long long *>(smem + L::SLOT_OFF + so * Sl::BYTES + Sl::ITEM_OFF) = -1;
                slot_publish();
                break;
            }
            fph ^= 1u << sq;
            const PairTile t = decode_pair(plan, item);
            const Board *__restrict__ B = t.B;
            const int i0 = t.i0, j0 = t.j0, kb = t.kb, ke = t.ke;
            const bool top = t.top;
            const int ps = t.bot ? kb : kb - 2, q0 = t.bot ? kb : kb - 1;
            const PairConst &pc = plan.pc;
            const int ix0 = pc.ix0, ix1 = pc.ix1, iy0 = pc.iy0, iy1 = pc.iy1, iz0 = pc.iz0, iz1 = pc.iz1;
            const int X = pc.pitch, ny = pc.ny;
            const long long P = pc.plane, NN = pc.nodes;
            const float2 Sx2 = make_float2(pc.S[0], pc.S[0]), Sy2 = make_float2(pc.S[1], pc.S[1]);
            const float2 Sz2 = make_float2(pc.S[2], pc.S[2]);
            const float2 nSx2 = make_float2(-pc.S[0], -pc.S[0]), nSy2 = make_float2(-pc.S[1], -pc.S[1]);
            const float2 nSz2 = make_float2(-pc.S[2], -pc.S[2]);
            const int id16 = pc.id16;
            const float4 *__restrict__ ctab = pc.ctab;
            int *const status = status0;
            T *const Mp = (T *)pc.mid;
            const int g = i0 - 2;
            const int ca = g + 2 * lx, cb = ca + 1;
            const int whi = min(i0 + kPairCols, ix1);
            const bool own_a = ca >= i0 && ca < whi, own_b = cb >= i0 && cb < whi;
            const bool slab_a = ca < ix0 && ca >= 0, slab_b = cb < ix0 && cb >= 0;
            const int ecol = (g - (g & ~(16 / St::ES - 1))) + 2 * lx;
            const int xc0 = id16 ? (g & ~7) : (g & ~15);
            const int ida = ca - xc0, idb = ida + 1;
            const int jr = j0 - 1 + 2 * w;     // first row of this warp
            // sources in the step-1 region, probes on owned nodes (rare: checked per item)
            bool src_here = false, probe_here = false;
            for (int s = 0; s < B->n_src; ++s) {
                const Source &S = B->src[s];
                src_here |= S.i >= g && S.i < g + 64 && S.j >= jr && S.j < jr + 2 && S.k >= q0 && S.k <= ke;
            }
            for (int s = 0; s < B->n_probe; ++s) {
                const Probe &Q = B->probe[s];
                probe_here |= Q.i >= i0 && Q.i < whi && Q.j >= jr && Q.j < jr + 2 && Q.k >= kb && Q.k < ke;
            }
            const double dt = B->dt;
            const long long step = t.step;

            float2 hk1x[2], hk1y[2];   // H~^{n+1/2} x, y of the previous plane
#pragma unroll
            for (int r = 0; r < 2; ++r) { hk1x[r] = make_float2(0.f, 0.f); hk1y[r] = make_float2(0.f, 0.f); }
            if (t.bot) {   // plane iz0 - 1 (z-UPML or slab) was written by the launches of step n
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const int j = jr + r;
                    if (j < 0 || j > ny) continue;
                    const T *gq = Mp + (long long)(iz0 - 1) * P + (long long)j * X;
                    if (ca >= 0 && ca < X) { hk1x[r].x = Io<T>::ld(gq + 3 * NN + ca); hk1y[r].x = Io<T>::ld(gq + 4 * NN + ca); }
                    if (cb >= 0 && cb < X) { hk1x[r].y = Io<T>::ld(gq + 3 * NN + cb); hk1y[r].y = Io<T>::ld(gq + 4 * NN + cb); }
                }
            }
            int s0 = sq;
            for (int k = ps;; ++k) {
                const bool pseudo = top && k == ke;
                const int s1 = s0 + 1 == NS ? 0 : s0 + 1;
                if (!pseudo) {
                    mbar_wait(&full[s1], (fph >> s1) & 1u, status, abort_flag);
                    fph ^= 1u << s1;
                }
                const bool wslot = k >= q0;
                unsigned char *sl = smem + L::SLOT_OFF + so * Sl::BYTES;
                if (wslot) {
                    slot_acquire();
                    if (k == q0 && w == 0 && lx == 0) *reinterpret_cast<volatile long long *>(sl + Sl::ITEM_OFF) = item;
                }
                const unsigned char *st0 = smem + s0 * St::BYTES, *st1 = smem + s1 * St::BYTES;
                if (pseudo) {
                    // plane iz1: E^{n+1} as the z-UPML launch of step n stored it (box rows from j0 - 1)
#pragma unroll
                    for (int r = 0; r < 2; ++r) {
                        const T *mt = reinterpret_cast<const T *>(st0 + St::H_OFF) + ecol + (2 * w + r) * EW;
                        T *se = reinterpret_cast<T *>(sl + Sl::E_OFF) + (2 * w + r) * OW + 2 * lx;
#pragma unroll
                        for (int c = 0; c < 3; ++c) Pair<T>::st(se + c * Sl::CS, Pair<T>::lds(mt + c * St::H_CS));
                    }
                } else {
                    // box rows from 2w: the row above the warp's rows (E and H~ boxes start at j0 - 2)
                    const T *E0 = reinterpret_cast<const T *>(st0 + St::E_OFF) + ecol + 2 * w * EW;
                    const T *E1 = reinterpret_cast<const T *>(st1 + St::E_OFF) + ecol + 2 * w * EW;
                    const T *H0 = reinterpret_cast<const T *>(st0 + St::H_OFF) + ecol + 2 * w * EW;
                    const unsigned char *C0 = st0 + St::C_OFF + 2 * w * (id16 ? 2 * kPairC16W : kPairC8W);
                    constexpr int ECS = St::E_CS, HCS = St::H_CS;
                    const bool full_plane = k >= q0;
                    float4 cea[2], ceb[2];
#pragma unroll
                    for (int r = 0; r < 2; ++r) {
                        const int ia = id16 ? (int)reinterpret_cast<const uint16_t *>(C0)[r * kPairC16W + ida]
                                            : (int)C0[r * kPairC8W + ida];
                        const int ib = id16 ? (int)reinterpret_cast<const uint16_t *>(C0)[r * kPairC16W + idb]
                                            : (int)C0[r * kPairC8W + idb];
                        cea[r] = __ldg(ctab + ia);
                        ceb[r] = __ldg(ctab + ib);
                        // the ids of the step-2 rows (slot id rows start at j0)
                        const int idr = 2 * w - 1 + r;
                        if (full_plane && idr >= 0 && idr < TY) {
                            if (id16)
                                *reinterpret_cast<uint32_t *>(sl + Sl::ID_OFF + (idr * OW + 2 * lx) * 2) =
                                    (uint32_t)ia | ((uint32_t)ib << 16);
                            else
                                *reinterpret_cast<uint16_t *>(sl + Sl::ID_OFF + idr * OW + 2 * lx) =
                                    (uint16_t)(ia | (ib << 8));
                        }
                    }
                    auto hrow = [&](int rr, float2 &ex, float2 &ey, float2 &ez, float2 &hx, float2 &hy, float2 &hz) {
                        ez = Pair<T>::lds(E0 + 2 * ECS + rr * EW);
                        ey = Pair<T>::lds(E0 + ECS + rr * EW);
                        ex = Pair<T>::lds(E0 + rr * EW);
                        const float2 ezu = Pair<T>::lds(E0 + 2 * ECS + (rr + 1) * EW);
                        const float2 exu = Pair<T>::lds(E0 + (rr + 1) * EW);
                        const float2 eyk = Pair<T>::lds(E1 + ECS + rr * EW), exk = Pair<T>::lds(E1 + rr * EW);
                        const float ez2 = cvt<T>(E0[2 * ECS + rr * EW + 2]), ey2 = cvt<T>(E0[ECS + rr * EW + 2]);
                        const float2 ezx = make_float2(ez.y, ez2), eyx = make_float2(ey.y, ey2);
                        const float2 scx = curl2v(ezu, ez, eyk, ey, Sy2, nSz2);
                        const float2 scy = curl2v(exk, ex, ezx, ez, Sz2, nSx2);
                        const float2 scz = curl2v(eyx, ey, exu, ex, Sx2, nSy2);
                        hx = sub2(Pair<T>::lds(H0 + rr * EW), scx);
                        hy = sub2(Pair<T>::lds(H0 + HCS + rr * EW), scy);
                        hz = sub2(Pair<T>::lds(H0 + 2 * HCS + rr * EW), scz);
                    };
                    // H~ outside the fused region (low x columns, low y rows) comes from the slab output in M
                    auto slab_fix = [&](int j, float2 &hx, float2 &hy, float2 &hz) {
                        if (j < 0 || j >= iy1) return;
                        const bool row_out = j < iy0;
                        const bool fa = (row_out || slab_a) && ca >= 0 && ca < X;
                        const bool fb = (row_out || slab_b) && cb >= 0 && cb < X;
                        if (!fa && !fb) return;
                        const T *gq = Mp + (long long)k * P + (long long)j * X;
                        if (fa) { hx.x = Io<T>::ld(gq + 3 * NN + ca); hy.x = Io<T>::ld(gq + 4 * NN + ca); hz.x = Io<T>::ld(gq + 5 * NN + ca); }
                        if (fb) { hx.y = Io<T>::ld(gq + 3 * NN + cb); hy.y = Io<T>::ld(gq + 4 * NN + cb); hz.y = Io<T>::ld(gq + 5 * NN + cb); }
                    };
                    float2 px, pz;   // H~x, H~z at (., j-1)
                    {
                        float2 ex, ey, ez, hy;
                        hrow(0, ex, ey, ez, px, hy, pz);
                        slab_fix(jr - 1, px, hy, pz);
                    }
#pragma unroll
                    for (int r = 0; r < 2; ++r) {
                        const int j = jr + r;
                        float2 ex, ey, ez, hx, hy, hz;
                        hrow(r + 1, ex, ey, ez, hx, hy, hz);
                        slab_fix(j, hx, hy, hz);
                        const float hyl = __shfl_up_sync(0xffffffffu, hy.y, 1);
                        const float hzl = __shfl_up_sync(0xffffffffu, hz.y, 1);
                        if (full_plane) {
                            const float2 hym = make_float2(hyl, hy.x), hzm = make_float2(hzl, hz.x);
                            const float2 scx = curl2v(hz, pz, hy, hk1y[r], Sy2, nSz2);
                            const float2 scy = curl2v(hx, hk1x[r], hz, hzm, Sz2, nSx2);
                            const float2 scz = curl2v(hy, hym, hx, px, Sx2, nSy2);
                            float2 exv = rnd2<T>(make_float2(__fmaf_rn(cea[r].x, scx.x, ex.x), __fmaf_rn(ceb[r].x, scx.y, ex.y)));
                            float2 eyv = rnd2<T>(make_float2(__fmaf_rn(cea[r].y, scy.x, ey.x), __fmaf_rn(ceb[r].y, scy.y, ey.y)));
                            float2 ezv = rnd2<T>(make_float2(__fmaf_rn(cea[r].z, scz.x, ez.x), __fmaf_rn(ceb[r].z, scz.y, ez.y)));
                            if (src_here) {   // Eq. 8 sources of step n on this row, in the order k_post applies them
                                for (int s = 0; s < B->n_src; ++s) {
                                    const Source &S = B->src[s];
                                    if (S.k != k || S.j != j || (S.i != ca && S.i != cb)) continue;
                                    const double wv = src_pulse(S, step, dt);
                                    float2 e = S.comp == 0 ? exv : (S.comp == 1 ? eyv : ezv);
                                    const float2 en = S.comp == 0 ? ex : (S.comp == 1 ? ey : ez);
                                    if (S.i == ca) e.x = rnd<T>(src_apply(S, wv, e.x, en.x));
                                    else e.y = rnd<T>(src_apply(S, wv, e.y, en.y));
                                    if (S.comp == 0) exv = e;
                                    else if (S.comp == 1) eyv = e;
                                    else ezv = e;
                                }
                            }
                            T *se = reinterpret_cast<T *>(sl + Sl::E_OFF) + (2 * w + r) * OW + 2 * lx;
                            Pair<T>::st(se, exv);
                            Pair<T>::st(se + Sl::CS, eyv);
                            Pair<T>::st(se + 2 * Sl::CS, ezv);
                            T *sh = reinterpret_cast<T *>(sl + Sl::H_OFF) + (2 * w + r) * OW + 2 * lx;
                            Pair<T>::st(sh, hx);
                            Pair<T>::st(sh + Sl::CS, hy);
                            Pair<T>::st(sh + 2 * Sl::CS, hz);
                            // the state n+1 of owned band nodes (and of probe and source edges) goes to M
                            if (k >= kb && k < ke && j >= j0 && j < j0 + TY && j < iy1) {
                                const bool ze = k == iz0 || k == iz1 - 1, zh = k == iz1 - 1;
                                const bool ye = j == iy0 || j == iy1 - 1, yh = j == iy1 - 1;
                                bool wea = own_a && (ze || ye || ca == ix0 || ca == ix1 - 1);
                                bool web = own_b && (ze || ye || cb == ix0 || cb == ix1 - 1);
                                const bool wha = own_a && (zh || yh || ca == ix1 - 1);
                                const bool whb = own_b && (zh || yh || cb == ix1 - 1);
                                if (probe_here)
                                    for (int s = 0; s < B->n_probe; ++s) {
                                        const Probe &Q = B->probe[s];
                                        if (Q.k == k && Q.j == j) { wea |= own_a && Q.i == ca; web |= own_b && Q.i == cb; }
                                    }
                                if (src_here)
                                    for (int s = 0; s < B->n_src; ++s) {
                                        const Source &S = B->src[s];
                                        if (S.k == k && S.j == j) { wea |= own_a && S.i == ca; web |= own_b && S.i == cb; }
                                    }
                                T *o = Mp + (long long)k * P + (long long)j * X + ca;
                                if (wea && web) {
                                    stg2(o, exv); stg2(o + NN, eyv); stg2(o + 2 * NN, ezv);
                                } else if (wea) {
                                    stg1(o, exv.x); stg1(o + NN, eyv.x); stg1(o + 2 * NN, ezv.x);
                                } else if (web) {
                                    stg1(o + 1, exv.y); stg1(o + NN + 1, eyv.y); stg1(o + 2 * NN + 1, ezv.y);
                                }
                                if (wha && whb) {
                                    stg2(o + 3 * NN, hx); stg2(o + 4 * NN, hy); stg2(o + 5 * NN, hz);
                                } else if (wha) {
                                    stg1(o + 3 * NN, hx.x); stg1(o + 4 * NN, hy.x); stg1(o + 5 * NN, hz.x);
                                } else if (whb) {
                                    stg1(o + 3 * NN + 1, hx.y); stg1(o + 4 * NN + 1, hy.y); stg1(o + 5 * NN + 1, hz.y);
                                }
                            }
                        }
                        hk1x[r] = hx;
                        hk1y[r] = hy;
                        px = hx;
                        pz = hz;
                    }
                }
                if (wslot) slot_publish();
                __syncwarp();
                if (lx == 0) mbar_arrive(&empty[s0]);
                s0 = s1;
                if (k == ke) break;
            }
            if (!top) {   // the E-only plane above the segment
                __syncwarp();
                if (lx == 0) mbar_arrive(&empty[s0]);
                s0 = s0 + 1 == NS ? 0 : s0 + 1;
            }
            sq = s0;
        }
        return;
    }

    // ---------------------------------------------------------------- step 2
    uint32_t ofph = 0;
    int so = 0;
    for (;;) {
        mbar_wait(&ofull[so], (ofph >> so) & 1u, status0, abort_flag);
        const long long item = *reinterpret_cast<volatile long long *>(smem + L::SLOT_OFF + so * Sl::BYTES + Sl::ITEM_OFF);
        if (item < 0) break;
        ofph ^= 1u << so;
        const PairTile t = decode_pair(plan, item);
        const Board *__restrict__ B = t.B;
        const int i0 = t.i0, j0 = t.j0, kb = t.kb, ke = t.ke;
        const int q0 = t.bot ? kb : kb - 1;
        const PairConst &pc = plan.pc;
        const int ix0 = pc.ix0, ix1 = pc.ix1, iy0 = pc.iy0, iy1 = pc.iy1, iz0 = pc.iz0;
        const int X = pc.pitch;
        const long long P = pc.plane, NN = pc.nodes;
        const float2 Sx2 = make_float2(pc.S[0], pc.S[0]), Sy2 = make_float2(pc.S[1], pc.S[1]);
        const float2 Sz2 = make_float2(pc.S[2], pc.S[2]);
        const float2 nSx2 = make_float2(-pc.S[0], -pc.S[0]), nSy2 = make_float2(-pc.S[1], -pc.S[1]);
        const float2 nSz2 = make_float2(-pc.S[2], -pc.S[2]);
        const int id16 = pc.id16;
        const float4 *__restrict__ ctab = pc.ctab;
        int *const status = status0;
        const int g = i0 - 2;
        const int ca = g + 2 * lx, cb = ca + 1;
        const int whi = min(i0 + kPairCols, ix1);
        const bool own_a = ca >= i0 && ca < whi, own_b = cb >= i0 && cb < whi;
        // stores: H~^{n+3/2} off the high x face, E^{n+2} off both x faces (the band's)
        const bool sha = own_a && ca != ix1 - 1, shb = own_b && cb != ix1 - 1;
        const bool sea = sha && ca != ix0, seb = shb && cb != ix0;
        const int jb = j0 + 2 * w;   // first row of this warp
        T *gp = (T *)B->f[t.out][0] + ((long long)q0 * P + (long long)jb * X + ca);
        float2 hk1x[2], hk1y[2];   // H~^{n+3/2} x, y of the previous plane
#pragma unroll
        for (int r = 0; r < 2; ++r) { hk1x[r] = make_float2(0.f, 0.f); hk1y[r] = make_float2(0.f, 0.f); }
        int o0 = so;
        for (int q = q0; q < ke; ++q, gp += P) {
            const int o1 = o0 + 1 == NO ? 0 : o0 + 1;
            mbar_wait(&ofull[o1], (ofph >> o1) & 1u, status, abort_flag);
            ofph ^= 1u << o1;
            const unsigned char *sl0 = smem + L::SLOT_OFF + o0 * Sl::BYTES, *sl1 = smem + L::SLOT_OFF + o1 * Sl::BYTES;
            // slot rows from 2w: the row above the warp's rows (slot rows start at j0 - 1)
            const T *E0 = reinterpret_cast<const T *>(sl0 + Sl::E_OFF) + 2 * lx + 2 * w * OW;
            const T *E1 = reinterpret_cast<const T *>(sl1 + Sl::E_OFF) + 2 * lx + 2 * w * OW;
            const T *H0 = reinterpret_cast<const T *>(sl0 + Sl::H_OFF) + 2 * lx + 2 * w * OW;
            constexpr int CS = Sl::CS;
            const bool hplane = q >= kb, eplane = q >= kb && q != iz0;
            float4 cea[2], ceb[2];
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int row = 2 * w + r;   // id rows of the slot start at j0
                int ia, ib;
                if (id16) {
                    const uint32_t v = *reinterpret_cast<const uint32_t *>(sl0 + Sl::ID_OFF + (row * OW + 2 * lx) * 2);
                    ia = (int)(v & 0xffffu); ib = (int)(v >> 16);
                } else {
                    const uint32_t v = *reinterpret_cast<const uint16_t *>(sl0 + Sl::ID_OFF + row * OW + 2 * lx);
                    ia = (int)(v & 0xffu); ib = (int)(v >> 8);
                }
                cea[r] = __ldg(ctab + ia);
                ceb[r] = __ldg(ctab + ib);
            }
            auto hrow = [&](int rr, float2 &ex, float2 &ey, float2 &ez, float2 &hx, float2 &hy, float2 &hz) {
                ez = Pair<T>::lds(E0 + 2 * CS + rr * OW);
                ey = Pair<T>::lds(E0 + CS + rr * OW);
                ex = Pair<T>::lds(E0 + rr * OW);
                const float2 ezu = Pair<T>::lds(E0 + 2 * CS + (rr + 1) * OW);
                const float2 exu = Pair<T>::lds(E0 + (rr + 1) * OW);
                const float2 eyk = Pair<T>::lds(E1 + CS + rr * OW), exk = Pair<T>::lds(E1 + rr * OW);
                const float ez2 = cvt<T>(E0[2 * CS + rr * OW + 2]), ey2 = cvt<T>(E0[CS + rr * OW + 2]);
                const float2 ezx = make_float2(ez.y, ez2), eyx = make_float2(ey.y, ey2);
                const float2 scx = curl2v(ezu, ez, eyk, ey, Sy2, nSz2);
                const float2 scy = curl2v(exk, ex, ezx, ez, Sz2, nSx2);
                const float2 scz = curl2v(eyx, ey, exu, ex, Sx2, nSy2);
                hx = sub2(Pair<T>::lds(H0 + rr * OW), scx);
                hy = sub2(Pair<T>::lds(H0 + CS + rr * OW), scy);
                hz = sub2(Pair<T>::lds(H0 + 2 * CS + rr * OW), scz);
            };
            float2 px, pz;
            {
                float2 ex, ey, ez, hy;
                hrow(0, ex, ey, ez, px, hy, pz);
            }
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int j = jb + r;
                float2 ex, ey, ez, hx, hy, hz;
                hrow(r + 1, ex, ey, ez, hx, hy, hz);
                const float hyl = __shfl_up_sync(0xffffffffu, hy.y, 1);
                const float hzl = __shfl_up_sync(0xffffffffu, hz.y, 1);
                if (hplane && j < iy1) {
                    T *o = gp + (long long)r * X;
                    const bool yh = j != iy1 - 1, ye = yh && j != iy0;
                    const bool ha = sha && yh, hb = shb && yh;
                    if (ha && hb) {
                        stg2(o + 3 * NN, hx); stg2(o + 4 * NN, hy); stg2(o + 5 * NN, hz);
                    } else if (ha) {
                        stg1(o + 3 * NN, hx.x); stg1(o + 4 * NN, hy.x); stg1(o + 5 * NN, hz.x);
                    } else if (hb) {
                        stg1(o + 3 * NN + 1, hx.y); stg1(o + 4 * NN + 1, hy.y); stg1(o + 5 * NN + 1, hz.y);
                    }
                    if (eplane) {
                        const float2 hym = make_float2(hyl, hy.x), hzm = make_float2(hzl, hz.x);
                        const float2 scx = curl2v(hz, pz, hy, hk1y[r], Sy2, nSz2);
                        const float2 scy = curl2v(hx, hk1x[r], hz, hzm, Sz2, nSx2);
                        const float2 scz = curl2v(hy, hym, hx, px, Sx2, nSy2);
                        const float2 exv = make_float2(__fmaf_rn(cea[r].x, scx.x, ex.x), __fmaf_rn(ceb[r].x, scx.y, ex.y));
                        const float2 eyv = make_float2(__fmaf_rn(cea[r].y, scy.x, ey.x), __fmaf_rn(ceb[r].y, scy.y, ey.y));
                        const float2 ezv = make_float2(__fmaf_rn(cea[r].z, scz.x, ez.x), __fmaf_rn(ceb[r].z, scz.y, ez.y));
                        const bool ea = sea && ye, eb = seb && ye;
                        if (ea && eb) {
                            stg2(o, exv); stg2(o + NN, eyv); stg2(o + 2 * NN, ezv);
                        } else if (ea) {
                            stg1(o, exv.x); stg1(o + NN, eyv.x); stg1(o + 2 * NN, ezv.x);
                        } else if (eb) {
                            stg1(o + 1, exv.y); stg1(o + NN + 1, eyv.y); stg1(o + 2 * NN + 1, ezv.y);
                        }
                    }
                }
                hk1x[r] = hx;
                hk1y[r] = hy;
                px = hx;
                pz = hz;
            }
            __syncwarp();
            if (lx == 0) mbar_arrive(&oempty[o0]);
            o0 = o1;
        }
        __syncwarp();
        if (lx == 0) mbar_arrive(&oempty[o0]);   // the slot of plane ke
        so = o0 + 1 == NO ? 0 : o0 + 1;
    }
}

// ------------------------------------------------------------------ slabs
// A slab thread marches kSlabKz consecutive nodes of its slab: along z for
// slabs more than one plane thick (an (i, j) column), along y for the two
// single-plane z slabs (an (i, k) column).  Consecutive threads take
// consecutive i, so rows are coalesced, and the per-column UPML factors and
// index arithmetic are paid once per column.
struct SlabCol {
    const Slab *sl;
    long long t;          // slab-local (aux) index of the first node; + tstep per node
    int tstep;
    bool ym;              // marching along y (else z)
    int i, j, k, count;   // first node, nodes to march
};

// Block set-up from the plan's per-block descriptor: the step counters, the
// slab's box and every set's field pointers are independent loads.
template <typename T>
__device__ __forceinline__ bool slab_locate(const Plan &plan, long long blk, const Board *&B, SlabCol &sc,
                                            Fields<T> &F)
{
    const SlabBlock d = plan.slab_blk[blk];
    B = d.B;
    const long long step = __ldg(d.step), stop = __ldg(d.stop);
    const Slab *sl = &B->slab[d.slab];
    const int ni = sl->ni, nj = sl->nj, i0 = sl->i0, j0 = sl->j0, k0 = sl->k0, k1 = sl->k1, j1 = sl->j1;
    const void *f0[6], *f1[6], *f2[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        f0[c] = B->f[0][c];
        f1[c] = B->f[1][c];
        f2[c] = B->f[2][c];
    }
    const int depth = B->tdepth;
    if (step >= stop) return false;
    const bool ym = (k1 - k0 == 1);
    const int nij = ni * nj;
    const int tt = d.t0 + (int)threadIdx.x;
    if (ym) {
        const int nrow = (nj + kSlabKz - 1) / kSlabKz;
        if (tt >= ni * nrow) return false;
        const int jr = tt / ni, ii = tt - jr * ni;
        sc.i = i0 + ii;
        sc.j = j0 + jr * kSlabKz;
        sc.k = k0;
        sc.count = min(kSlabKz, j1 - sc.j);
        sc.t = (long long)jr * kSlabKz * ni + ii;
        sc.tstep = ni;
    } else {
        const int nkz = (k1 - k0 + kSlabKz - 1) / kSlabKz;
        if (tt >= nij * nkz) return false;
        const int kz = tt / nij, ij = tt - kz * nij;
        const int jj = ij / ni;
        sc.i = i0 + (ij - jj * ni);
        sc.j = j0 + jj;
        sc.k = k0 + kz * kSlabKz;
        sc.count = min(kSlabKz, k1 - sc.k);
        sc.t = (long long)kz * kSlabKz * nij + ij;
        sc.tstep = nij;
    }
    sc.ym = ym;
    sc.sl = sl;
    const int si = set_of(depth, step), so = set_of(depth, step + 1);
    auto pick = [&](int set, int c) -> const void * { return set == 0 ? f0[c] : (set == 1 ? f1[c] : f2[c]); };
    F.ex = (const T *)pick(si, 0); F.ey = (const T *)pick(si, 1); F.ez = (const T *)pick(si, 2);
    F.hx = (const T *)pick(si, 3); F.hy = (const T *)pick(si, 4); F.hz = (const T *)pick(si, 5);
    F.oex = (T *)pick(so, 0); F.oey = (T *)pick(so, 1); F.oez = (T *)pick(so, 2);
    F.ohx = (T *)pick(so, 3); F.ohy = (T *)pick(so, 4); F.ohz = (T *)pick(so, 5);
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

// The slab kernels issue every load of a node unconditionally, with the
// offsets of neighbours that do not exist (i = nx, j = ny, k = nz, or the
// image across an outer wall) clamped to an in-bounds node; only the stores
// are conditional.  A thread streams the inputs of its next nodes into a
// per-thread ring of shared-memory slots with cp.async (one commit group
// per node), so several nodes' loads are in flight while it updates the
// current one, without holding them in registers.

// cp.async of the 32-bit word at src (4-byte aligned) into shared memory.
__device__ __forceinline__ void cp_word(float *dst, const void *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Storage element <-> 32-bit word: a 16-bit element is copied with its
// neighbour (the aligned word holding it) and picked by its index parity.
// Field arrays start 128-byte aligned and node offsets keep the element
// index, so the parity of the node index selects the half.
template <typename T>
struct Word;
template <>
struct Word<float> {
    static __device__ __forceinline__ const void *at(const float *p) { return p; }
    static __device__ __forceinline__ float get(float w, long long) { return w; }
};
template <>
struct Word<__half> {
    static __device__ __forceinline__ const void *at(const __half *p)
    {
        return (const void *)((uintptr_t)p & ~(uintptr_t)3);
    }
    static __device__ __forceinline__ float get(float w, long long e)
    {
        const unsigned b = __float_as_uint(w);
        return __half2float(__ushort_as_half((unsigned short)((e & 1) ? b >> 16 : b & 0xffffu)));
    }
};

// Coefficient id of node idx from the word holding it (8- or 16-bit ids).
__device__ __forceinline__ const void *cid_word(const void *cid, int id16, long long idx)
{
    return id16 ? (const void *)((uintptr_t)((const uint16_t *)cid + idx) & ~(uintptr_t)3)
                : (const void *)((uintptr_t)((const uint8_t *)cid + idx) & ~(uintptr_t)3);
}
__device__ __forceinline__ int cid_get(int id16, float w, long long idx)
{
    const unsigned b = __float_as_uint(w);
    return id16 ? (int)((idx & 1) ? b >> 16 : b & 0xffffu) : (int)((b >> (8 * (int)(idx & 3))) & 0xffu);
}

// One row of a 1D UPML factor table through the read-only cache (the
// tables are 16-byte aligned, one Coef per position).
__device__ __forceinline__ Coef ldcoef(const Coef *p)
{
    const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
    return Coef{v.x, v.y, v.z, v.w};
}

// Ring slots per thread (nodes in flight + 1), words per node and resident
// blocks per SM of the two slab kernels; the rings are sized so that the
// blocks' shared memory fits an SM.  With 128-thread blocks, four nodes in
// flight per thread at the same occupancy measured 2 % faster than three
// with 256-thread blocks.
constexpr int kSlabHStages = 5, kSlabHWords = 15, kSlabHBlocks = 5;
constexpr int kSlabEStages = 5, kSlabEWords = 16, kSlabEBlocks = 4;
constexpr int kSlabHSmem = kSlabHStages * kSlabHWords * kSlabThreads * 4;
constexpr int kSlabESmem = kSlabEStages * kSlabEWords * kSlabThreads * 4;
static_assert(kSlabHBlocks * (kSlabHSmem + 1024) <= 232448 && kSlabEBlocks * (kSlabESmem + 1024) <= 232448,
              "slab rings exceed an SM's shared memory");

// Slot w of node m in a thread's ring of S slots of NW words (words of one
// slot are kSlabThreads apart, so a warp's accesses to a word are conflict-free).
template <int S, int NW>
__device__ __forceinline__ float *ring_at(float *my, int m, int w)
{
    return my + ((m % S) * NW + w) * kSlabThreads;
}

enum SlabHWord { hEYC, hEXC, hEYU, hEXU, hEZC, hEZJ, hEZI, hEYI, hEXJ, hHX, hHY, hHZ, hBX, hBY, hBZ };

template <typename T>
__global__ void __launch_bounds__(kSlabThreads, kSlabHBlocks) k_slab_h(Plan plan)
{
    extern __shared__ float slab_ring[];
    float *const my = slab_ring + threadIdx.x;
    for (long long blk = blockIdx.x; blk < plan.n_slab; blk += gridDim.x) {
        const Board *B;
        SlabCol sc;
        Fields<T> F;
        if (!slab_locate(plan, blk, B, sc, F)) continue;
        const int i = sc.i, ny = B->ny, nz = B->nz;
        const int X = B->pitch;
        const long long P = B->plane;
        const float Sx = B->S[0], Sy = B->S[1], Sz = B->S[2];
        const Slab &sl = *sc.sl;
        float *const ax = sl.aux[3], *const ay = sl.aux[4], *const az = sl.aux[5];
        const bool xin = i < B->nx;
        const int di = xin ? 1 : 0;   // clamped +x neighbour offset
        // x factors fixed along the column: H_x (x integer), H_y, H_z (x half)
        const Coef x0 = B->cw[0][0][i], x1 = B->cw[0][1][i];
        const int j0 = sc.j, k0 = sc.k, cnt = sc.count;
        const bool ym = sc.ym;
        const long long idx0 = (long long)k0 * P + (long long)j0 * X + i;
        const long long didx = ym ? X : P;
        // y and z factors: only the marching axis' change from node to node
        const Coef *const cy0 = B->cw[1][0], *const cy1 = B->cw[1][1];
        const Coef *const cz0 = B->cw[2][0], *const cz1 = B->cw[2][1];
        Coef y0 = ldcoef(cy0 + j0), y1 = ldcoef(cy1 + j0), z0 = ldcoef(cz0 + k0), z1 = ldcoef(cz1 + k0);
        // issue the loads of node m (empty group past the column's end)
        auto issue = [&](int m) {
            if (m < cnt) {
                const long long idx = idx0 + m * didx, t = sc.t + (long long)m * sc.tstep;
                const int j = ym ? j0 + m : j0, k = ym ? k0 : k0 + m;
                const int dj = j < ny ? X : 0;
                const long long dk = k < nz ? P : 0;
                if (ym || m == 0) {   // marching z, E_y and E_x at the node are the previous +z loads
                    cp_word(ring_at<kSlabHStages, kSlabHWords>(my, m, hEYC), Word<T>::at(F.ey + idx));
                    cp_word(ring_at<kSlabHStages, kSlabHWords>(my, m, hEXC), Word<T>::at(F.ex + idx));
                }
                cp_word(ring_at<kSlabHStages, kSlabHWords>(my, m, hEYU), Word<T>::at(F.ey + idx + dk));
                cp_word(ring_at<kSlabHStages, kSlabHWords>(my, m, hEXU), Word<T>::at(F.ex + idx + dk));
                cp_word(ring_at<kSlabHStages, kSlabHWords>(my, m, hEZC), Word<T>::at(F.ez + idx));
                cp_word(ring_at<kSlabHStages, kSlabHWords>(my, m, hEZJ), Word<T>::at(F.ez + idx + dj));
                cp_word(ring_at<kSlabHStages, kSlabHWords>(my, m, hEZI), Word<T>::at(F.ez + idx + di));
                cp_word(ring_at<kSlabHStages, kSlabHWords>(my, m, hEYI), Word<T>::at(F.ey + idx + di));
                cp_word(ring_at<kSlabHStages, kSlabHWords>(my, m, hEXJ), Word<T>::at(F.ex + idx + dj));
                cp_word(ring_at<kSlabHStages, kSlabHWords>(my, m, hHX), Word<T>::at(F.hx + idx));
                cp_word(ring_at<kSlabHStages, kSlabHWords>(my, m, hHY), Word<T>::at(F.hy + idx));
                cp_word(ring_at<kSlabHStages, kSlabHWords>(my, m, hHZ), Word<T>::at(F.hz + idx));
                if (ax) cp_word(ring_at<kSlabHStages, kSlabHWords>(my, m, hBX), ax + t);
                if (ay) cp_word(ring_at<kSlabHStages, kSlabHWords>(my, m, hBY), ay + t);
                if (az) cp_word(ring_at<kSlabHStages, kSlabHWords>(my, m, hBZ), az + t);
            }
            cp_commit();
        };
#pragma unroll
        for (int m = 0; m < kSlabHStages - 1; ++m) issue(m);
        float eyc = 0.f, exc = 0.f;   // E_y, E_x at the node (carried along z)
#pragma unroll
        for (int m = 0; m < kSlabKz; ++m) {
            if (m >= cnt) break;
            issue(m + kSlabHStages - 1);
            cp_wait<kSlabHStages - 1>();
            const long long idx = idx0 + m * didx, t = sc.t + (long long)m * sc.tstep;
            const int j = ym ? j0 + m : j0, k = ym ? k0 : k0 + m;
            const int dj = j < ny ? X : 0;
            const long long dk = k < nz ? P : 0;
            auto w = [&](int word) { return *ring_at<kSlabHStages, kSlabHWords>(my, m, word); };
            if (ym || m == 0) {
                eyc = Word<T>::get(w(hEYC), idx);
                exc = Word<T>::get(w(hEXC), idx);
            }
            const float eyu = Word<T>::get(w(hEYU), idx + dk), exu = Word<T>::get(w(hEXU), idx + dk);
            const float ezc = Word<T>::get(w(hEZC), idx);
            const float ezj = Word<T>::get(w(hEZJ), idx + dj), ezi = Word<T>::get(w(hEZI), idx + di);
            const float eyi = Word<T>::get(w(hEYI), idx + di), exj = Word<T>::get(w(hEXJ), idx + dj);
            const float hxo = Word<T>::get(w(hHX), idx), hyo = Word<T>::get(w(hHY), idx);
            const float hzo = Word<T>::get(w(hHZ), idx);
            const bool yin = j < ny, zin = k < nz;
            if (m > 0) {
                if (ym) { y0 = ldcoef(cy0 + j); y1 = ldcoef(cy1 + j); }
                else { z0 = ldcoef(cz0 + k); z1 = ldcoef(cz1 + k); }
            }
            float bn;
            if (yin && zin) {   // H_x(i, j+1/2, k+1/2)
                const float h = upml_h2(hxo, curl2(ezj, ezc, eyu, eyc, Sy, Sz), y1, z1, x0, ax != nullptr,
                                        ax ? w(hBX) : 0.f, bn);
                Io<T>::st(F.ohx + idx, h);
                if (ax) ax[t] = bn;
            }
            if (xin && zin) {   // H_y(i+1/2, j, k+1/2)
                const float h = upml_h2(hyo, curl2(exu, exc, ezi, ezc, Sz, Sx), z1, x1, y0, ay != nullptr,
                                        ay ? w(hBY) : 0.f, bn);
                Io<T>::st(F.ohy + idx, h);
                if (ay) ay[t] = bn;
            }
            if (xin && yin) {   // H_z(i+1/2, j+1/2, k)
                const float h = upml_h2(hzo, curl2(eyi, eyc, exj, exc, Sx, Sy), x1, y1, z0, az != nullptr,
                                        az ? w(hBZ) : 0.f, bn);
                Io<T>::st(F.ohz + idx, h);
                if (az) az[t] = bn;
            }
            eyc = eyu;
            exc = exu;
        }
        cp_wait<0>();   // no copy into the ring may be outstanding when the next block reuses it
    }
}

// Factor of the image of tangential H~ across an outer wall for a neighbour
// `outside` the grid (PMC: odd mirror, -1; PEC: 0).
__device__ __forceinline__ float hsign(bool outside, int wall) { return outside ? (wall == 1 ? -1.0f : 0.0f) : 1.0f; }

// Ring words of a slab E node: H~ at the node and at its -x, -y, -z
// neighbours (each loaded once; a neighbour across the low wall is clamped to
// the node itself, and the image of H~ across a high wall is the -x/-y/-z
// neighbour's value, picked after the load), E^n, the D~ auxiliaries, the id.
enum SlabEWord { eHZ, eHZJ, eHZI, eHY, eHYI, eHYK, eHX, eHXJ, eHXK, eEX, eEY, eEZ, eDX, eDY, eDZ, eID };

template <typename T>
__global__ void __launch_bounds__(kSlabThreads, kSlabEBlocks) k_slab_e(Plan plan)
{
    extern __shared__ float slab_ring[];
    float *const my = slab_ring + threadIdx.x;
    for (long long blk = blockIdx.x; blk < plan.n_slab; blk += gridDim.x) {
        const Board *B;
        SlabCol sc;
        Fields<T> F;
        if (!slab_locate(plan, blk, B, sc, F)) continue;
        const int i = sc.i;
        const int nx = B->nx, ny = B->ny, nz = B->nz;
        const int X = B->pitch;
        const long long P = B->plane;
        const float Sx = B->S[0], Sy = B->S[1], Sz = B->S[2];
        const Slab &sl = *sc.sl;
        float *const ax = sl.aux[0], *const ay = sl.aux[1], *const az = sl.aux[2];
        const int *wl = B->wall;
        const int w2 = wl[2], w3 = wl[3], w4 = wl[4], w5 = wl[5];
        // images across the x walls (fixed along the column)
        const bool xhi = i == nx, xlo = i == 0;
        const float sxh = hsign(xhi, wl[1]), sxl = hsign(xlo, wl[0]);
        const int ox0 = xlo ? 0 : -1;   // offset of H at i-1 (clamped at the low wall)
        // x factors fixed along the column: E_x (x half), E_y, E_z (x integer)
        const Coef x1 = B->cw[0][1][i], x0 = B->cw[0][0][i];
        const int j0 = sc.j, k0 = sc.k, cnt = sc.count;
        const bool ym = sc.ym;
        const long long idx0 = (long long)k0 * P + (long long)j0 * X + i;
        const long long didx = ym ? X : P;
        const Coef *const cy0 = B->cw[1][0], *const cy1 = B->cw[1][1];
        const Coef *const cz0 = B->cw[2][0], *const cz1 = B->cw[2][1];
        Coef y0 = ldcoef(cy0 + j0), y1 = ldcoef(cy1 + j0), z0 = ldcoef(cz0 + k0), z1 = ldcoef(cz1 + k0);
        const void *const cid = B->cid;
        const int id16 = B->id16;
        const float4 *const ctab = B->ctab;
        auto issue = [&](int m) {
            if (m < cnt) {
                const long long idx = idx0 + m * didx, t = sc.t + (long long)m * sc.tstep;
                const int j = ym ? j0 + m : j0, k = ym ? k0 : k0 + m;
                const int oy0 = j == 0 ? 0 : -X;
                const long long oz0 = k == 0 ? 0 : -P;
                cp_word(ring_at<kSlabEStages, kSlabEWords>(my, m, eID), cid_word(cid, id16, idx));
                cp_word(ring_at<kSlabEStages, kSlabEWords>(my, m, eHZ), Word<T>::at(F.ohz + idx));
                cp_word(ring_at<kSlabEStages, kSlabEWords>(my, m, eHZJ), Word<T>::at(F.ohz + idx + oy0));
                cp_word(ring_at<kSlabEStages, kSlabEWords>(my, m, eHZI), Word<T>::at(F.ohz + idx + ox0));
                cp_word(ring_at<kSlabEStages, kSlabEWords>(my, m, eHY), Word<T>::at(F.ohy + idx));
                cp_word(ring_at<kSlabEStages, kSlabEWords>(my, m, eHYI), Word<T>::at(F.ohy + idx + ox0));
                cp_word(ring_at<kSlabEStages, kSlabEWords>(my, m, eHX), Word<T>::at(F.ohx + idx));
                cp_word(ring_at<kSlabEStages, kSlabEWords>(my, m, eHXJ), Word<T>::at(F.ohx + idx + oy0));
                if (ym || m == 0) {   // marching z, H~y and H~x at -z are the previous node's values
                    cp_word(ring_at<kSlabEStages, kSlabEWords>(my, m, eHYK), Word<T>::at(F.ohy + idx + oz0));
                    cp_word(ring_at<kSlabEStages, kSlabEWords>(my, m, eHXK), Word<T>::at(F.ohx + idx + oz0));
                }
                cp_word(ring_at<kSlabEStages, kSlabEWords>(my, m, eEX), Word<T>::at(F.ex + idx));
                cp_word(ring_at<kSlabEStages, kSlabEWords>(my, m, eEY), Word<T>::at(F.ey + idx));
                cp_word(ring_at<kSlabEStages, kSlabEWords>(my, m, eEZ), Word<T>::at(F.ez + idx));
                if (ax) cp_word(ring_at<kSlabEStages, kSlabEWords>(my, m, eDX), ax + t);
                if (ay) cp_word(ring_at<kSlabEStages, kSlabEWords>(my, m, eDY), ay + t);
                if (az) cp_word(ring_at<kSlabEStages, kSlabEWords>(my, m, eDZ), az + t);
            }
            cp_commit();
        };
#pragma unroll
        for (int m = 0; m < kSlabEStages - 1; ++m) issue(m);
        float hyk = 0.f, hxk = 0.f;   // H~y, H~x at -z (carried along z)
#pragma unroll
        for (int m = 0; m < kSlabKz; ++m) {
            if (m >= cnt) break;
            issue(m + kSlabEStages - 1);
            cp_wait<kSlabEStages - 1>();
            const long long idx = idx0 + m * didx, t = sc.t + (long long)m * sc.tstep;
            const int j = ym ? j0 + m : j0, k = ym ? k0 : k0 + m;
            const int oy0 = j == 0 ? 0 : -X;
            const long long oz0 = k == 0 ? 0 : -P;
            auto w = [&](int word) { return *ring_at<kSlabEStages, kSlabEWords>(my, m, word); };
            const bool yhi = j == ny, ylo = j == 0, zhi = k == nz, zlo = k == 0;
            const float syh = hsign(yhi, w3), syl = hsign(ylo, w2), szh = hsign(zhi, w5), szl = hsign(zlo, w4);
            const float4 ce = __ldg(ctab + cid_get(id16, w(eID), idx));
            if (m > 0) {
                if (ym) { y0 = ldcoef(cy0 + j); y1 = ldcoef(cy1 + j); }
                else { z0 = ldcoef(cz0 + k); z1 = ldcoef(cz1 + k); }
            }
            if (ym || m == 0) {
                hyk = Word<T>::get(w(eHYK), idx + oz0);
                hxk = Word<T>::get(w(eHXK), idx + oz0);
            }
            const float hz = Word<T>::get(w(eHZ), idx), hzj = Word<T>::get(w(eHZJ), idx + oy0);
            const float hzi = Word<T>::get(w(eHZI), idx + ox0);
            const float hy = Word<T>::get(w(eHY), idx), hyi = Word<T>::get(w(eHYI), idx + ox0);
            const float hx = Word<T>::get(w(eHX), idx), hxj = Word<T>::get(w(eHXJ), idx + oy0);
            float dn;
            if (i < nx) {   // E_x(i+1/2, j, k)
                const float e = upml_e2(Word<T>::get(w(eEX), idx),
                                        curl2(syh * (yhi ? hzj : hz), syl * hzj, szh * (zhi ? hyk : hy), szl * hyk,
                                              Sy, Sz),
                                        ce.x, y0, z0, x1, ax != nullptr, ax ? w(eDX) : 0.f, dn);
                Io<T>::st(F.oex + idx, e);
                if (ax) ax[t] = dn;
            }
            if (j < ny) {   // E_y(i, j+1/2, k)
                const float e = upml_e2(Word<T>::get(w(eEY), idx),
                                        curl2(szh * (zhi ? hxk : hx), szl * hxk, sxh * (xhi ? hzi : hz), sxl * hzi,
                                              Sz, Sx),
                                        ce.y, z0, x0, y1, ay != nullptr, ay ? w(eDY) : 0.f, dn);
                Io<T>::st(F.oey + idx, e);
                if (ay) ay[t] = dn;
            }
            if (k < nz) {   // E_z(i, j, k+1/2)
                const float e = upml_e2(Word<T>::get(w(eEZ), idx),
                                        curl2(sxh * (xhi ? hyi : hy), sxl * hyi, syh * (yhi ? hxj : hx), syl * hxj,
                                              Sx, Sy),
                                        ce.z, x0, y0, z1, az != nullptr, az ? w(eDZ) : 0.f, dn);
                Io<T>::st(F.oez + idx, e);
                if (az) az[t] = dn;
            }
            hyk = hy;   // the next node (k + 1 <= nz) reads H at k
            hxk = hx;
        }
        cp_wait<0>();
    }
}

// ------------------------------------------------------------------ sources, probes
template <typename T>
__global__ void k_post(Plan plan)
{
    const int b = blockIdx.x;
    if (b >= plan.nb) return;
    Board *B = plan.boards[b];
    // What does not depend on the step is loaded before the step counter, so
    // the descriptors, the field pointers and the counters arrive together
    // (this kernel is a short chain of dependent loads between two launches).
    const int tid = threadIdx.x;
    const int n_src = B->n_src, n_probe = B->n_probe, n_total = B->n_total;
    const bool par_src = B->src_distinct != 0;
    const Source *const src = B->src;
    const Probe *const probe = B->probe;
    const double dt = B->dt;
    const float scale = B->scale;
    void *fp[3][3];
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int c = 0; c < 3; ++c) fp[q][c] = B->f[q][c];
    const int depth = B->tdepth;
    const bool skip_i = plan.first_of_pair != 0;
    Source s0;
    Probe q0;
    if (tid < n_src) s0 = src[tid];
    if (tid < n_probe) q0 = probe[tid];
    const long long step = *((volatile long long *)B->step);
    if (step >= *((volatile long long *)B->stop)) return;
    const int out = set_of(depth, step + 1), in = set_of(depth, step);
    auto field = [&](int set, int comp) -> T * {
        void *const *f = set == 0 ? fp[0] : (set == 1 ? fp[1] : fp[2]);
        return (T *)(comp == 0 ? f[0] : comp == 1 ? f[1] : f[2]);
    };
    // sources on distinct edges are independent: one thread each; sources
    // sharing an edge are applied in order by thread 0.  On the first step of
    // a two-step pass the pass has applied the sources inside I already.
    if (par_src || tid == 0) {
        for (int s = par_src ? tid : 0; s < n_src; s += par_src ? (int)blockDim.x : 1) {
            const Source S = (par_src && s == tid) ? s0 : src[s];
            if (skip_i && in_interior(B, S.i, S.j, S.k)) continue;
            const double w = src_pulse(S, step, dt);
            T *e = field(out, S.comp) + S.node;
            Io<T>::st(e, src_apply(S, w, Io<T>::ldw(e), Io<T>::ldw((const T *)field(in, S.comp) + S.node)));
        }
    }
    __syncthreads();
    const bool rec = step < (long long)n_total;
    for (int p = tid; p < n_probe; p += blockDim.x) {
        const Probe Q = p == tid ? q0 : probe[p];
        const float v = Io<T>::ldw((const T *)field(out, Q.comp) + Q.node) * scale;
        if (rec) B->trace[(long long)p * n_total + step] = v;
        if (!isfinite(v)) atomicOr(B->status, 1);
    }
    __syncthreads();
    if (tid == 0) *((volatile long long *)B->step) = step + 1;
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
    const int pin = set_of(B->tdepth, step - 1), pout = set_of(B->tdepth, step);
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

// ------------------------------------------------------------------ failure detection
// Self-test of the bounded wait: an mbarrier that nothing arrives on, waited
// on with the same bounded poll as the fused kernel, must give up, set
// status bit 1 (value 2) and return, leaving the context usable.
__global__ void k_wait_selftest(int *status, uint32_t max_polls)
{
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_wait(&bar, 0, status, &abort_flag, max_polls);
}

cudaError_t launch_wait_selftest(int *status, unsigned max_polls, cudaStream_t st)
{
    k_wait_selftest<<<1, 32, 0, st>>>(status, max_polls);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ launchers
// Fused-kernel configurations: W compute warps x 62 columns by TY rows, an
// NS-stage ring; ZP selects the z-UPML launch.
constexpr int kFusedStages = 3;

template <typename T, int TY, int W, bool ZP, int R>
struct FusedCfg {
    static constexpr int NS = kFusedStages;
    using L = FusedLayout<T, TY, W, NS, ZP, R>;
    static dim3 block() { return dim3(32, W * R + 1); }
    static int grid()
    {
        static int g = 0;
        if (!g) {
            int dev = 0, sms = 0, per = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fused<T, TY, W, NS, ZP, R>, 32 * (W * R + 1),
                                                          L::BYTES);
            g = (sms > 0 ? sms : 152) * (per > 0 ? per : 1);
        }
        return g;
    }
    static cudaError_t set_limit()
    {
        return cudaFuncSetAttribute(k_fused<T, TY, W, NS, ZP, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    L::BYTES);
    }
    static void launch(const Plan &plan, cudaStream_t st)
    {
        const long long n = ZP ? plan.n_zp : plan.n_int;
        if (n <= 0) return;
        const int g = (int)(n < grid() ? n : grid());
        Plan p = plan;
        p.slots = grid();
        k_fused<T, TY, W, NS, ZP, R><<<g, block(), L::BYTES, st>>>(p);
    }
};

// Supported fused tiles (tile_x columns x tile_y rows): 62x4 and 124x4 (one
// compute warp per 62 columns), 62x8 (four compute warps of two rows sharing
// the stage) and 124x8 (two compute warps of four rows per 62 columns).
template <typename T, bool ZP>
static void launch_fused(const Plan &plan, cudaStream_t st)
{
    const int key = plan.tile_x * 16 + plan.tile_y;
    switch (key) {
    case 62 * 16 + 8: FusedCfg<T, 8, 1, ZP, 4>::launch(plan, st); break;
    case 124 * 16 + 4: FusedCfg<T, 4, 2, ZP, 1>::launch(plan, st); break;
    case 124 * 16 + 8: FusedCfg<T, 8, 2, ZP, 2>::launch(plan, st); break;
    default: FusedCfg<T, 4, 1, ZP, 1>::launch(plan, st); break;
    }
}

// Two-step pass: two blocks per SM (shared memory), one launch per pair of steps.
template <typename T>
struct PairCfg {
    using L = PairLayout<T>;
    static dim3 block() { return dim3(32, kPairW1 + kPairW2 + 1); }
    static int grid()
    {
        static int g = 0;
        if (!g) {
            int dev = 0, sms = 0, per = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pair<T>, L::THREADS, L::BYTES);
            g = (sms > 0 ? sms : 152) * (per > 0 ? per : 1);
        }
        return g;
    }
    static cudaError_t set_limit()
    {
        return cudaFuncSetAttribute(k_pair<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, L::BYTES);
    }
    static void launch(const Plan &plan, cudaStream_t st)
    {
        if (plan.n_pair <= 0) return;
        const int g = (int)(plan.n_pair < grid() ? plan.n_pair : grid());
        Plan p = plan;
        p.slots = grid();
        k_pair<T><<<g, block(), L::BYTES, st>>>(p);
    }
};

// Slab kernels launch one block per descriptor (grid-striding past this).
constexpr long long kMaxGrid = 1 << 20;

template <typename T>
static cudaError_t phase_t(const Plan &plan, int phase, int grid_cap, cudaStream_t st)
{
    switch (phase) {
    case kPhaseSlabH:
        if (plan.n_slab > 0)
            k_slab_h<T><<<(int)(plan.n_slab < kMaxGrid ? plan.n_slab : kMaxGrid), kSlabThreads, kSlabHSmem, st>>>(plan);
        break;
    case kPhaseFusedZ:
        if (plan.n_zp > 0) {
            cudaMemsetAsync(plan.work + 1, 0, sizeof(int), st);
            launch_fused<T, true>(plan, st);
        }
        break;
    case kPhaseInterior:
        if (plan.n_int > 0) {
            cudaMemsetAsync(plan.work, 0, sizeof(int), st);
            launch_fused<T, false>(plan, st);
        }
        break;
    case kPhaseSlabE:
        if (plan.n_slab > 0)
            k_slab_e<T><<<(int)(plan.n_slab < kMaxGrid ? plan.n_slab : kMaxGrid), kSlabThreads, kSlabESmem, st>>>(plan);
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
    default: return phase_t<float>(plan, phase, grid_cap, st);
    }
}

// The nine launches of a pair of steps n, n+1 (n even, depth 2), numbered
// 0..8 (see the two-step pass): slab H, z-UPML, the pass, slab E, post (its
// interior sources skipped), slab H with the band's H boxes, z-UPML, slab E
// with the band's E boxes, post.  kPairPhase names the phase each belongs to.
template <typename T>
static cudaError_t pair_t(const Plan &plan, int idx, int grid_cap, cudaStream_t st)
{
    Plan p = plan;
    switch (idx) {
    case 2:
        if (plan.n_pair > 0) {
            cudaMemsetAsync(plan.work + 2, 0, sizeof(int), st);
            PairCfg<T>::launch(plan, st);
        }
        return cudaGetLastError();
    case 4: p.first_of_pair = 1; return phase_t<T>(p, kPhasePost, grid_cap, st);
    case 5:   // the band's H+E blocks sit just before the slab blocks in the table
        p.slab_blk -= plan.n_band_h;
        p.n_slab += plan.n_band_h;
        return phase_t<T>(p, kPhaseSlabH, grid_cap, st);
    case 7:   // and its E-only blocks before those
        p.slab_blk -= plan.n_band;
        p.n_slab += plan.n_band;
        return phase_t<T>(p, kPhaseSlabE, grid_cap, st);
    default: return phase_t<T>(p, kPairPhase[idx], grid_cap, st);
    }
}

cudaError_t launch_pair_part(const Plan &plan, int prec, int idx, int grid_cap, cudaStream_t st)
{
    switch (prec) {
    case kFP16: return pair_t<__half>(plan, idx, grid_cap, st);
    default: return pair_t<float>(plan, idx, grid_cap, st);
    }
}

cudaError_t launch_pair(const Plan &plan, int prec, int grid_cap, cudaStream_t st)
{
    for (int i = 0; i < kPairLaunches; ++i) {
        cudaError_t e = launch_pair_part(plan, prec, i, grid_cap, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
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
    cudaError_t e[11] = {PairCfg<T>::set_limit(),
                         cudaFuncSetAttribute(k_slab_h<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSlabHSmem),
                         cudaFuncSetAttribute(k_slab_e<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSlabESmem),
                         FusedCfg<T, 4, 1, false, 1>::set_limit(), FusedCfg<T, 8, 1, false, 4>::set_limit(),
                         FusedCfg<T, 4, 2, false, 1>::set_limit(), FusedCfg<T, 8, 2, false, 2>::set_limit(),
                         FusedCfg<T, 4, 1, true, 1>::set_limit(),  FusedCfg<T, 8, 1, true, 4>::set_limit(),
                         FusedCfg<T, 4, 2, true, 1>::set_limit(),  FusedCfg<T, 8, 2, true, 2>::set_limit()};
    for (cudaError_t x : e)
        if (x != cudaSuccess) return x;
    return cudaSuccess;
}

cudaError_t fused_set_smem_limits()
{
    cudaError_t a = limits_t<float>(), b = limits_t<__half>();
    return a != cudaSuccess ? a : b;
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
    default: k_energy<float><<<n_part, 256, 0, st>>>(b_dev, partials); break;
    }
    k_energy_final<<<1, 256, 0, st>>>(partials, n_part, out2);
    return cudaGetLastError();
}

}  // namespace fdtd
