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
    return ((long long)(k - k0) * (B->iy1 - B->iy0) + (j - B->iy0)) * (long long)(B->ix1 - B->ix0) + (i - B->ix0);
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

// Tiled fused H+E kernel over the fused region.  A CTA owns a 32 x TY tile of
// (i, j) columns and marches a z-segment.  Per plane k it keeps E^n of planes
// k and k+1 (tile plus one-node halo) in shared memory, computes H~^{n+1/2}(k)
// for the tile plus the low-x column and low-y row it needs (recomputed from
// the same inputs when they lie in the fused region, read from the slab
// kernel's output otherwise), then E^{n+1}(k) for the tile.  E^n of plane k+2
// and the tile's H~^{n-1/2}(k+1) are prefetched into registers while plane k
// is computed.
template <typename T, int TY>
__global__ void __launch_bounds__(32 * TY, 512 / (32 * TY)) k_fused(Plan plan)
{
    constexpr int NT = 32 * TY;
    constexpr int EW = 34, EH = TY + 2, EPL = EW * EH;
    constexpr int NE = (3 * EPL + NT - 1) / NT;
    constexpr int HW = 33, HH = TY + 1;
    constexpr int HCW = TY > 1 ? 1 : 0;          // warp computing the low-x halo column
    __shared__ float sE[3][3][EH][EW];
    __shared__ float sH[3][HH][HW];
    const int lx = threadIdx.x, ly = threadIdx.y, tid = ly * 32 + lx;

    for (long long item = blockIdx.x; item < plan.n_int; item += gridDim.x) {
        const int b = find_board(plan.int_prefix, plan.nb, item);
        const Board *__restrict__ B = plan.boards[b];
        if (!board_active(B)) continue;
        const long long step = *((volatile long long *)B->step);
        const int par = (int)(step & 1);
        const long long local = item - __ldg(plan.int_prefix + b);
        const int nx = B->nx, ny = B->ny, nz = B->nz;
        const int ix0 = B->ix0, ix1 = B->ix1, iy0 = B->iy0, iy1 = B->iy1;
        const int ntx = (ix1 - ix0 + 31) / 32, nty = (iy1 - iy0 + TY - 1) / TY;
        const int tx = (int)(local % ntx);
        const long long rest = local / ntx;
        const int ty = (int)(rest % nty), tz = (int)(rest / nty);
        const int i0 = ix0 + tx * 32, j0 = iy0 + ty * TY;
        const int kb = 1 + tz * plan.zseg, ke = min(kb + plan.zseg, nz);
        const int i = i0 + lx, j = j0 + ly;
        const bool own = i < ix1 && j < iy1;
        const int X = B->pitch;
        const long long P = B->plane;
        const float Sx = B->S[0], Sy = B->S[1], Sz = B->S[2];
        const Fields<T> F(B, par);
        const Coef *__restrict__ czi = B->cw[2][0];
        const Coef *__restrict__ czh = B->cw[2][1];

        // halo duties: row (i, j0-1) by warp 0, column (i0-1, j0+lx) by warp HCW lanes < TY
        const bool row_duty = (ly == 0) && (i < ix1);
        const bool row_calc = row_duty && (j0 - 1 >= iy0);
        const bool col_duty = (ly == HCW) && (lx < TY) && (j0 + lx < iy1);
        const bool col_calc = col_duty && (i0 - 1 >= ix0);
        const int cj = j0 + lx;                          // column-halo node (i0-1, cj)

        auto load_plane = [&](int kp, float (&r)[NE]) {
#pragma unroll
            for (int u = 0; u < NE; ++u) {
                const int f = tid + u * NT;
                float v = 0.f;
                if (f < 3 * EPL) {
                    const int c = f / EPL, rr = f - c * EPL, sy = rr / EW, sx = rr - sy * EW;
                    const int gi = i0 - 1 + sx, gj = j0 - 1 + sy;
                    if (gi <= nx && gj <= ny && kp <= nz) {
                        const T *src = c == 0 ? F.ex : (c == 1 ? F.ey : F.ez);
                        v = Io<T>::ld(src + ((unsigned)kp * (unsigned)P + (unsigned)(gj * X + gi)));
                    }
                }
                r[u] = v;
            }
        };
        auto store_plane = [&](int stg, const float (&r)[NE]) {
#pragma unroll
            for (int u = 0; u < NE; ++u) {
                const int f = tid + u * NT;
                if (f < 3 * EPL) {
                    const int c = f / EPL, rr = f - c * EPL, sy = rr / EW, sx = rr - sy * EW;
                    sE[stg][c][sy][sx] = r[u];
                }
            }
        };

        // per-plane operands of this thread (current and prefetched next plane)
        struct Ops {
            float hx, hy, hz;        // own H~^{n-1/2}
            float rhx, rhz;          // row halo H~ (old, or new if not recomputed)
            float chy, chz;          // column halo H~
            float dy, dz, by, bz;    // own auxiliaries (z-UPML planes)
            float rbz, cby, cbz;     // halo auxiliaries
            int cid;
        };
        auto fetch = [&](int k, Ops &o) {
            const int zb = zbox_of(B, k);
            const long long q = (long long)k * P + (long long)j * X + i;
            if (own) {
                o.hx = Io<T>::ld(F.hx + q); o.hy = Io<T>::ld(F.hy + q); o.hz = Io<T>::ld(F.hz + q);
                o.cid = cid_at(B, q);
                if (zb) {
                    const long long a = zaux_index(B, zb, i, j, k);
                    o.dy = B->zD[zb - 1][0][a]; o.dz = B->zD[zb - 1][1][a];
                    o.by = __ldg(B->zB[zb - 1][0][par] + a); o.bz = __ldg(B->zB[zb - 1][1][par] + a);
                }
            }
            if (row_duty) {
                const long long r = (long long)k * P + (long long)(j0 - 1) * X + i;
                if (row_calc) {
                    o.rhx = Io<T>::ld(F.hx + r); o.rhz = Io<T>::ld(F.hz + r);
                    if (zb) o.rbz = __ldg(B->zB[zb - 1][1][par] + zaux_index(B, zb, i, j0 - 1, k));
                } else {
                    o.rhx = Io<T>::ld(F.ohx + r); o.rhz = Io<T>::ld(F.ohz + r);
                }
            }
            if (col_duty) {
                const long long r = (long long)k * P + (long long)cj * X + (i0 - 1);
                if (col_calc) {
                    o.chy = Io<T>::ld(F.hy + r); o.chz = Io<T>::ld(F.hz + r);
                    if (zb) {
                        const long long a = zaux_index(B, zb, i0 - 1, cj, k);
                        o.cby = __ldg(B->zB[zb - 1][0][par] + a); o.cbz = __ldg(B->zB[zb - 1][1][par] + a);
                    }
                } else {
                    o.chy = Io<T>::ld(F.ohy + r); o.chz = Io<T>::ld(F.ohz + r);
                }
            }
        };

        // own H~x, H~y at plane kb-1 (needed by E(kb))
        float hxm = 0.f, hym = 0.f;
        if (own) {
            const long long q = (long long)(kb - 1) * P + (long long)j * X + i;
            if (kb - 1 >= 1) {
                const int zb = zbox_of(B, kb - 1);
                ZCoef z;
                z.zi = czi[kb - 1]; z.zh = czh[kb - 1];
                const float scx = curl2(Io<T>::ld(F.ez + q + X), Io<T>::ld(F.ez + q), Io<T>::ld(F.ey + q + P),
                                        Io<T>::ld(F.ey + q), Sy, Sz);
                const float scy = curl2(Io<T>::ld(F.ex + q + P), Io<T>::ld(F.ex + q), Io<T>::ld(F.ez + q + 1),
                                        Io<T>::ld(F.ez + q), Sz, Sx);
                float Bo = 0.f, Bn;
                if (zb) Bo = __ldg(B->zB[zb - 1][0][par] + zaux_index(B, zb, i, j, kb - 1));
                hxm = fused_hx(Io<T>::ld(F.hx + q), scx, zb, z);
                hym = fused_hy(Io<T>::ld(F.hy + q), scy, zb, z, Bo, Bn);
            } else {
                hxm = Io<T>::ld(F.ohx + q);
                hym = Io<T>::ld(F.ohy + q);
            }
        }
        {
            float r[NE];
            load_plane(kb, r);
            store_plane(kb % 3, r);
            load_plane(kb + 1, r);
            store_plane((kb + 1) % 3, r);
        }
        Ops cur, nxt;
        fetch(kb, cur);
        __syncthreads();

        for (int k = kb; k < ke; ++k) {
            const int s0 = k % 3, s1 = (k + 1) % 3, s2 = (k + 2) % 3;
            const bool more = (k + 1 < ke);
            float rE[NE];
            if (more) {
                load_plane(k + 2, rE);
                fetch(k + 1, nxt);
            }
            const int zb = zbox_of(B, k);
            ZCoef z;
            if (zb) { z.zi = czi[k]; z.zh = czh[k]; }
            const int sx = lx + 1, sy = ly + 1;
            float hxv = 0.f, hyv = 0.f, hzv = 0.f, nby = 0.f, nbz = 0.f;
            if (own) {
                const float scx = curl2(sE[s0][2][sy + 1][sx], sE[s0][2][sy][sx], sE[s1][1][sy][sx], sE[s0][1][sy][sx], Sy, Sz);
                const float scy = curl2(sE[s1][0][sy][sx], sE[s0][0][sy][sx], sE[s0][2][sy][sx + 1], sE[s0][2][sy][sx], Sz, Sx);
                const float scz = curl2(sE[s0][1][sy][sx + 1], sE[s0][1][sy][sx], sE[s0][0][sy + 1][sx], sE[s0][0][sy][sx], Sx, Sy);
                hxv = fused_hx(cur.hx, scx, zb, z);
                hyv = fused_hy(cur.hy, scy, zb, z, cur.by, nby);
                hzv = fused_hz(cur.hz, scz, zb, z, cur.bz, nbz);
                sH[0][sy][sx] = hxv; sH[1][sy][sx] = hyv; sH[2][sy][sx] = hzv;
            }
            if (row_duty) {   // node (i, j0-1): smem row sy = 0
                if (row_calc) {
                    const float scx = curl2(sE[s0][2][1][sx], sE[s0][2][0][sx], sE[s1][1][0][sx], sE[s0][1][0][sx], Sy, Sz);
                    const float scz = curl2(sE[s0][1][0][sx + 1], sE[s0][1][0][sx], sE[s0][0][1][sx], sE[s0][0][0][sx], Sx, Sy);
                    float d;
                    sH[0][0][sx] = fused_hx(cur.rhx, scx, zb, z);
                    sH[2][0][sx] = fused_hz(cur.rhz, scz, zb, z, cur.rbz, d);
                } else {
                    sH[0][0][sx] = cur.rhx;
                    sH[2][0][sx] = cur.rhz;
                }
            }
            if (col_duty) {   // node (i0-1, j0+lx): smem column sx = 0, row lx+1
                const int cy = lx + 1;
                if (col_calc) {
                    const float scy = curl2(sE[s1][0][cy][0], sE[s0][0][cy][0], sE[s0][2][cy][1], sE[s0][2][cy][0], Sz, Sx);
                    const float scz = curl2(sE[s0][1][cy][1], sE[s0][1][cy][0], sE[s0][0][cy + 1][0], sE[s0][0][cy][0], Sx, Sy);
                    float d;
                    sH[1][cy][0] = fused_hy(cur.chy, scy, zb, z, cur.cby, d);
                    sH[2][cy][0] = fused_hz(cur.chz, scz, zb, z, cur.cbz, d);
                } else {
                    sH[1][cy][0] = cur.chy;
                    sH[2][cy][0] = cur.chz;
                }
            }
            __syncthreads();
            if (own) {
                const long long q = (long long)k * P + (long long)j * X + i;
                const float4 ce = __ldg(B->ctab + cur.cid);
                const float scx = curl2(sH[2][sy][sx], sH[2][sy - 1][sx], hyv, hym, Sy, Sz);
                const float scy = curl2(hxv, hxm, sH[2][sy][sx], sH[2][sy][sx - 1], Sz, Sx);
                const float scz = curl2(sH[1][sy][sx], sH[1][sy][sx - 1], sH[0][sy][sx], sH[0][sy - 1][sx], Sx, Sy);
                float exv, eyv, ezv;
                if (!zb) {
                    exv = __fmaf_rn(ce.x, scx, sE[s0][0][sy][sx]);
                    eyv = __fmaf_rn(ce.y, scy, sE[s0][1][sy][sx]);
                    ezv = __fmaf_rn(ce.z, scz, sE[s0][2][sy][sx]);
                } else {
                    float nd, ndy, ndz;
                    exv = upml_e2(sE[s0][0][sy][sx], scx, ce.x, kOne, z.zi, kOne, false, 0.f, nd);
                    eyv = upml_e2(sE[s0][1][sy][sx], scy, ce.y, z.zi, kOne, kOne, true, cur.dy, ndy);
                    ezv = upml_e2(sE[s0][2][sy][sx], scz, ce.z, kOne, kOne, z.zh, true, cur.dz, ndz);
                    const long long a = zaux_index(B, zb, i, j, k);
                    B->zD[zb - 1][0][a] = ndy;
                    B->zD[zb - 1][1][a] = ndz;
                    B->zB[zb - 1][0][par ^ 1][a] = nby;
                    B->zB[zb - 1][1][par ^ 1][a] = nbz;
                }
                Io<T>::st(F.ohx + q, hxv);
                Io<T>::st(F.ohy + q, hyv);
                Io<T>::st(F.ohz + q, hzv);
                Io<T>::st(F.oex + q, exv);
                Io<T>::st(F.oey + q, eyv);
                Io<T>::st(F.oez + q, ezv);
            }
            hxm = hxv;
            hym = hyv;
            if (more) {
                store_plane(s2, rE);
                cur = nxt;
            }
            __syncthreads();
        }
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
template <typename T>
static cudaError_t phase_t(const Plan &plan, int phase, int grid_cap, cudaStream_t st)
{
    switch (phase) {
    case kPhaseSlabH:
        if (plan.n_slab > 0)
            k_slab_h<T><<<(int)(plan.n_slab < grid_cap ? plan.n_slab : grid_cap), kSlabThreads, 0, st>>>(plan);
        break;
    case kPhaseInterior:
        if (plan.n_int > 0) {
            const int g = (int)(plan.n_int < grid_cap ? plan.n_int : grid_cap);
            if (plan.tile_y == 2) k_fused<T, 2><<<g, dim3(32, 2), 0, st>>>(plan);
            else if (plan.tile_y == 8) k_fused<T, 8><<<g, dim3(32, 8), 0, st>>>(plan);
            else k_fused<T, 4><<<g, dim3(32, 4), 0, st>>>(plan);
        }
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
