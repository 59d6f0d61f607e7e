// fdtd_internal.h -- device-side data layout shared by the kernels and the C-ABI.
//
// Normalised unknowns.  The kernels advance E/s and eta0*H/s (s a power-of-two
// storage scale, 1 in FP32 mode), so the curl updates read
//   H~ <- H~ - (S_{w+1} dE_{w+2} - S_{w+2} dE_{w+1}),   S_w = c dt / d_w,
//   E  <- E  + (1/eps_r) (S_{w+1} dH~_{w+2} - S_{w+2} dH~_{w+1})
// and the Gedney D/B recurrences of the UPML (Eqs. 1-4, graded by Eq. 5) use
// per-position factors with q = sigma dt / (2 eps0):
//   b1 = (kappa - q)/(kappa + q), g = 1/(kappa + q), ap = kappa + q, am = kappa - q
//   D~' = b1_{w+1} D~ + g_{w+1} (S curl H~)_w
//   E'  = b1_{w+2} E  + (1/eps_r) g_{w+2} (ap_w D~' - am_w D~)
// (B~/H~ alike with a minus on the curl).  In the model space b1 = g = ap =
// am = 1 and both reduce to plain Yee.
//
// Memory layout in HBM: every field component is a [nz+1][ny+1][pitch] array
// (x fastest, pitch an odd multiple of 32 elements, see row_pitch),
// indexed by the node its Yee sample starts at; samples that do not exist stay
// zero.  Fields live in two or three sets: a step reads the set holding the
// current state and writes another (see set_of).
// One uint8 per node (uint16 when a geometry has more than 256) selects a row
// (ce_x, ce_y, ce_z) = 1/eps_r of its three E edges (0 on PEC) of a table.
// UPML factors are 1D per axis at integer and half positions.
//
// Which auxiliaries are stored.  With H~' = b1_{w+2} H~ + g_{w+2} (ap_w B~' -
// am_w B~) and B~' = b1_{w+1} B~ - g_{w+1} S curl: if the factors along w are
// trivial (ap = am = 1) and at most one of w+1, w+2 is graded, B~' - B~ is a
// known multiple of the curl or H~ - B~ is constant in time (zero, since both
// start at zero), so the component updates as the lossy Yee form
// H~' = (b1_{w+1} b1_{w+2}) H~ - (g_{w+1} g_{w+2}) S curl with no auxiliary
// (one of each product is exactly 1).  Likewise E' = (b1 b1) E + ce (g g) S curl
// (E - ce D~ is constant).  An auxiliary is kept only where the factors along
// w are graded or both w+1 and w+2 are.
//
// Work split.  The fused region F = [ix0,ix1) x [iy0,iy1) x [zlo,nz) (the
// columns outside the x/y UPML, minus the outer z planes; zlo = 0 under a
// z-UPML, whose PEC wall plane k = 0 the z-UPML launch works) is updated by
// one fused H+E kernel that marches z; its z-UPML planes ([zlo,iz0) and
// [iz1,nz)) have sigma_z only, so they carry D~z (updated in place) and B~z
// (ping-ponged, since neighbouring tiles recompute halo H from it) in compact
// [k][j][i] boxes.  Everything else (x/y UPML slabs with their
// edges and corners, and the outer z planes) is updated by generic slab
// kernels whose auxiliary D~/B~ live in compact [k][j][i] boxes per slab, only
// for components whose recurrence there is not trivial.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fdtd {

constexpr int kMaxSlab = 32;
// Row pitch of the field, id and diagnostic arrays (elements): nx + 1 rounded
// up to a multiple of 32, then to an odd multiple of 32, so that FP32 rows
// start 128-byte aligned and span an odd number of 128-byte lines (consecutive
// rows and planes then spread over the memory partitions; measured 0.4 % on
// the 880x680x100 board against a pitch of an even number of lines).
inline int row_pitch(int nx)
{
    int p = (nx + 1 + 31) / 32 * 32;
    if (((p / 32) & 1) == 0) p += 32;
    return p;
}
constexpr int kMaxCombo = 256;
constexpr int kMaxCombo16 = 65536;

enum Prec : int { kFP32 = 0, kFP16 = 1 };

// Per-position UPML factors (b1, g, ap, am).
struct Coef {
    float b1, g, ap, am;
};

struct Slab {
    int i0, i1, j0, j1, k0, k1;   // node box, half-open
    int ni, nj;                   // i1 - i0, j1 - j0
    long long n;                  // nodes in the box
    long long block0;             // first slab-kernel block of this slab (board-local)
                                  // (blocks cover ni * nj * ceil(nk / kSlabKz) threads, or
                                  // ni * ceil(nj / kSlabKz) for a single plane)
    float *aux[6];                // D~x, D~y, D~z, B~x, B~y, B~z or nullptr
};

enum SourceKind : int { kSrcCurrent = 0, kSrcResistiveVoltage = 1 };

struct Source {
    long long node;               // linear node index
    int comp;                     // 0..2
    int kind;                     // SourceKind
    int i, j, k, pad;             // the node
    double J0, t0, tau;           // Eq. 8 pulse (amplitude J0 [A/m^2], or V0 [V] for a voltage source)
    double coef;                  // current: ce * dt / (eps0 s), E/s -= coef * J
    double beta, gam;             // voltage: E' = (E_plain - beta E - gam Vs) / (1 + beta) (gam includes 1/s)
    double rs;                    // voltage: series resistance [ohm]
};

struct Probe {
    long long node;
    int comp;
    int i, j, k;                  // the node
};

// Everything a kernel needs about one board; lives in device memory.
struct Board {
    int nx, ny, nz;
    int pitch;
    long long plane;              // pitch * (ny + 1)
    long long nodes;              // plane * (nz + 1)
    int prec;
    int pad0;
    void *f[3][6];                // [set][Ex, Ey, Ez, Hx, Hy, Hz]; set 2 only with two-step passes
    int tdepth;                   // steps per interior pass: 1, or 2 (time blocking, see set_of)
    int pair_ok;                  // the two-step pass can run on this board (set 2 and its maps exist)
    const void *cid;              // combo id per node (uint8, or uint16 if id16)
    int id16;
    int pad2;
    const float4 *ctab;           // combo table rows (ce_x, ce_y, ce_z, 0)
    const Coef *cw[3][2];         // [axis][0: integer, 1: half] positions
    float S[3];                   // c dt / d_w
    float scale;                  // physical = stored * scale (E); H = stored * scale / eta0
    int wall[6];
    int depth[6];                 // UPML cells per face
    int ix0, ix1, iy0, iy1, iz0, iz1;   // fused xy box; non-UPML z range [iz0, iz1)
    int zlo;                            // first plane of the fused region: 0 under a z-UPML (PEC wall), else 1
    // z-UPML boxes of the fused region: [0] k in [zlo, iz0), [1] k in [iz1, nz);
    // element (i, j, k) at ((k - k0) * (iy1 - iy0) + j - iy0) * zpitch + i - ix0.
    // With sigma_z alone, B~x, B~y and D~x, D~y need no storage (see the
    // auxiliary rule below); B~z and D~z are kept.
    float *zD[2];                 // [box]         D~z
    float *zB[2][2];              // [box][parity] B~z
    int zpitch;                   // row pitch of the z-UPML boxes (multiple of 8)
    int tm_tx, tm_ty;             // tile shape the tensor maps were encoded for
    const CUtensorMap *tm;        // kNumMaps TMA descriptors (see tm_* below)
    int n_slab;
    int slab_blocks;              // slab-kernel blocks for this board
    // Band boxes (slab[n_slab], ...): the one-node outer layer of the interior
    // region I = [ix0,ix1) x [iy0,iy1) x [iz0,iz1) whose second step a
    // two-step pass cannot finish.  The first n_band_h boxes (the high x and y
    // layers) need H and E, the rest E only; their blocks follow the slab
    // blocks, H+E boxes first.
    int n_band, n_band_h;
    int band_blocks, band_h_blocks;
    Slab slab[kMaxSlab];
    long long *step;              // completed steps (device counter)
    long long *stop;              // inactive once *step >= *stop
    int n_src;
    int n_probe;
    int src_distinct;             // no two sources share an edge
    int pad3;
    const Source *src;
    const Probe *probe;
    double dt;
    float *trace;                 // [n_probe][n_total]
    int n_total;                  // DFT length N (0: no recording)
    int n_bins;
    double *dft;                  // [n_probe][n_bins][2]
    long long *dft_done;          // samples already folded into dft
    int *status;                  // bit 0: non-finite probe sample seen; bit 1: a bounded wait
                                  // gave up; bit 2: tile / tensor-map mismatch (item skipped)
    int pad1;
};

// One slab-kernel block of a plan: everything its threads need to start
// loading, so a block's set-up is one table read plus loads that do not
// depend on one another.
struct SlabBlock {
    const Board *B;
    const long long *step, *stop;   // the board's step counters
    int slab;                       // slab index within the board
    int t0;                         // first slab-local thread of the block
};

// Field set that holds the state after n steps (E^n and H~^{n-1/2}).  With
// depth 1 the sets alternate.  With depth 2 the states after an even number
// of steps alternate between sets 0 and 1 and odd states use set 2, so one
// pass can read the state n (even) and write the state n + 2 into the other
// of sets 0 and 1 while the slab kernels keep the state n + 1 in set 2.
__host__ __device__ inline int set_of(int depth, long long n)
{
    return depth == 2 ? ((n & 1) ? 2 : (int)((n >> 1) & 1)) : (int)(n & 1);
}

// Constants of the single board a two-step pass works on, carried in the
// plan (kernel parameters) so that the pass reads them from the constant
// bank instead of holding them in registers.
struct PairConst {
    float S[3];
    int ix0, ix1, iy0, iy1, iz0, iz1;
    int ny, pitch, id16, pad;
    long long plane, nodes;
    const float4 *ctab;
    void *mid;                    // component 0 of field set 2
};

// How a depth-2 board runs n steps from step s: one single step to reach an
// even step, then pairs (one two-step pass each), then one or two single
// steps, so that the last step is a single one and the states after the
// last two steps are complete in memory.
struct PairSplit {
    int lead, pairs, tail;
};
inline PairSplit pair_split(long long s, int n)
{
    PairSplit p{0, 0, 0};
    if (n <= 0) return p;
    int left = n;
    if (s & 1) {
        p.lead = 1;
        --left;
    }
    p.pairs = left >= 3 ? (left - 1) / 2 : 0;
    p.tail = left - 2 * p.pairs;
    return p;
}

// Renaming of the field sets when the blocking depth changes from d0 to d1
// after n steps: the new set x is the old set perm[x], so that the states
// after steps n and n - 1 sit where set_of(d1, .) expects them (the third set
// takes the spare one).
inline void rename_sets(int d0, int d1, long long n, int perm[3])
{
    const int a = set_of(d0, n), b = set_of(d0, n - 1), x = set_of(d1, n), y = set_of(d1, n - 1);
    int spare = 0;
    while (spare == a || spare == b) ++spare;
    perm[x] = a;
    perm[y] = b;
    perm[3 - x - y] = spare;
}

// A launch plan over one or more boards: per-phase work-item prefix sums.
struct Plan {
    int nb;
    int tile_x, tile_y, zseg;     // interior tile (threads in x, y) and z-segment
    Board *const *boards;         // [nb] device pointers
    const long long *int_prefix;  // [nb + 1] interior-kernel items (planes [iz0, iz1))
    const long long *zp_prefix;   // [nb + 1] z-UPML-kernel items (planes [zlo, iz0) and [iz1, nz))
    const long long *slab_prefix; // [nb + 1] slab blocks
    const SlabBlock *slab_blk;    // [n_slab] per-block descriptors
    const long long *dft_prefix;  // [nb + 1] DFT warps
    long long n_int, n_zp, n_slab, n_dft;
    int *work;                    // fused-kernel work counters [interior, z-UPML, two-step] (zeroed before every launch)
    int slots;                    // resident blocks of the fused launch (set by its launcher; orders the items)
    // two-step passes (single-board plans of a depth-2 board)
    long long n_pair;             // two-step items (60 x 8 tiles x z segments of pair_zseg planes)
    int pair_zseg;
    int first_of_pair;            // k_post: the step is the first of a two-step pass (its sources
                                  // inside I were applied by the pass)
    long long n_band_h, n_band;   // band blocks just before slab_blk[0] (E-only first, then H+E; second step of a pair)
    PairConst pc;
};

// TMA descriptor slots of a board (3D maps: x, y, plane).
__host__ __device__ constexpr int tm_e(int set, int c) { return set * 3 + c; }               // E   box_e  x (TY+2)
__host__ __device__ constexpr int tm_h(int set, int c) { return 9 + set * 3 + c; }           // H   box_h  x (TY+1)
constexpr int kTmCid = 18;                                                // ids box_c* x TY
__host__ __device__ constexpr int tm_zd(int box) { return 19 + box; }                         // D~z box_a  x TY
__host__ __device__ constexpr int tm_zb(int box, int par) { return 21 + box * 2 + par; }        // B~z box_a  x (TY+1)
// two-step pass (60 x 8 tiles): E^n and H~^{n-1/2} of sets 0/1 with two halo
// rows below and two (E) or one (H~) above, E^{n+1} of set 2 and the ids with
// one halo row each side
__host__ __device__ constexpr int tp_e(int set, int c) { return 25 + set * 3 + c; }          // E   kPairEW x (8+4)
__host__ __device__ constexpr int tp_h(int set, int c) { return 31 + set * 3 + c; }          // H   kPairEW x (8+3)
__host__ __device__ constexpr int tp_t(int c) { return 37 + c; }                             // E   kPairEW x (8+2), set 2
constexpr int kTpCid = 40;                                                // ids kPairC*W x (8+2)
constexpr int kNumMaps = 41;
constexpr int kPairCols = 60, kPairRows = 8;
constexpr int kPairEW = 72, kPairC8W = 80, kPairC16W = 72;
// TMA box widths for a tile of tx columns (x rounded down to 16 bytes)
__host__ __device__ constexpr int box_up(int x, int m) { return (x + m - 1) / m * m; }
__host__ __device__ constexpr int box_e(int tx) { return box_up(tx + 9, 8); }
__host__ __device__ constexpr int box_h(int tx) { return box_up(tx + 8, 8); }
__host__ __device__ constexpr int box_c8(int tx) { return box_up(tx + 15, 16); }
__host__ __device__ constexpr int box_c16(int tx) { return box_up(tx + 7, 8); }
__host__ __device__ constexpr int box_a(int tx) { return box_up(tx + 5, 4); }

// The fused kernel instantiated for tile_x x tile_y columns stages TMA boxes
// whose sizes are baked into the board's tensor maps (tm_tx x tm_ty).  A
// kernel whose tile differs from the maps' would copy boxes past its shared
// memory stage, so every plan build checks the agreement on the host (no
// device work), and the kernels re-check it per work item (status bit 4).
inline bool fused_maps_match(const Board &h, int tile_x, int tile_y)
{
    if (h.ix1 <= h.ix0 || h.iy1 <= h.iy0) return true;   // no fused region: no maps are used
    return h.tm != nullptr && h.tm_tx == tile_x && h.tm_ty == tile_y;
}

constexpr int kSlabThreads = 128;
constexpr int kSlabKz = 8;          // planes per slab-kernel thread
constexpr int kDftProbeGroup = 4;

enum Phase : int { kPhaseSlabH = 0, kPhaseFusedZ = 1, kPhaseInterior = 2, kPhaseSlabE = 3, kPhasePost = 4, kNumPhases = 5 };

// Launchers (fdtd_kernels.cu).  All enqueue on `st`.
cudaError_t launch_phase(const Plan &plan, int prec, int phase, int grid_cap, cudaStream_t st);
cudaError_t launch_step(const Plan &plan, int prec, int grid_cap, cudaStream_t st);
// A pair of steps with the two-step pass (depth-2 board, even step); or one of its nine launches.
constexpr int kPairLaunches = 9;
constexpr int kPairPhase[kPairLaunches] = {kPhaseSlabH, kPhaseFusedZ, kPhaseInterior, kPhaseSlabE, kPhasePost,
                                           kPhaseSlabH, kPhaseFusedZ, kPhaseSlabE,    kPhasePost};
cudaError_t launch_pair(const Plan &plan, int prec, int grid_cap, cudaStream_t st);
cudaError_t launch_pair_part(const Plan &plan, int prec, int idx, int grid_cap, cudaStream_t st);
cudaError_t launch_dft(const Plan &plan, int grid_cap, cudaStream_t st);
cudaError_t launch_set_i64(long long *p, long long v, cudaStream_t st);
cudaError_t launch_energy(const Board *b_dev, const Board &b_host, double *partials, int n_part,
                          double *out2, cudaStream_t st);
int energy_partials(const Board &b_host);
bool fused_tile_supported(int tile_x, int tile_y);
// Record the message returned by fdtd_last_error on this thread; returns code.
int set_error(int code, const char *msg);
cudaError_t fused_set_smem_limits();
cudaError_t launch_wait_selftest(int *status, unsigned max_polls, cudaStream_t st);

}  // namespace fdtd
