/*
 * fdtd.h -- C-ABI of libfdtd.so: a 3D Yee-grid FDTD solver with a Gedney
 * D/B-form UPML for PCB power/ground structures, computed by hand-written CUDA
 * kernels for sm_103a (GB300).
 *
 * The method ("A Time Domain Approach to Power Integrity for Printed Circuit
 * Boards"): Maxwell's curl equations on the Yee grid of Fig. 2, leapfrog in
 * time (Model section), terminated by a uniaxial PML (Eqs. 1-4) graded by
 * Eq. 5 and backed by a PEC wall; time step bounded by Eq. 7; power and
 * ground planes are perfect conductors (tangential E = 0); excitation by the
 * current pulse of Eq. 8; probe time series reduced to spectra (Results
 * section: FFT of the ground-plane E_z).
 *
 * Conventions used by every call:
 *  - Cells (i, j, k), 0 <= i < nx, 0 <= j < ny, 0 <= k < nz.  Volumes given by
 *    the caller are [nz][ny][nx], x fastest.
 *  - An E edge is named by the node it starts at and its direction:
 *    (i, j, k, FDTD_X) is E_x(i+1/2, j, k), FDTD_Y is E_y(i, j+1/2, k),
 *    FDTD_Z is E_z(i, j, k+1/2).  Node indices run 0..n (inclusive).
 *  - Units: SI (metres, seconds, A/m^2, V/m).
 *  - Host pointers are read during the call only (copied); the library owns
 *    all device memory it allocates, and frees it in fdtd_destroy.
 *  - Every call returns FDTD_OK (0) or a negative fdtd_status; none aborts or
 *    throws.  Work is queued asynchronously on the context's stream: a CUDA
 *    error raised by queued kernels is reported by the next call that
 *    synchronises (fdtd_sync, fdtd_probe_spectra, fdtd_probe_trace,
 *    fdtd_get_field, fdtd_diagnostics).
 *  - A context is not thread-safe; use one context per host thread/stream.
 */
#ifndef FDTD_H
#define FDTD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FDTD_OK = 0,
    FDTD_EINVAL = -1,     /* invalid argument (message from fdtd_last_error) */
    FDTD_ENOMEM = -2,     /* device or host allocation failed */
    FDTD_ECUDA = -3,      /* a CUDA runtime call or kernel failed */
    FDTD_EUNSTABLE = -4,  /* NaN/Inf detected in the fields */
    FDTD_ETIMEOUT = -5,   /* a bounded device-side wait gave up */
    FDTD_ESTATE = -6      /* call not valid in the context's current state */
} fdtd_status;

enum { FDTD_FP32 = 0, FDTD_FP16_STORE = 1 };
enum { FDTD_WALL_PEC = 0, FDTD_WALL_PMC = 1 };
enum { FDTD_X = 0, FDTD_Y = 1, FDTD_Z = 2 };
enum { FDTD_EX = 0, FDTD_EY = 1, FDTD_EZ = 2, FDTD_HX = 3, FDTD_HY = 4, FDTD_HZ = 5 };

typedef struct fdtd_ctx fdtd_ctx;      /* one board, owned by the library */
typedef struct fdtd_batch fdtd_batch;  /* a set of boards stepped together */

/* Grid (Model section; anisotropic cells, the paper's key modification of its
 * base code).  dt <= 0 selects dt = courant * Eq. 7 with v = c. */
typedef struct {
    int nx, ny, nz;
    double dx, dy, dz;
    double courant;
    double dt;
} fdtd_grid;

/* UPML (Eqs. 1-5): depth in cells on faces -x,+x,-y,+y,-z,+z; polynomial
 * order m and kappa_max of Eq. 5; sigma_max = -(m+1) ln(R0) / (2 eta0 d) for
 * a layer of thickness d.  wall[f] is the outer boundary of face f: PEC
 * (tangential E = 0) or PMC (tangential H = 0); a face with depth > 0 must be
 * PEC (the UPML is backed by a perfect conductor, Model section). */
typedef struct {
    int depth[6];
    double m;
    double R0;
    double kappa_max;
    int wall[6];
} fdtd_boundary;

/* PEC region (Results section: planes modelled as perfect conductors): the
 * half-open cell range [i0,i1) x [j0,j1) x [k0,k1); every E edge on the
 * closed node box [i0,i1] x [j0,j1] x [k0,k1] is held at zero.  k1 == k0
 * gives a zero-thickness sheet on node plane k0. */
typedef struct {
    int i0, i1, j0, j1, k0, k1;
} fdtd_box;

/* Read-only facts about a context (for bindings and benchmarks). */
typedef struct {
    int nx, ny, nz;
    double dt;                 /* seconds */
    long long step;            /* leapfrog steps completed (device counter, synchronised read) */
    int n_sources, n_probes;
    int n_total_steps;         /* DFT length N set by fdtd_set_spectrum (0 if unset) */
    int n_bins;                /* DFT bins q = 0..n_bins-1, f_q = q / (N dt) */
    int precision;
    long long interior_nodes;  /* nodes updated by the fused interior kernel */
    long long fused_upml_nodes;/* of those, nodes in z-UPML planes (carry D~z and B~z) */
    long long slab_nodes;      /* nodes updated by the UPML/boundary slab kernels */
    long long device_bytes;    /* device memory held */
    int n_combo;               /* distinct per-node E-coefficient triples */
    long long slab_aux_values; /* auxiliary D~/B~ values held by the slabs (read and written once per step) */
    int pitch;                 /* row pitch of the device field and id arrays, elements (nx + 1 rounded up) */
    int depth;                 /* leapfrog steps per interior pass in effect: 1, or 2 (time blocking) */
} fdtd_info_t;

/* Create a board (Model section, Fig. 1).
 *  grid      grid size, cell sizes [m], Courant number or explicit dt.
 *  mat_ids   host [nz][ny][nx] material index per cell (copied).
 *  eps_r     host [n_mat] relative permittivity per material (> 0).  The
 *            permittivity of an E edge is the mean over the cells sharing it.
 *  pec       host [n_pec] PEC boxes, or NULL if n_pec == 0.
 *  pec_mask  optional host [nz][ny][nx]: nonzero cells are PEC (each acts as a
 *            1x1x1 box); may be NULL.
 *  bnd       UPML depths, grading and outer walls.
 *  precision FDTD_FP32, or FDTD_FP16_STORE (fields stored as FP16 with a
 *            power-of-two scale, arithmetic in FP32; UPML auxiliary D/B
 *            always FP32).  Any other value is FDTD_EINVAL.
 *  stream    cudaStream_t the context enqueues on; NULL makes the library
 *            create (and later destroy) its own non-blocking stream.
 *  out       receives the context.
 * The per-node coefficient ids are built as in fdtd_set_materials: uint8
 * for up to 256 distinct edge coefficient triples, uint16 beyond.
 * Errors: FDTD_EINVAL for bad sizes or walls, a material id outside eps_r,
 * more than 65536 distinct edge coefficient triples, a PMC face with UPML;
 * FDTD_ENOMEM; FDTD_ECUDA. */
int fdtd_create(const fdtd_grid *grid, const uint8_t *mat_ids, const double *eps_r, int n_mat,
                const fdtd_box *pec, int n_pec, const uint8_t *pec_mask,
                const fdtd_boundary *bnd, int precision, void *stream, fdtd_ctx **out);

/* Add a current source (Eq. 8, square restored in the exponent):
 * J(t) = J0 ((t - t0)/tau) exp(-((t - t0)/tau)^2) [A/m^2] on E edge
 * (i, j, k, comp), applied at t = (n + 1/2) dt as E -= dt J / eps.  Several
 * sources may share an edge (they add).  The edge must lie outside the UPML
 * and must not be PEC (FDTD_EINVAL).  Only before the first fdtd_step
 * (FDTD_ESTATE).  src_id may be NULL. */
int fdtd_set_source(fdtd_ctx *ctx, int i, int j, int k, int comp, double J0, double t0, double tau,
                    int *src_id);

/* Add a resistive voltage source on an E edge (Results section: the Table 1
 * run drives the board with V0 = 5 V through Rs = 10 ohm, implemented with
 * semi-implicit update coefficients; the pulse has the shape of Eq. 8,
 * Vs(t) = V0 ((t - t0)/tau) exp(-((t - t0)/tau)^2) at t = (n + 1/2) dt).
 * Vs in series with Rs drives the current I = (l E^{n+1/2} + Vs)/Rs through
 * the edge (l its length, E^{n+1/2} the mean of E^n and E^{n+1}), which
 * enters Ampere's law as curl H - I/A (A = cell volume / l); Vs is the
 * open-circuit voltage of the edge's lower node over its upper one.
 * Rs = +infinity leaves the edge open.  Same edge rules as fdtd_set_source
 * (exists, outside the UPML, not PEC); only before the first step.
 * *src_id (optional) receives the index among all sources. */
int fdtd_set_voltage_source(fdtd_ctx *ctx, int i, int j, int k, int comp, double V0, double t0, double tau,
                            double Rs, int *src_id);

/* Add a probe on E edge (i, j, k, comp): samples E^{n+1} after every step
 * (Results section: ground-plane E_z).  Only before the first fdtd_step. */
int fdtd_add_probe(fdtd_ctx *ctx, int i, int j, int k, int comp, int *probe_id);

/* Set the spectrum: the first n_total_steps samples of every probe are kept
 * (FP32 trace) and accumulated into a running DFT in FP64,
 * X_p(f_q) = dt sum_{n < N} x_p^n exp(-j 2 pi q n / N), f_q = q / (N dt),
 * for f_q <= f_max (f_max <= 0: all bins up to Nyquist, N/2 + 1).  Samples
 * after step N are not recorded.  Only before the first fdtd_step. */
int fdtd_set_spectrum(fdtd_ctx *ctx, double f_max, int n_total_steps);

/* Advance n >= 0 leapfrog steps (H^{n+1/2} from E^n, then E^{n+1} from
 * H^{n+1/2} and J^{n+1/2}, then probes and DFT).  Asynchronous on the
 * context's stream; fields stay on the device between calls. */
int fdtd_step(fdtd_ctx *ctx, int n);

/* fdtd_step with every phase launched directly (no CUDA graph) and timed
 * with CUDA events on the context's stream: phase_ms[0..5] receive the summed
 * device time [ms] of the UPML/boundary slab H kernel, the fused H+E kernel
 * over the z-UPML planes of the interior columns, the fused H+E kernel over
 * the interior planes, the slab E kernel, the source/probe kernel and the
 * running-DFT update over the n steps.  Synchronises.  phase_ms (6 doubles)
 * may not be NULL. */
int fdtd_step_profiled(fdtd_ctx *ctx, int n, double *phase_ms);

/* Copy the running DFT to host out[P][Q][2] (re, im), P = probes, Q = bins;
 * requires max_bins >= Q.  *n_bins receives Q.  Synchronises the stream. */
int fdtd_probe_spectra(fdtd_ctx *ctx, double *out, int max_bins, int *n_bins);

/* Copy the FP32 trace of one probe (V/m, samples 0..len-1) to host out.
 * *len receives min(recorded samples, max_len).  Synchronises. */
int fdtd_probe_trace(fdtd_ctx *ctx, int probe, float *out, int max_len, int *len);

/* Copy one field component to host out[(nz+1)(ny+1)(nx+1)] as FP32 in SI
 * units (E in V/m, H in A/m), node layout [k][j][i]; entries where the
 * component does not exist are 0.  field is FDTD_EX..FDTD_HZ; E is E^{n},
 * H is H^{n-1/2} after n steps.  Synchronises. */
int fdtd_get_field(fdtd_ctx *ctx, int field, float *out);

/* Copy one node plane k (0 <= k <= nz) of a field component to host
 * out[(ny+1)(nx+1)] as FP32 in SI units, layout [j][i], with the conventions
 * of fdtd_get_field: headless snapshots, e.g. of the ground-plane E_z of the
 * Results section's Figs. 3-4.  Synchronises. */
int fdtd_get_plane(fdtd_ctx *ctx, int field, int k, float *out);

/* Discrete energy W = 1/2 V (sum eps E^{n-1}.E^{n-1} + sum mu0 H^{n-3/2}.H^{n-1/2})
 * of the last completed step (exactly conserved by the Yee scheme in a
 * lossless closed box) and max |div B| [T/m] over cells outside the UPML,
 * both reduced in FP64 on the device.  Needs at least one step.  Either
 * output may be NULL.  Synchronises. */
int fdtd_diagnostics(fdtd_ctx *ctx, double *energy, double *max_div_b);

/* Zero all fields, UPML auxiliaries, traces, DFT accumulators and the step
 * counter (sources, probes and geometry stay).  Asynchronous. */
int fdtd_reset(fdtd_ctx *ctx);

/* Checkpoint.  fdtd_save copies the whole solver state to host memory: both
 * field parities, every UPML auxiliary, the probe traces, the running-DFT
 * accumulators and the step counters (the Model section's leapfrog state at
 * step n), after a small header that identifies the board.  With buf == NULL
 * or cap < the size, nothing is copied and *size receives the bytes needed
 * (FDTD_OK).  The caller owns buf.  Synchronises.  Not for a context that is
 * in a batch (FDTD_ESTATE).
 * fdtd_load restores such a checkpoint into a context created from the same
 * problem (grid, boundary, precision, materials, sources, probes, spectrum);
 * a header that does not match returns FDTD_EINVAL and leaves the context
 * unchanged.  Stepping a restored context continues bitwise as the saved
 * one would have (fields and traces; the FP64 spectra agree to rounding,
 * since the running DFT folds samples at chunk boundaries).  Synchronises. */
int fdtd_save(fdtd_ctx *ctx, void *buf, size_t cap, size_t *size);
int fdtd_load(fdtd_ctx *ctx, const void *buf, size_t size);

/* Failure-detection self-test of the bounded device waits.  Launches one
 * block on `stream` (NULL: the default stream) that waits on an mbarrier no
 * one arrives at, with the fused kernel's bounded poll (max_polls polls,
 * 0 = the fused kernel's limit).  The wait must give up and report it:
 * returns FDTD_ETIMEOUT (the expected result), FDTD_OK if the wait did not
 * time out, or FDTD_ECUDA.  Nothing faults, traps or hangs, and the device
 * stays usable.  Allocates one int and frees it.  Synchronises. */
int fdtd_selftest_wait_timeout(void *stream, unsigned max_polls);

/* Replace the material ids of the board (same eps_r table, PEC and ports),
 * rebuilding the per-node edge coefficient ids on the host (in parallel) and
 * copying them to the device, then reset.  The host id buffers (3 bytes per
 * node of the largest board seen) are a process-wide scratch kept for reuse;
 * calls from several threads take turns on it.  Returns FDTD_EINVAL for a
 * material id outside eps_r or more than 65536 distinct coefficient triples,
 * FDTD_ENOMEM if the scratch cannot grow. */
int fdtd_set_materials(fdtd_ctx *ctx, const uint8_t *mat_ids);

/* Halo exchange for one board split into sub-boards along an axis (one
 * sub-board per GPU, or several on one GPU).  On the Yee grid of Fig. 2 the
 * curl of the Model section's leapfrog reaches one node plane, so sub-boards
 * that share one cell layer stay exact if, after every step, each receives
 * from its neighbour the E components tangential to the cut on the node
 * plane it cannot compute itself (its outer wall plane there); H on the
 * shared layer is recomputed on both sides from those E values.
 * The plane is node plane `plane` (0 <= plane <= n along `axis`, 0 = x,
 * 1 = y, 2 = z) of the components in comp_mask (bit f for FDTD_EX..FDTD_HZ),
 * in the context's current state (E^n and H^{n-1/2} after n steps), in its
 * storage type (FP32, or FP16 with the context's scale).
 *  fdtd_halo_pack    copies the plane into dev_buf, a caller-owned device
 *                    buffer of (number of components) x (the two other node
 *                    counts) elements, component-major, rows along x (for a
 *                    y plane: [comp][nz+1][nx+1]).
 *  fdtd_halo_unpack  copies such a buffer back into the plane.
 *  fdtd_halo_copy    copies the plane of src into plane dst_plane of dst
 *                    (contexts on the same or on different devices, same
 *                    storage type and scale, same extents on the other two
 *                    axes, same step count), after the work queued on src's
 *                    stream, on dst's stream.
 * All three are asynchronous on the context's stream (dst's for the copy).
 * Errors: FDTD_EINVAL (bad axis, plane, mask, shapes, NULL buffer),
 * FDTD_ESTATE (a context in a batch; contexts at different steps). */
int fdtd_halo_pack(fdtd_ctx *ctx, int axis, int plane, unsigned comp_mask, void *dev_buf);
int fdtd_halo_unpack(fdtd_ctx *ctx, int axis, int plane, unsigned comp_mask, const void *dev_buf);
int fdtd_halo_copy(fdtd_ctx *dst, int dst_plane, fdtd_ctx *src, int src_plane, int axis, unsigned comp_mask);

/* Host only: the per-node edge coefficients fdtd_create builds for a
 * geometry (arguments as in fdtd_create), without touching a device.  The
 * coefficient of an E edge is 1/eps_r with eps_r the mean over the cells
 * sharing the edge; it is 0 on PEC edges and on edges tangential to a PEC
 * wall.  ids: host [nz+1][ny+1][nx+1] (caller-owned) receives the node's row
 * in table; table: host [max_rows][4] (caller-owned) receives the distinct
 * (ce_x, ce_y, ce_z, 0) rows in order of first appearance by plane; *n_rows
 * their count.  Entries of edges that do not exist (i = nx for x edges, and so
 * on) are 0.  Errors: as fdtd_create, and FDTD_EINVAL when the table needs
 * more than max_rows rows (at most 65536). */
int fdtd_node_coefficients(const fdtd_grid *grid, const uint8_t *mat_ids, const double *eps_r, int n_mat,
                           const fdtd_box *pec, int n_pec, const uint8_t *pec_mask, const fdtd_boundary *bnd,
                           uint16_t *ids, float *table, int max_rows, int *n_rows);

/* Host only: the device memory [bytes] a board needs, without touching a
 * device: what fdtd_create allocates for the grid and boundary (fields of
 * two field sets in the given precision, per-node coefficient ids counted at
 * 16 bits with a 65536-row table, the 1D UPML factors, the auxiliaries of the
 * UPML boxes as fdtd_create lays them out, counters and scratch), plus what
 * the first step adds: the tensor maps, n_sources sources, n_probes probes
 * with traces of n_total_steps samples and the running DFT's bins up to f_max
 * (as in fdtd_set_spectrum).  An upper bound on fdtd_info's device_bytes by at
 * most one byte per node and the table's 1 MB (8-bit ids when at most 256
 * edge coefficient triples occur), at depth 1 (fdtd_tuning: depth 2 adds a
 * third field set).  Serves admission by memory budget.
 * Errors: FDTD_EINVAL for the cases fdtd_create refuses on grid, boundary or
 * precision. */
int fdtd_device_bytes(const fdtd_grid *grid, const fdtd_boundary *bnd, int precision, int n_sources, int n_probes,
                      int n_total_steps, double f_max, long long *bytes);

/* Fill *info (synchronises to read the step counter). */
int fdtd_info(fdtd_ctx *ctx, fdtd_info_t *info);

/* Wait for all queued work; returns the first CUDA error or NaN/Inf found
 * by the stability check (FDTD_EUNSTABLE). */
int fdtd_sync(fdtd_ctx *ctx);

/* Release the context and its device memory (synchronises first). */
void fdtd_destroy(fdtd_ctx *ctx);

/* Static text for a status code. */
const char *fdtd_strerror(int code);

/* Text of the last FDTD_EINVAL / FDTD_ECUDA raised on this host thread. */
const char *fdtd_last_error(void);

/* Discrete field energy and max |div B| of fields the caller owns, with no
 * device allocation.  The paper has no counterpart: this is a service for
 * callers that cannot allocate device memory when they need the check --
 * code under a fixed memory budget or pool that must not grow, real-time
 * loops that forbid allocator calls, hosts that hand the library only
 * pre-registered buffers.  It computes the same quantities as
 * fdtd_diagnostics, from raw arrays:
 *  fields   9 device pointers to FP32 [nz+1][ny+1][pitch] arrays (x fastest,
 *           node layout as fdtd_get_field): E^n x,y,z [V/m], H^{n-1/2} x,y,z
 *           and H^{n+1/2} x,y,z [A/m]
 *  eps_r    3 device pointers to the per-edge relative permittivity of the
 *           E_x, E_y, E_z edges in the same layout, or NULL (all 1)
 *  nx,ny,nz cells; pitch >= nx+1 elements; dx,dy,dz cell sizes [m]
 *  upml_depth  6 UPML depths (NULL: none), each >= 0 and the two of an axis
 *           summing to at most its cells (else FDTD_EINVAL): div B is taken
 *           over the cells outside them
 *  stream   cudaStream_t to run on (NULL: legacy default stream)
 *  energy, max_div_b  host outputs [J] and [T/m] (either may be NULL); a NaN
 *           in H^{n+1/2} inside the window makes max_div_b NaN
 * Scratch space is a fixed static device array that each GPU loading the
 * library holds until exit; grids above 33,554,432 nodes are rejected with
 * FDTD_EINVAL.  The first call on a device (and the first after a
 * cudaDeviceReset) resolves the array's device address with that device
 * current, so it should come before any stream capture.  All calls share the
 * array: calls whose work overlaps on the GPU race.  The call copies its two
 * results to host memory and synchronises the stream before returning;
 * errors as the other calls (message from fdtd_last_error). */
int fdtd_energy_static(const float *const fields[9], const float *const eps_r[3], int nx, int ny, int nz,
                       int pitch, double dx, double dy, double dz, const int upml_depth[6], void *stream,
                       double *energy, double *max_div_b);

/* ---------------- batching (many boards, one launch per phase) -------------
 * A batch steps many boards with one kernel launch per phase (UPML H, interior
 * fused H+E, UPML E, sources/probes) over a packed list of (board, tile) work
 * items, replayed as one CUDA graph per chunk of steps.  Each board's
 * arithmetic is identical to stepping it alone.  Boards keep their own device
 * state and may join or leave between calls.  All boards must share the
 * batch's stream (the batch uses its own; member contexts must not be
 * stepped on their own while in a batch). */

/* Create an empty batch on stream (NULL: own stream). */
int fdtd_batch_create(void *stream, fdtd_batch **out);

/* Add a board that will run n_steps more steps (its ports and spectrum must
 * be set).  FDTD_EINVAL if it is already in a batch. */
int fdtd_batch_add(fdtd_batch *b, fdtd_ctx *ctx, int n_steps);

/* Remove a board (its state stays valid; synchronises the batch stream). */
int fdtd_batch_remove(fdtd_batch *b, fdtd_ctx *ctx);

/* Advance every member by min(n, its remaining steps); members that reach
 * their target stop while the others continue.  *n_done (may be NULL)
 * receives the number of members that have no steps left. */
int fdtd_batch_step(fdtd_batch *b, int n, int *n_done);

/* Remaining steps of one member (synchronises). */
int fdtd_batch_remaining(fdtd_batch *b, fdtd_ctx *ctx, long long *remaining);

/* Wait for the batch stream. */
int fdtd_batch_sync(fdtd_batch *b);

/* Destroy the batch (members stay alive and are detached). */
void fdtd_batch_destroy(fdtd_batch *b);

/* Tuning knobs of the kernels (autotuner): the fused-kernel tile (tile_x
 * columns: 62 or 124, i.e. one or two strips of 62 columns; tile_y rows: 4
 * or 8; a 62x8 tile is worked by four compute warps of 2 rows, a 124x8 tile
 * by two warps of 4 rows per strip; default 62x8), the z-segment length
 * (planes one tile marches before the next work item; default 10) and the
 * number of steps per CUDA graph (default 16).  depth is the number of
 * leapfrog steps one sweep over the interior region advances (time blocking,
 * Model section: the leapfrog's H and E updates of two steps in one pass):
 * 1 (default) or 2.  With depth 2 a single board keeps a third field set
 * (6 x nodes more field values) and runs pairs of steps as one two-step
 * interior pass plus the slab, z-UPML and source launches of both steps.
 * With FP32 storage the results are bit-identical to depth 1.  With FP16
 * storage the E update of the interior region's one-node outer layer reads
 * the stored (FP16) H~ where depth 1 uses the unrounded value, a difference at
 * the storage rounding level.  Depth 2 takes effect on boards
 * whose interior spans at least 3 nodes per axis, whose fused region starts
 * at an even x, and whose top wall is a z-UPML or PEC (fdtd_info reports the
 * depth in effect); batches run depth 1.  pair_zseg is the z-segment length
 * of the two-step pass (default 38, >= 2).  Values <= 0 keep the current
 * setting; unsupported tiles are rejected with FDTD_EINVAL.  Applies to
 * launches queued afterwards. */
typedef struct {
    int tile_x, tile_y, zseg, graph_chunk;
    int depth, pair_zseg;
} fdtd_tuning;

int fdtd_set_tuning(fdtd_ctx *ctx, const fdtd_tuning *t);
int fdtd_batch_set_tuning(fdtd_batch *b, const fdtd_tuning *t);

#ifdef __cplusplus
}
#endif

#endif /* FDTD_H */
