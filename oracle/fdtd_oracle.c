/*
 * fdtd_oracle.c -- plain, slow, FP64 CPU FDTD used ONLY as test infrastructure.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg (and
 * `bench.py --impl reference`) may build, load or call this file.  The CUDA
 * library never links or calls it, and it shares no code with the CUDA path:
 * the only common thing is the seeded Problem description (geometry, ports).
 *
 * What it computes (paper: Model section, Eqs. 1-5, 7, 8; Results section):
 *  - Yee grid (Fig. 2): E_x(i+1/2,j,k), E_y(i,j+1/2,k), E_z(i,j,k+1/2),
 *    H_x(i,j+1/2,k+1/2), H_y(i+1/2,j,k+1/2), H_z(i+1/2,j+1/2,k); all fields
 *    start at zero; leapfrog in time, H at half steps (Model section).
 *  - Unified UPML treatment everywhere (Eqs. 1-4): every E component carries
 *    its D and every H component its B; in the model space sigma=0, kappa=1 so
 *    the two-step update reduces to plain Yee.  Eq. 4 is discretised with
 *    central differences in time and the time average of the sigma term:
 *       kappa_y dD_x/dt + sigma_y/eps0 D_x = (curl H)_x - J_x
 *       kappa_x dD_x/dt + sigma_x/eps0 D_x = eps (kappa_z dE_x/dt + sigma_z/eps0 E_x)
 *    (the second from D_x = eps (s_z/s_x) E_x), cyclic in x->y->z; the same
 *    two-step process gives B then H with mu0 in place of eps.
 *  - Polynomial grading (Eq. 5) with rho measured from the UPML interface,
 *    sigma_max = -(m+1) ln(R0) / (2 eta0 d) (the paper gives no sigma_max;
 *    this is the usual choice for a target reflection R0), outer wall PEC.
 *  - Time step from Eq. 7 with v = c (fastest medium) times a Courant number.
 *  - PEC sheets: tangential E held at zero on every edge of a PEC box
 *    (Results: the planes are perfect conductors).  Outer faces are PEC
 *    (tangential E = 0) or PMC (odd mirror of tangential H across the wall).
 *  - Current source (Eq. 8): J(t) = J0 ((t-t0)/tau) exp(-((t-t0)/tau)^2) at
 *    t = (n+1/2) dt on one E edge, entering Ampere's law as curl H - J.
 *  - Resistive voltage source (Results section: V0 and Rs on one E edge, the
 *    same pulse shape): a voltage Vs(t) in series with Rs across the edge of
 *    length l and cross-section A = V/l.  Its current I = (l E + Vs)/Rs at
 *    n+1/2, with E^{n+1/2} = (E^n + E^{n+1})/2, enters Ampere's law as
 *    curl H - I/A, which is solved for E^{n+1} at that edge (so Vs is the
 *    open-circuit voltage of the edge's lower node over its upper one:
 *    E = -Vs/l when no current flows).  Edges must lie outside the UPML.
 *  - Probes sample E^{n+1}; running DFT X(f_q) = dt sum_n x^n exp(-j 2 pi q n/N)
 *    in FP64 (Results section: FFT of the ground-plane E_z).
 *  - Diagnostics: discrete energy W^n = 1/2 V (sum eps E^n.E^n +
 *    sum mu0 H^{n-1/2}.H^{n+1/2}) (samples on the outer node planes weighted by
 *    their half dual cell) and max |div B| over cells outside the UPML.
 *
 * Pins (tests/test_oracle_*.py): cavity closed form of Eq. 9 (PMC side walls)
 * and the Yee dispersion relation, energy conservation and the discrete energy
 * balance with a source, div B = 0 to round-off, UPML reflection below -40 dB,
 * running DFT = FFT, superposition, mirror symmetry, Table 1 of the paper.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define PI 3.14159265358979323846
static const double C0 = 299792458.0;            /* speed of light, m/s */
static const double MU0 = 4.0e-7 * PI;           /* H/m */
#define EPS0 (1.0 / (MU0 * C0 * C0))             /* F/m */
#define ETA0 (MU0 * C0)                          /* ohm */

enum { WALL_PEC = 0, WALL_PMC = 1 };

typedef struct {
    int nx, ny, nz;
    double dx, dy, dz;
    double courant;
    double dt;                      /* > 0 overrides courant */
    const uint8_t *mat;             /* [nz][ny][nx] cell material ids */
    const double *eps_r;            /* [n_mat] */
    int n_mat;
    const int32_t *pec_boxes;       /* [n_pec][6] i0,i1,j0,j1,k0,k1 (cells, half-open) */
    int n_pec;
    int upml_depth[6];              /* -x,+x,-y,+y,-z,+z */
    double upml_m, upml_R0, upml_kappa_max;
    int walls[6];
    const int32_t *src;             /* [n_src][4] i,j,k,comp */
    const double *src_prm;          /* [n_src][3] J0, t0, tau */
    int n_src;
    const int32_t *probe;           /* [n_probe][4] */
    int n_probe;
    int n_steps;
    int n_bins;
    int n_threads;
    const int32_t *vsrc;            /* [n_vsrc][4] i,j,k,comp */
    const double *vsrc_prm;         /* [n_vsrc][4] V0 [V], t0, tau [s], Rs [ohm] */
    int n_vsrc;
} oracle_problem;

typedef struct {
    double dt;                      /* out */
    double *trace;                  /* [n_probe][n_steps] or NULL */
    double *dft;                    /* [n_probe][n_bins][2] or NULL */
    double *energy;                 /* [n_steps] or NULL */
    double *divb;                   /* [n_steps] or NULL */
    double *src_wave;               /* [n_steps] or NULL: J^{n+1/2} of source 0 */
    double *fields;                 /* [6][(nz+1)(ny+1)(nx+1)] or NULL */
    double *vsrc_current;           /* [n_steps] or NULL: I^{n+1/2} of voltage source 0 [A] */
} oracle_outputs;

/* Eq. 9: resonant frequency of the PEC/PMC cavity model of a board. */
double oracle_cavity_fr(int m, int n, double Lx, double Ly, double Lz, double eps_r)
{
    double a = m / (2.0 * (Lx + Lz / 2.0));
    double b = n / (2.0 * (Ly + Lz / 2.0));
    return C0 / sqrt(eps_r) * sqrt(a * a + b * b);
}

/* Eq. 7 with v = c: the largest stable time step of the grid. */
double oracle_cfl_dt(double dx, double dy, double dz)
{
    return 1.0 / (C0 * sqrt(1.0 / (dx * dx) + 1.0 / (dy * dy) + 1.0 / (dz * dz)));
}

/* Eq. 8 (square restored in the exponent, (t-t0)/tau in front). */
double oracle_pulse(double J0, double t0, double tau, double t)
{
    double u = (t - t0) / tau;
    return J0 * u * exp(-u * u);
}

/* Eq. 5 grading at coordinate x (in cells; half-integers allowed) along an
 * axis of N cells with UPML depth dlo / dhi cells on its low / high faces. */
static void grade(double x, int N, int dlo, int dhi, double smax_lo, double smax_hi,
                  double m, double kmax, double *sigma, double *kappa)
{
    *sigma = 0.0;
    *kappa = 1.0;
    if (dlo > 0 && x < dlo) {
        double r = pow((dlo - x) / dlo, m);
        *sigma = r * smax_lo;
        *kappa = 1.0 + (kmax - 1.0) * r;
    } else if (dhi > 0 && x > N - dhi) {
        double r = pow((x - (N - dhi)) / dhi, m);
        *sigma = r * smax_hi;
        *kappa = 1.0 + (kmax - 1.0) * r;
    }
}

/* Per-axis time-stepping factors at one position (from Eq. 4 discretised). */
typedef struct { double ca, cb, cp, cm; } tcoef;

static tcoef tc(double sigma, double kappa, double dt)
{
    tcoef c;
    double p = 2.0 * EPS0 * kappa + sigma * dt;
    double q = 2.0 * EPS0 * kappa - sigma * dt;
    c.ca = q / p;               /* multiplies the old value */
    c.cb = 2.0 * EPS0 * dt / p; /* multiplies the curl */
    c.cp = p;                   /* new-value factor in the D->E / B->H step */
    c.cm = q;                   /* old-value factor */
    return c;
}

/* H component c at index (i,j,k), where one index may lie one step outside the
 * component's range: across a PMC wall the tangential H is mirrored with a
 * sign change (so it vanishes on the wall); across a PEC wall it is zero (the
 * E edge being updated is then PEC anyway). */
static inline double hget(double *const H[3], int c, int i, int j, int k, int nx, int ny, int nz,
                          const int walls[6])
{
    const int NX = nx + 1, NY = ny + 1;
    int hi[3];
    hi[0] = (c == 0) ? nx : nx - 1;
    hi[1] = (c == 1) ? ny : ny - 1;
    hi[2] = (c == 2) ? nz : nz - 1;
    if (i >= 0 && j >= 0 && k >= 0 && i <= hi[0] && j <= hi[1] && k <= hi[2])
        return H[c][((size_t)k * NY + j) * NX + i];
    int idx[3] = {i, j, k};
    for (int a = 0; a < 3; a++) {
        if (idx[a] < 0) {
            if (walls[2 * a] != WALL_PMC) return 0.0;
            idx[a] = 0;
            return -H[c][((size_t)idx[2] * NY + idx[1]) * NX + idx[0]];
        }
        if (idx[a] > hi[a]) {
            if (walls[2 * a + 1] != WALL_PMC) return 0.0;
            idx[a] = hi[a];
            return -H[c][((size_t)idx[2] * NY + idx[1]) * NX + idx[0]];
        }
    }
    return H[c][((size_t)k * NY + j) * NX + i];
}

/* Dual-cell weight of a field sample in the discrete energy: a component that
 * sits on a node plane (integer position along an axis) at the first or last
 * node of that axis owns only half a dual cell along it.  E_c is integer along
 * the two axes other than c; H_c only along axis c. */
static double dualw(int c, int is_h, int i, int j, int k, int nx, int ny, int nz)
{
    const int idx[3] = {i, j, k}, N[3] = {nx, ny, nz};
    double w = 1.0;
    for (int a = 0; a < 3; a++) {
        int integer_axis = is_h ? (a == c) : (a != c);
        if (integer_axis && (idx[a] == 0 || idx[a] == N[a])) w *= 0.5;
    }
    return w;
}

int oracle_run(const oracle_problem *P, oracle_outputs *O)
{
    const int nx = P->nx, ny = P->ny, nz = P->nz;
    const int NX = nx + 1, NY = ny + 1, NZ = nz + 1;
    const size_t nn = (size_t)NX * NY * NZ;
    const double dx = P->dx, dy = P->dy, dz = P->dz;
    const double dt = P->dt > 0 ? P->dt : P->courant * oracle_cfl_dt(dx, dy, dz);
    const double V = dx * dy * dz;
    const int nt = P->n_threads > 0 ? P->n_threads : 1;
    (void)nt;
    O->dt = dt;
    if (nx < 1 || ny < 1 || nz < 1) return -1;
    for (int f = 0; f < 6; f++)
        if (P->upml_depth[f] > 0 && P->walls[f] != WALL_PEC) return -2;

#define AT(a, i, j, k) (a)[((size_t)(k) * NY + (j)) * NX + (i)]

    double *E[3], *H[3], *D[3], *B[3], *J[3], *epsE[3];
    uint8_t *pec[3];
    for (int c = 0; c < 3; c++) {
        E[c] = calloc(nn, sizeof(double));
        H[c] = calloc(nn, sizeof(double));
        D[c] = calloc(nn, sizeof(double));
        B[c] = calloc(nn, sizeof(double));
        J[c] = calloc(nn, sizeof(double));
        epsE[c] = calloc(nn, sizeof(double));
        pec[c] = calloc(nn, 1);
        if (!E[c] || !H[c] || !D[c] || !B[c] || !J[c] || !epsE[c] || !pec[c]) return -3;
    }

    /* --- edge permittivity: mean of the existing cells sharing the edge --- */
#define EPSCELL(i, j, k) (P->eps_r[P->mat[((size_t)(k) * ny + (j)) * nx + (i)]])
    for (int k = 0; k <= nz; k++)
        for (int j = 0; j <= ny; j++)
            for (int i = 0; i <= nx; i++) {
                double s; int n;
                if (i < nx) {   /* E_x: cells (i, j-1..j, k-1..k) */
                    s = 0; n = 0;
                    for (int b = k - 1; b <= k; b++)
                        for (int a = j - 1; a <= j; a++)
                            if (a >= 0 && a < ny && b >= 0 && b < nz) { s += EPSCELL(i, a, b); n++; }
                    AT(epsE[0], i, j, k) = s / n;
                }
                if (j < ny) {   /* E_y: cells (i-1..i, j, k-1..k) */
                    s = 0; n = 0;
                    for (int b = k - 1; b <= k; b++)
                        for (int a = i - 1; a <= i; a++)
                            if (a >= 0 && a < nx && b >= 0 && b < nz) { s += EPSCELL(a, j, b); n++; }
                    AT(epsE[1], i, j, k) = s / n;
                }
                if (k < nz) {   /* E_z: cells (i-1..i, j-1..j, k) */
                    s = 0; n = 0;
                    for (int b = j - 1; b <= j; b++)
                        for (int a = i - 1; a <= i; a++)
                            if (a >= 0 && a < nx && b >= 0 && b < ny) { s += EPSCELL(a, b, k); n++; }
                    AT(epsE[2], i, j, k) = s / n;
                }
            }

    /* --- PEC edges: every edge on the closed node box of a PEC cell box --- */
    for (int b = 0; b < P->n_pec; b++) {
        const int32_t *q = P->pec_boxes + 6 * b;
        int i0 = q[0], i1 = q[1], j0 = q[2], j1 = q[3], k0 = q[4], k1 = q[5];
        for (int k = k0; k <= k1; k++)
            for (int j = j0; j <= j1; j++)
                for (int i = i0; i <= i1; i++) {
                    if (i < 0 || j < 0 || k < 0 || i > nx || j > ny || k > nz) continue;
                    if (i < i1 && i < nx) AT(pec[0], i, j, k) = 1;
                    if (j < j1 && j < ny) AT(pec[1], i, j, k) = 1;
                    if (k < k1 && k < nz) AT(pec[2], i, j, k) = 1;
                }
    }
    /* PEC outer walls: tangential E on the face is zero */
    for (int k = 0; k <= nz; k++)
        for (int j = 0; j <= ny; j++)
            for (int i = 0; i <= nx; i++) {
                int onx = (i == 0 && P->walls[0] == WALL_PEC) || (i == nx && P->walls[1] == WALL_PEC);
                int ony = (j == 0 && P->walls[2] == WALL_PEC) || (j == ny && P->walls[3] == WALL_PEC);
                int onz = (k == 0 && P->walls[4] == WALL_PEC) || (k == nz && P->walls[5] == WALL_PEC);
                if (ony || onz) AT(pec[0], i, j, k) = 1;
                if (onx || onz) AT(pec[1], i, j, k) = 1;
                if (onx || ony) AT(pec[2], i, j, k) = 1;
            }

    /* --- Eq. 5 grading per axis at integer (node) and half (mid) positions --- */
    const int Nw[3] = {nx, ny, nz};
    const double dw[3] = {dx, dy, dz};
    tcoef *ci[3], *chf[3];   /* ci[w][i]: at node i; chf[w][i]: at i+1/2 */
    for (int w = 0; w < 3; w++) {
        int dlo = P->upml_depth[2 * w], dhi = P->upml_depth[2 * w + 1];
        double lnR = log(P->upml_R0);
        double smax_lo = dlo > 0 ? -(P->upml_m + 1.0) * lnR / (2.0 * ETA0 * dlo * dw[w]) : 0.0;
        double smax_hi = dhi > 0 ? -(P->upml_m + 1.0) * lnR / (2.0 * ETA0 * dhi * dw[w]) : 0.0;
        ci[w] = malloc(sizeof(tcoef) * (Nw[w] + 1));
        chf[w] = malloc(sizeof(tcoef) * (Nw[w] + 1));
        for (int i = 0; i <= Nw[w]; i++) {
            double s, kk;
            grade((double)i, Nw[w], dlo, dhi, smax_lo, smax_hi, P->upml_m, P->upml_kappa_max, &s, &kk);
            ci[w][i] = tc(s, kk, dt);
            grade(i + 0.5, Nw[w], dlo, dhi, smax_lo, smax_hi, P->upml_m, P->upml_kappa_max, &s, &kk);
            chf[w][i] = tc(s, kk, dt);
        }
    }

    /* --- H neighbour fetch with the outer-wall rule for indices one past the grid --- */
#define HGET(c, i, j, k) hget(H, c, i, j, k, nx, ny, nz, P->walls)

    /* --- voltage-source edges: existing, outside the UPML, not PEC, Rs > 0 --- */
    int bad = 0;
    double *ve_old = calloc(P->n_vsrc > 0 ? P->n_vsrc : 1, sizeof(double));
    double *vd_old = calloc(P->n_vsrc > 0 ? P->n_vsrc : 1, sizeof(double));
    if (!ve_old || !vd_old) bad = -3;
    for (int s = 0; s < P->n_vsrc && !bad; s++) {
        const int32_t *q = P->vsrc + 4 * s;
        const int id[3] = {q[0], q[1], q[2]}, c = q[3];
        if (c < 0 || c > 2) { bad = -4; break; }
        for (int w = 0; w < 3; w++) {
            const int hi = w == c ? Nw[w] - 1 : Nw[w];
            if (id[w] < 0 || id[w] > hi) bad = -4;
        }
        if (bad) break;
        for (int w = 0; w < 3; w++) {
            double sg, kp;
            const int dlo = P->upml_depth[2 * w], dhi = P->upml_depth[2 * w + 1];
            grade(id[w] + (w == c ? 0.5 : 0.0), Nw[w], dlo, dhi, 1.0, 1.0, P->upml_m, P->upml_kappa_max, &sg, &kp);
            if (sg != 0.0 || kp != 1.0) bad = -4;
        }
        if (AT(pec[c], id[0], id[1], id[2])) bad = -5;
        if (!(P->vsrc_prm[4 * s + 3] > 0.0)) bad = -6;
    }

    const int Q = P->n_bins;
    const int N = bad ? 0 : P->n_steps;
    for (int n = 0; n < N; n++) {
        /* ---- electric energy of E^n ---- */
        double we = 0.0, wh = 0.0;
        if (O->energy) {
            #pragma omp parallel for num_threads(nt) reduction(+ : we) schedule(static)
            for (int k = 0; k <= nz; k++)
                for (int j = 0; j <= ny; j++)
                    for (int i = 0; i <= nx; i++)
                        for (int c = 0; c < 3; c++) {
                            double e = AT(E[c], i, j, k);
                            if (e != 0.0) we += dualw(c, 0, i, j, k, nx, ny, nz) * EPS0 * AT(epsE[c], i, j, k) * e * e;
                        }
        }

        /* ---- B^{n+1/2}, H^{n+1/2} from E^n (Faraday with UPML) ---- */
        #pragma omp parallel for num_threads(nt) reduction(+ : wh) schedule(static)
        for (int k = 0; k <= nz; k++)
            for (int j = 0; j <= ny; j++)
                for (int i = 0; i <= nx; i++) {
                    if (j < ny && k < nz) {  /* H_x(i, j+1/2, k+1/2): B axis y, H axis z, B->H axis x */
                        double curl = (AT(E[2], i, j + 1, k) - AT(E[2], i, j, k)) / dy
                                    - (AT(E[1], i, j, k + 1) - AT(E[1], i, j, k)) / dz;
                        tcoef a = chf[1][j], b = chf[2][k], c = ci[0][i];
                        double Bo = AT(B[0], i, j, k);
                        double Bn = a.ca * Bo - a.cb * curl;
                        double Ho = AT(H[0], i, j, k);
                        double Hn = b.ca * Ho + (c.cp * Bn - c.cm * Bo) / (MU0 * b.cp);
                        AT(B[0], i, j, k) = Bn; AT(H[0], i, j, k) = Hn;
                        wh += dualw(0, 1, i, j, k, nx, ny, nz) * MU0 * Ho * Hn;
                    }
                    if (i < nx && k < nz) {  /* H_y(i+1/2, j, k+1/2): B axis z, H axis x, B->H axis y */
                        double curl = (AT(E[0], i, j, k + 1) - AT(E[0], i, j, k)) / dz
                                    - (AT(E[2], i + 1, j, k) - AT(E[2], i, j, k)) / dx;
                        tcoef a = chf[2][k], b = chf[0][i], c = ci[1][j];
                        double Bo = AT(B[1], i, j, k);
                        double Bn = a.ca * Bo - a.cb * curl;
                        double Ho = AT(H[1], i, j, k);
                        double Hn = b.ca * Ho + (c.cp * Bn - c.cm * Bo) / (MU0 * b.cp);
                        AT(B[1], i, j, k) = Bn; AT(H[1], i, j, k) = Hn;
                        wh += dualw(1, 1, i, j, k, nx, ny, nz) * MU0 * Ho * Hn;
                    }
                    if (i < nx && j < ny) {  /* H_z(i+1/2, j+1/2, k): B axis x, H axis y, B->H axis z */
                        double curl = (AT(E[1], i + 1, j, k) - AT(E[1], i, j, k)) / dx
                                    - (AT(E[0], i, j + 1, k) - AT(E[0], i, j, k)) / dy;
                        tcoef a = chf[0][i], b = chf[1][j], c = ci[2][k];
                        double Bo = AT(B[2], i, j, k);
                        double Bn = a.ca * Bo - a.cb * curl;
                        double Ho = AT(H[2], i, j, k);
                        double Hn = b.ca * Ho + (c.cp * Bn - c.cm * Bo) / (MU0 * b.cp);
                        AT(B[2], i, j, k) = Bn; AT(H[2], i, j, k) = Hn;
                        wh += dualw(2, 1, i, j, k, nx, ny, nz) * MU0 * Ho * Hn;
                    }
                }
        if (O->energy) O->energy[n] = 0.5 * V * (we + wh);

        /* ---- div B over cells outside the UPML ---- */
        if (O->divb) {
            double mx = 0.0;
            int xlo = P->upml_depth[0], xhi = nx - P->upml_depth[1];
            int ylo = P->upml_depth[2], yhi = ny - P->upml_depth[3];
            int zlo = P->upml_depth[4], zhi = nz - P->upml_depth[5];
            for (int k = zlo; k < zhi; k++)
                for (int j = ylo; j < yhi; j++)
                    for (int i = xlo; i < xhi; i++) {
                        double dv = (AT(B[0], i + 1, j, k) - AT(B[0], i, j, k)) / dx
                                  + (AT(B[1], i, j + 1, k) - AT(B[1], i, j, k)) / dy
                                  + (AT(B[2], i, j, k + 1) - AT(B[2], i, j, k)) / dz;
                        if (fabs(dv) > mx) mx = fabs(dv);
                    }
            O->divb[n] = mx;
        }

        /* ---- source currents J^{n+1/2} (Eq. 8) ---- */
        double t_half = (n + 0.5) * dt;
        for (int s = 0; s < P->n_src; s++) {
            const int32_t *q = P->src + 4 * s;
            AT(J[q[3]], q[0], q[1], q[2]) = 0.0;
        }
        for (int s = 0; s < P->n_src; s++) {
            const int32_t *q = P->src + 4 * s;
            const double *pr = P->src_prm + 3 * s;
            double js = oracle_pulse(pr[0], pr[1], pr[2], t_half);
            AT(J[q[3]], q[0], q[1], q[2]) += js;
            if (s == 0 && O->src_wave) O->src_wave[n] = js;
        }

        /* E^n and D^n on the voltage-source edges (their update is redone below) */
        for (int s = 0; s < P->n_vsrc; s++) {
            const int32_t *q = P->vsrc + 4 * s;
            ve_old[s] = AT(E[q[3]], q[0], q[1], q[2]);
            vd_old[s] = AT(D[q[3]], q[0], q[1], q[2]);
        }

        /* ---- D^{n+1}, E^{n+1} from H^{n+1/2} and J^{n+1/2} (Ampere with UPML) ---- */
        #pragma omp parallel for num_threads(nt) schedule(static)
        for (int k = 0; k <= nz; k++)
            for (int j = 0; j <= ny; j++)
                for (int i = 0; i <= nx; i++) {
                    if (i < nx) {  /* E_x(i+1/2, j, k): D axis y, E axis z, D->E axis x */
                        if (AT(pec[0], i, j, k)) { AT(E[0], i, j, k) = 0.0; AT(D[0], i, j, k) = 0.0; }
                        else {
                            double curl = (HGET(2, i, j, k) - HGET(2, i, j - 1, k)) / dy
                                        - (HGET(1, i, j, k) - HGET(1, i, j, k - 1)) / dz;
                            tcoef a = ci[1][j], b = ci[2][k], c = chf[0][i];
                            double Do = AT(D[0], i, j, k);
                            double Dn = a.ca * Do + a.cb * (curl - AT(J[0], i, j, k));
                            double eps = EPS0 * AT(epsE[0], i, j, k);
                            AT(E[0], i, j, k) = b.ca * AT(E[0], i, j, k) + (c.cp * Dn - c.cm * Do) / (eps * b.cp);
                            AT(D[0], i, j, k) = Dn;
                        }
                    }
                    if (j < ny) {  /* E_y(i, j+1/2, k): D axis z, E axis x, D->E axis y */
                        if (AT(pec[1], i, j, k)) { AT(E[1], i, j, k) = 0.0; AT(D[1], i, j, k) = 0.0; }
                        else {
                            double curl = (HGET(0, i, j, k) - HGET(0, i, j, k - 1)) / dz
                                        - (HGET(2, i, j, k) - HGET(2, i - 1, j, k)) / dx;
                            tcoef a = ci[2][k], b = ci[0][i], c = chf[1][j];
                            double Do = AT(D[1], i, j, k);
                            double Dn = a.ca * Do + a.cb * (curl - AT(J[1], i, j, k));
                            double eps = EPS0 * AT(epsE[1], i, j, k);
                            AT(E[1], i, j, k) = b.ca * AT(E[1], i, j, k) + (c.cp * Dn - c.cm * Do) / (eps * b.cp);
                            AT(D[1], i, j, k) = Dn;
                        }
                    }
                    if (k < nz) {  /* E_z(i, j, k+1/2): D axis x, E axis y, D->E axis z */
                        if (AT(pec[2], i, j, k)) { AT(E[2], i, j, k) = 0.0; AT(D[2], i, j, k) = 0.0; }
                        else {
                            double curl = (HGET(1, i, j, k) - HGET(1, i - 1, j, k)) / dx
                                        - (HGET(0, i, j, k) - HGET(0, i, j - 1, k)) / dy;
                            tcoef a = ci[0][i], b = ci[1][j], c = chf[2][k];
                            double Do = AT(D[2], i, j, k);
                            double Dn = a.ca * Do + a.cb * (curl - AT(J[2], i, j, k));
                            double eps = EPS0 * AT(epsE[2], i, j, k);
                            AT(E[2], i, j, k) = b.ca * AT(E[2], i, j, k) + (c.cp * Dn - c.cm * Do) / (eps * b.cp);
                            AT(D[2], i, j, k) = Dn;
                        }
                    }
                }

        /* ---- resistive voltage sources: Ampere at the edge with the lumped
         *      current I = (l E^{n+1/2} + Vs)/Rs, solved for E^{n+1} ---- */
        for (int s = 0; s < P->n_vsrc; s++) {
            const int32_t *q = P->vsrc + 4 * s;
            const double *pr = P->vsrc_prm + 4 * s;
            const int i = q[0], j = q[1], k = q[2], c = q[3];
            double curl;
            if (c == 0) curl = (HGET(2, i, j, k) - HGET(2, i, j - 1, k)) / dy - (HGET(1, i, j, k) - HGET(1, i, j, k - 1)) / dz;
            else if (c == 1) curl = (HGET(0, i, j, k) - HGET(0, i, j, k - 1)) / dz - (HGET(2, i, j, k) - HGET(2, i - 1, j, k)) / dx;
            else curl = (HGET(1, i, j, k) - HGET(1, i - 1, j, k)) / dx - (HGET(0, i, j, k) - HGET(0, i, j - 1, k)) / dy;
            const double l = c == 0 ? dx : (c == 1 ? dy : dz);
            const double A = V / l, R = pr[3];
            const double eps = EPS0 * AT(epsE[c], i, j, k);
            const double vs = oracle_pulse(pr[0], pr[1], pr[2], t_half);
            const double rhs_j = curl - AT(J[c], i, j, k);
            /* eps (E' - E)/dt = rhs_j - (l (E + E')/2 + vs) / (R A) */
            const double a = dt * l / (2.0 * eps * R * A);
            const double Eo = ve_old[s];
            const double En = ((1.0 - a) * Eo + dt / eps * rhs_j - dt * vs / (eps * R * A)) / (1.0 + a);
            const double I = (l * 0.5 * (Eo + En) + vs) / R;
            AT(E[c], i, j, k) = En;
            AT(D[c], i, j, k) = vd_old[s] + dt * (rhs_j - I / A);
            if (s == 0 && O->vsrc_current) O->vsrc_current[n] = I;
        }

        /* ---- probes and running DFT of E^{n+1} ---- */
        for (int p = 0; p < P->n_probe; p++) {
            const int32_t *q = P->probe + 4 * p;
            double x = AT(E[q[3]], q[0], q[1], q[2]);
            if (O->trace) O->trace[(size_t)p * N + n] = x;
            if (O->dft) {
                for (int b = 0; b < Q; b++) {
                    long long r = ((long long)b * n) % N;
                    double ph = -2.0 * PI * (double)r / (double)N;
                    O->dft[((size_t)p * Q + b) * 2 + 0] += dt * x * cos(ph);
                    O->dft[((size_t)p * Q + b) * 2 + 1] += dt * x * sin(ph);
                }
            }
        }
    }

    if (O->fields) {
        for (int c = 0; c < 3; c++) {
            memcpy(O->fields + (size_t)c * nn, E[c], nn * sizeof(double));
            memcpy(O->fields + (size_t)(3 + c) * nn, H[c], nn * sizeof(double));
        }
    }
    for (int c = 0; c < 3; c++) {
        free(E[c]); free(H[c]); free(D[c]); free(B[c]); free(J[c]); free(epsE[c]); free(pec[c]);
        free(ci[c]); free(chf[c]);
    }
    free(ve_old);
    free(vd_old);
    return bad;
#undef AT
}
