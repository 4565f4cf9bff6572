/*
 * md_oracle.c -- plain, slow, FP64 CPU reference ("the oracle") for one MD timestep of a
 * short-range pair potential, as described in Bailey et al., "RUMD: A general purpose molecular
 * dynamics package optimized to utilize GPU hardware down to a few thousand particles".
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke check and bench.py's CPU
 * baseline may load this library.  It shares no code, header or constant with the CUDA path.
 *
 * What it computes (each function names the passage it follows):
 *   - Lennard-Jones 12-6 pair potential with per type-pair (eps, sigma, rc), cut off with the
 *     "shifted potential" method (Sec. 2, "Pair potentials": truncation plus a shift of the
 *     potential so that it is continuous at rc).
 *   - Forces, per-particle energy and virial by the plain definition: a full double loop over
 *     all pairs under the minimum-image convention in a cubic periodic box.  The per-particle
 *     energy is half the pair sum (the halving of Fig. 2 for a full, both-directions sum).
 *   - Leapfrog NVE and Nose-Hoover NVT integration (Sec. 2, "Integrators"; the paper names the
 *     integrators but prints no equations: the discretisation used is listed below).
 *   - Brute-force Verlet neighbour sets: j is a neighbour of i iff j != i and the squared
 *     distance is strictly below (rc_ab + s)^2 (Sec. 3 and Figs. 3-4), in FP64 and in the
 *     bit-defined fixed-point arithmetic of the mixed-precision position mirror.
 *   - Optionally, a Coulomb term between charged particles cut off with the shifted-force method
 *     (Sec. 9 "Electrostatics": the molten-salt benchmark uses Coulomb forces with a large
 *     shifted-force cutoff instead of a mesh/Ewald method).
 *   - A textbook linked-cell FP64 force routine (Sec. 6 cell-index method, cells of edge >= rc,
 *     27-cell stencil) used only for large-N baselines; it must equal the double loop.
 *
 * Readings where the paper is silent (stated once here, used consistently):
 *   u(r)   = 4 eps [(sigma/r)^12 - (sigma/r)^6],  u_SP(r) = u(r) - u(rc) for r < rc, else 0.
 *   Shifted force (Sec. 2: "truncation plus shift of the pair force ... a linear term in the
 *   potential"): u_SF(r) = u(r) - u(rc) + (r - rc) F(rc), |F|_SF(r) = F(r) - F(rc), with
 *   F(r) = -u'(r), for r < rc.
 *   Coulomb, shifted force (charges q in units of sqrt(4 pi eps0 eps sigma), as Sec. 9 states):
 *   u_C(r) = q_a q_b [1/r - 1/rc_C + (r - rc_C)/rc_C^2],  |F|_C(r) = q_a q_b [1/r^2 - 1/rc_C^2]
 *   for r < rc_C (the shifted-force construction above applied to u = q_a q_b / r); the LJ term
 *   keeps its own rc_ab.
 *   F_ij   = (24 eps / r^2) [2 (sigma/r)^12 - (sigma/r)^6] r_ij,  r_ij = r_i - r_j (min image,
 *            d -= L * round(d / L), round half away from zero).
 *   u_i    = 1/2 sum_j u_SP(r_ij);  w_i = 1/2 * 1/3 sum_j r_ij . F_ij;  U = sum u_i, W = sum w_i.
 *   NVE    : v_{n+1/2} = v_{n-1/2} + dt F_n / m;  r_{n+1} = r_n + dt v_{n+1/2}.
 *   NVT    : g = 3N - 3, K0 = g T0 / 2,
 *            xi_n = xi_{n-1} + dt (K_{n-1/2} / K0 - 1) / tau^2,
 *            v_{n+1/2} = [(1 - xi_n dt/2) v_{n-1/2} + dt F_n / m] / (1 + xi_n dt/2),
 *            r_{n+1} = r_n + dt v_{n+1/2}.
 *            Conserved: H = U + K + g T0 (tau^2 xi^2 / 2 + sum_k xi_k dt).
 *   Fixed-point neighbour arithmetic (the mixed-precision mirror): each coordinate is a 32-bit
 *   unsigned integer q with q L / 2^32 the position, so one period is 2^32 units; per axis
 *   d = (float)(int32)(q_j - q_i) (the 32-bit difference is the nearest periodic image; the
 *   conversion rounds to nearest), then dist2 = ((dx*dx + dy*dy) + dz*dz) * ps2 in float, each
 *   product and sum rounded separately (no fused multiply-add), with ps2 = (float)((L / 2^32)^2),
 *   compared with the FP32 threshold (float)((rc_ab + s)^2).
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fno-fast-math -fPIC -shared (see build.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAX_TYPES 8

int or_version(void) { return 4; }

void or_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int or_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------------------------------
 * Pair potential (Sec. 2 "Pair potentials", LJ 12-6 with the shifted-potential or the
 * shifted-force cutoff).  Returns u and the scalar fs with F_ij = fs * r_ij.  r2 < rc^2.
 * ------------------------------------------------------------------------------------------- */
static int g_cutoff = 0;   /* 0: shifted potential, 1: shifted force */

void or_set_cutoff(int method) { g_cutoff = method; }
int or_get_cutoff(void) { return g_cutoff; }

static void lj_sp(double r2, double eps, double sig, double rc, double *u, double *fs) {
    double sr2 = sig * sig / r2;
    double sr6 = sr2 * sr2 * sr2;
    double sc2 = sig * sig / (rc * rc);
    double sc6 = sc2 * sc2 * sc2;
    *u = 4.0 * eps * (sr6 * sr6 - sr6) - 4.0 * eps * (sc6 * sc6 - sc6);
    *fs = 24.0 * eps * (2.0 * sr6 * sr6 - sr6) / r2;
    if (g_cutoff == 1) {
        double r = sqrt(r2);
        double frc = 24.0 * eps * (2.0 * sc6 * sc6 - sc6) / rc;   /* F(rc) = -u'(rc) */
        *u += (r - rc) * frc;
        *fs -= frc / r;
    }
}

/* Coulomb shifted-force setting (Sec. 9): per-type charges and the Coulomb cutoff rc_C;
 * rc_C <= 0 switches the term off (the default). */
static double g_q[OR_MAX_TYPES];
static double g_rcc = 0.0;

void or_set_coulomb(int nt, const double *q, double rcc) {
    for (int t = 0; t < OR_MAX_TYPES; ++t) g_q[t] = (q && t < nt) ? q[t] : 0.0;
    g_rcc = (q && rcc > 0.0) ? rcc : 0.0;
}
double or_get_coulomb_rc(void) { return g_rcc; }

static void coulomb_sf(double r2, double qq, double rcc, double *u, double *fs) {
    double r = sqrt(r2);
    *u = qq * (1.0 / r - 1.0 / rcc + (r - rcc) / (rcc * rcc));
    *fs = qq * (1.0 / r2 - 1.0 / (rcc * rcc)) / r;    /* F_ij = fs * r_ij */
}

/* All pair terms between types ti, tj at squared distance r2: LJ within rc_ab, Coulomb within
 * rc_C.  Adds to *u and *fs; returns 1 if any term is inside its cutoff. */
static int pair_terms(double r2, int ti, int tj, int nt, const double *eps, const double *sig,
                      const double *rc, double *u, double *fs) {
    int p = ti * nt + tj, any = 0;
    *u = 0.0; *fs = 0.0;
    if (r2 < rc[p] * rc[p]) {
        lj_sp(r2, eps[p], sig[p], rc[p], u, fs);
        any = 1;
    }
    if (g_rcc > 0.0 && r2 < g_rcc * g_rcc) {
        double uc, fc;
        coulomb_sf(r2, g_q[ti] * g_q[tj], g_rcc, &uc, &fc);
        *u += uc; *fs += fc;
        any = 1;
    }
    return any;
}

/* Largest cutoff of any term (the linked-cell edge). */
static double max_cutoff(int nt, const double *rc) {
    double m = g_rcc;
    for (int p = 0; p < nt * nt; ++p) if (rc[p] > m) m = rc[p];
    return m;
}

/* Exported for closed-form tests: Coulomb shifted-force pair energy and force magnitude. */
void or_coulomb_pair(double r, double qq, double rcc, double *u, double *fmag) {
    if (r >= rcc) { *u = 0.0; *fmag = 0.0; return; }
    double fs;
    coulomb_sf(r * r, qq, rcc, u, &fs);
    *fmag = fs * r;
}

/* Exported for closed-form tests: pair energy and force magnitude along r at distance r. */
void or_pair(double r, double eps, double sig, double rc, double *u_sp, double *fmag) {
    if (r >= rc) { *u_sp = 0.0; *fmag = 0.0; return; }
    double u, fs;
    lj_sp(r * r, eps, sig, rc, &u, &fs);
    *u_sp = u;
    *fmag = fs * r;
}

static inline double min_image(double d, double L) { return d - L * round(d / L); }

/* Contribution of all j to particle i (plain definition, Sec. 5 / Fig. 2 semantics). */
static void one_particle(int i, int n, const double *pos, const int *type, double L, int nt,
                         const double *eps, const double *sig, const double *rc,
                         double *fi, double *ui, double *wi) {
    double fx = 0, fy = 0, fz = 0, u = 0, w = 0;
    const double xi = pos[3 * i], yi = pos[3 * i + 1], zi = pos[3 * i + 2];
    const int ti = type[i];
    for (int j = 0; j < n; ++j) {
        if (j == i) continue;
        double dx = min_image(xi - pos[3 * j], L);
        double dy = min_image(yi - pos[3 * j + 1], L);
        double dz = min_image(zi - pos[3 * j + 2], L);
        double r2 = dx * dx + dy * dy + dz * dz;
        double uu, fs;
        if (pair_terms(r2, ti, type[j], nt, eps, sig, rc, &uu, &fs)) {
            fx += fs * dx; fy += fs * dy; fz += fs * dz;
            u += uu;
            w += fs * r2;
        }
    }
    fi[0] = fx; fi[1] = fy; fi[2] = fz;
    *ui = 0.5 * u;
    *wi = 0.5 * w / 3.0;
}

/* Forces, per-particle energies and virials; UW[0] = U, UW[1] = W.  O(N^2), FP64. */
int or_forces(int n, const double *pos, const int *type, double L, int nt, const double *eps,
              const double *sig, const double *rc, double *f, double *u, double *w, double *UW) {
    if (n < 0 || nt < 1 || nt > OR_MAX_TYPES || !(L > 0)) return 1;
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < n; ++i)
        one_particle(i, n, pos, type, L, nt, eps, sig, rc, f + 3 * i, u + i, w + i);
    double U = 0, W = 0;
    for (int i = 0; i < n; ++i) { U += u[i]; W += w[i]; }
    if (UW) { UW[0] = U; UW[1] = W; }
    return 0;
}

/* Same quantities for a listed subset of particles only (for sampled checks at large N). */
int or_forces_subset(int n, const double *pos, const int *type, double L, int nt,
                     const double *eps, const double *sig, const double *rc, int nsub,
                     const int *idx, double *f, double *u, double *w) {
    if (n < 0 || nt < 1 || nt > OR_MAX_TYPES || !(L > 0)) return 1;
    for (int k = 0; k < nsub; ++k) if (idx[k] < 0 || idx[k] >= n) return 2;
#pragma omp parallel for schedule(dynamic, 4)
    for (int k = 0; k < nsub; ++k)
        one_particle(idx[k], n, pos, type, L, nt, eps, sig, rc, f + 3 * k, u + k, w + k);
    return 0;
}

/* ---------------------------------------------------------------------------------------------
 * Linked-cell FP64 force routine (textbook cell-index method of Sec. 6 with cell edge >= rc_max,
 * 27 cells).  Only used where the O(N^2) loop is too slow; tests pin it to or_forces.
 * ------------------------------------------------------------------------------------------- */
static inline int cell_of(double x, double L, int nc) {
    double s = x - L * floor(x / L);               /* wrap into [0, L) */
    int c = (int)(s / L * nc);
    if (c >= nc) c = nc - 1;
    if (c < 0) c = 0;
    return c;
}

int or_forces_cells(int n, const double *pos, const int *type, double L, int nt,
                    const double *eps, const double *sig, const double *rc, double *f, double *u,
                    double *w, double *UW) {
    if (n < 0 || nt < 1 || nt > OR_MAX_TYPES || !(L > 0)) return 1;
    double rcmax = max_cutoff(nt, rc);
    int nc = (int)floor(L / rcmax);
    if (nc < 3) return or_forces(n, pos, type, L, nt, eps, sig, rc, f, u, w, UW);
    long ncell = (long)nc * nc * nc;
    int *head = (int *)malloc(sizeof(int) * ncell);
    int *next = (int *)malloc(sizeof(int) * (n > 0 ? n : 1));
    int *cid = (int *)malloc(sizeof(int) * 3 * (n > 0 ? n : 1));
    if (!head || !next || !cid) { free(head); free(next); free(cid); return 3; }
    for (long c = 0; c < ncell; ++c) head[c] = -1;
    for (int i = n - 1; i >= 0; --i) {
        int cx = cell_of(pos[3 * i], L, nc), cy = cell_of(pos[3 * i + 1], L, nc),
            cz = cell_of(pos[3 * i + 2], L, nc);
        cid[3 * i] = cx; cid[3 * i + 1] = cy; cid[3 * i + 2] = cz;
        long c = ((long)cz * nc + cy) * nc + cx;
        next[i] = head[c];
        head[c] = i;
    }
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < n; ++i) {
        double fx = 0, fy = 0, fz = 0, uu = 0, ww = 0;
        const double xi = pos[3 * i], yi = pos[3 * i + 1], zi = pos[3 * i + 2];
        const int ti = type[i];
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int cx = (cid[3 * i] + dx + nc) % nc, cy = (cid[3 * i + 1] + dy + nc) % nc,
                        cz = (cid[3 * i + 2] + dz + nc) % nc;
                    for (int j = head[((long)cz * nc + cy) * nc + cx]; j >= 0; j = next[j]) {
                        if (j == i) continue;
                        double ddx = min_image(xi - pos[3 * j], L);
                        double ddy = min_image(yi - pos[3 * j + 1], L);
                        double ddz = min_image(zi - pos[3 * j + 2], L);
                        double r2 = ddx * ddx + ddy * ddy + ddz * ddz;
                        double e, fs;
                        if (pair_terms(r2, ti, type[j], nt, eps, sig, rc, &e, &fs)) {
                            fx += fs * ddx; fy += fs * ddy; fz += fs * ddz;
                            uu += e;
                            ww += fs * r2;
                        }
                    }
                }
        f[3 * i] = fx; f[3 * i + 1] = fy; f[3 * i + 2] = fz;
        u[i] = 0.5 * uu;
        w[i] = 0.5 * ww / 3.0;
    }
    double U = 0, W = 0;
    for (int i = 0; i < n; ++i) { U += u[i]; W += w[i]; }
    if (UW) { UW[0] = U; UW[1] = W; }
    free(head); free(next); free(cid);
    return 0;
}

/* ---------------------------------------------------------------------------------------------
 * Leapfrog NVE / Nose-Hoover NVT (Sec. 2 "Integrators"; equations are the readings above).
 *
 * pos: (n,3) UNWRAPPED positions r_n (in/out); vel: (n,3) velocities v_{n-1/2} (in/out).
 * state[4] (in/out): xi_{n-1}, K_{n-1/2}, sum_k xi_k dt, have_K (0 => K_{n-1/2} is computed
 * from vel on entry).  log: nsteps rows of 10 doubles:
 *   U_n, W_n, K_{n-1/2}, K_{n+1/2}, xi_n, sum xi dt, P_x, P_y, P_z (momentum of v_{n+1/2}), H_n
 * where H_n = U_n + (K_{n-1/2} + K_{n+1/2})/2 (+ thermostat terms for NVT).
 * integrator: 0 = NVE, 1 = Nose-Hoover.  use_cells: 1 selects or_forces_cells.
 * ------------------------------------------------------------------------------------------- */
int or_run(int n, double *pos, double *vel, const int *type, double L, int nt, const double *eps,
           const double *sig, const double *rc, const double *mass, int integrator, double dt,
           double T0, double tau, double *state, int nsteps, double *log, int use_cells) {
    if (n < 2 || nt < 1 || nt > OR_MAX_TYPES || !(L > 0) || !(dt > 0)) return 1;
    if (integrator == 1 && !(tau > 0 && T0 > 0)) return 1;
    double *f = (double *)malloc(sizeof(double) * 3 * n);
    double *u = (double *)malloc(sizeof(double) * n);
    double *w = (double *)malloc(sizeof(double) * n);
    if (!f || !u || !w) { free(f); free(u); free(w); return 3; }
    const double g = 3.0 * n - 3.0;
    const double K0 = 0.5 * g * T0;
    double xi = state[0], Kprev = state[1], xint = state[2];
    if (state[3] == 0.0) {
        Kprev = 0;
        for (int i = 0; i < n; ++i) {
            double m = mass[type[i]];
            Kprev += 0.5 * m * (vel[3 * i] * vel[3 * i] + vel[3 * i + 1] * vel[3 * i + 1] +
                                vel[3 * i + 2] * vel[3 * i + 2]);
        }
    }
    for (int s = 0; s < nsteps; ++s) {
        double UW[2];
        int rcode = use_cells ? or_forces_cells(n, pos, type, L, nt, eps, sig, rc, f, u, w, UW)
                              : or_forces(n, pos, type, L, nt, eps, sig, rc, f, u, w, UW);
        if (rcode) { free(f); free(u); free(w); return rcode; }
        double a = 1.0, b = 1.0;
        if (integrator == 1) {
            xi = xi + dt * (Kprev / K0 - 1.0) / (tau * tau);
            xint += xi * dt;
            a = 1.0 - 0.5 * xi * dt;
            b = 1.0 / (1.0 + 0.5 * xi * dt);
        }
        double K = 0, px = 0, py = 0, pz = 0;
        for (int i = 0; i < n; ++i) {
            double m = mass[type[i]];
            for (int c = 0; c < 3; ++c) {
                double v = vel[3 * i + c];
                v = (integrator == 1) ? (a * v + dt * f[3 * i + c] / m) * b : v + dt * f[3 * i + c] / m;
                vel[3 * i + c] = v;
                pos[3 * i + c] += dt * v;
            }
            double vx = vel[3 * i], vy = vel[3 * i + 1], vz = vel[3 * i + 2];
            K += 0.5 * m * (vx * vx + vy * vy + vz * vz);
            px += m * vx; py += m * vy; pz += m * vz;
        }
        if (log) {
            double *row = log + 10 * (long)s;
            row[0] = UW[0]; row[1] = UW[1]; row[2] = Kprev; row[3] = K; row[4] = xi;
            row[5] = xint; row[6] = px; row[7] = py; row[8] = pz;
            double H = UW[0] + 0.5 * (Kprev + K);
            if (integrator == 1) H += g * T0 * (0.5 * tau * tau * xi * xi + xint);
            row[9] = H;
        }
        Kprev = K;
    }
    state[0] = xi; state[1] = Kprev; state[2] = xint; state[3] = 1.0;
    free(f); free(u); free(w);
    return 0;
}

/* ---------------------------------------------------------------------------------------------
 * Brute-force Verlet neighbour sets (Secs. 3, 6; Figs. 3-4): j in nbl(i) iff j != i and
 * dist2 < (rc_{t_i t_j} + s)^2, strict.  Full list (both directions).  list is row-major
 * (n, maxn) with ascending j; counts[i] is the true count even when it exceeds maxn.
 * thr2[p] = (rc_p + s)^2 for type pair p.
 * ------------------------------------------------------------------------------------------- */
int or_neighbors_fp64(int n, const double *pos, const int *type, double L, int nt,
                      const double *thr2, int maxn, int *counts, int *list) {
    if (n < 0 || nt < 1 || nt > OR_MAX_TYPES || !(L > 0) || maxn < 0) return 1;
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < n; ++i) {
        int c = 0;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            double dx = min_image(pos[3 * j] - pos[3 * i], L);
            double dy = min_image(pos[3 * j + 1] - pos[3 * i + 1], L);
            double dz = min_image(pos[3 * j + 2] - pos[3 * i + 2], L);
            double d2 = dx * dx + dy * dy + dz * dz;
            if (d2 < thr2[type[i] * nt + type[j]]) {
                if (c < maxn) list[(long)i * maxn + c] = j;
                ++c;
            }
        }
        counts[i] = c;
    }
    return 0;
}

/* Fixed-point mode: same rule, in the bit-defined arithmetic of the fixed-point mirror stated in
 * the header.  q is (n,3) uint32; ps2 = (float)((L / 2^32)^2); thr2f[p] = (float)((rc_p + s)^2). */
static inline float fixed_d(uint32_t a, uint32_t b) {
    const uint32_t u = a - b;     /* modulo 2^32 */
    const int32_t d = (int32_t)u; /* two's complement: the nearest image */
    return (float)d;
}

int or_neighbors_fixed(int n, const uint32_t *q, const int *type, float ps2, int nt,
                       const float *thr2f, int maxn, int *counts, int *list) {
    if (n < 0 || nt < 1 || nt > OR_MAX_TYPES || !(ps2 > 0) || maxn < 0) return 1;
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < n; ++i) {
        int c = 0;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            const float dx = fixed_d(q[3 * j], q[3 * i]);
            const float dy = fixed_d(q[3 * j + 1], q[3 * i + 1]);
            const float dz = fixed_d(q[3 * j + 2], q[3 * i + 2]);
            float d2 = dx * dx;
            d2 = d2 + dy * dy;
            d2 = d2 + dz * dz;
            d2 = d2 * ps2;
            if (d2 < thr2f[type[i] * nt + type[j]]) {
                if (c < maxn) list[(long)i * maxn + c] = j;
                ++c;
            }
        }
        counts[i] = c;
    }
    return 0;
}
