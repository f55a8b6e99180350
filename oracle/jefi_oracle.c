/*
 * jefi_oracle.c -- plain FP64 CPU oracle for the discretised Jefimenko sum.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the GPU library is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may build, load
 * or call it; the library never does.  It shares no code, header or table
 * with the CUDA path.
 *
 * What it computes (paper, Sec. 2.2, Eqs. E-1, B-1, tr-1): for every
 * observation point r and time t, a midpoint sum over the source cells r'
 * of the retarded terms
 *
 *   E += k_e dV [ D (rho/R^3 + drho/(c R^2)) - dJ/(c^2 R) ]
 *   B += k_b dV [ (J/R^3 + dJ/(c R^2)) x D ]          D = r - r', R = |D|
 *
 * (paper Eqs. E and B, continuous form, written with general k_e, k_b, c;
 * the paper's units are k_e = k_b = 1/(4 pi), c = 1).  The sources are read
 * at the time slice the retarded time t_r = t - R/c falls in (Eq. tr-1):
 *
 *   n = floor(((t - t0) - R/c) / dt),      slice n holds the source at t0 + n dt,
 *
 * and the time derivative is the backward difference of Eq. E-1,
 * (f[n] - f[n-1]) / dt, with f[-1] = 0, unless the caller supplies the
 * derivatives.  Sources are zero before the first slice (n < 0), as in the
 * paper's step-on test sources (Sec. 3.1, 3.2).
 *
 * Coarse screening (paper Sec. 2.1 and Sec. 3, screening volume delta^3): a
 * pair contributes nothing when |D_a| <= delta_a on all three axes.
 *
 * Exact floating-point sequence (the slot index must be reproducible):
 *   x_i   = lo + (i + 0.5) * d             (product rounded, then sum rounded)
 *   D_a   = xo_a - xs_a
 *   S     = (Dx*Dx + Dy*Dy) + Dz*Dz        (each product rounded, no FMA)
 *   R     = sqrt(S)                         (correctly rounded)
 *   T     = t - t0
 *   n     = floor((T - R / c) / dt)
 * Build with -O2 -ffp-contract=off and without -ffast-math.
 *
 * Sums over source cells are Neumaier-compensated; an optional output gives
 * the sum of |term| per component for error diagnostics.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL 1
#define ORACLE_ENOTYET 3

/* Cell centre of index i on an axis with origin lo and spacing d
 * (cell-centred grid: 15 cells over [-3,3] with cell 0.4 in Sec. 3.1). */
double oracle_cell_center(double lo, double d, int64_t i) {
    double off = ((double)i + 0.5) * d;
    return lo + off;
}

/* Squared distance in the fixed order (Dx*Dx + Dy*Dy) + Dz*Dz. */
static double sq_dist(double dx, double dy, double dz) {
    double sx = dx * dx;
    double sy = dy * dy;
    double sz = dz * dz;
    double sxy = sx + sy;
    return sxy + sz;
}

/* Retarded slice index of Eq. tr-1 for a pair at squared distance S,
 * with T = t - t0 already formed. */
int64_t oracle_slot_from_s(double S, double T, double c, double dt) {
    double R = sqrt(S);
    double q = R / c;
    double u = (T - q) / dt;
    return (int64_t)floor(u);
}

/* Slots of explicit pairs: xo[k], xs[k] are 3-vectors. */
void oracle_pair_slots(int64_t n_pairs, const double* xo, const double* xs,
                       double t, double t0, double c, double dt, int64_t* out) {
    double T = t - t0;
    for (int64_t k = 0; k < n_pairs; ++k) {
        double dx = xo[3 * k + 0] - xs[3 * k + 0];
        double dy = xo[3 * k + 1] - xs[3 * k + 1];
        double dz = xo[3 * k + 2] - xs[3 * k + 2];
        out[k] = oracle_slot_from_s(sq_dist(dx, dy, dz), T, c, dt);
    }
}

/* Neumaier compensated accumulator. */
typedef struct { double s, c; } nsum;

static void nadd(nsum* a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x))
        a->c += (a->s - t) + x;
    else
        a->c += (x - t) + a->s;
    a->s = t;
}

static double nval(const nsum* a) { return a->s + a->c; }

/*
 * Fields at one time t for every observation point.
 *
 * src_n[3], src_lo[3], src_d[3]  source grid (cell-centred, x fastest)
 * obs[n_obs][3]                  observation points (FP64)
 * n_slices                       history length: slices 0 .. n_slices-1
 * rho[n_slices][Ns], J[n_slices][Ns][3]   sources, cell index x fastest
 * drho, dJ                       NULL -> backward difference; else supplied
 *                                derivatives with the same layout
 * screen[3]                      screening half-widths (>= 0)
 * E, B [n_obs][3]                outputs
 * absE, absB [n_obs][3]          optional sums of |term| (may be NULL)
 * slot_range[2]                  optional: min and max slot used by any
 *                                unscreened pair (may be NULL)
 * Returns ORACLE_ENOTYET if some pair needs a slice >= n_slices.
 */
int oracle_fields(const int32_t* src_n, const double* src_lo, const double* src_d,
                  int64_t n_obs, const double* obs,
                  int64_t n_slices, const double* rho, const double* J,
                  const double* drho, const double* dJ,
                  double c, double k_e, double k_b, double dt, double t0,
                  const double* screen, double t,
                  double* E, double* B, double* absE, double* absB,
                  int64_t* slot_range, int nthreads) {
    if (!(c > 0.0) || !(dt > 0.0) || n_slices < 0) return ORACLE_EINVAL;
    const int64_t nx = src_n[0], ny = src_n[1], nz = src_n[2];
    const int64_t Ns = nx * ny * nz;
    const double dV = src_d[0] * src_d[1] * src_d[2];
    const double T = t - t0;
    int err = ORACLE_OK;
    int64_t gmin = INT64_MAX, gmax = INT64_MIN;

    double* xs = (double*)malloc(sizeof(double) * (size_t)(nx > 0 ? nx : 1));
    double* ys = (double*)malloc(sizeof(double) * (size_t)(ny > 0 ? ny : 1));
    double* zs = (double*)malloc(sizeof(double) * (size_t)(nz > 0 ? nz : 1));
    for (int64_t i = 0; i < nx; ++i) xs[i] = oracle_cell_center(src_lo[0], src_d[0], i);
    for (int64_t i = 0; i < ny; ++i) ys[i] = oracle_cell_center(src_lo[1], src_d[1], i);
    for (int64_t i = 0; i < nz; ++i) zs[i] = oracle_cell_center(src_lo[2], src_d[2], i);

#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4) reduction(min : gmin) reduction(max : gmax) \
    num_threads(nthreads > 0 ? nthreads : omp_get_max_threads())
#endif
    for (int64_t o = 0; o < n_obs; ++o) {
        const double xo = obs[3 * o + 0], yo = obs[3 * o + 1], zo = obs[3 * o + 2];
        nsum e[3] = {{0, 0}, {0, 0}, {0, 0}};
        nsum b[3] = {{0, 0}, {0, 0}, {0, 0}};
        double ae[3] = {0, 0, 0}, ab[3] = {0, 0, 0};
        for (int64_t k = 0; k < nz; ++k) {
            const double dz = zo - zs[k];
            for (int64_t j = 0; j < ny; ++j) {
                const double dy = yo - ys[j];
                for (int64_t i = 0; i < nx; ++i) {
                    const double dx = xo - xs[i];
                    /* coarse screening: skip when inside the delta box */
                    if (fabs(dx) <= screen[0] && fabs(dy) <= screen[1] && fabs(dz) <= screen[2])
                        continue;
                    const double S = sq_dist(dx, dy, dz);
                    const double R = sqrt(S);
                    const int64_t n = (int64_t)floor((T - R / c) / dt);
                    if (n < 0) continue; /* no source before the first slice */
                    if (n >= n_slices) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
                        err = ORACLE_ENOTYET;
                        continue;
                    }
                    if (n < gmin) gmin = n;
                    if (n > gmax) gmax = n;
                    const int64_t cell = (k * ny + j) * nx + i;
                    const double* Jn = J + 3 * (n * Ns + cell);
                    const double r_n = rho[n * Ns + cell];
                    double dr, dj[3];
                    if (drho != NULL) {
                        dr = drho[n * Ns + cell];
                    } else {
                        const double r_prev = (n >= 1) ? rho[(n - 1) * Ns + cell] : 0.0;
                        dr = (r_n - r_prev) / dt;
                    }
                    if (dJ != NULL) {
                        for (int a = 0; a < 3; ++a) dj[a] = dJ[3 * (n * Ns + cell) + a];
                    } else {
                        for (int a = 0; a < 3; ++a) {
                            const double jp = (n >= 1) ? J[3 * ((n - 1) * Ns + cell) + a] : 0.0;
                            dj[a] = (Jn[a] - jp) / dt;
                        }
                    }
                    const double R2 = R * R;
                    const double R3 = R2 * R;
                    const double D[3] = {dx, dy, dz};
                    /* E: D (rho/R^3 + drho/(c R^2)) - dJ/(c^2 R) */
                    const double sc = r_n / R3 + dr / (c * R2);
                    double te[3];
                    for (int a = 0; a < 3; ++a) te[a] = D[a] * sc - dj[a] / (c * c * R);
                    /* B: V x D with V = J/R^3 + dJ/(c R^2) */
                    double V[3];
                    for (int a = 0; a < 3; ++a) V[a] = Jn[a] / R3 + dj[a] / (c * R2);
                    double tb[3];
                    tb[0] = V[1] * D[2] - V[2] * D[1];
                    tb[1] = V[2] * D[0] - V[0] * D[2];
                    tb[2] = V[0] * D[1] - V[1] * D[0];
                    for (int a = 0; a < 3; ++a) {
                        nadd(&e[a], te[a]);
                        nadd(&b[a], tb[a]);
                        ae[a] += fabs(te[a]);
                        ab[a] += fabs(tb[a]);
                    }
                }
            }
        }
        for (int a = 0; a < 3; ++a) {
            E[3 * o + a] = k_e * dV * nval(&e[a]);
            B[3 * o + a] = k_b * dV * nval(&b[a]);
            if (absE) absE[3 * o + a] = fabs(k_e * dV) * ae[a];
            if (absB) absB[3 * o + a] = fabs(k_b * dV) * ab[a];
        }
    }
    free(xs);
    free(ys);
    free(zs);
    if (slot_range) {
        slot_range[0] = gmin;
        slot_range[1] = gmax;
    }
    return err;
}

/*
 * Second-order variant (opt-in in the library): the same sum, with the
 * sources read at the retarded time itself instead of at the slice it falls
 * in.  With u = ((t - t0) - R/c) / dt (the floor argument above, same FP64
 * sequence), n = floor(u) and w = u - n:
 *
 *   f(t_r)  = (1 - w) f[n] + w f[n+1]                  linear interpolation
 *   f'(t_r) = (1 - w) f'[n] + w f'[n+1]
 *
 * where f'[k] is the supplied derivative or the central difference
 * (f[k+1] - f[k-1]) / (2 dt).  Slices before the first are zero, values and
 * derivatives alike: f[k] = f'[k] = 0 for k < 0 (so f'[0] = f[1] / (2 dt)).
 * Linear interpolation and the central difference are both exact for
 * sources linear in time, and the interpolated central difference is exact
 * for sources quadratic in time.
 *
 * Needs slices up to n+1 (supplied) or n+2 (central); returns
 * ORACLE_ENOTYET otherwise.  Arguments as oracle_fields.
 */
static double hist_at(const double* f, int64_t stride, int64_t k, int64_t cell, int comp) {
    return k < 0 ? 0.0 : f[(k * stride + cell) * (comp < 0 ? 1 : 3) + (comp < 0 ? 0 : comp)];
}

int oracle_fields_interp(const int32_t* src_n, const double* src_lo, const double* src_d,
                         int64_t n_obs, const double* obs,
                         int64_t n_slices, const double* rho, const double* J,
                         const double* drho, const double* dJ,
                         double c, double k_e, double k_b, double dt, double t0,
                         const double* screen, double t,
                         double* E, double* B, int nthreads) {
    if (!(c > 0.0) || !(dt > 0.0) || n_slices < 0) return ORACLE_EINVAL;
    const int64_t nx = src_n[0], ny = src_n[1], nz = src_n[2];
    const int64_t Ns = nx * ny * nz;
    const double dV = src_d[0] * src_d[1] * src_d[2];
    const double T = t - t0;
    const int supplied = drho != NULL && dJ != NULL;
    const int64_t need_ahead = supplied ? 1 : 2;   /* last slice read beyond n */
    int err = ORACLE_OK;

#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads > 0 ? nthreads : omp_get_max_threads())
#endif
    for (int64_t o = 0; o < n_obs; ++o) {
        const double xo = obs[3 * o + 0], yo = obs[3 * o + 1], zo = obs[3 * o + 2];
        nsum e[3] = {{0, 0}, {0, 0}, {0, 0}};
        nsum b[3] = {{0, 0}, {0, 0}, {0, 0}};
        for (int64_t k = 0; k < nz; ++k) {
            const double dz = zo - oracle_cell_center(src_lo[2], src_d[2], k);
            for (int64_t j = 0; j < ny; ++j) {
                const double dy = yo - oracle_cell_center(src_lo[1], src_d[1], j);
                for (int64_t i = 0; i < nx; ++i) {
                    const double dx = xo - oracle_cell_center(src_lo[0], src_d[0], i);
                    if (fabs(dx) <= screen[0] && fabs(dy) <= screen[1] && fabs(dz) <= screen[2])
                        continue;
                    const double S = sq_dist(dx, dy, dz);
                    const double R = sqrt(S);
                    const double u = (T - R / c) / dt;
                    const double fl = floor(u);
                    const int64_t n = (int64_t)fl;
                    const double w = u - fl;
                    if (n + 1 < 0) continue; /* both slices before the first */
                    if (n + need_ahead >= n_slices) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
                        err = ORACLE_ENOTYET;
                        continue;
                    }
                    const int64_t cell = (k * ny + j) * nx + i;
                    /* source values and derivatives at slices n and n+1 */
                    double r2[2], j2[2][3], dr2[2], dj2[2][3];
                    for (int s = 0; s < 2; ++s) {
                        const int64_t m = n + s;
                        r2[s] = hist_at(rho, Ns, m, cell, -1);
                        for (int a = 0; a < 3; ++a) j2[s][a] = hist_at(J, Ns, m, cell, a);
                        if (m < 0) {
                            dr2[s] = 0.0;
                            for (int a = 0; a < 3; ++a) dj2[s][a] = 0.0;
                        } else if (supplied) {
                            dr2[s] = hist_at(drho, Ns, m, cell, -1);
                            for (int a = 0; a < 3; ++a) dj2[s][a] = hist_at(dJ, Ns, m, cell, a);
                        } else {
                            dr2[s] = (hist_at(rho, Ns, m + 1, cell, -1) - hist_at(rho, Ns, m - 1, cell, -1)) /
                                     (2.0 * dt);
                            for (int a = 0; a < 3; ++a)
                                dj2[s][a] = (hist_at(J, Ns, m + 1, cell, a) - hist_at(J, Ns, m - 1, cell, a)) /
                                            (2.0 * dt);
                        }
                    }
                    const double r_n = (1.0 - w) * r2[0] + w * r2[1];
                    const double dr = (1.0 - w) * dr2[0] + w * dr2[1];
                    double Jn[3], dj[3];
                    for (int a = 0; a < 3; ++a) {
                        Jn[a] = (1.0 - w) * j2[0][a] + w * j2[1][a];
                        dj[a] = (1.0 - w) * dj2[0][a] + w * dj2[1][a];
                    }
                    const double R2 = R * R;
                    const double R3 = R2 * R;
                    const double D[3] = {dx, dy, dz};
                    const double sc = r_n / R3 + dr / (c * R2);
                    double V[3], te[3], tb[3];
                    for (int a = 0; a < 3; ++a) {
                        te[a] = D[a] * sc - dj[a] / (c * c * R);
                        V[a] = Jn[a] / R3 + dj[a] / (c * R2);
                    }
                    tb[0] = V[1] * D[2] - V[2] * D[1];
                    tb[1] = V[2] * D[0] - V[0] * D[2];
                    tb[2] = V[0] * D[1] - V[1] * D[0];
                    for (int a = 0; a < 3; ++a) {
                        nadd(&e[a], te[a]);
                        nadd(&b[a], tb[a]);
                    }
                }
            }
        }
        for (int a = 0; a < 3; ++a) {
            E[3 * o + a] = k_e * dV * nval(&e[a]);
            B[3 * o + a] = k_b * dV * nval(&b[a]);
        }
    }
    return err;
}

/*
 * Every pair's slot for a small problem: out[n_obs][Ns] (cell index x
 * fastest); screened pairs get INT64_MIN.  Used to check slot selection
 * pair by pair.
 */
void oracle_all_slots(const int32_t* src_n, const double* src_lo, const double* src_d,
                      int64_t n_obs, const double* obs, double c, double dt, double t0,
                      const double* screen, double t, int64_t* out, int nthreads) {
    const int64_t nx = src_n[0], ny = src_n[1], nz = src_n[2];
    const int64_t Ns = nx * ny * nz;
    const double T = t - t0;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : omp_get_max_threads())
#endif
    for (int64_t o = 0; o < n_obs; ++o) {
        for (int64_t k = 0; k < nz; ++k) {
            const double dz = obs[3 * o + 2] - oracle_cell_center(src_lo[2], src_d[2], k);
            for (int64_t j = 0; j < ny; ++j) {
                const double dy = obs[3 * o + 1] - oracle_cell_center(src_lo[1], src_d[1], j);
                for (int64_t i = 0; i < nx; ++i) {
                    const double dx = obs[3 * o + 0] - oracle_cell_center(src_lo[0], src_d[0], i);
                    const int64_t cell = (k * ny + j) * nx + i;
                    if (fabs(dx) <= screen[0] && fabs(dy) <= screen[1] && fabs(dz) <= screen[2]) {
                        out[o * Ns + cell] = INT64_MIN;
                        continue;
                    }
                    out[o * Ns + cell] = oracle_slot_from_s(sq_dist(dx, dy, dz), T, c, dt);
                }
            }
        }
    }
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
