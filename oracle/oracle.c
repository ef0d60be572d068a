/*
 * Plain FP64 CPU oracle for the on-the-fly property path of
 * "DL_POLY 5: Calculation of system properties on the fly for very large
 * systems via massive parallelism" (arXiv 2503.07526).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * statement of what the GPU library computes.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or helper with the CUDA library, and the
 * library never calls it.
 *
 * Contents, each written from the paper's definition:
 *   - shifted Lennard-Jones pair forces with per-particle energy and virial
 *     (stress tensor, Sec. 2.3 Eq. (stress); per-particle split of the heat
 *     flux, Sec. 2.3 heat-flux equation), by brute force over all pairs and
 *     by link cells (Sec. 1: DL_POLY's linked cells);
 *   - velocity-Verlet NVE stepping (Sec. 1);
 *   - the per-step system stress tensor and heat flux (Sec. 2.3);
 *   - the multiple-tau correlator update and readout (Sec. 2.2, Appendix D
 *     Algorithms 1 and 2), with the readings listed below;
 *   - the direct correlation estimator (Sec. 2.2 Eq. (cor));
 *   - trapezoid Green-Kubo integration (Sec. 2.3 Eqs. (visc), (therm)).
 *
 * Readings of the paper where it is garbled or silent:
 *   R1  Alg. 1 uses one name for the ring and its insert pointer; the number
 *       of valid lags is the number of samples the level has received,
 *       capped at p (a product is formed only when the older sample exists).
 *   R2  Alg. 1 "accumulate"/"accumulator" is one accumulator.
 *   R3  A level passes the mean of its accumulator on when exactly m samples
 *       have been accumulated (the prose says every m steps), not m+1.
 *   R4  Level 1 correlates lags 0..p-1; higher levels lags floor(p/m)..p-1
 *       (the "i == 1" test is read as "level == 1", matching Alg. 2).
 *   R5  The product is the older x times the newer y, as in Eq. (cor)
 *       (X(s) Y(s+l)); for autocorrelations the order does not matter.
 *   R6  Alg. 2 reads levels 2..blocksUsed after level 1 (level 1's upper
 *       lags are not read twice).  Times are lag * m^(level-1) in units of
 *       the correlator's update interval.
 *   R7  Samples passed on past the last level are dropped (Alg. 1 returns).
 *   R8  Eq. (stress) sums over ordered pairs i, j != i; the pair virial
 *       carries a factor 1/2 (each unordered pair once), fixed by the strain
 *       derivative of the energy.  sigma is the pressure tensor.
 *   R9  The per-particle potential energy in the heat flux is half of each
 *       pair energy (equal split); the per-particle virial is
 *       W_i = 1/2 sum_j r_ij (x) f_ij, so 1/2 sum_j (f_ij . v_i) r_ij = W_i v_i.
 *   R10 The potential is truncated at rc and shifted in energy (force
 *       unshifted) when shift != 0.
 *
 * Array conventions: positions, velocities and forces are component-major
 * [3][n]; per-particle virials and stress tensors are [6] in the order
 * xx, yy, zz, xy, xz, yz.  Units are whatever the caller uses (LJ reduced
 * units in the tests: eps = sigma = m = kB = 1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOMEM -2

/* ---------------------------------------------------------------- pairs */

/* Shifted 12-6 Lennard-Jones: U(r) = 4 eps [(s/r)^12 - (s/r)^6] - U(rc),
 * fs = -U'(r)/r, so that the force on i from j is f_ij = fs * r_ij with
 * r_ij = r_i - r_j. */
static void lj_pair(double r2, double eps, double sig, double ushift,
                    double *u, double *fs) {
  double sr2 = sig * sig / r2;
  double sr6 = sr2 * sr2 * sr2;
  double sr12 = sr6 * sr6;
  *u = 4.0 * eps * (sr12 - sr6) - ushift;
  *fs = 24.0 * eps * (2.0 * sr12 - sr6) / r2;
}

static double lj_energy_at(double r, double eps, double sig) {
  double sr = sig / r;
  double sr6 = pow(sr, 6.0);
  return 4.0 * eps * (sr6 * sr6 - sr6);
}

/* Adds the contribution of neighbour j (displacement d = r_i - r_j) to
 * particle i's force, energy and virial (R8, R9). */
static void add_pair(double dx, double dy, double dz, double rc2, double eps,
                     double sig, double ushift, double *fi, double *ei,
                     double *wi) {
  double r2 = dx * dx + dy * dy + dz * dz;
  if (r2 >= rc2) return;
  double u, fs;
  lj_pair(r2, eps, sig, ushift, &u, &fs);
  double fx = fs * dx, fy = fs * dy, fz = fs * dz;
  fi[0] += fx;
  fi[1] += fy;
  fi[2] += fz;
  *ei += 0.5 * u;
  wi[0] += 0.5 * dx * fx;
  wi[1] += 0.5 * dy * fy;
  wi[2] += 0.5 * dz * fz;
  wi[3] += 0.5 * dx * fy;
  wi[4] += 0.5 * dx * fz;
  wi[5] += 0.5 * dy * fz;
}

static double min_image(double d, double L) { return d - L * nearbyint(d / L); }

/* All ordered pairs i != j, minimum image when periodic (requires rc < L/2).
 * F [3][n], epot [n], W [6][n] are overwritten. */
int orc_lj_brute(int64_t n, const double *r, double L, int periodic,
                 double eps, double sig, double rc, int shift, double *F,
                 double *epot, double *W) {
  if (n < 0 || rc <= 0.0 || (periodic && !(rc < 0.5 * L))) return ORC_EINVAL;
  double rc2 = rc * rc;
  double ushift = shift ? lj_energy_at(rc, eps, sig) : 0.0;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < n; ++i) {
    double fi[3] = {0, 0, 0}, ei = 0.0, wi[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      double dx = r[i] - r[j];
      double dy = r[n + i] - r[n + j];
      double dz = r[2 * n + i] - r[2 * n + j];
      if (periodic) {
        dx = min_image(dx, L);
        dy = min_image(dy, L);
        dz = min_image(dz, L);
      }
      add_pair(dx, dy, dz, rc2, eps, sig, ushift, fi, &ei, wi);
    }
    for (int a = 0; a < 3; ++a) F[a * n + i] = fi[a];
    epot[i] = ei;
    for (int a = 0; a < 6; ++a) W[a * n + i] = wi[a];
  }
  return ORC_OK;
}

static double wrap_box(double x, double L) {
  double y = x - L * floor(x / L);
  if (y >= L) y -= L; /* x = -tiny rounds to L */
  return y;
}

/* Link cells (the classic head / next lists) on a periodic cubic box with
 * nc = floor(L / rc) >= 3 cells per side.  Same outputs as orc_lj_brute. */
int orc_lj_cells(int64_t n, const double *r, double L, double eps, double sig,
                 double rc, int shift, double *F, double *epot, double *W) {
  if (n < 0 || rc <= 0.0) return ORC_EINVAL;
  int nc = (int)floor(L / rc);
  if (nc < 3) return ORC_EINVAL;
  double edge = L / nc;
  int64_t ncell = (int64_t)nc * nc * nc;
  int64_t *head = malloc(sizeof(int64_t) * ncell);
  int64_t *next = malloc(sizeof(int64_t) * (n > 0 ? n : 1));
  int64_t *cell = malloc(sizeof(int64_t) * (n > 0 ? n : 1));
  if (!head || !next || !cell) {
    free(head); free(next); free(cell);
    return ORC_ENOMEM;
  }
  for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
  for (int64_t i = 0; i < n; ++i) {
    int ci[3];
    for (int a = 0; a < 3; ++a) {
      ci[a] = (int)floor(wrap_box(r[a * n + i], L) / edge);
      if (ci[a] >= nc) ci[a] = nc - 1;
    }
    cell[i] = ((int64_t)ci[2] * nc + ci[1]) * nc + ci[0];
    next[i] = head[cell[i]];
    head[cell[i]] = i;
  }
  double rc2 = rc * rc;
  double ushift = shift ? lj_energy_at(rc, eps, sig) : 0.0;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < n; ++i) {
    int64_t c = cell[i];
    int cx = (int)(c % nc), cy = (int)((c / nc) % nc), cz = (int)(c / ((int64_t)nc * nc));
    double fi[3] = {0, 0, 0}, ei = 0.0, wi[6] = {0, 0, 0, 0, 0, 0};
    for (int oz = -1; oz <= 1; ++oz)
      for (int oy = -1; oy <= 1; ++oy)
        for (int ox = -1; ox <= 1; ++ox) {
          int jx = (cx + ox + nc) % nc, jy = (cy + oy + nc) % nc, jz = (cz + oz + nc) % nc;
          int64_t cj = ((int64_t)jz * nc + jy) * nc + jx;
          for (int64_t j = head[cj]; j >= 0; j = next[j]) {
            if (j == i) continue;
            double dx = min_image(r[i] - r[j], L);
            double dy = min_image(r[n + i] - r[n + j], L);
            double dz = min_image(r[2 * n + i] - r[2 * n + j], L);
            add_pair(dx, dy, dz, rc2, eps, sig, ushift, fi, &ei, wi);
          }
        }
    for (int a = 0; a < 3; ++a) F[a * n + i] = fi[a];
    epot[i] = ei;
    for (int a = 0; a < 6; ++a) W[a * n + i] = wi[a];
  }
  free(head); free(next); free(cell);
  return ORC_OK;
}

/* For tests of reduced-precision forces: per atom, the number of
 * neighbours whose distance lies within band of rc, where the truncated
 * force jumps by |f(rc)| and a rounded distance may fall on either side of
 * the cutoff (both results are then valid).  Link cells as above, at least
 * rc + band wide, so that a pair up to rc + band apart lies in neighbouring
 * cells. */
int orc_lj_near_cutoff(int64_t n, const double *r, double L, double rc, double band,
                       int32_t *count) {
  if (n < 0 || rc <= 0.0 || band < 0.0 || !(L > 0.0)) return ORC_EINVAL;
  int nc = (int)floor(L / (rc + band));
  if (nc < 3) {  /* a box under three cells wide: every pair */
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
      int32_t k = 0;
      for (int64_t j = 0; j < n; ++j) {
        if (j == i) continue;
        double dx = min_image(r[i] - r[j], L);
        double dy = min_image(r[n + i] - r[n + j], L);
        double dz = min_image(r[2 * n + i] - r[2 * n + j], L);
        if (fabs(sqrt(dx * dx + dy * dy + dz * dz) - rc) <= band) ++k;
      }
      count[i] = k;
    }
    return ORC_OK;
  }
  double edge = L / nc;
  int64_t ncell = (int64_t)nc * nc * nc;
  int64_t *head = malloc(sizeof(int64_t) * ncell);
  int64_t *next = malloc(sizeof(int64_t) * (n > 0 ? n : 1));
  int64_t *cell = malloc(sizeof(int64_t) * (n > 0 ? n : 1));
  if (!head || !next || !cell) {
    free(head); free(next); free(cell);
    return ORC_ENOMEM;
  }
  for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
  for (int64_t i = 0; i < n; ++i) {
    int ci[3];
    for (int a = 0; a < 3; ++a) {
      ci[a] = (int)floor(wrap_box(r[a * n + i], L) / edge);
      if (ci[a] >= nc) ci[a] = nc - 1;
    }
    cell[i] = ((int64_t)ci[2] * nc + ci[1]) * nc + ci[0];
    next[i] = head[cell[i]];
    head[cell[i]] = i;
  }
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < n; ++i) {
    int64_t c = cell[i];
    int cx = (int)(c % nc), cy = (int)((c / nc) % nc), cz = (int)(c / ((int64_t)nc * nc));
    int32_t k = 0;
    for (int oz = -1; oz <= 1; ++oz)
      for (int oy = -1; oy <= 1; ++oy)
        for (int ox = -1; ox <= 1; ++ox) {
          int jx = (cx + ox + nc) % nc, jy = (cy + oy + nc) % nc, jz = (cz + oz + nc) % nc;
          for (int64_t j = head[((int64_t)jz * nc + jy) * nc + jx]; j >= 0; j = next[j]) {
            if (j == i) continue;
            double dx = min_image(r[i] - r[j], L);
            double dy = min_image(r[n + i] - r[n + j], L);
            double dz = min_image(r[2 * n + i] - r[2 * n + j], L);
            double d = sqrt(dx * dx + dy * dy + dz * dz);
            if (fabs(d - rc) <= band) ++k;
          }
        }
    count[i] = k;
  }
  free(head); free(next); free(cell);
  return ORC_OK;
}

/* ------------------------------------------------- system observables */

#define ORC_NOBS 12 /* U, K, T, sigma[6] (xx yy zz xy xz yz), q[3] */

/* Sec. 2.3: V sigma_ab = sum_i m v_a v_b + sum_i W_i,ab (R8);
 * V q = sum_i (E_i v_i + W_i v_i) with E_i = m v_i^2 / 2 + epot_i (R9).
 * T = 2K / (3n - 3) with kB = 1 (momentum-conserving NVE). */
void orc_observables(int64_t n, double V, const double *mass_of,
                     const double *v, const double *epot, const double *W,
                     double *obs) {
  double U = 0, K = 0, s[6] = {0, 0, 0, 0, 0, 0}, q[3] = {0, 0, 0};
  for (int64_t i = 0; i < n; ++i) {
    double m = mass_of[i];
    double vx = v[i], vy = v[n + i], vz = v[2 * n + i];
    double ke = 0.5 * m * (vx * vx + vy * vy + vz * vz);
    double Ei = ke + epot[i];
    double w[6];
    for (int a = 0; a < 6; ++a) w[a] = W[a * n + i];
    U += epot[i];
    K += ke;
    s[0] += m * vx * vx + w[0];
    s[1] += m * vy * vy + w[1];
    s[2] += m * vz * vz + w[2];
    s[3] += m * vx * vy + w[3];
    s[4] += m * vx * vz + w[4];
    s[5] += m * vy * vz + w[5];
    /* W_i v_i with the symmetric W_i */
    q[0] += Ei * vx + w[0] * vx + w[3] * vy + w[4] * vz;
    q[1] += Ei * vy + w[3] * vx + w[1] * vy + w[5] * vz;
    q[2] += Ei * vz + w[4] * vx + w[5] * vy + w[2] * vz;
  }
  obs[0] = U;
  obs[1] = K;
  obs[2] = (n > 1) ? 2.0 * K / (3.0 * (double)n - 3.0) : 0.0;
  for (int a = 0; a < 6; ++a) obs[3 + a] = s[a] / V;
  for (int a = 0; a < 3; ++a) obs[9 + a] = q[a] / V;
}

/* --------------------------------------------- multiple-tau correlator */

/* State of one correlator over ns series pushed in lockstep (Alg. 1).
 * Series are split into ng = ns / gs contiguous groups of gs series; the lag
 * sums of a group add its series' products, so a group's readout is the
 * mean over its series (the atom average of the VAF, Sec. 2.7).  The ring,
 * pointer, counters and counts are those Alg. 1 keeps per block; the ones
 * that do not depend on the data are stored once, since every series of a
 * correlator receives its samples at the same steps. */
typedef struct {
  int b, p, m, cross;
  int64_t ns, gs, ng;
  double *shx, *shy;  /* [b][p][ns] ring of x and y (shy == shx if !cross) */
  double *accx, *accy;/* [b][ns] block accumulators */
  double *tmpx, *tmpy;/* [b][ns] means passed on to the next block */
  int64_t *nacc;      /* [b] samples in the accumulator */
  int *ptr;           /* [b] next ring slot */
  int64_t *nrecv;     /* [b] samples received by the block */
  double *values;     /* [ng][b][p] lag sums */
  int64_t *count;     /* [b][p] products per lag (per series) */
  int blocks_used;
} orc_corr;

void orc_corr_free(orc_corr *c) {
  if (!c) return;
  free(c->shx);
  if (c->cross) free(c->shy);
  free(c->accx);
  if (c->cross) free(c->accy);
  free(c->tmpx);
  if (c->cross) free(c->tmpy);
  free(c->nacc); free(c->ptr); free(c->nrecv); free(c->values); free(c->count);
  free(c);
}

orc_corr *orc_corr_new(int b, int p, int m, int64_t ns, int64_t gs, int cross) {
  if (b < 1 || p < 2 || m < 1 || m > p || ns < 1 || gs < 1 || ns % gs) return NULL;
  orc_corr *c = calloc(1, sizeof(orc_corr));
  if (!c) return NULL;
  c->b = b; c->p = p; c->m = m; c->cross = cross ? 1 : 0;
  c->ns = ns; c->gs = gs; c->ng = ns / gs;
  size_t ring = (size_t)b * p * ns, lvl = (size_t)b * ns;
  c->shx = calloc(ring, sizeof(double));
  c->shy = c->cross ? calloc(ring, sizeof(double)) : c->shx;
  c->accx = calloc(lvl, sizeof(double));
  c->accy = c->cross ? calloc(lvl, sizeof(double)) : c->accx;
  c->tmpx = calloc(lvl, sizeof(double));
  c->tmpy = c->cross ? calloc(lvl, sizeof(double)) : c->tmpx;
  c->nacc = calloc(b, sizeof(int64_t));
  c->ptr = calloc(b, sizeof(int));
  c->nrecv = calloc(b, sizeof(int64_t));
  c->values = calloc((size_t)c->ng * b * p, sizeof(double));
  c->count = calloc((size_t)b * p, sizeof(int64_t));
  if (!c->shx || !c->shy || !c->accx || !c->accy || !c->tmpx || !c->tmpy ||
      !c->nacc || !c->ptr || !c->nrecv || !c->values || !c->count) {
    orc_corr_free(c);
    return NULL;
  }
  return c;
}

/* Alg. 1 for block k (0-based) with one new sample per series. */
static void corr_update(orc_corr *c, int k, const double *x, const double *y) {
  if (k >= c->b) return; /* R7 */
  const int64_t ns = c->ns;
  const int p = c->p;
  if (k + 1 > c->blocks_used) c->blocks_used = k + 1;
  int slot = c->ptr[k];
  double *rx = c->shx + ((size_t)k * p + slot) * ns;
  double *ry = c->shy + ((size_t)k * p + slot) * ns;
  for (int64_t s = 0; s < ns; ++s) rx[s] = x[s];
  if (c->cross)
    for (int64_t s = 0; s < ns; ++s) ry[s] = y[s];
  c->nrecv[k] += 1;
  double *ax = c->accx + (size_t)k * ns, *ay = c->accy + (size_t)k * ns;
  for (int64_t s = 0; s < ns; ++s) ax[s] += x[s];
  if (c->cross)
    for (int64_t s = 0; s < ns; ++s) ay[s] += y[s];
  c->nacc[k] += 1;
  if (c->nacc[k] == c->m) { /* R3 */
    double *mx = c->tmpx + (size_t)k * ns, *my = c->tmpy + (size_t)k * ns;
    for (int64_t s = 0; s < ns; ++s) mx[s] = ax[s] / (double)c->m;
    if (c->cross)
      for (int64_t s = 0; s < ns; ++s) my[s] = ay[s] / (double)c->m;
    corr_update(c, k + 1, mx, my);
    for (int64_t s = 0; s < ns; ++s) ax[s] = 0.0;
    if (c->cross)
      for (int64_t s = 0; s < ns; ++s) ay[s] = 0.0;
    c->nacc[k] = 0;
  }
  int lo = (k == 0) ? 0 : p / c->m; /* R4 */
  for (int lag = lo; lag < p; ++lag) {
    if ((int64_t)lag >= c->nrecv[k]) break; /* R1: older sample must exist */
    int j = ((slot - lag) % p + p) % p;
    const double *ox = c->shx + ((size_t)k * p + j) * ns; /* older x (R5) */
    for (int64_t g = 0; g < c->ng; ++g) {
      double acc = 0.0;
      const int64_t s0 = g * c->gs, s1 = s0 + c->gs;
#pragma omp parallel for reduction(+ : acc) if (c->gs > 65536)
      for (int64_t s = s0; s < s1; ++s) acc += ox[s] * ry[s];
      c->values[((size_t)g * c->b + k) * p + lag] += acc;
    }
    c->count[(size_t)k * p + lag] += 1;
  }
  c->ptr[k] = (slot + 1) % p;
}

/* Pushes one sample of every series into block 1.  y may be NULL for an
 * autocorrelator (cross == 0); it must be NULL or equal to x then. */
int orc_corr_push(orc_corr *c, const double *x, const double *y) {
  if (!c || !x) return ORC_EINVAL;
  if (c->cross && !y) return ORC_EINVAL;
  corr_update(c, 0, x, c->cross ? y : x);
  return ORC_OK;
}

/* Alg. 2 for group g (R6): writes up to cap (time, value) pairs with
 * value = lag sum / (count * gs); returns the number of points (or the
 * number needed when cap is too small, as a negative count). */
int64_t orc_corr_read(const orc_corr *c, int64_t g, double *times,
                      double *values, int64_t cap) {
  if (!c || g < 0 || g >= c->ng) return 0;
  int64_t npts = 0;
  const int p = c->p;
  for (int k = 0; k < c->blocks_used; ++k) {
    int lo = (k == 0) ? 0 : p / c->m;
    double scale = pow((double)c->m, (double)k);
    for (int lag = lo; lag < p; ++lag) {
      int64_t cnt = c->count[(size_t)k * p + lag];
      if (cnt <= 0) continue;
      if (npts < cap) {
        times[npts] = lag * scale;
        values[npts] = c->values[((size_t)g * c->b + k) * p + lag] /
                       ((double)cnt * (double)c->gs);
      }
      ++npts;
    }
  }
  return npts <= cap ? npts : -npts;
}

/* Raw state for tests: lag sums [ng][b][p] and counts [b][p]. */
void orc_corr_raw(const orc_corr *c, double *values, int64_t *count,
                  int *blocks_used) {
  memcpy(values, c->values, sizeof(double) * (size_t)c->ng * c->b * c->p);
  memcpy(count, c->count, sizeof(int64_t) * (size_t)c->b * c->p);
  *blocks_used = c->blocks_used;
}

/* Eq. (cor): C(l) = 1/(S-l) sum_{s=1}^{S-l} X(s) Y(s+l), for l = 0..L-1. */
int orc_direct_corr(int64_t S, const double *x, const double *y, int64_t L,
                    double *out) {
  if (L > S) return ORC_EINVAL;
  for (int64_t l = 0; l < L; ++l) {
    double acc = 0.0;
    for (int64_t s = 0; s < S - l; ++s) acc += x[s] * y[s + l];
    out[l] = acc / (double)(S - l);
  }
  return ORC_OK;
}

/* ----------------------------------------------------- Green-Kubo */

/* Integral of the piecewise-linear interpolant through (t_i, c_i) from t_0
 * to min(t_cut, t_{n-1}) (trapezoid rule, Sec. 2.3 "numerical
 * integration"), times prefactor.  running[i] (optional) is the integral
 * from t_0 to t_i, times prefactor, for every i. */
int orc_gk_trapz(int64_t n, const double *t, const double *c, double t_cut,
                 double prefactor, double *integral, double *running) {
  if (n < 1) return ORC_EINVAL;
  for (int64_t i = 1; i < n; ++i)
    if (!(t[i] > t[i - 1])) return ORC_EINVAL;
  double acc = 0.0, cut = 0.0;
  int done = 0;
  if (running) running[0] = 0.0;
  if (t_cut <= t[0]) done = 1;
  for (int64_t i = 1; i < n; ++i) {
    double h = t[i] - t[i - 1];
    if (!done && t_cut < t[i]) {
      double frac = (t_cut - t[i - 1]) / h;
      double ccut = c[i - 1] + frac * (c[i] - c[i - 1]);
      cut = acc + 0.5 * (t_cut - t[i - 1]) * (c[i - 1] + ccut);
      done = 1;
    }
    acc += 0.5 * h * (c[i - 1] + c[i]);
    if (running) running[i] = prefactor * acc;
  }
  if (!done) cut = acc;
  *integral = prefactor * cut;
  return ORC_OK;
}

/* ------------------------------------------------ velocity Verlet NVE */

typedef struct {
  int64_t n;
  double L, eps, sig, rc, dt;
  int shift, use_cells;
  double *r, *v, *F, *epot, *W, *mass_of;
  int64_t step;
  double obs[ORC_NOBS];
} orc_md;

void orc_md_free(orc_md *h) {
  if (!h) return;
  free(h->r); free(h->v); free(h->F); free(h->epot); free(h->W); free(h->mass_of);
  free(h);
}

static int md_forces(orc_md *h) {
  if (h->use_cells)
    return orc_lj_cells(h->n, h->r, h->L, h->eps, h->sig, h->rc, h->shift, h->F, h->epot, h->W);
  return orc_lj_brute(h->n, h->r, h->L, 1, h->eps, h->sig, h->rc, h->shift, h->F, h->epot, h->W);
}

/* Copies the inputs; computes the forces and observables at t = 0. */
orc_md *orc_md_new(int64_t n, double L, const double *r, const double *v,
                   const int32_t *type, int ntypes, const double *mass,
                   double eps, double sig, double rc, int shift, double dt,
                   int use_cells) {
  if (n < 2 || L <= 0.0 || ntypes < 1) return NULL;
  orc_md *h = calloc(1, sizeof(orc_md));
  if (!h) return NULL;
  h->n = n; h->L = L; h->eps = eps; h->sig = sig; h->rc = rc; h->dt = dt;
  h->shift = shift; h->use_cells = use_cells;
  h->r = malloc(sizeof(double) * 3 * n);
  h->v = malloc(sizeof(double) * 3 * n);
  h->F = malloc(sizeof(double) * 3 * n);
  h->epot = malloc(sizeof(double) * n);
  h->W = malloc(sizeof(double) * 6 * n);
  h->mass_of = malloc(sizeof(double) * n);
  if (!h->r || !h->v || !h->F || !h->epot || !h->W || !h->mass_of) {
    orc_md_free(h);
    return NULL;
  }
  memcpy(h->r, r, sizeof(double) * 3 * n);
  memcpy(h->v, v, sizeof(double) * 3 * n);
  for (int64_t i = 0; i < n; ++i) {
    int t = type ? type[i] : 0;
    if (t < 0 || t >= ntypes) { orc_md_free(h); return NULL; }
    h->mass_of[i] = mass[t];
  }
  if (md_forces(h) != ORC_OK) { orc_md_free(h); return NULL; }
  orc_observables(n, L * L * L, h->mass_of, h->v, h->epot, h->W, h->obs);
  return h;
}

/* nsteps of velocity Verlet (kick, drift, forces, kick), then the system
 * observables of the new state.  After each step, the scalar correlator cs
 * (6 series: sigma_xy, sigma_xz, sigma_yz, q_x, q_y, q_z) receives a sample
 * every us steps and the velocity correlator cv (3n series, component-major
 * v_x of every atom, then v_y, then v_z) every uv steps; either may be
 * NULL.  obs_out (optional) receives ORC_NOBS values per step. */
int orc_md_step(orc_md *h, int64_t nsteps, orc_corr *cs, int64_t us,
                orc_corr *cv, int64_t uv, double *obs_out) {
  const int64_t n = h->n;
  const double dt = h->dt, V = h->L * h->L * h->L;
  if ((cs && (cs->ns != 6 || us < 1)) || (cv && (cv->ns != 3 * n || uv < 1)))
    return ORC_EINVAL;
  for (int64_t s = 0; s < nsteps; ++s) {
    for (int64_t i = 0; i < n; ++i)
      for (int a = 0; a < 3; ++a) {
        h->v[a * n + i] += 0.5 * dt * h->F[a * n + i] / h->mass_of[i];
        h->r[a * n + i] += dt * h->v[a * n + i];
        h->r[a * n + i] = wrap_box(h->r[a * n + i], h->L);
      }
    int rc = md_forces(h);
    if (rc != ORC_OK) return rc;
    for (int64_t i = 0; i < n; ++i)
      for (int a = 0; a < 3; ++a)
        h->v[a * n + i] += 0.5 * dt * h->F[a * n + i] / h->mass_of[i];
    orc_observables(n, V, h->mass_of, h->v, h->epot, h->W, h->obs);
    h->step += 1;
    if (obs_out) memcpy(obs_out + s * ORC_NOBS, h->obs, sizeof(double) * ORC_NOBS);
    if (cs && h->step % us == 0) {
      double x[6] = {h->obs[6], h->obs[7], h->obs[8], h->obs[9], h->obs[10], h->obs[11]};
      orc_corr_push(cs, x, NULL);
    }
    if (cv && h->step % uv == 0) orc_corr_push(cv, h->v, NULL);
  }
  return ORC_OK;
}

void orc_md_get(const orc_md *h, double *r, double *v, double *F, double *epot,
                double *W, double *obs) {
  const int64_t n = h->n;
  if (r) memcpy(r, h->r, sizeof(double) * 3 * n);
  if (v) memcpy(v, h->v, sizeof(double) * 3 * n);
  if (F) memcpy(F, h->F, sizeof(double) * 3 * n);
  if (epot) memcpy(epot, h->epot, sizeof(double) * n);
  if (W) memcpy(W, h->W, sizeof(double) * 6 * n);
  if (obs) memcpy(obs, h->obs, sizeof(double) * ORC_NOBS);
}

/* Multiplies every velocity by lam (the velocity-rescaling equilibration
 * used before correlated runs) and refreshes the observables. */
void orc_md_scale_velocities(orc_md *h, double lam) {
  for (int64_t i = 0; i < 3 * h->n; ++i) h->v[i] *= lam;
  orc_observables(h->n, h->L * h->L * h->L, h->mass_of, h->v, h->epot, h->W, h->obs);
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Sets the number of OpenMP threads of the following calls (timing only:
 * every per-atom result is computed by one thread whatever the count). */
void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
