/*
 * FP64 CPU oracle for model-based AR-OAM inversion (Li et al., arXiv:2009.10173).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header, table or constant generator
 * with the CUDA path.
 *
 * What it computes, each in the plainest form that follows the paper:
 *   - the sensor-surface patches of Eq. 3 (sub-elements x_j with areas dx_j),
 *     laid out as rings uniform in polar angle with 8*u_r patches per ring
 *     (reading of the unspecified patch layout; axial symmetry, Results);
 *   - the per-position model slab of Eq. 4 (A_s = sum_j A_j dx_j), with the
 *     point-voxel reading of Eq. 1: a voxel at distance d from patch j adds
 *     (dx_j / d) * de/dtau(tau - D_j) to the signal, D_j = fs*(d/c - t0), where
 *     e is the electrical impulse response (Gaussian-windowed cosine) and the
 *     time derivative of Eq. 1 is moved onto e (arbitrary units, Eq. 2);
 *   - the forward operator A and its transpose as lateral correlations of that
 *     slab with the volume ("two coordinate systems", Efficient reconstruction
 *     based on scanning symmetries), zero outside the scan and voxel grids.
 *
 * Lengths enter in metres and are converted to millimetres so that a weight
 * dx_j/d_j is in mm.  All arithmetic is IEEE double; the build uses
 * -ffp-contract=off so that x86 and Arm hosts produce the same bits.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
  double focal_m, aperture_m, hole_m, c_mps;
  double fc_hz, frac_bw, trunc_sigma;
  double dx_m, dy_m, dz_m, z0_rel_m, fs_hz, t0_s; /* t0_s: NaN = automatic */
  int32_t n_patches, px, py, nz, nt, win;
} orc_params;

enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_EWINDOW = -2, ORC_ENOMEM = -3 };

/* ------------------------------------------------------------------------ */
/* Sensor surface patches (Eq. 3).                                          */
/* The spherical cap of radius F and aperture D (optional central hole h)   */
/* spans polar angles [asin(h/2F), asin(D/2F)] about the acoustic axis.     */
/* Rings are uniform in polar angle (at most M/8 of them); ring r gets 8*u_r patches with */
/* sum u_r = M/8, each ring at least one unit and the rest shared in        */
/* proportion to ring area by largest remainder (ties to the inner ring).   */
/* Patch j: unit normal n_j (pointing from the surface to the focus is -n), */
/* surface point q_j = -F n_j about the focus, area w_j.                    */
/* ------------------------------------------------------------------------ */
int orc_patch_count_rings(const orc_params *p) {
  double F = p->focal_m, D = p->aperture_m, h = p->hole_m;
  int M = p->n_patches;
  if (!(F > 0) || !(D > 0) || !(D < 2 * F) || h < 0 || !(h < D) || M <= 0 || M % 8)
    return ORC_EINVAL;
  double tmin = asin(h / (2 * F)), tmax = asin(D / (2 * F));
  double atot = 2 * M_PI * F * F * (cos(tmin) - cos(tmax));
  long nr = lround((tmax - tmin) * F * sqrt((double)M / atot));
  if (nr < 1) nr = 1;
  if (nr > M / 8) nr = M / 8; /* every ring needs at least one unit of 8 patches */
  return (int)nr;
}

int orc_patches(const orc_params *p, double *nx, double *ny, double *nz, double *w) {
  int nr = orc_patch_count_rings(p);
  if (nr < 0) return nr;
  double F = p->focal_m, D = p->aperture_m, h = p->hole_m;
  int M = p->n_patches, U = M / 8;
  double tmin = asin(h / (2 * F)), tmax = asin(D / (2 * F));
  double atot = 2 * M_PI * F * F * (cos(tmin) - cos(tmax));
  double *ar = malloc(sizeof(double) * nr), *frac = malloc(sizeof(double) * nr);
  int *u = malloc(sizeof(int) * nr), *bonus = calloc(nr, sizeof(int));
  if (!ar || !frac || !u || !bonus) { free(ar); free(frac); free(u); free(bonus); return ORC_ENOMEM; }
  int rest = U - nr, given = 0;
  for (int r = 0; r < nr; ++r) {
    double t0 = tmin + (tmax - tmin) * r / nr, t1 = tmin + (tmax - tmin) * (r + 1) / nr;
    ar[r] = 2 * M_PI * F * F * (cos(t0) - cos(t1));
    double q = rest * ar[r] / atot;
    double f = floor(q);
    u[r] = 1 + (int)f;
    frac[r] = q - f;
    given += (int)f;
  }
  for (int left = rest - given; left > 0; --left) { /* largest remainder, ties to lower r */
    int best = -1;
    for (int r = 0; r < nr; ++r)
      if (!bonus[r] && (best < 0 || frac[r] > frac[best])) best = r;
    bonus[best] = 1;
    u[best] += 1;
  }
  int j = 0;
  for (int r = 0; r < nr; ++r) {
    double t0 = tmin + (tmax - tmin) * r / nr, t1 = tmin + (tmax - tmin) * (r + 1) / nr;
    double ct = 0.5 * (cos(t0) + cos(t1));
    double st = sqrt(1.0 - ct * ct);
    int n = 8 * u[r];
    for (int m = 0; m < n; ++m, ++j) {
      double phi = (m + 0.5) * 2 * M_PI / n;
      nx[j] = st * cos(phi);
      ny[j] = st * sin(phi);
      nz[j] = ct;
      w[j] = ar[r] / n;
    }
  }
  free(ar); free(frac); free(u); free(bonus);
  return j; /* == M */
}

/* ------------------------------------------------------------------------ */
/* Electrical impulse response and its time derivative, in sample units.    */
/* e(tau) = exp(-tau^2 / (2 s^2)) cos(w tau), s = fs / (2 pi sf),           */
/* sf = fc * frac_bw / (2 sqrt(2 ln 2)) (the -6 dB amplitude width of the   */
/* Gaussian spectrum equals frac_bw * fc), w = 2 pi fc / fs;                 */
/* zero for |tau| > trunc_sigma * s.                                        */
/* ------------------------------------------------------------------------ */
static void eir_consts(const orc_params *p, double *sig, double *om, double *cut) {
  double sf = p->fc_hz * p->frac_bw / (2.0 * sqrt(2.0 * log(2.0)));
  *sig = p->fs_hz / (2 * M_PI * sf);
  *om = 2 * M_PI * p->fc_hz / p->fs_hz;
  *cut = p->trunc_sigma * (*sig);
}

double orc_eir(const orc_params *p, double tau) {
  double s, w, cut;
  eir_consts(p, &s, &w, &cut);
  if (fabs(tau) > cut) return 0.0;
  return exp(-tau * tau / (2 * s * s)) * cos(w * tau);
}

double orc_eir_dot(const orc_params *p, double tau) {
  double s, w, cut;
  eir_consts(p, &s, &w, &cut);
  if (fabs(tau) > cut) return 0.0;
  double g = exp(-tau * tau / (2 * s * s));
  return -g * ((tau / (s * s)) * cos(w * tau) + w * sin(w * tau));
}

/* ------------------------------------------------------------------------ */
/* Geometry.  Origin at the focus of the sensor at scan position (0,0), z   */
/* into depth.  The voxel at tap (b, a), depth k sits at                    */
/* r = (a dx, b dy, z0_rel + k dz); its distance to patch j is |r - q_j|.   */
/* ------------------------------------------------------------------------ */
static double dist(const orc_params *p, double rx, double ry, double rz,
                   double nx, double ny, double nz) {
  double F = p->focal_m;
  double ex = rx + F * nx, ey = ry + F * ny, ez = rz + F * nz;
  return sqrt(ex * ex + ey * ey + ez * ez);
}

typedef struct {
  int M;
  double *nx, *ny, *nz, *w;
} patchset;

static int load_patches(const orc_params *p, patchset *ps) {
  ps->M = p->n_patches;
  ps->nx = malloc(sizeof(double) * 4 * (size_t)ps->M);
  if (!ps->nx) return ORC_ENOMEM;
  ps->ny = ps->nx + ps->M; ps->nz = ps->ny + ps->M; ps->w = ps->nz + ps->M;
  int r = orc_patches(p, ps->nx, ps->ny, ps->nz, ps->w);
  if (r < 0) { free(ps->nx); return r; }
  return ORC_OK;
}

/* Minimum and maximum distance over every slab voxel and patch. */
int orc_distance_range(const orc_params *p, double *dmin, double *dmax) {
  patchset ps;
  int rc = load_patches(p, &ps);
  if (rc) return rc;
  int R = (p->win - 1) / 2, W = p->win;
  double lo = INFINITY, hi = -INFINITY;
#pragma omp parallel for reduction(min : lo) reduction(max : hi) schedule(static)
  for (int t = 0; t < W * W; ++t) {
    int b = t / W - R, a = t % W - R;
    for (int k = 0; k < p->nz; ++k)
      for (int j = 0; j < ps.M; ++j) {
        double d = dist(p, a * p->dx_m, b * p->dy_m, p->z0_rel_m + k * p->dz_m,
                        ps.nx[j], ps.ny[j], ps.nz[j]);
        if (d < lo) lo = d;
        if (d > hi) hi = d;
      }
  }
  free(ps.nx);
  *dmin = lo; *dmax = hi;
  return ORC_OK;
}

/* Time origin.  The paper does not state one; sample n is at time
 * t0 + n/fs with t0 = (floor(fs dmin / c - T s) - 2) / fs, and the window
 * must hold the latest arrival: fs (dmax/c - t0) + T s < Nt. */
int orc_t0(const orc_params *p, double *t0) {
  if (p->win < 1 || p->win % 2 == 0 || p->nz < 1 || p->nt < 1 || !(p->fs_hz > 0) ||
      !(p->c_mps > 0) || !(p->trunc_sigma > 0) || !(p->fc_hz > 0) || !(p->frac_bw > 0))
    return ORC_EINVAL;
  double dmin, dmax, s, w, cut;
  int rc = orc_distance_range(p, &dmin, &dmax);
  if (rc) return rc;
  eir_consts(p, &s, &w, &cut);
  double t = isnan(p->t0_s) ? (floor(p->fs_hz * dmin / p->c_mps - cut) - 2.0) / p->fs_hz : p->t0_s;
  if (p->fs_hz * (dmin / p->c_mps - t) - cut < 0) return ORC_EWINDOW;
  if (p->fs_hz * (dmax / p->c_mps - t) + cut >= p->nt) return ORC_EWINDOW;
  *t0 = t;
  return ORC_OK;
}

/* Accumulate one voxel's signal (Eq. 3 summed over patches) into out[0..nt). */
static void voxel_signal(const orc_params *p, const patchset *ps, double t0,
                         double rx, double ry, double rz, double *out) {
  double s, w, cut;
  eir_consts(p, &s, &w, &cut);
  for (int j = 0; j < ps->M; ++j) {
    double d = dist(p, rx, ry, rz, ps->nx[j], ps->ny[j], ps->nz[j]);
    double Dj = p->fs_hz * (d / p->c_mps - t0);
    double wt = ps->w[j] / d * 1e3; /* mm^2 / mm */
    int n0 = (int)ceil(Dj - cut), n1 = (int)floor(Dj + cut);
    if (n0 < 0) n0 = 0;
    if (n1 > p->nt - 1) n1 = p->nt - 1;
    for (int n = n0; n <= n1; ++n) out[n] += wt * orc_eir_dot(p, n - Dj);
  }
}

/* One slab column S[b, a, k, 0..nt) (Eq. 4). */
int orc_slab_column(const orc_params *p, double t0, int b, int a, int k, double *out) {
  patchset ps;
  int rc = load_patches(p, &ps);
  if (rc) return rc;
  memset(out, 0, sizeof(double) * p->nt);
  voxel_signal(p, &ps, t0, a * p->dx_m, b * p->dy_m, p->z0_rel_m + k * p->dz_m, out);
  free(ps.nx);
  return ORC_OK;
}

/* Whole slab S[win][win][nz][nt]. */
int orc_slab(const orc_params *p, double t0, double *S) {
  patchset ps;
  int rc = load_patches(p, &ps);
  if (rc) return rc;
  int R = (p->win - 1) / 2, W = p->win;
  size_t nt = p->nt;
  memset(S, 0, sizeof(double) * (size_t)W * W * p->nz * nt);
#pragma omp parallel for schedule(dynamic)
  for (int c = 0; c < W * W * p->nz; ++c) {
    int t = c / p->nz, k = c % p->nz;
    int b = t / W - R, a = t % W - R;
    voxel_signal(p, &ps, t0, a * p->dx_m, b * p->dy_m, p->z0_rel_m + k * p->dz_m, S + (size_t)c * nt);
  }
  free(ps.nx);
  return ORC_OK;
}

/* Slab at one time sample n for every tap and depth: out[win][win][nz]. */
int orc_slab_time_slice(const orc_params *p, double t0, int n, double *out) {
  patchset ps;
  int rc = load_patches(p, &ps);
  if (rc) return rc;
  int R = (p->win - 1) / 2, W = p->win;
  double s, w, cut;
  eir_consts(p, &s, &w, &cut);
#pragma omp parallel for schedule(dynamic)
  for (int c = 0; c < W * W * p->nz; ++c) {
    int t = c / p->nz, k = c % p->nz;
    int b = t / W - R, a = t % W - R;
    double acc = 0;
    for (int j = 0; j < ps.M; ++j) {
      double d = dist(p, a * p->dx_m, b * p->dy_m, p->z0_rel_m + k * p->dz_m, ps.nx[j], ps.ny[j], ps.nz[j]);
      double tau = n - p->fs_hz * (d / p->c_mps - t0);
      if (fabs(tau) <= cut) acc += ps.w[j] / d * 1e3 * orc_eir_dot(p, tau);
    }
    out[c] = acc;
  }
  free(ps.nx);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Forward operator A (Eq. 4 applied through the scanning symmetry):        */
/*   s[y][x][n] = sum_{b,a,k} S[b,a,k,n] H[y+b][x+a][k],                    */
/* H = 0 outside the grid.  Layouts: H[py][px][nz], s[py][px][nt].          */
/* Columns that are zero outside [first,last] contribute exact zeros, so    */
/* the loop visits only that range (no change to any sum).                  */
/* ------------------------------------------------------------------------ */
static void column_ranges(const double *S, size_t ncol, int nt, int *first, int *last) {
  for (size_t c = 0; c < ncol; ++c) {
    const double *col = S + c * nt;
    int f = nt, l = -1;
    for (int n = 0; n < nt; ++n)
      if (col[n] != 0.0) { if (f == nt) f = n; l = n; }
    first[c] = f; last[c] = l;
  }
}

int orc_forward(const double *S, int win, int nz, int nt, int py, int px, const double *H, double *s) {
  int R = (win - 1) / 2;
  size_t ncol = (size_t)win * win * nz;
  int *first = malloc(sizeof(int) * ncol), *last = malloc(sizeof(int) * ncol);
  if (!first || !last) { free(first); free(last); return ORC_ENOMEM; }
  column_ranges(S, ncol, nt, first, last);
#pragma omp parallel for schedule(dynamic)
  for (int pos = 0; pos < py * px; ++pos) {
    int y = pos / px, x = pos % px;
    double *out = s + (size_t)pos * nt;
    for (int n = 0; n < nt; ++n) out[n] = 0.0;
    for (int b = -R; b <= R; ++b) {
      if (y + b < 0 || y + b >= py) continue;
      for (int a = -R; a <= R; ++a) {
        if (x + a < 0 || x + a >= px) continue;
        const double *h = H + ((size_t)(y + b) * px + (x + a)) * nz;
        for (int k = 0; k < nz; ++k) {
          size_t c = ((size_t)(b + R) * win + (a + R)) * nz + k;
          const double *col = S + c * nt;
          for (int n = first[c]; n <= last[c]; ++n) out[n] += col[n] * h[k];
        }
      }
    }
  }
  free(first); free(last);
  return ORC_OK;
}

/* Transpose: H[y][x][k] = sum_{b,a,n} S[b,a,k,n] s[y-b][x-a][n]. */
int orc_adjoint(const double *S, int win, int nz, int nt, int py, int px, const double *s, double *H) {
  int R = (win - 1) / 2;
  size_t ncol = (size_t)win * win * nz;
  int *first = malloc(sizeof(int) * ncol), *last = malloc(sizeof(int) * ncol);
  if (!first || !last) { free(first); free(last); return ORC_ENOMEM; }
  column_ranges(S, ncol, nt, first, last);
#pragma omp parallel for schedule(dynamic)
  for (int pos = 0; pos < py * px; ++pos) {
    int y = pos / px, x = pos % px;
    double *out = H + (size_t)pos * nz;
    for (int k = 0; k < nz; ++k) out[k] = 0.0;
    for (int b = -R; b <= R; ++b) {
      if (y - b < 0 || y - b >= py) continue;
      for (int a = -R; a <= R; ++a) {
        if (x - a < 0 || x - a >= px) continue;
        const double *sig = s + ((size_t)(y - b) * px + (x - a)) * nt;
        for (int k = 0; k < nz; ++k) {
          size_t c = ((size_t)(b + R) * win + (a + R)) * nz + k;
          const double *col = S + c * nt;
          double acc = 0.0;
          for (int n = first[c]; n <= last[c]; ++n) acc += col[n] * sig[n];
          out[k] += acc;
        }
      }
    }
  }
  free(first); free(last);
  return ORC_OK;
}

/* Forward output at chosen (position, sample) pairs, from time slices of the
 * slab: s[y][x][n] = sum_{b,a,k} slice_n[b][a][k] H[y+b][x+a][k].  slices
 * holds one [win][win][nz] slice per entry of which[]. */
int orc_forward_at(const double *slices, int win, int nz, int py, int px, const double *H,
                   int count, const int *ys, const int *xs, const int *which, double *out) {
  int R = (win - 1) / 2;
  for (int i = 0; i < count; ++i) {
    const double *sl = slices + (size_t)which[i] * win * win * nz;
    double acc = 0.0;
    int y = ys[i], x = xs[i];
    for (int b = -R; b <= R; ++b) {
      if (y + b < 0 || y + b >= py) continue;
      for (int a = -R; a <= R; ++a) {
        if (x + a < 0 || x + a >= px) continue;
        const double *h = H + ((size_t)(y + b) * px + (x + a)) * nz;
        const double *c = sl + ((size_t)(b + R) * win + (a + R)) * nz;
        for (int k = 0; k < nz; ++k) acc += c[k] * h[k];
      }
    }
    out[i] = acc;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Exact lateral-FFT restatement of A and A^T.                              */
/* Both operators are 2-D correlations over the scan grid, so with the      */
/* volume and the signals zero-padded to P x P (P >= max(py, px) + R, so    */
/* that no circular wrap reaches the output window) the correlation theorem */
/* gives, per depth k and sample n,                                         */
/*   A:    s^_n(v,u)  = sum_k conj(S^_{k,n}(v,u)) H^_k(v,u)                 */
/*   A^T:  H^_k(v,u)  = sum_n      S^_{k,n}(v,u)  s^_n(v,u)                 */
/* where X^ is the 2-D DFT over (y, x) (textbook Cooley-Tukey radix-2 below) */
/* and S_{k,n} holds S[b][a][k][n] at (b mod P, a mod P).                   */
/* ------------------------------------------------------------------------ */

static int is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

/* In-place radix-2 decimation-in-time FFT of n complex values spaced by
 * `stride`: X[f] = sum_j x[j] exp(sign * 2 pi i j f / n), unscaled. */
static void fft1(double *re, double *im, int n, int stride, int sign) {
  for (int i = 1, j = 0; i < n; ++i) { /* bit-reversal permutation */
    int bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) {
      double t = re[(size_t)i * stride]; re[(size_t)i * stride] = re[(size_t)j * stride]; re[(size_t)j * stride] = t;
      t = im[(size_t)i * stride]; im[(size_t)i * stride] = im[(size_t)j * stride]; im[(size_t)j * stride] = t;
    }
  }
  for (int len = 2; len <= n; len <<= 1) {
    const int half = len >> 1;
    for (int q = 0; q < half; ++q) {
      const double ang = sign * 2.0 * M_PI * (double)q / (double)len;
      const double wr = cos(ang), wi = sin(ang);
      for (int s0 = 0; s0 < n; s0 += len) {
        const size_t i0 = (size_t)(s0 + q) * stride, i1 = (size_t)(s0 + q + half) * stride;
        const double xr = re[i1] * wr - im[i1] * wi, xi = re[i1] * wi + im[i1] * wr;
        re[i1] = re[i0] - xr; im[i1] = im[i0] - xi;
        re[i0] += xr; im[i0] += xi;
      }
    }
  }
}

/* 2-D transform of a P x P row-major array (rows then columns). */
static void fft2(double *re, double *im, int P, int sign) {
  for (int r = 0; r < P; ++r) fft1(re + (size_t)r * P, im + (size_t)r * P, P, 1, sign);
  for (int c = 0; c < P; ++c) fft1(re + c, im + c, P, P, sign);
}

/* Exposed for the tests: one 1-D transform of n values (n a power of two). */
int orc_fft(double *re, double *im, int n, int sign) {
  if (!is_pow2(n) || (sign != 1 && sign != -1)) return ORC_EINVAL;
  fft1(re, im, n, 1, sign);
  return ORC_OK;
}

/* The 2-D DFT of one slab slice S[.][.][k][n] placed at (b mod P, a mod P). */
int orc_slab_dft(const double *S, int win, int nz, int nt, int k, int n, int P, double *re, double *im) {
  const int R = (win - 1) / 2;
  if (!is_pow2(P) || P < win) return ORC_EINVAL;
  memset(re, 0, sizeof(double) * P * P);
  memset(im, 0, sizeof(double) * P * P);
  for (int b = -R; b <= R; ++b)
    for (int a = -R; a <= R; ++a)
      re[(size_t)((b + P) % P) * P + (a + P) % P] = S[(((size_t)(b + R) * win + (a + R)) * nz + k) * nt + n];
  fft2(re, im, P, -1);
  return ORC_OK;
}

static int fft_pad_ok(int P, int R, int py, int px) {
  return is_pow2(P) && P >= py + R && P >= px + R;
}

/* Does any tap of slab column (k, n) differ from zero? */
static int slice_nonzero(const double *S, int win, int nz, int nt, int k, int n) {
  for (int t = 0; t < win * win; ++t)
    if (S[((size_t)t * nz + k) * nt + n] != 0.0) return 1;
  return 0;
}

int orc_forward_fft(const double *S, int win, int nz, int nt, int py, int px, int P, const double *H, double *s) {
  const int R = (win - 1) / 2;
  const size_t PP = (size_t)P * P;
  if (!fft_pad_ok(P, R, py, px)) return ORC_EINVAL;
  double *Hr = calloc(PP * nz, sizeof(double)), *Hi = calloc(PP * nz, sizeof(double));
  if (!Hr || !Hi) { free(Hr); free(Hi); return ORC_ENOMEM; }
  for (int k = 0; k < nz; ++k) {
    for (int y = 0; y < py; ++y)
      for (int x = 0; x < px; ++x) Hr[k * PP + (size_t)y * P + x] = H[((size_t)y * px + x) * nz + k];
    fft2(Hr + k * PP, Hi + k * PP, P, -1);
  }
  int rc = ORC_OK;
#pragma omp parallel
  {
    double *sr = malloc(sizeof(double) * PP), *si = malloc(sizeof(double) * PP);
    double *tr = malloc(sizeof(double) * PP), *ti = malloc(sizeof(double) * PP);
    if (!sr || !si || !tr || !ti) {
#pragma omp atomic write
      rc = ORC_ENOMEM;
    } else {
#pragma omp for schedule(dynamic)
      for (int n = 0; n < nt; ++n) {
        memset(sr, 0, sizeof(double) * PP);
        memset(si, 0, sizeof(double) * PP);
        for (int k = 0; k < nz; ++k) {
          if (!slice_nonzero(S, win, nz, nt, k, n)) continue;
          orc_slab_dft(S, win, nz, nt, k, n, P, tr, ti);
          const double *hr = Hr + k * PP, *hi = Hi + k * PP;
          for (size_t f = 0; f < PP; ++f) { /* conj(S^) * H^ */
            sr[f] += tr[f] * hr[f] + ti[f] * hi[f];
            si[f] += tr[f] * hi[f] - ti[f] * hr[f];
          }
        }
        fft2(sr, si, P, +1);
        for (int y = 0; y < py; ++y)
          for (int x = 0; x < px; ++x) s[((size_t)y * px + x) * nt + n] = sr[(size_t)y * P + x] / (double)PP;
      }
    }
    free(sr); free(si); free(tr); free(ti);
  }
  free(Hr); free(Hi);
  return rc;
}

int orc_adjoint_fft(const double *S, int win, int nz, int nt, int py, int px, int P, const double *s, double *H) {
  const int R = (win - 1) / 2;
  const size_t PP = (size_t)P * P;
  if (!fft_pad_ok(P, R, py, px)) return ORC_EINVAL;
  double *Sr = calloc(PP * nt, sizeof(double)), *Si = calloc(PP * nt, sizeof(double));
  if (!Sr || !Si) { free(Sr); free(Si); return ORC_ENOMEM; }
  for (int n = 0; n < nt; ++n) {
    for (int y = 0; y < py; ++y)
      for (int x = 0; x < px; ++x) Sr[n * PP + (size_t)y * P + x] = s[((size_t)y * px + x) * nt + n];
    fft2(Sr + n * PP, Si + n * PP, P, -1);
  }
  int rc = ORC_OK;
#pragma omp parallel
  {
    double *hr = malloc(sizeof(double) * PP), *hi = malloc(sizeof(double) * PP);
    double *tr = malloc(sizeof(double) * PP), *ti = malloc(sizeof(double) * PP);
    if (!hr || !hi || !tr || !ti) {
#pragma omp atomic write
      rc = ORC_ENOMEM;
    } else {
#pragma omp for schedule(dynamic)
      for (int k = 0; k < nz; ++k) {
        memset(hr, 0, sizeof(double) * PP);
        memset(hi, 0, sizeof(double) * PP);
        for (int n = 0; n < nt; ++n) {
          if (!slice_nonzero(S, win, nz, nt, k, n)) continue;
          orc_slab_dft(S, win, nz, nt, k, n, P, tr, ti);
          const double *xr = Sr + n * PP, *xi = Si + n * PP;
          for (size_t f = 0; f < PP; ++f) { /* S^ * s^ */
            hr[f] += tr[f] * xr[f] - ti[f] * xi[f];
            hi[f] += tr[f] * xi[f] + ti[f] * xr[f];
          }
        }
        fft2(hr, hi, P, +1);
        for (int y = 0; y < py; ++y)
          for (int x = 0; x < px; ++x) H[((size_t)y * px + x) * nz + k] = hr[(size_t)y * P + x] / (double)PP;
      }
    }
    free(hr); free(hi); free(tr); free(ti);
  }
  free(Sr); free(Si);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Lateral-FFT restatement with the slab's spectrum computed once.          */
/* Same correlation-theorem identities as above; the spectrum of every     */
/* slab slice (k, n) inside depth k's band is transformed once per model    */
/* and kept, so an application costs the input and output transforms and  */
/* the spectral sums only.  Depth k's band [klo, klo + klen) is the union,  */
/* over taps and patches, of the samples each patch's EIR window can reach */
/* (all other samples of depth k are exactly zero).  The slab is real, so  */
/* its spectrum is Hermitian: only columns u = 0 .. P/2 are stored, and    */
/* an output spectrum (also of real data) is completed from those columns  */
/* by X(v, u) = conj(X(-v, -u)) before the inverse transform.               */
/* ------------------------------------------------------------------------ */

/* Depth k's band: the union over taps and patches of the patch's EIR      */
/* window [ceil(D_j - cut), floor(D_j + cut)], clipped to [0, nt).         */
int orc_depth_band(const orc_params *p, double t0, int k, int *klo, int *klen) {
  patchset ps;
  int rc = load_patches(p, &ps);
  if (rc) return rc;
  int R = (p->win - 1) / 2;
  double s, w, cut;
  eir_consts(p, &s, &w, &cut);
  int lo = p->nt, hi = -1, W = p->win;
#pragma omp parallel for reduction(min : lo) reduction(max : hi) schedule(static)
  for (int t = 0; t < W * W; ++t) {
    int b = t / W - R, a = t % W - R;
    for (int j = 0; j < ps.M; ++j) {
        double d = dist(p, a * p->dx_m, b * p->dy_m, p->z0_rel_m + k * p->dz_m, ps.nx[j], ps.ny[j], ps.nz[j]);
        double Dj = p->fs_hz * (d / p->c_mps - t0);
        int n0 = (int)ceil(Dj - cut), n1 = (int)floor(Dj + cut);
        if (n0 < 0) n0 = 0;
        if (n1 > p->nt - 1) n1 = p->nt - 1;
        if (n0 > n1) continue;
        if (n0 < lo) lo = n0;
        if (n1 > hi) hi = n1;
    }
  }
  free(ps.nx);
  if (hi < lo) { *klo = 0; *klen = 0; } else { *klo = lo; *klen = hi - lo + 1; }
  return ORC_OK;
}

/* Half spectra of the slab slices (k, n), n in [klo, klo + klen):          */
/* re/im[(n - klo)][v][u], v in [0, P), u in [0, P/2], of the 2-D DFT of    */
/* S[.][.][k][n] placed at (b mod P, a mod P) (sign -1, unscaled).          */
/* symmetric != 0 evaluates Eq. 3 only for one tap per orbit of the patch   */
/* set's symmetries -- (b, a) ~ (+-b, +-a), and (a, b) when dx == dy         */
/* (axial symmetry, Results) -- and copies that column to the orbit's other */
/* taps; the direct evaluation of those taps sums the same terms in another */
/* order, so the two agree to rounding.                                     */
int orc_spectrum_depth(const orc_params *p, double t0, int k, int P, int klo, int klen, int symmetric,
                       double *re, double *im) {
  int R = (p->win - 1) / 2, W = p->win;
  if (!is_pow2(P) || P < W || klo < 0 || klen < 0 || klo + klen > p->nt) return ORC_EINVAL;
  patchset ps;
  int rc = load_patches(p, &ps);
  if (rc) return rc;
  const size_t nt = p->nt, PP = (size_t)P * P, Q = P / 2 + 1;
  double *cols = calloc((size_t)W * W * nt, sizeof(double)); /* S[b][a][k][0..nt) */
  if (!cols) { free(ps.nx); return ORC_ENOMEM; }
  const int swap = symmetric && p->dx_m == p->dy_m;
#pragma omp parallel for schedule(dynamic)
  for (int t = 0; t < W * W; ++t) {
    int b = t / W - R, a = t % W - R;
    if (symmetric && (b < 0 || a < 0 || (swap && a > b))) continue; /* not an orbit representative */
    voxel_signal(p, &ps, t0, a * p->dx_m, b * p->dy_m, p->z0_rel_m + k * p->dz_m, cols + (size_t)t * nt);
  }
  free(ps.nx);
  if (symmetric)
    for (int t = 0; t < W * W; ++t) {
      int b = abs(t / W - R), a = abs(t % W - R);
      if (swap && a > b) { int x = a; a = b; b = x; }
      int rep = (b + R) * W + (a + R);
      if (rep != t) memcpy(cols + (size_t)t * nt, cols + (size_t)rep * nt, sizeof(double) * nt);
    }
#pragma omp parallel
  {
    double *tr = malloc(sizeof(double) * PP), *ti = malloc(sizeof(double) * PP);
    if (!tr || !ti) {
#pragma omp atomic write
      rc = ORC_ENOMEM;
    } else {
#pragma omp for schedule(dynamic)
      for (int i = 0; i < klen; ++i) {
        int n = klo + i;
        memset(tr, 0, sizeof(double) * PP);
        memset(ti, 0, sizeof(double) * PP);
        for (int b = -R; b <= R; ++b)
          for (int a = -R; a <= R; ++a)
            tr[(size_t)((b + P) % P) * P + (a + P) % P] = cols[((size_t)(b + R) * W + (a + R)) * nt + n];
        fft2(tr, ti, P, -1);
        double *dr = re + (size_t)i * P * Q, *di = im + (size_t)i * P * Q;
        for (int v = 0; v < P; ++v)
          for (size_t u = 0; u < Q; ++u) {
            dr[(size_t)v * Q + u] = tr[(size_t)v * P + u];
            di[(size_t)v * Q + u] = ti[(size_t)v * P + u];
          }
      }
    }
    free(tr); free(ti);
  }
  free(cols);
  return rc;
}

/* Complete a half spectrum (columns 0..P/2) of real data to all P columns  */
/* and transform back (sign +1); out[y][x] = Re / P^2 for y < py, x < px.    */
static void half_inverse(const double *hr, const double *hi, int P, double *tr, double *ti) {
  const size_t Q = P / 2 + 1;
  for (int v = 0; v < P; ++v)
    for (int u = 0; u < P; ++u) {
      size_t d = (size_t)v * P + u;
      if ((size_t)u < Q) {
        tr[d] = hr[(size_t)v * Q + u];
        ti[d] = hi[(size_t)v * Q + u];
      } else { /* X(v, u) = conj(X(-v, -u)) */
        size_t sidx = (size_t)((P - v) % P) * Q + (size_t)(P - u);
        tr[d] = hr[sidx];
        ti[d] = -hi[sidx];
      }
    }
  fft2(tr, ti, P, +1);
}

/* A H from the stored half spectra.  klo/klen: per-depth bands; koff[k]:   */
/* index of depth k's first slice in re/im (slices of P x (P/2+1)).         */
int orc_forward_spec(const double *re, const double *im, const int *klo, const int *klen, const long long *koff,
                     int nz, int nt, int P, int R, int py, int px, const double *H, double *s) {
  const size_t PP = (size_t)P * P, Q = P / 2 + 1, PQ = (size_t)P * Q;
  if (!fft_pad_ok(P, R, py, px)) return ORC_EINVAL;
  double *Hr = malloc(sizeof(double) * PQ * nz), *Hi = malloc(sizeof(double) * PQ * nz);
  if (!Hr || !Hi) { free(Hr); free(Hi); return ORC_ENOMEM; }
  int rc = ORC_OK;
#pragma omp parallel
  {
    double *tr = malloc(sizeof(double) * PP), *ti = malloc(sizeof(double) * PP);
    double *ar = malloc(sizeof(double) * PQ), *ai = malloc(sizeof(double) * PQ);
    if (!tr || !ti || !ar || !ai) {
#pragma omp atomic write
      rc = ORC_ENOMEM;
    } else {
#pragma omp for schedule(dynamic)
      for (int k = 0; k < nz; ++k) { /* H^_k, half spectrum */
        memset(tr, 0, sizeof(double) * PP);
        memset(ti, 0, sizeof(double) * PP);
        for (int y = 0; y < py; ++y)
          for (int x = 0; x < px; ++x) tr[(size_t)y * P + x] = H[((size_t)y * px + x) * nz + k];
        fft2(tr, ti, P, -1);
        for (int v = 0; v < P; ++v)
          for (size_t u = 0; u < Q; ++u) {
            Hr[k * PQ + (size_t)v * Q + u] = tr[(size_t)v * P + u];
            Hi[k * PQ + (size_t)v * Q + u] = ti[(size_t)v * P + u];
          }
      }
#pragma omp for schedule(dynamic)
      for (int n = 0; n < nt; ++n) {
        int any = 0;
        memset(ar, 0, sizeof(double) * PQ);
        memset(ai, 0, sizeof(double) * PQ);
        for (int k = 0; k < nz; ++k) {
          if (n < klo[k] || n >= klo[k] + klen[k]) continue;
          any = 1;
          const double *sr = re + (size_t)(koff[k] + (n - klo[k])) * PQ, *si = im + (size_t)(koff[k] + (n - klo[k])) * PQ;
          const double *hr = Hr + k * PQ, *hi = Hi + k * PQ;
          for (size_t f = 0; f < PQ; ++f) { /* conj(S^) * H^ */
            ar[f] += sr[f] * hr[f] + si[f] * hi[f];
            ai[f] += sr[f] * hi[f] - si[f] * hr[f];
          }
        }
        if (!any) {
          for (int y = 0; y < py; ++y)
            for (int x = 0; x < px; ++x) s[((size_t)y * px + x) * nt + n] = 0.0;
          continue;
        }
        half_inverse(ar, ai, P, tr, ti);
        for (int y = 0; y < py; ++y)
          for (int x = 0; x < px; ++x) s[((size_t)y * px + x) * nt + n] = tr[(size_t)y * P + x] / (double)PP;
      }
    }
    free(tr); free(ti); free(ar); free(ai);
  }
  free(Hr); free(Hi);
  return rc;
}

/* A^T s from the stored half spectra. */
int orc_adjoint_spec(const double *re, const double *im, const int *klo, const int *klen, const long long *koff,
                     int nz, int nt, int P, int R, int py, int px, const double *s, double *H) {
  const size_t PP = (size_t)P * P, Q = P / 2 + 1, PQ = (size_t)P * Q;
  if (!fft_pad_ok(P, R, py, px)) return ORC_EINVAL;
  int nlo = nt, nhi = 0; /* samples some band reaches */
  for (int k = 0; k < nz; ++k)
    if (klen[k] > 0) {
      if (klo[k] < nlo) nlo = klo[k];
      if (klo[k] + klen[k] > nhi) nhi = klo[k] + klen[k];
    }
  const int NS = nhi > nlo ? nhi - nlo : 0;
  double *Sr = malloc(sizeof(double) * PQ * (NS ? NS : 1)), *Si = malloc(sizeof(double) * PQ * (NS ? NS : 1));
  if (!Sr || !Si) { free(Sr); free(Si); return ORC_ENOMEM; }
  int rc = ORC_OK;
#pragma omp parallel
  {
    double *tr = malloc(sizeof(double) * PP), *ti = malloc(sizeof(double) * PP);
    double *ar = malloc(sizeof(double) * PQ), *ai = malloc(sizeof(double) * PQ);
    if (!tr || !ti || !ar || !ai) {
#pragma omp atomic write
      rc = ORC_ENOMEM;
    } else {
#pragma omp for schedule(dynamic)
      for (int i = 0; i < NS; ++i) { /* s^_n, half spectrum */
        int n = nlo + i;
        memset(tr, 0, sizeof(double) * PP);
        memset(ti, 0, sizeof(double) * PP);
        for (int y = 0; y < py; ++y)
          for (int x = 0; x < px; ++x) tr[(size_t)y * P + x] = s[((size_t)y * px + x) * nt + n];
        fft2(tr, ti, P, -1);
        for (int v = 0; v < P; ++v)
          for (size_t u = 0; u < Q; ++u) {
            Sr[i * PQ + (size_t)v * Q + u] = tr[(size_t)v * P + u];
            Si[i * PQ + (size_t)v * Q + u] = ti[(size_t)v * P + u];
          }
      }
#pragma omp for schedule(dynamic)
      for (int k = 0; k < nz; ++k) {
        if (klen[k] == 0) {
          for (int y = 0; y < py; ++y)
            for (int x = 0; x < px; ++x) H[((size_t)y * px + x) * nz + k] = 0.0;
          continue;
        }
        memset(ar, 0, sizeof(double) * PQ);
        memset(ai, 0, sizeof(double) * PQ);
        for (int n = klo[k]; n < klo[k] + klen[k]; ++n) {
          const double *sr = re + (size_t)(koff[k] + (n - klo[k])) * PQ, *si = im + (size_t)(koff[k] + (n - klo[k])) * PQ;
          const double *xr = Sr + (size_t)(n - nlo) * PQ, *xi = Si + (size_t)(n - nlo) * PQ;
          for (size_t f = 0; f < PQ; ++f) { /* S^ * s^ */
            ar[f] += sr[f] * xr[f] - si[f] * xi[f];
            ai[f] += sr[f] * xi[f] + si[f] * xr[f];
          }
        }
        half_inverse(ar, ai, P, tr, ti);
        for (int y = 0; y < py; ++y)
          for (int x = 0; x < px; ++x) H[((size_t)y * px + x) * nz + k] = tr[(size_t)y * P + x] / (double)PP;
      }
    }
    free(tr); free(ti); free(ar); free(ai);
  }
  free(Sr); free(Si);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* The paper's own discretisation of Eq. 1 (Methods, Forward modeling, with  */
/* its ref. [33]): the absorbed energy between voxel centres is the         */
/* trilinear interpolation of the voxel values, i.e. each voxel carries the */
/* tent phi(x) = L(x/dx) L(y/dy) L(z/dz), L(u) = max(0, 1 - |u|); the       */
/* surface integral of Eq. 1 over the sphere |x - x'| = ct is taken of that */
/* interpolant, and the time derivative by a central finite difference on   */
/* the sample grid.                                                          */
/*                                                                           */
/* Over one tent's support (a few micrometres) the sphere of radius ct      */
/* (millimetres) is a plane to within its sagitta (< 1e-3 voxel here), so    */
/* the integral of the tent over the sphere is its planar Radon transform   */
/*   R(s) = int phi(x) delta(e.x - s) dx                                     */
/* along the unit normal e = (v - x)/|v - x| at s = ct - |v - x|.  Each     */
/* factor L(x/dx) projects to a hat of half-width a = |e_x| dx and area dx, */
/* a hat is (1/a) times the convolution of two boxes of width a, and the    */
/* convolution of n boxes of widths c_i is                                   */
/*   sum over sigma in {+-1}^n of prod(sigma) (s + sum sigma_i c_i / 2)_+^(n-1) / (n-1)! */
/* (truncated powers).  An axis with a < 1e-3 max(a) (e nearly orthogonal to */
/* it) projects to a spike of mass d, so its two boxes are dropped and its  */
/* mass multiplies the rest (error ~ (a / max a)^2 < 1e-6).                  */
/* ------------------------------------------------------------------------ */
double orc_tent_radon(double dx, double dy, double dz, double ex, double ey, double ez, double s) {
  const double d[3] = {dx, dy, dz}, e[3] = {fabs(ex), fabs(ey), fabs(ez)};
  double a[3], amax = 0.0;
  for (int i = 0; i < 3; ++i) {
    a[i] = e[i] * d[i];
    if (a[i] > amax) amax = a[i];
  }
  double c[6], scale = 1.0;
  int n = 0;
  for (int i = 0; i < 3; ++i) {
    if (a[i] < 1e-3 * amax) {
      scale *= d[i];  /* spike of mass d */
    } else {
      c[n++] = a[i];
      c[n++] = a[i];
      scale *= d[i] / (a[i] * a[i]);
    }
  }
  double fact = 1.0; /* (n-1)! */
  for (int i = 2; i < n; ++i) fact *= i;
  double sum = 0.0;
  for (int mask = 0; mask < (1 << n); ++mask) {
    double x = s, sign = 1.0;
    for (int i = 0; i < n; ++i) {
      if (mask & (1 << i)) { x -= 0.5 * c[i]; sign = -sign; }
      else x += 0.5 * c[i];
    }
    if (x > 0.0) sum += sign * pow(x, n - 1);
  }
  return scale * sum / fact;
}

/* One slab column of the discretised model, S33[b, a, k, 0..nt):            */
/*   I_j(m)  = R_j(c t_m - r_j) / (c t_m),  t_m = t0 + m / fs  (r_j = |v - q_j|, */
/*             lengths in mm; e_j the unit vector from patch j to the voxel) */
/*   D_j(m)  = (I_j(m + 1) - I_j(m - 1)) / 2           (central difference)  */
/*   S33(n)  = sum_j w_j sum_m e(n - m) D_j(m)          (EIR sampled at whole */
/*             samples, e(tau) of the point model, zero beyond trunc_sigma)  */
/* Arbitrary units as Eq. 2; for a tent much smaller than a wavelength and   */
/* samples much finer than the tent it tends to (V fs / c) times the point-  */
/* voxel column, V = dx dy dz the tent's volume.                             */
int orc_slab33_column(const orc_params *p, double t0, int b, int a, int k, double *out) {
  patchset ps;
  int rc = load_patches(p, &ps);
  if (rc) return rc;
  double sg, om, cut;
  eir_consts(p, &sg, &om, &cut);
  const int T = (int)floor(cut);
  const int nt = p->nt;
  double *D = calloc((size_t)nt + 2, sizeof(double)); /* D[m + 1], m in [-1, nt] */
  double *e = malloc(sizeof(double) * (2 * (size_t)T + 1));
  if (!D || !e) { free(D); free(e); free(ps.nx); return ORC_ENOMEM; }
  for (int m = -T; m <= T; ++m) e[m + T] = orc_eir(p, (double)m);
  memset(out, 0, sizeof(double) * nt);
  const double F = p->focal_m * 1e3, ddx = p->dx_m * 1e3, ddy = p->dy_m * 1e3, ddz = p->dz_m * 1e3;
  const double vx = a * ddx, vy = b * ddy, vz = (p->z0_rel_m + k * p->dz_m) * 1e3;
  const double c_mm = p->c_mps * 1e3, h = ddx + ddy + ddz; /* support half-width bound along any e */
  for (int j = 0; j < ps.M; ++j) {
    const double qx = -F * ps.nx[j], qy = -F * ps.ny[j], qz = -F * ps.nz[j];
    const double ux = vx - qx, uy = vy - qy, uz = vz - qz;
    const double r = sqrt(ux * ux + uy * uy + uz * uz);
    const double ex = ux / r, ey = uy / r, ez = uz / r;
    /* samples m with |c t_m - r| < h carry the tent */
    const int m0 = (int)floor(p->fs_hz * ((r - h) / c_mm - t0)) - 1;
    const int m1 = (int)ceil(p->fs_hz * ((r + h) / c_mm - t0)) + 1;
    memset(D, 0, sizeof(double) * ((size_t)nt + 2));
    for (int m = (m0 < -1 ? -1 : m0); m <= (m1 > nt ? nt : m1); ++m) {
      /* D(m) = (I(m+1) - I(m-1)) / 2 */
      const double rho1 = c_mm * (t0 + (m + 1) / p->fs_hz), rho0 = c_mm * (t0 + (m - 1) / p->fs_hz);
      const double i1 = orc_tent_radon(ddx, ddy, ddz, ex, ey, ez, rho1 - r) / rho1;
      const double i0 = orc_tent_radon(ddx, ddy, ddz, ex, ey, ez, rho0 - r) / rho0;
      D[m + 1] = 0.5 * (i1 - i0);
    }
    const double wj = ps.w[j] * 1e6; /* mm^2 */
    const int n0 = (m0 - T < 0 ? 0 : m0 - T), n1 = (m1 + T > nt - 1 ? nt - 1 : m1 + T);
    for (int n = n0; n <= n1; ++n) { /* D is zero outside [m0, m1] */
      double acc = 0.0;
      for (int m = n - T; m <= n + T; ++m) {
        if (m < -1 || m > nt) continue;
        acc += e[n - m + T] * D[m + 1];
      }
      out[n] += wj * acc;
    }
  }
  free(D); free(e); free(ps.nx);
  return ORC_OK;
}
