/*
 * FP64 CPU oracle for Lyman-alpha skewer synthesis (arXiv 2310.18996).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, __graft_entry__.smoke() and
 * bench.py's cpu_baseline / reference legs; never by the product library.
 * Plain loops, double precision, no blocking or fusion beyond what each
 * definition states.  Citations name the paper's sections and equations.
 *
 * Readings of points the paper leaves open (kept identical in the CUDA
 * library, which implements them independently):
 *  - cosmology: flat LCDM of Table 1, Omega_L = 1 - Omega_M, no radiation;
 *  - growth G(z): linear growing mode, normalised to G(0) = 1;
 *  - pixel grid: global, pixel J at comoving distance (J + 1/2) dr, a skewer
 *    takes the pixels with r_lo <= r_J < r_hi of its forest window;
 *  - interpolation: trilinear between voxel centres (i + 1/2) cell, periodic;
 *  - small-scale field: independent realisation per segment of n_fft pixels
 *    aligned to the skewer start, Philox4x32-10 noise, Box-Muller normals
 *    (the Nyquist mode takes the counter-0 words that mode 0 leaves unused);
 *  - a, b, c: ln a, b, c linear in z between nodes, clamped at the ends;
 *  - rebin: box-car mean of R consecutive pixels, incomplete tail dropped.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* Gauss-Legendre rule, computed once from the Legendre recurrence.          */
/* ------------------------------------------------------------------------ */
#define GL_N 20
static double gl_x[GL_N], gl_w[GL_N];
static int gl_ready = 0;

static void gl_init(void) {
  if (gl_ready) return;
#pragma omp critical(orc_gl_init)
  {
    if (!gl_ready) {
      for (int i = 0; i < GL_N; ++i) {
        /* Newton on P_n(x) from the Chebyshev-like first guess. */
        double x = cos(M_PI * (i + 0.75) / (GL_N + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
          double p0 = 1.0, p1 = x;
          for (int k = 2; k <= GL_N; ++k) {
            double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
          }
          dp = GL_N * (x * p1 - p0) / (x * x - 1.0);
          double dx = p1 / dp;
          x -= dx;
          if (fabs(dx) < 1e-16) break;
        }
        gl_x[i] = x;
        gl_w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
      }
      gl_ready = 1;
    }
  }
}

/* Composite Gauss-Legendre of f over [lo, hi] with `pieces` equal panels. */
static double gl_integrate(double (*f)(double, double), double par, double lo, double hi,
                           int pieces) {
  gl_init();
  double h = (hi - lo) / pieces, sum = 0.0;
  for (int p = 0; p < pieces; ++p) {
    double a = lo + p * h, mid = a + 0.5 * h, half = 0.5 * h, s = 0.0;
    for (int i = 0; i < GL_N; ++i) s += gl_w[i] * f(par, mid + half * gl_x[i]);
    sum += s * half;
  }
  return sum;
}

/* ------------------------------------------------------------------------ */
/* Cosmology (Sec. 2, Table 1).                                              */
/* ------------------------------------------------------------------------ */
double orc_hubble_e(double om, double z) {
  double zp = 1.0 + z;
  return sqrt(om * zp * zp * zp + (1.0 - om));
}

static double inv_e(double om, double z) { return 1.0 / orc_hubble_e(om, z); }

/* D_C(z) = (c/H0) int_0^z dz'/E(z').  Checkpoints every 0.1 in z, each the
   integral from the previous checkpoint, then one panel to z. */
#define DC_STEP 0.1
#define DC_MAXCK 200
static double dc_ck_om = -1.0;
static double dc_ck[DC_MAXCK + 1];

static void dc_checkpoints(double om) {
  if (dc_ck_om == om) return;
#pragma omp critical(orc_dc_init)
  {
    if (dc_ck_om != om) {
      dc_ck[0] = 0.0;
      for (int i = 1; i <= DC_MAXCK; ++i)
        dc_ck[i] = dc_ck[i - 1] + gl_integrate(inv_e, om, (i - 1) * DC_STEP, i * DC_STEP, 2);
      dc_ck_om = om;
    }
  }
}

double orc_comoving_distance(double om, double z) {
  if (z <= 0.0) return 0.0;
  dc_checkpoints(om);
  int i = (int)floor(z / DC_STEP);
  if (i > DC_MAXCK) i = DC_MAXCK;
  double z0 = i * DC_STEP;
  double tail = (z > z0) ? gl_integrate(inv_e, om, z0, z, 2) : 0.0;
  return ORC_C_OVER_H0 * (dc_ck[i] + tail);
}

/* Inverse of D_C: bracket on the checkpoints, then Newton with dD/dz = c/(H0 E). */
double orc_z_of_distance(double om, double r) {
  if (r <= 0.0) return 0.0;
  dc_checkpoints(om);
  int i = 0;
  while (i < DC_MAXCK && ORC_C_OVER_H0 * dc_ck[i + 1] < r) ++i;
  double lo = i * DC_STEP, hi = (i + 1) * DC_STEP;
  double z = 0.5 * (lo + hi);
  for (int it = 0; it < 60; ++it) {
    double f = orc_comoving_distance(om, z) - r;
    double step = f * orc_hubble_e(om, z) / ORC_C_OVER_H0;
    double zn = z - step;
    if (zn <= lo || zn >= hi) { /* keep the iterate inside the bracket */
      if (f > 0) hi = z; else lo = z;
      zn = 0.5 * (lo + hi);
    } else {
      if (f > 0) hi = z; else lo = z;
    }
    if (fabs(zn - z) < 1e-15 * (1.0 + z)) { z = zn; break; }
    z = zn;
  }
  return z;
}

/* Linear growing mode D(a) = (5 Om/2) E(a) int_0^a da'/(a' E(a'))^3, with
   a' = s^2 so that the integrand 2 s^4 / (Om + OL s^6)^{3/2} is smooth. */
static double growth_integrand(double om, double s) {
  double s2 = s * s, s6 = s2 * s2 * s2;
  double q = om + (1.0 - om) * s6;
  return 2.0 * s2 * s2 / (q * sqrt(q));
}

static double growth_unnormalised(double om, double a) {
  double ea = sqrt(om / (a * a * a) + (1.0 - om));
  return ea * gl_integrate(growth_integrand, om, 0.0, sqrt(a), 8);
}

double orc_growth(double om, double z) {
  return growth_unnormalised(om, 1.0 / (1.0 + z)) / growth_unnormalised(om, 1.0);
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, Salmon, Moraes, Dror & Shaw (SC'11): ten rounds of a       */
/* multiply-hi/lo S-box with a Weyl-sequence key schedule.                   */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Box-Muller: u = (x + 1/2) 2^-32 in (0,1); two independent N(0,1). */
void orc_box_muller(uint32_t xu1, uint32_t xu2, double *e1, double *e2) {
  double u1 = ((double)xu1 + 0.5) * 0x1p-32;
  double u2 = ((double)xu2 + 0.5) * 0x1p-32;
  double rad = sqrt(-2.0 * log(u1));
  *e1 = rad * cos(2.0 * M_PI * u2);
  *e2 = rad * sin(2.0 * M_PI * u2);
}

/* White noise of a synthetic box (Sec. 2.1 draws the Gaussian boxes from    */
/* white noise): voxel v = (z n + y) n + x; Philox4x32-10 with key (seed low, */
/* seed high) and counter (g low, g high, 0, 0), g = v / 4; words (0, 1)     */
/* give voxels 4g, 4g + 1 and words (2, 3) voxels 4g + 2, 4g + 3 through     */
/* Box-Muller.                                                               */
void orc_box_noise(uint64_t seed, int32_t n, double *out) {
  const int64_t nv = (int64_t)n * n * n;
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int64_t g = 0; 4 * g < nv; ++g) {
    const uint32_t ctr[4] = {(uint32_t)g, (uint32_t)((uint64_t)g >> 32), 0u, 0u};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    double e[4];
    orc_box_muller(w[0], w[1], &e[0], &e[1]);
    orc_box_muller(w[2], w[3], &e[2], &e[3]);
    for (int q = 0; q < 4 && 4 * g + q < nv; ++q) out[4 * g + q] = e[q];
  }
}

/* Quasars from three lognormal quasar-density boxes (Sec. 2.2, App. A), one */
/* voxel at a time in the order of the paper's recipe.  Writes the accept     */
/* probability P and the uniform u0 of every voxel (n^3 each) and the ids and */
/* positions of the accepted voxels (at most capacity); returns the count.    */
static double orc_bias(const double *bl, double z) { return bl[0] * pow((1.0 + z) / (1.0 + bl[1]), bl[2]); }

int64_t orc_qso_draw(double omega_m, const float *b1, const float *b2, const float *b3, int32_t stride, int32_t n,
                     double cell, const double origin[3], const double zq[3], const double bl[3], double xi_m5,
                     const double *nbar, int32_t n_nbar, double nbar_z0, double nbar_dz, uint64_t seed,
                     double *p_out, double *u_out, uint64_t *ids, double *pos, int64_t capacity) {
  const int64_t nv = (int64_t)n * n * n;
  const float *box[3] = {b1, b2, b3};
  double sig2[3];
  for (int i = 0; i < 3; ++i) {
    double s = 0.0;
    for (int64_t v = 0; v < nv; ++v) s += (double)box[i][v * stride] * (double)box[i][v * stride];
    sig2[i] = s / (double)nv;
  }
  double xi0[3], bz[3];
  for (int i = 0; i < 3; ++i) {
    const double g = orc_growth(omega_m, zq[i]);
    bz[i] = orc_bias(bl, zq[i]);
    xi0[i] = bz[i] * bz[i] * g * g * xi_m5;
  }
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  int64_t count = 0;
  for (int64_t v = 0; v < nv; ++v) {
    const int64_t x = v % n, y = (v / n) % n, zz = v / ((int64_t)n * n);
    const double c[3] = {origin[0] + (x + 0.5) * cell, origin[1] + (y + 0.5) * cell, origin[2] + (zz + 0.5) * cell};
    const double r = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    const double z = orc_z_of_distance(omega_m, r), g = orc_growth(omega_m, z), b = orc_bias(bl, z);
    double a[3], xi[3];
    for (int i = 0; i < 3; ++i) {
      a[i] = b * (1.0 + zq[i]) / (bz[i] * (1.0 + z));
      xi[i] = pow(1.0 + xi0[i], a[i] * a[i]) - 1.0;
    }
    const double t12 = (z - zq[0]) / (zq[1] - zq[0]), t23 = (z - zq[1]) / (zq[2] - zq[1]);
    const double xi12 = (1.0 - t12) * xi[0] + t12 * xi[1], xi23 = (1.0 - t23) * xi[1] + t23 * xi[2];
    const double xmod = b * b * g * g * xi_m5;
    double lam = fabs(xi12 - xi23) > 0.0 ? (xmod - xi23) / (xi12 - xi23) : 0.5;
    lam = lam < 0.0 ? 0.0 : (lam > 1.0 ? 1.0 : lam);
    const double w[3] = {lam * (1.0 - t12), lam * t12 + (1.0 - lam) * (1.0 - t23), (1.0 - lam) * t23};
    double p = 0.0, ep = 0.0;
    for (int i = 0; i < 3; ++i) {
      p += w[i] * exp(a[i] * (double)box[i][v * stride]);
      ep += w[i] * exp(0.5 * a[i] * a[i] * sig2[i]);
    }
    double nb = 0.0;
    const double s = (z - nbar_z0) / nbar_dz;
    if (s >= 0.0 && s <= (double)(n_nbar - 1)) {
      int j = (int)floor(s);
      if (j > n_nbar - 2) j = n_nbar - 2;
      nb = nbar[j] + (s - j) * (nbar[j + 1] - nbar[j]);
    }
    double P = ep > 0.0 ? nb * cell * cell * cell * (p > 0.0 ? p : 0.0) / ep : 0.0;
    if (P > 1.0) P = 1.0;
    const uint32_t ctr[4] = {(uint32_t)v, (uint32_t)((uint64_t)v >> 32), 0x51534Fu, 0u};
    uint32_t wd[4];
    orc_philox4x32_10(ctr, key, wd);
    const double u0 = ((double)wd[0] + 0.5) * 0x1p-32;
    if (p_out) p_out[v] = P;
    if (u_out) u_out[v] = u0;
    if (u0 < P) {
      if (count < capacity) {
        ids[count] = (uint64_t)v;
        pos[3 * count + 0] = origin[0] + (x + ((double)wd[1] + 0.5) * 0x1p-32) * cell;
        pos[3 * count + 1] = origin[1] + (y + ((double)wd[2] + 0.5) * 0x1p-32) * cell;
        pos[3 * count + 2] = origin[2] + (zz + ((double)wd[3] + 0.5) * 0x1p-32) * cell;
      }
      ++count;
    }
  }
  return count;
}

/* ------------------------------------------------------------------------ */
/* Discrete Fourier transforms written as their defining sums.               */
/* ------------------------------------------------------------------------ */
/* X_m = sum_j x_j exp(-2 pi i m j / n), m = 0..n/2 */
void orc_dft_forward_real(const double *x, int32_t n, double *re, double *im) {
  for (int32_t m = 0; m <= n / 2; ++m) {
    double sr = 0.0, si = 0.0;
    for (int32_t j = 0; j < n; ++j) {
      double ang = 2.0 * M_PI * (double)(((int64_t)m * j) % n) / n;
      sr += x[j] * cos(ang);
      si -= x[j] * sin(ang);
    }
    re[m] = sr;
    im[m] = si;
  }
}

/* x_j = (1/n) sum_{m=0}^{n-1} X_m exp(+2 pi i m j / n) with X_{n-m} = conj X_m;
   inputs are X_0..X_{n/2}; the imaginary parts of X_0 and X_{n/2} are unused. */
void orc_dft_inverse_hermitian(const double *re, const double *im, int32_t n, double *x) {
  for (int32_t j = 0; j < n; ++j) {
    double s = 0.0;
    for (int32_t m = 0; m < n; ++m) {
      double xr, xi;
      if (m == 0 || m == n / 2) {
        xr = re[m];
        xi = 0.0;
      } else if (m < n / 2) {
        xr = re[m];
        xi = im[m];
      } else {
        xr = re[n - m];
        xi = -im[n - m];
      }
      double ang = 2.0 * M_PI * (double)(((int64_t)m * j) % n) / n;
      s += xr * cos(ang) - xi * sin(ang);
    }
    x[j] = s / n;
  }
}

/* ------------------------------------------------------------------------ */
/* Geometry (Sec. 2.3 pixels of 0.2 Mpc/h; Sec. 2.4 unperturbed z for lambda) */
/* ------------------------------------------------------------------------ */
int orc_geometry(const orc_cfg *cfg, const double q[3], int32_t *j_lo, int32_t *npix,
                 double *z_q) {
  double rq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
  double zq = orc_z_of_distance(cfg->omega_m, rq);
  if (z_q) *z_q = zq;
  *j_lo = 0;
  *npix = 0;
  double z_lo = (1.0 + zq) * cfg->lrf_min / cfg->lambda_lya - 1.0;
  double z_hi = (1.0 + zq) * cfg->lrf_max / cfg->lambda_lya - 1.0;
  if (cfg->lobs_min > 0.0) {
    double zc = cfg->lobs_min / cfg->lambda_lya - 1.0;
    if (z_lo < zc) z_lo = zc;
  }
  if (z_lo < 0.0) z_lo = 0.0;
  if (!(z_hi > z_lo)) return 0;
  double r_lo = orc_comoving_distance(cfg->omega_m, z_lo);
  double r_hi = orc_comoving_distance(cfg->omega_m, z_hi);
  /* pixels J with r_lo <= (J + 1/2) dr < r_hi */
  int64_t jl = (int64_t)ceil(r_lo / cfg->dr - 0.5);
  int64_t jh = (int64_t)ceil(r_hi / cfg->dr - 0.5);
  int64_t n = jh - jl;
  if (n < 0) n = 0;
  if (cfg->n_max > 0 && n > cfg->n_max) {
    jl = jh - cfg->n_max; /* keep the red end, drop blue pixels */
    n = cfg->n_max;
  }
  if (n < cfg->n_min) n = 0;
  *j_lo = (int32_t)jl;
  *npix = (int32_t)n;
  return 0;
}

double orc_pixel_z(const orc_cfg *cfg, int64_t j) {
  return orc_z_of_distance(cfg->omega_m, ((double)j + 0.5) * cfg->dr);
}

/* ------------------------------------------------------------------------ */
/* Trilinear interpolation between voxel centres, periodic box.              */
/* c is the continuous coordinate in cell units (voxel i spans [i, i+1)).    */
/* ------------------------------------------------------------------------ */
static int64_t wrap(int64_t i, int32_t n) {
  int64_t r = i % n;
  return r < 0 ? r + n : r;
}

double orc_trilinear(const float *box, int32_t n, const double c[3]) {
  double base[3], t[3];
  for (int d = 0; d < 3; ++d) {
    double s = c[d] - 0.5;
    base[d] = floor(s);
    t[d] = s - base[d];
  }
  double v = 0.0;
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        double w = (dx ? t[0] : 1.0 - t[0]) * (dy ? t[1] : 1.0 - t[1]) *
                   (dz ? t[2] : 1.0 - t[2]);
        int64_t ix = wrap((int64_t)base[0] + dx, n);
        int64_t iy = wrap((int64_t)base[1] + dy, n);
        int64_t iz = wrap((int64_t)base[2] + dz, n);
        v += w * (double)box[ix + (int64_t)n * (iy + (int64_t)n * iz)];
      }
  return v;
}

/* Gaussian-kernel average (Sec. 2.3): voxels ic-3..ic+3 per axis around the */
/* voxel ic = floor(c) containing the point, weight exp(-|d|^2/2) with d the  */
/* distance to the voxel centre (i + 1/2) in cell units, normalised.          */
double orc_gauss7(const float *box, int32_t n, const double c[3]) {
  int64_t ic[3];
  for (int d = 0; d < 3; ++d) ic[d] = (int64_t)floor(c[d]);
  double v = 0.0, wsum = 0.0;
  for (int64_t kz = ic[2] - 3; kz <= ic[2] + 3; ++kz)
    for (int64_t ky = ic[1] - 3; ky <= ic[1] + 3; ++ky)
      for (int64_t kx = ic[0] - 3; kx <= ic[0] + 3; ++kx) {
        double dx = ((double)kx + 0.5) - c[0];
        double dy = ((double)ky + 0.5) - c[1];
        double dz = ((double)kz + 0.5) - c[2];
        double w = exp(-0.5 * (dx * dx + dy * dy + dz * dz));
        int64_t ix = wrap(kx, n), iy = wrap(ky, n), iz = wrap(kz, n);
        v += w * (double)box[ix + (int64_t)n * (iy + (int64_t)n * iz)];
        wsum += w;
      }
  return v / wsum;
}

/* ------------------------------------------------------------------------ */
/* Small-scale field delta_S (Sec. 2.3): Gaussian modes times sqrt(P_S),     */
/* inverse Fourier transform.  Mode m of segment `seg` of quasar `id`:       */
/*   Philox key (seed, id & 0xffffffff); for 0 < m < n/2 counter             */
/*   (m >> 1, seg, id >> 32, 0), words (0,1) for even m and (2,3) for odd m; */
/*   the Nyquist mode m = n/2 takes words (0,1) of counter 0, the pair no    */
/*   other mode uses (X_0 = 0).  Box-Muller gives (e1, e2);                  */
/*   X_m = A_m (e1 + i e2)/sqrt(2) for 0 < m < n/2, X_{n/2} = A e1,          */
/*   A_m = sqrt(n P_S(k_m) / dr).                                            */
/* ------------------------------------------------------------------------ */
/* P_S(k_m) of a segment whose window starts at global pixel j0 */
static double small_scale_power(const orc_cfg *cfg, int32_t m, int64_t j0) {
  int32_t h = cfg->n_fft / 2 + 1;
  if (cfg->p_s_nodes <= 1) return cfg->p_s[m];
  double zs = 0.0;
  for (int64_t j = j0; j < j0 + cfg->n_fft; ++j) zs += orc_pixel_z(cfg, j);
  zs /= cfg->n_fft;
  int32_t k = cfg->p_s_nodes;
  if (zs <= cfg->p_s_z[0]) return cfg->p_s[m];
  if (zs >= cfg->p_s_z[k - 1]) return cfg->p_s[(int64_t)(k - 1) * h + m];
  int32_t i = 0;
  while (i + 2 < k && zs >= cfg->p_s_z[i + 1]) ++i;
  double w = (zs - cfg->p_s_z[i]) / (cfg->p_s_z[i + 1] - cfg->p_s_z[i]);
  return (1.0 - w) * cfg->p_s[(int64_t)i * h + m] + w * cfg->p_s[(int64_t)(i + 1) * h + m];
}

void orc_small_scale_modes(const orc_cfg *cfg, uint64_t id, int32_t seg, int64_t j0, double *re,
                           double *im) {
  int32_t n = cfg->n_fft;
  re[0] = 0.0;
  im[0] = 0.0;
  for (int32_t m = 1; m <= n / 2; ++m) {
    uint32_t c = (m < n / 2) ? (uint32_t)(m >> 1) : 0u;
    uint32_t ctr[4] = {c, (uint32_t)seg, (uint32_t)(id >> 32), 0u};
    uint32_t key[2] = {cfg->seed, (uint32_t)(id & 0xffffffffu)};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    int pair = (m < n / 2 && (m & 1)) ? 2 : 0;
    double e1, e2;
    orc_box_muller(w[pair], w[pair + 1], &e1, &e2);
    double amp = sqrt((double)n * small_scale_power(cfg, m, j0) / cfg->dr);
    if (m < n / 2) {
      re[m] = amp * e1 / sqrt(2.0);
      im[m] = amp * e2 / sqrt(2.0);
    } else {
      re[m] = amp * e1;
      im[m] = 0.0;
    }
  }
}

void orc_small_scale_segment(const orc_cfg *cfg, uint64_t id, int32_t seg, int64_t j0, double *out) {
  int32_t n = cfg->n_fft;
  double *re = (double *)malloc(sizeof(double) * (n / 2 + 1));
  double *im = (double *)malloc(sizeof(double) * (n / 2 + 1));
  orc_small_scale_modes(cfg, id, seg, j0, re, im);
  orc_dft_inverse_hermitian(re, im, n, out);
  free(re);
  free(im);
}

/* ------------------------------------------------------------------------ */
/* One skewer (Eq. gfield inputs): growth-scaled delta_L and eta_par at each */
/* pixel, and delta_S.                                                       */
/* ------------------------------------------------------------------------ */
int orc_skewer_fields(const orc_cfg *cfg, const float *dbox, const float *ebox,
                      const double q[3], uint64_t id, int32_t j_lo, int32_t npix,
                      double *delta_lg, double *eta_g, double *delta_s) {
  double rq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
  double u[3] = {q[0] / rq, q[1] / rq, q[2] / rq};
  int32_t nf = cfg->n_fft;
  double *seg = (double *)malloc(sizeof(double) * nf);
  int32_t cur = -1;
  for (int32_t j = 0; j < npix; ++j) {
    int64_t J = (int64_t)j_lo + j;
    double r = ((double)J + 0.5) * cfg->dr;
    double c[3];
    for (int d = 0; d < 3; ++d) c[d] = (r * u[d] - cfg->origin[d]) / cfg->cell;
    double zj = orc_z_of_distance(cfg->omega_m, r);
    double g = orc_growth(cfg->omega_m, zj);
    if (delta_lg)
      delta_lg[j] = g * (cfg->interp ? orc_gauss7(dbox, cfg->n, c) : orc_trilinear(dbox, cfg->n, c));
    if (eta_g) {
      if (cfg->eta_mode) {
        /* eta_par = u_p u_q eta_pq over the symmetric tensor (Eq. eta) */
        static const int pq[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
        const int64_t n3 = (int64_t)cfg->n * cfg->n * cfg->n;
        double e = 0.0;
        for (int k = 0; k < 6; ++k) {
          const float *bk = ebox + k * n3;
          double v = cfg->interp ? orc_gauss7(bk, cfg->n, c) : orc_trilinear(bk, cfg->n, c);
          double w = u[pq[k][0]] * u[pq[k][1]] * (pq[k][0] == pq[k][1] ? 1.0 : 2.0);
          e += w * v;
        }
        eta_g[j] = g * e;
      } else {
        eta_g[j] = g * (cfg->interp ? orc_gauss7(ebox, cfg->n, c) : orc_trilinear(ebox, cfg->n, c));
      }
    }
    if (delta_s) {
      if (j / nf != cur) {
        cur = j / nf;
        orc_small_scale_segment(cfg, id, cur, (int64_t)j_lo + (int64_t)cur * nf, seg);
      }
      delta_s[j] = seg[j % nf];
    }
  }
  free(seg);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* FGPA, Eq. (FGPA): F = exp(-a exp(b (delta + c eta))).                     */
/* ------------------------------------------------------------------------ */
void orc_fgpa_params(const orc_nodes *nd, double z, double *a, double *b, double *c) {
  int k = nd->count;
  double la, bb, cc;
  if (z <= nd->z[0]) {
    la = nd->ln_a[0]; bb = nd->b[0]; cc = nd->c[0];
  } else if (z >= nd->z[k - 1]) {
    la = nd->ln_a[k - 1]; bb = nd->b[k - 1]; cc = nd->c[k - 1];
  } else {
    int i = 0;
    while (!(z >= nd->z[i] && z < nd->z[i + 1])) ++i;
    double w = (z - nd->z[i]) / (nd->z[i + 1] - nd->z[i]);
    la = (1.0 - w) * nd->ln_a[i] + w * nd->ln_a[i + 1];
    bb = (1.0 - w) * nd->b[i] + w * nd->b[i + 1];
    cc = (1.0 - w) * nd->c[i] + w * nd->c[i + 1];
  }
  *a = exp(la);
  *b = bb;
  *c = cc;
}

double orc_fgpa(double a, double b, double c, double delta, double eta) {
  return exp(-a * exp(b * (delta + c * eta)));
}

/* ------------------------------------------------------------------------ */
/* Batch driver.                                                             */
/* ------------------------------------------------------------------------ */
int64_t orc_run_skewers(const orc_cfg *cfg, const float *dbox, const float *ebox,
                        const double *qpos, const uint64_t *ids, int64_t nq,
                        const orc_nodes *nodes, int32_t rebin, int32_t *j_lo,
                        int32_t *npix, int64_t *offsets, double *delta_tot, double *eta,
                        double *flux_fine, int64_t *offsets_out, double *flux_out,
                        int32_t n_threads) {
  if (rebin < 1) return -1;
  gl_init();
  dc_checkpoints(cfg->omega_m);
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads > 0 ? n_threads : 1)
  for (int64_t i = 0; i < nq; ++i) orc_geometry(cfg, qpos + 3 * i, &j_lo[i], &npix[i], NULL);
  offsets[0] = 0;
  for (int64_t i = 0; i < nq; ++i) offsets[i + 1] = offsets[i] + npix[i];
  if (offsets_out) {
    offsets_out[0] = 0;
    for (int64_t i = 0; i < nq; ++i) offsets_out[i + 1] = offsets_out[i] + npix[i] / rebin;
  }
  if (!delta_tot) return offsets[nq];
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads > 0 ? n_threads : 1)
  for (int64_t i = 0; i < nq; ++i) {
    int32_t n = npix[i];
    if (n == 0) continue;
    double *dl = (double *)malloc(sizeof(double) * n);
    double *ds = (double *)malloc(sizeof(double) * n);
    double *et = eta + offsets[i];
    orc_skewer_fields(cfg, dbox, ebox, qpos + 3 * i, ids[i], j_lo[i], n, dl, et, ds);
    for (int32_t j = 0; j < n; ++j) delta_tot[offsets[i] + j] = dl[j] + ds[j];
    if (flux_fine || flux_out) {
      double *ff = (double *)malloc(sizeof(double) * n);
      for (int32_t j = 0; j < n; ++j) {
        double zj = orc_pixel_z(cfg, (int64_t)j_lo[i] + j);
        double a, b, c;
        orc_fgpa_params(nodes, zj, &a, &b, &c);
        ff[j] = orc_fgpa(a, b, c, delta_tot[offsets[i] + j], et[j]);
        if (flux_fine) flux_fine[offsets[i] + j] = ff[j];
      }
      if (flux_out) {
        int32_t no = n / rebin;
        for (int32_t k = 0; k < no; ++k) {
          double s = 0.0;
          for (int32_t r = 0; r < rebin; ++r) s += ff[k * rebin + r];
          flux_out[offsets_out[i] + k] = s / rebin;
        }
      }
      free(ff);
    }
    free(dl);
    free(ds);
  }
  return offsets[nq];
}

/* ------------------------------------------------------------------------ */
/* Statistics (Sec. 4.1 delta_q = F/Fbar - 1; P1D of the flux).              */
/* ------------------------------------------------------------------------ */
void orc_stats_zero(orc_stats *st) { memset(st, 0, sizeof(*st)); }

static int zbin_of(const orc_bins *bins, double z) {
  double f = floor((z - bins->z_lo) / bins->dz);
  if (f < 0.0 || f >= bins->n_z) return -1;
  return (int)f;
}

/* flux_out: output-resolution flux (offsets_out); delta/eta: fine-resolution
   fields (offsets_fine) averaged over the same R pixels, or NULL. */
int orc_stats_accumulate(const orc_cfg *cfg, const orc_bins *bins, int32_t rebin,
                         const int32_t *j_lo, const int64_t *offsets_fine,
                         const int64_t *offsets_out, int64_t nq, const double *flux_out,
                         const double *delta_fine, const double *eta_fine, orc_stats *st) {
  if ((delta_fine || eta_fine) && !offsets_fine) return -1;
  int32_t np = bins->n_fft;
  int32_t half = np / 2;
  if (bins->n_z > ORC_MAX_ZBINS || bins->n_k > ORC_MAX_KBINS || half % bins->n_k) return -1;
  double *zbar = NULL, *xr = (double *)malloc(sizeof(double) * (half + 1)),
         *xi = (double *)malloc(sizeof(double) * (half + 1));
  for (int64_t q = 0; q < nq; ++q) {
    int64_t nout = offsets_out[q + 1] - offsets_out[q];
    int64_t fine_off = offsets_fine ? offsets_fine[q] : 0;
    /* output pixel k covers fine pixels k R .. k R + R - 1 */
    zbar = (double *)realloc(zbar, sizeof(double) * (nout > 0 ? nout : 1));
    for (int64_t k = 0; k < nout; ++k) {
      double zs = 0.0, ds = 0.0, es = 0.0;
      for (int32_t r = 0; r < rebin; ++r) {
        int64_t jf = k * rebin + r;
        zs += orc_pixel_z(cfg, (int64_t)j_lo[q] + jf);
        if (delta_fine) ds += delta_fine[fine_off + jf];
        if (eta_fine) es += eta_fine[fine_off + jf];
      }
      zbar[k] = zs / rebin;
      double d = ds / rebin, e = es / rebin, f = flux_out[offsets_out[q] + k];
      int zb = zbin_of(bins, zbar[k]);
      if (zb < 0) continue;
      double *s = st->sums[zb];
      s[0] += 1.0;
      s[1] += f;
      s[2] += f * f;
      s[3] += d;
      s[4] += e;
      s[5] += d * d;
      s[6] += e * e;
      s[7] += d * e;
      s[8] += f * d;
      s[9] += f * e;
    }
    /* P1D: full segments of np output pixels aligned to the skewer start */
    int64_t nseg = nout / np;
    for (int64_t sgi = 0; sgi < nseg; ++sgi) {
      double zm = 0.0;
      for (int32_t j = 0; j < np; ++j) zm += zbar[sgi * np + j];
      zm /= np;
      int zb = zbin_of(bins, zm);
      if (zb < 0) continue;
      orc_dft_forward_real(flux_out + offsets_out[q] + sgi * np, np, xr, xi);
      double scale = (double)rebin * cfg->dr / np;
      for (int32_t m = 1; m <= half; ++m) {
        double p = scale * (xr[m] * xr[m] + xi[m] * xi[m]);
        int kb = (int)(((int64_t)(m - 1) * bins->n_k) / half);
        st->p1d_sum[zb][kb] += p;
      }
      st->n_seg[zb] += 1.0;
    }
  }
  free(zbar);
  free(xr);
  free(xi);
  return 0;
}

void orc_stats_finalize(const orc_bins *bins, orc_stats *st) {
  int32_t half = bins->n_fft / 2;
  double per_bin = (double)half / bins->n_k;
  for (int zb = 0; zb < bins->n_z; ++zb) {
    double *s = st->sums[zb];
    double n = s[0];
    if (n <= 0.0) continue;
    double fbar = s[1] / n;
    st->mean_flux[zb] = fbar;
    double varf = s[2] / n - fbar * fbar;
    st->sigma_f[zb] = varf > 0.0 ? sqrt(varf) : 0.0;
    double md = s[3] / n, me = s[4] / n;
    double cdd = s[5] / n - md * md, cee = s[6] / n - me * me, cde = s[7] / n - md * me;
    double vfd = s[8] / n - fbar * md, vfe = s[9] / n - fbar * me;
    double det = cdd * cee - cde * cde;
    if (det != 0.0) {
      double kd = (cee * vfd - cde * vfe) / det;
      double ke = (cdd * vfe - cde * vfd) / det;
      st->b_f[zb] = kd / fbar;
      st->beta_f[zb] = kd != 0.0 ? ke / kd : 0.0;
    }
    for (int kb = 0; kb < bins->n_k; ++kb) {
      if (st->n_seg[zb] > 0.0) {
        st->p1d_f[zb][kb] = st->p1d_sum[zb][kb] / (st->n_seg[zb] * per_bin);
        st->p1d_df[zb][kb] = st->p1d_f[zb][kb] / (fbar * fbar);
      }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Surrogate MLP (no counterpart in the paper): 4 -> 128 -> 128 -> 128 -> 35, */
/* GELU(x) = x Phi(x) on the hidden layers, linear output, mean squared      */
/* error; backward pass by the chain rule written out layer by layer.        */
/* ------------------------------------------------------------------------ */
static const int mlp_dims[5] = {4, 128, 128, 128, 35};

/* Phi(x) = erfc(-x/sqrt 2)/2 keeps full relative accuracy in the negative tail */
double orc_gelu(double x) { return 0.5 * x * erfc(-x / sqrt(2.0)); }

static double gelu_deriv(double x) {
  return 0.5 * erfc(-x / sqrt(2.0)) + x * exp(-0.5 * x * x) / sqrt(2.0 * M_PI);
}

static void mlp_offsets(int64_t w_off[4], int64_t b_off[4]) {
  int64_t o = 0;
  for (int l = 0; l < 4; ++l) {
    w_off[l] = o;
    o += (int64_t)mlp_dims[l + 1] * mlp_dims[l];
    b_off[l] = o;
    o += mlp_dims[l + 1];
  }
}

/* The value as a tensor-core operand in BF16: rounded to FP32 (nearest even),
   then to the 8 significant bits of BF16 (nearest even on the dropped 16
   bits of the FP32 word).  Finite inputs only. */
double orc_bf16(double x) {
  float f = (float)x;
  uint32_t u;
  memcpy(&u, &f, sizeof u);
  const uint32_t lsb = (u >> 16) & 1u;
  u = (u + 0x7FFFu + lsb) & 0xFFFF0000u;
  memcpy(&f, &u, sizeof f);
  return (double)f;
}

/* forward of one sample; z[l], h[l] hold layer l's pre- and post-activation.
   bf16: the hidden activations are stored as BF16 operands (h[l] rounded);
   the output layer stays unrounded. */
static void mlp_sample(const double *p, const double *x, double z[4][128], double h[4][128],
                       double *y, int bf16) {
  int64_t wo[4], bo[4];
  mlp_offsets(wo, bo);
  const double *in = x;
  for (int l = 0; l < 4; ++l) {
    int ni = mlp_dims[l], no = mlp_dims[l + 1];
    for (int j = 0; j < no; ++j) {
      double s = p[bo[l] + j];
      for (int k = 0; k < ni; ++k) s += p[wo[l] + (int64_t)j * ni + k] * in[k];
      z[l][j] = s;
      h[l][j] = (l < 3) ? orc_gelu(s) : s;
      if (bf16 && l < 3) h[l][j] = orc_bf16(h[l][j]);
    }
    in = h[l];
  }
  for (int j = 0; j < mlp_dims[4]; ++j) y[j] = h[3][j];
}

void orc_mlp_forward(const double *params, const double *x, int64_t n, double *y, int bf16) {
  double z[4][128], h[4][128];
  for (int64_t s = 0; s < n; ++s) mlp_sample(params, x + 4 * s, z, h, y + 35 * s, bf16);
}

/* Adam (Kingma & Ba 2015, Algorithm 1), step t >= 1 on n parameters:
   m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
   m_hat = m / (1 - b1^t), v_hat = v / (1 - b2^t),
   p <- p - lr m_hat / (sqrt(v_hat) + eps). */
void orc_adam_step(double *p, double *m, double *v, const double *g, int64_t n, int64_t t, double lr,
                   double b1, double b2, double eps) {
  const double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
  for (int64_t i = 0; i < n; ++i) {
    m[i] = b1 * m[i] + (1.0 - b1) * g[i];
    v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
    const double mh = m[i] / c1, vh = v[i] / c2;
    p[i] -= lr * mh / (sqrt(vh) + eps);
  }
}

/* bf16: the backward operands of the tensor-core products are BF16 too: the
   output gradient dy and every dz = dh * GELU'(z) are rounded before they
   enter the weight gradients, the bias gradients and the next dh. */
double orc_mlp_loss_grad(const double *params, const double *x, const double *t, int64_t n,
                         double *grad, int bf16) {
  int64_t wo[4], bo[4];
  mlp_offsets(wo, bo);
  if (grad) memset(grad, 0, sizeof(double) * ORC_MLP_NPARAM);
  double z[4][128], h[4][128], y[35], dz[128], dh[128];
  double loss = 0.0;
  const double scale = 1.0 / ((double)n * 35.0);
  for (int64_t s = 0; s < n; ++s) {
    const double *xs = x + 4 * s;
    mlp_sample(params, xs, z, h, y, bf16);
    for (int j = 0; j < 35; ++j) {
      double r = y[j] - t[35 * s + j];
      loss += r * r * scale;
      dz[j] = 2.0 * r * scale; /* d loss / d y (output layer is linear) */
      if (bf16) dz[j] = orc_bf16(dz[j]);
    }
    if (!grad) continue;
    for (int l = 3; l >= 0; --l) {
      int ni = mlp_dims[l], no = mlp_dims[l + 1];
      const double *in = (l > 0) ? h[l - 1] : xs;
      for (int j = 0; j < no; ++j) {
        grad[bo[l] + j] += dz[j];
        for (int k = 0; k < ni; ++k) grad[wo[l] + (int64_t)j * ni + k] += dz[j] * in[k];
      }
      if (l == 0) break;
      for (int k = 0; k < ni; ++k) {
        double a = 0.0;
        for (int j = 0; j < no; ++j) a += params[wo[l] + (int64_t)j * ni + k] * dz[j];
        dh[k] = a;
      }
      for (int k = 0; k < ni; ++k) {
        dz[k] = dh[k] * gelu_deriv(z[l - 1][k]);
        if (bf16) dz[k] = orc_bf16(dz[k]);
      }
    }
  }
  return loss;
}
