/*
 * FP64 CPU oracle for Lyman-alpha skewer synthesis (arXiv 2310.18996).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / --impl reference legs of bench.py may load this library.
 * It shares no code, header, table or constant generator with the CUDA
 * library in paper_2310_18996_gb300/, and neither side includes the other.
 *
 * Every routine is a plain, slow, direct transcription of a definition:
 * quadrature for the cosmology, the Philox4x32-10 round function, the
 * Box-Muller map, an O(N^2) discrete Fourier transform, trilinear weights
 * written out corner by corner, and straight loops for the statistics.
 * All floating point is double precision; box values are FP32 inputs that
 * are promoted on read.
 */
#ifndef MK_ORACLE_H
#define MK_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_C_OVER_H0 2997.92458 /* c / H0 in Mpc/h (H0 = 100 h km/s/Mpc) */
#define ORC_MAX_NODES 32
#define ORC_MAX_ZBINS 32
#define ORC_MAX_KBINS 64
#define ORC_NSUM 10

/* Everything the method needs to turn a catalogue and a box into skewers. */
typedef struct orc_cfg {
  double omega_m;    /* flat LCDM, Omega_L = 1 - Omega_M, no radiation (Table 1) */
  double lambda_lya; /* Lya rest wavelength [Angstrom] */
  /* box: n^3 cells of side `cell`, x fastest, periodic; origin = corner */
  int32_t n;
  double cell;
  double origin[3]; /* box corner in the observer frame [Mpc/h]; observer at 0 */
  /* line-of-sight pixels */
  double dr;               /* pixel length [Mpc/h] (Sec. 2.3: 0.2) */
  double lrf_min, lrf_max; /* rest-frame forest window [Angstrom] */
  double lobs_min;         /* observed-frame lower cut [Angstrom], <= 0: none */
  int32_t n_min, n_max;    /* skewers shorter than n_min get n = 0; n_max > 0
                              truncates at the blue end */
  /* small-scale field (Sec. 2.3): segments of n_fft pixels */
  int32_t n_fft;
  const double *p_s; /* n_fft/2+1 samples P_S(k_m), k_m = 2 pi m/(n_fft dr) */
  uint32_t seed;
  /* interpolation of delta_L and eta at a pixel: 0 trilinear between voxel
     centres, 1 the Gaussian-kernel average over 7^3 voxels of Sec. 2.3 */
  int32_t interp;
  /* eta_par at a pixel: 0 the single box ebox taken as the line-of-sight
     gradient; 1 ebox holds the six boxes eta_pq (xx, yy, zz, xy, xz, yz, each
     n^3, consecutive) and eta_par = u_p u_q eta_pq with u the unit vector to
     the quasar (Eq. eta) */
  int32_t eta_mode;
  /* z-dependent small-scale power (Sec. 2.6 tunes P_s per z_t): p_s_nodes >= 2
     tables at increasing p_s_z, p_s holding p_s_nodes x (n_fft/2+1) values;
     a segment takes P_s linearly interpolated in z (clamped) at the mean
     pixel z of its n_fft-pixel window.  p_s_nodes <= 1: one table for all z. */
  int32_t p_s_nodes;
  const double *p_s_z;
} orc_cfg;

/* FGPA parameter nodes (Sec. 2.5: tuned at a few z, interpolated between). */
typedef struct orc_nodes {
  int32_t count;
  double z[ORC_MAX_NODES];
  double ln_a[ORC_MAX_NODES];
  double b[ORC_MAX_NODES];
  double c[ORC_MAX_NODES];
} orc_nodes;

/* Statistic binning: n_z redshift bins [z_lo + i dz, z_lo + (i+1) dz). */
typedef struct orc_bins {
  int32_t n_z;
  double z_lo, dz;
  int32_t n_k;   /* equal-count linear k bins over m = 1..n_fft/2 */
  int32_t n_fft; /* P1D segment length in output pixels */
} orc_bins;

/* Raw FP64 sums and the finalised statistics. Sum index order:
   0 n, 1 F, 2 F^2, 3 d, 4 e, 5 d^2, 6 e^2, 7 d e, 8 F d, 9 F e
   where d = delta_tot and e = eta (both growth scaled). */
typedef struct orc_stats {
  double sums[ORC_MAX_ZBINS][ORC_NSUM];
  double p1d_sum[ORC_MAX_ZBINS][ORC_MAX_KBINS];
  double n_seg[ORC_MAX_ZBINS];
  double mean_flux[ORC_MAX_ZBINS];
  double sigma_f[ORC_MAX_ZBINS];
  double p1d_f[ORC_MAX_ZBINS][ORC_MAX_KBINS];
  double p1d_df[ORC_MAX_ZBINS][ORC_MAX_KBINS];
  double b_f[ORC_MAX_ZBINS];
  double beta_f[ORC_MAX_ZBINS];
} orc_stats;

/* ---- cosmology (Table 1, flat LCDM) ---- */
double orc_hubble_e(double omega_m, double z);
double orc_comoving_distance(double omega_m, double z);
double orc_z_of_distance(double omega_m, double r);
double orc_growth(double omega_m, double z);

/* ---- Philox4x32-10 (Salmon et al. 2011) and Box-Muller ---- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void orc_box_muller(uint32_t xu1, uint32_t xu2, double *e1, double *e2);
void orc_box_noise(uint64_t seed, int32_t n, double *out);
int64_t orc_qso_draw(double omega_m, const float *b1, const float *b2, const float *b3, int32_t stride, int32_t n,
                     double cell, const double origin[3], const double zq[3], const double bl[3], double xi_m5,
                     const double *nbar, int32_t n_nbar, double nbar_z0, double nbar_dz, uint64_t seed,
                     double *p_out, double *u_out, uint64_t *ids, double *pos, int64_t capacity);

/* ---- discrete Fourier transforms, O(N^2) ---- */
void orc_dft_forward_real(const double *x, int32_t n, double *re, double *im);
void orc_dft_inverse_hermitian(const double *re, const double *im, int32_t n, double *x);

/* ---- geometry of one quasar line of sight ---- */
int orc_geometry(const orc_cfg *cfg, const double q[3], int32_t *j_lo, int32_t *npix,
                 double *z_q);
double orc_pixel_z(const orc_cfg *cfg, int64_t j);

/* ---- trilinear interpolation of a periodic box (c in cell units) ---- */
double orc_trilinear(const float *box, int32_t n, const double c[3]);

/* ---- Gaussian-kernel average of a periodic box (Sec. 2.3): the 7^3 voxels
   centred on the voxel containing c, weighted by exp(-d^2 / 2) with d the
   distance from c to the voxel centre in cell units (sigma = one voxel side),
   weights normalised to sum 1 ---- */
double orc_gauss7(const float *box, int32_t n, const double c[3]);

/* ---- small-scale modes and field of one segment ---- */
/* j0: the first global pixel of the segment's window (j_lo + seg n_fft); it
   only matters with a z-dependent P_s */
void orc_small_scale_modes(const orc_cfg *cfg, uint64_t id, int32_t seg, int64_t j0, double *re,
                           double *im);
void orc_small_scale_segment(const orc_cfg *cfg, uint64_t id, int32_t seg, int64_t j0, double *out);

/* ---- one skewer: growth-scaled delta_L, eta and delta_S per pixel ---- */
int orc_skewer_fields(const orc_cfg *cfg, const float *dbox, const float *ebox,
                      const double q[3], uint64_t id, int32_t j_lo, int32_t npix,
                      double *delta_lg, double *eta_g, double *delta_s);

/* ---- FGPA parameters at z and the transform ---- */
void orc_fgpa_params(const orc_nodes *nodes, double z, double *a, double *b, double *c);
double orc_fgpa(double a, double b, double c, double delta, double eta);

/* ---- batch driver: geometry, fields, flux, rebin; ragged outputs ----
   offsets has nq+1 entries. Pass NULL outputs to size only. Returns total
   fine pixels (>= 0) or -1 on error. */
int64_t orc_run_skewers(const orc_cfg *cfg, const float *dbox, const float *ebox,
                        const double *qpos, const uint64_t *ids, int64_t nq,
                        const orc_nodes *nodes, int32_t rebin, int32_t *j_lo,
                        int32_t *npix, int64_t *offsets, double *delta_tot, double *eta,
                        double *flux_fine, int64_t *offsets_out, double *flux_out,
                        int32_t n_threads);

/* ---- statistics over ragged flux (output resolution R) ---- */
void orc_stats_zero(orc_stats *st);
int orc_stats_accumulate(const orc_cfg *cfg, const orc_bins *bins, int32_t rebin,
                         const int32_t *j_lo, const int64_t *offsets_fine,
                         const int64_t *offsets_out, int64_t nq, const double *flux_out,
                         const double *delta_fine, const double *eta_fine, orc_stats *st);
void orc_stats_finalize(const orc_bins *bins, orc_stats *st);

/* ---- surrogate MLP 4 -> 128 -> 128 -> 128 -> 35 with GELU hidden units ----
   Parameters in order W0 [128x4], b0, W1 [128x128], b1, W2 [128x128], b2,
   W3 [35x128], b3, each W row-major [out][in]; 38179 values. */
#define ORC_MLP_NPARAM 38179
/* bf16 != 0: the hidden activations are rounded to BF16 (the operands the
   tensor cores take in training); bf16 = 0: plain FP64 throughout. */
void orc_mlp_forward(const double *params, const double *x, int64_t n, double *y, int bf16);
/* mean squared error over n samples and 35 outputs, and its gradient; with
   bf16 the backward operands dy and dz are rounded to BF16 as well */
double orc_mlp_loss_grad(const double *params, const double *x, const double *t, int64_t n,
                         double *grad, int bf16);
double orc_gelu(double x);
/* x rounded to FP32, then to BF16 (round to nearest even at both steps) */
double orc_bf16(double x);
/* one Adam step (Kingma & Ba 2015, Algorithm 1) at step t >= 1 */
void orc_adam_step(double *p, double *m, double *v, const double *g, int64_t n, int64_t t, double lr,
                   double b1, double b2, double eps);

#ifdef __cplusplus
}
#endif
#endif
