/*
 * mockskewer: GB300 (sm_103a) library for Lyman-alpha forest skewer synthesis,
 * the transmission step of the mock method of Etourneau, Le Goff, Rich et al.,
 * "Mock data sets for the eBOSS and DESI Lyman-alpha forest surveys"
 * (arXiv 2310.18996).
 *
 * For every quasar line of sight the library
 *   1. places pixels of length dr on the line from the quasar to the observer
 *      over the rest-frame forest window (Sec. 2.3, pixels of 0.2 Mpc/h; the
 *      pixel wavelength uses the unperturbed redshift, Sec. 2.4),
 *   2. interpolates the density box delta and the line-of-sight
 *      velocity-gradient box eta_par at each pixel (Sec. 2.3; trilinear),
 *   3. scales both by the linear growth factor G(z) of the pixel (Sec. 2.1),
 *   4. adds the small-scale field delta_S, an independent Gaussian
 *      realisation per line of sight with power P_S (Sec. 2.3),
 *   5. applies the FGPA, F = exp[-a(z) exp(b(z) g)], g = delta + c(z) eta_par
 *      (Eq. FGPA, Sec. 2.4), with a, b, c interpolated between redshift nodes
 *      (Sec. 2.6),
 *   6. rebins to spectral pixels, and
 *   7. accumulates FP64 statistics: mean flux and sigma_F per z bin, the 1D
 *      flux power spectrum P1D (Sec. 2.6, Sec. 4.1 for delta_F = F/Fbar - 1),
 *      and the regression of F on (delta, eta) that gives b_F and beta_F.
 *
 * Conventions common to every call
 *   - Distances are comoving Mpc/h, wavelengths Angstrom.  The observer sits
 *     at the origin of the frame in which quasar positions are given.
 *   - Pixel J of the global grid is centred at comoving distance (J + 1/2) dr.
 *     A skewer holds the consecutive pixels j_lo .. j_lo + n - 1 whose centres
 *     r satisfy r_lo <= r < r_hi, r_lo/r_hi the distances of the forest
 *     window's ends; pixel 0 is the bluest (nearest the observer).
 *   - Ragged per-pixel arrays are dense: skewer i owns entries
 *     offsets[i] .. offsets[i+1] - 1, offsets[i+1] - offsets[i] = n_i.
 *   - "d_" arguments are device pointers on the context's device, "h_"
 *     arguments host pointers.  Large buffers are always allocated and owned
 *     by the caller; the library owns only its tables, a statistics
 *     workspace, captured graphs and a device error word.
 *   - Calls are asynchronous on the context's stream unless stated.  Device
 *     side range failures (an output larger than its stated capacity, a
 *     pixel outside the redshift tables) set the error word; the next
 *     synchronising call (mk_sync, mk_stats, mk_run, a size query) returns
 *     MK_ERANGE and clears it.
 *   - Return codes: MK_OK = 0, or one of the MK_E* codes below.  No call
 *     aborts or throws; mk_last_error() gives the message of the last failure.
 */
#ifndef MOCKSKEWER_H
#define MOCKSKEWER_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MK_OK 0
#define MK_EINVAL 1   /* bad argument: NULL pointer, size, unsupported option */
#define MK_ECUDA 2    /* a CUDA runtime call failed */
#define MK_ENOMEM 3   /* the library could not allocate its own workspace */
#define MK_ETIMEOUT 4 /* a bounded device wait gave up */
#define MK_ERANGE 5   /* a device-side bound check failed */

#define MK_MAX_NODES 32
#define MK_MAX_ZBINS 32
#define MK_MAX_KBINS 64
#define MK_MAX_CHUNKS 64   /* slices of mk_run_host */
#define MK_HOST_COPY_STREAMS 2
#define MK_NSUM 10

#define MK_BOX_PLANAR 0      /* two FP32 arrays, delta and eta, index x + n (y + n z) */
#define MK_BOX_INTERLEAVED 1 /* one FP32 array of (delta, eta) pairs, same index order */
#define MK_BOX_PADDED 2      /* (delta, eta) pairs on (n+1)^3 points, index x + (n+1) (y + (n+1) z);
                                plane, row and column n repeat index 0 (periodic ghost layer) */
#define MK_BOX_HALO 3        /* (delta, eta) pairs on (n+6)^3 points for x, y, z in [-3, n+3),
                                index (x+3) + (n+6) ((y+3) + (n+6) (z+3)), periodic copies
                                (required by MK_INTERP_GAUSS7, usable by trilinear) */

#define MK_BOX_TENSOR 4      /* delta and the six velocity-gradient boxes of Eq. eta, 8 floats
                                per point {delta, eta_xx, eta_yy, eta_zz, eta_xy, eta_xz, eta_yz, 0}
                                on (n+1)^3 points as MK_BOX_PADDED, 16-byte aligned; each sight
                                line takes eta_par = u_p u_q eta_pq (trilinear only) */

/* Interpolation of delta_L and eta at a pixel (mk_skewer_params.interp). */
#define MK_INTERP_TRILINEAR 0 /* between the 8 surrounding voxel centres */
#define MK_INTERP_GAUSS7 1    /* Sec. 2.3: Gaussian-kernel average over the 7^3 voxels around
                                 the voxel containing the pixel, sigma = one voxel side,
                                 weights normalised; needs an MK_BOX_HALO box */

/* mk_run flags */
#define MK_STORE_FIELDS 1u /* write delta_tot and eta (pre-FGPA skewers) */
#define MK_STORE_FLUX 2u   /* write F */
#define MK_STATS 4u        /* accumulate and return statistics */
#define MK_AUTOTUNE 8u     /* time the admissible launch shapes on this call's inputs the first
                              time a kernel variant runs, and keep the fastest for the context */
#define MK_GRAPH 16u       /* run the step (geometry, scan, fused kernel, statistics readback)
                              as a captured CUDA graph, re-captured when an argument changes */

typedef struct mk_ctx mk_ctx; /* opaque, library-owned */
typedef struct mk_box mk_box; /* opaque, refers to caller-owned device memory */

/* Flat LCDM cosmology (Table 1: Omega_M = 0.3147); Omega_L = 1 - Omega_M. */
typedef struct mk_cosmo {
  double omega_m;
  double lambda_lya; /* Lya rest wavelength [Angstrom], 1215.67 */
} mk_cosmo;

/* Box of n^3 cubic cells (n a power of two, 2..2048), periodic. */
typedef struct mk_box_desc {
  int32_t n;
  int32_t layout;   /* MK_BOX_PLANAR, MK_BOX_INTERLEAVED, MK_BOX_PADDED, MK_BOX_HALO or MK_BOX_TENSOR */
  double cell;      /* cell side [Mpc/h] */
  double origin[3]; /* corner of the box in the observer frame [Mpc/h] */
} mk_box_desc;

/* One quasar: position in the observer frame and a catalogue id that keys its
   small-scale noise (the same id gives the same delta_S in any batch). */
typedef struct mk_qso {
  double pos[3];
  uint64_t id;
} mk_qso;

/* Per-skewer record written by mk_make_skewers / mk_run (device memory). */
typedef struct mk_skewer {
  int64_t offset;  /* first pixel in the ragged arrays */
  int32_t n;       /* pixels */
  int32_t j_lo;    /* global index of pixel 0 */
  int64_t p0[3];   /* cell coordinate of pixel 0 minus 1/2, fixed point 2^-44 */
  int64_t step[3]; /* per-pixel step of that coordinate, fixed point 2^-44 */
  uint64_t id;
} mk_skewer;

typedef struct mk_skewer_params {
  double dr;               /* pixel length [Mpc/h] (paper: 0.2) */
  double lrf_min, lrf_max; /* rest-frame forest window [Angstrom] (1040, 1200) */
  double lobs_min;         /* observed-frame lower cut [Angstrom]; <= 0: none */
  int32_t n_min;           /* skewers with fewer pixels get n = 0 */
  int32_t n_max;           /* > 0: keep at most n_max pixels, dropping blue ones */
  int32_t n_fft;           /* delta_S segment length: power of two, 256..2048 */
  uint32_t seed;           /* small-scale noise seed */
  const double *h_p_s;     /* n_fft/2 + 1 values P_S(k_m), k_m = 2 pi m/(n_fft dr) */
  int32_t interp;          /* MK_INTERP_TRILINEAR (0) or MK_INTERP_GAUSS7 */
  /* z-dependent small-scale power (Sec. 2.6 tunes P_s at each z_t): with
     p_s_nodes >= 2, h_p_s holds p_s_nodes tables of n_fft/2 + 1 values at the
     increasing redshifts h_p_s_z, and a segment takes P_s linearly
     interpolated in z (clamped) at the mean z of the n_fft pixels of its
     window (global pixels j_lo + s n_fft onwards).  0 or 1: one table. */
  int32_t p_s_nodes;       /* 0 .. MK_MAX_NODES */
  const double *h_p_s_z;
} mk_skewer_params;

/* FGPA nodes: ln a, b, c at increasing z, linear in z between nodes, clamped
   outside (Sec. 2.6 tunes at a few z_t and interpolates). */
typedef struct mk_fgpa_nodes {
  int32_t count; /* 1..MK_MAX_NODES */
  double z[MK_MAX_NODES];
  double ln_a[MK_MAX_NODES];
  double b[MK_MAX_NODES];
  double c[MK_MAX_NODES];
} mk_fgpa_nodes;

/* Statistic bins: n_z redshift bins [z_lo + i dz, z_lo + (i+1) dz); P1D on
   segments of n_fft output pixels aligned to the skewer start (incomplete
   tail segments dropped), modes m = 1..n_fft/2 in n_k equal-count bins. */
typedef struct mk_stat_bins {
  int32_t n_z;   /* 1..MK_MAX_ZBINS */
  double z_lo, dz;
  int32_t n_k;   /* divides n_fft/2, <= MK_MAX_KBINS */
  int32_t n_fft; /* power of two, 256..2048 */
} mk_stat_bins;

/* Statistics (host memory).  sums[z][i], i = 0 count, 1 F, 2 F^2, 3 d, 4 e,
   5 d^2, 6 e^2, 7 d e, 8 F d, 9 F e, with d = delta_tot and e = eta of the
   pixel.  p1d_sum: sum over segments of (dr_out/N) |X_m|^2 per k bin.
   mean_flux = F-bar, sigma_f, p1d_f = P1D_F (per mode average), p1d_df =
   P1D_F / F-bar^2, b_f = k_d/F-bar and beta_f = k_e/k_d from the least squares
   fit F ~ F0 + k_d d + k_e e in each z bin. */
typedef struct mk_stats_out {
  double sums[MK_MAX_ZBINS][MK_NSUM];
  double p1d_sum[MK_MAX_ZBINS][MK_MAX_KBINS];
  double n_seg[MK_MAX_ZBINS];
  double mean_flux[MK_MAX_ZBINS];
  double sigma_f[MK_MAX_ZBINS];
  double p1d_f[MK_MAX_ZBINS][MK_MAX_KBINS];
  double p1d_df[MK_MAX_ZBINS][MK_MAX_KBINS];
  double b_f[MK_MAX_ZBINS];
  double beta_f[MK_MAX_ZBINS];
} mk_stats_out;

/* ---------------------------------------------------------------- context */

/* Create a context on `device` using `cuda_stream` (a cudaStream_t, borrowed;
   NULL = legacy default stream).  Builds the cosmology tables of `cosmo`
   (Sec. 2, Table 1) on the host in FP64.  Synchronous.  *out is NULL on error. */
int mk_create(mk_ctx **out, int device, void *cuda_stream, const mk_cosmo *cosmo);

/* Release everything the context owns (not caller buffers).  NULL is a no-op. */
void mk_destroy(mk_ctx *ctx);

/* The context's FP64 cosmology at redshift z (Sec. 2, Table 1): comoving
   distance D_C(z) in h^-1 Mpc and linear growth G(z), G(0) = 1.  Host only.
   MK_EINVAL for z outside [0, 12) or NULL outputs. */
int mk_cosmo_eval(mk_ctx *ctx, double z, double *d_c, double *growth);

/* Message of the last failing call on this context ("" if none).  The string
   is owned by the context and valid until its next call. */
const char *mk_last_error(const mk_ctx *ctx);

/* Change the stream later calls are issued on (borrowed). */
int mk_set_stream(mk_ctx *ctx, void *cuda_stream);

/* Wait for the context's stream and report (then clear) device-side errors. */
int mk_sync(mk_ctx *ctx);

/* ---------------------------------------------------------------- boxes */

/* Register a box held in caller-owned device memory (Sec. 2.1: the density
   box delta_m and the velocity-gradient box, here the single line-of-sight
   component eta_par).  MK_BOX_PLANAR: d_delta and d_eta each n^3 floats.
   MK_BOX_INTERLEAVED: d_delta holds 2 n^3 floats (delta, eta) per cell and
   d_eta must be NULL.  MK_BOX_PADDED / MK_BOX_HALO: d_delta holds the pairs of
   that layout (8-byte aligned), d_eta NULL.  MK_BOX_TENSOR: d_delta holds
   8 (n+1)^3 floats (16-byte aligned), d_eta NULL.  The memory must outlive the box.  Synchronous. */
int mk_load_box(mk_ctx *ctx, mk_box **out, const mk_box_desc *desc, const float *d_delta,
                const float *d_eta);
void mk_free_box(mk_box *box);

/* Interleave two planar boxes into d_out (2 n_voxels floats, caller-owned). */
int mk_pack_box(mk_ctx *ctx, int64_t n_voxels, const float *d_delta, const float *d_eta,
                float *d_out);

/* Pack two planar n^3 boxes into the MK_BOX_PADDED layout: d_out (caller-owned,
   8-byte aligned) receives 2 (n+1)^3 floats.  The paper stores plain periodic
   boxes (Sec. 2.1); the ghost layer is a storage choice of this library, so
   that the fused kernel reads the 8 corners of a cell at fixed offsets.
   Asynchronous on the context stream.  MK_EINVAL for n outside [2, 2048] or
   not a power of two, or NULL pointers. */
int mk_pack_box_padded(mk_ctx *ctx, int32_t n, const float *d_delta, const float *d_eta, float *d_out);

/* Pack two planar n^3 boxes into the MK_BOX_HALO layout: d_out (caller-owned,
   8-byte aligned) receives 2 (n+6)^3 floats.  The margin of 3 periodic copies
   lets the 7^3 Gaussian-kernel average of Sec. 2.3 read its 49 x-rows without
   index wrap.  No counterpart in the paper (a storage choice).  Asynchronous
   on the context stream.  MK_EINVAL as mk_pack_box_padded. */
int mk_pack_box_halo(mk_ctx *ctx, int32_t n, const float *d_delta, const float *d_eta, float *d_out);

/* Pack delta (n^3 floats) and the six planar boxes eta_pq (6 n^3 floats in
   the order xx, yy, zz, xy, xz, yz; Eq. eta) into the MK_BOX_TENSOR layout:
   d_out (caller-owned, 16-byte aligned) receives 8 (n+1)^3 floats.  The paper
   keeps the six boxes separately (Sec. 2.1); one 32-byte record per point
   lets a corner be read with two 16-byte loads.  Asynchronous on the context
   stream.  MK_EINVAL as mk_pack_box_padded, or d_out not 16-byte aligned. */
int mk_pack_box_tensor(mk_ctx *ctx, int32_t n, const float *d_delta, const float *d_eta6, float *d_out);

/* Synthesise the Gaussian boxes of Sec. 2.1 on the device: delta with power
   spectrum P(k) (Eq. deltaL) and the velocity-gradient boxes
   eta_pq = -k_p k_q / k^2 delta in Fourier space (Eq. eta with f = 1 and the
   sign of this library's single-box contract), straight into a box layout.
     white noise: voxel v = (z n + y) n + x; Philox4x32-10, key (seed low 32
       bits, seed high 32 bits), counter (v/4 low, v/4 high, 0, 0); words (0, 1)
       give voxels 4(v/4) and +1, words (2, 3) voxels +2 and +3 (Box-Muller,
       u = (x + 1/2) 2^-32);
     modes: DFT(delta)_k = DFT(noise)_k sqrt(P(|k|) / cell^3), with the k = 0
       mode and every mode with an index n/2 on an axis set to 0; k along an
       axis at index j is 2 pi (j or j - n) / (n cell);
     P(k): h_pk[i] at k = i dk, i < n_pk (2 .. 2^24), linear in between, 0 beyond.
   n: 128, 256, 512, 1024 or 2048 (a 2048^3 box and its padded copy take
   137 GB, in core on one GPU).  layout and d_out (caller-owned device memory):
     MK_BOX_PLANAR: delta alone, n^3 floats (eta_xx is dropped; the
       quasar-density boxes of mk_draw_qso need no eta);
     MK_BOX_INTERLEAVED: (delta, eta_xx) pairs, 2 n^3 floats (d_out may be d_work);
     MK_BOX_PADDED, MK_BOX_HALO: as mk_pack_box_padded / mk_pack_box_halo;
     MK_BOX_TENSOR: as mk_pack_box_tensor, and d_spec (2 n^3 floats) keeps the
       delta modes between the four inverse transforms (NULL otherwise).
   d_work: 2 n^3 floats of caller-owned scratch, 16-byte aligned, overwritten;
   it must not overlap d_out (except INTERLEAVED in place) or d_spec.
   Asynchronous on the context stream (the P(k) upload waits for the
   stream's earlier work).  MK_EINVAL for a bad size, layout, table or pointer. */
int mk_synth_box(mk_ctx *ctx, int32_t n, double cell, uint64_t seed, const double *h_pk, int32_t n_pk, double dk,
                 int32_t layout, float *d_work, float *d_spec, float *d_out);

/* ------------------------------------------- quasars from lognormal fields (Sec. 2.2, App. A) */

/* Correlation function of an isotropic power spectrum (host, FP64):
   xi(r) = (1 / 2 pi^2) int P(k) k^2 j0(k r) dk, the integral taken by the
   trapezoid rule on the table k_i = i dk, i < n_pk; j0(x) = sin(x)/x.  MK_EINVAL for n_pk < 2,
   dk <= 0 or NULL pointers. */
int mk_xi_of_pk(const double *h_pk, int32_t n_pk, double dk, const double *h_r, int32_t n_r, double *h_xi);

/* Power spectrum of the Gaussian field whose exponential has correlation
   B xi_m(r) (Sec. 2.2: P_q is the Fourier transform of ln[1 + b_q^2 xi_m]; with
   the growth of App. A, B = b_q^2(z_i) G^2(z_i)):
     xi_m on r_j = j pi / ((n_pk - 1) dk), j < n_pk (mk_xi_of_pk);
     h_pq[i] = 4 pi int ln(1 + B xi_m(r)) r^2 j0(k_i r) dr, trapezoid on r_j,
     set to 0 where the finite sums ring below 0.
   Host, FP64.  MK_EINVAL for B < 0, NULL pointers, n_pk < 2 or dk <= 0, or if
   1 + B xi_m <= 0 somewhere. */
int mk_lognormal_pk(const double *h_pk, int32_t n_pk, double dk, double B, double *h_pq);

/* Parameters of the quasar draw (Sec. 2.2 and App. A). */
typedef struct mk_qso_draw_params {
  int32_t n;           /* box side (voxels, a power of two <= 2048), box index [z][y][x] */
  double cell;         /* voxel side, h^-1 Mpc */
  double origin[3];    /* box corner relative to the observer */
  double z_box[3];     /* redshifts z_1 < z_2 < z_3 of the three quasar-density boxes */
  double bias[3];      /* b_q(z) = bias[0] ((1 + z) / (1 + bias[1]))^bias[2] */
  double xi_m5;        /* xi_m(5 h^-1 Mpc) of the z = 0 matter spectrum */
  const double *h_nbar; /* mean density, quasars per (h^-1 Mpc)^3, at z = nbar_z0 + j nbar_dz */
  int32_t n_nbar;      /* 0 outside the table, linear inside */
  double nbar_z0, nbar_dz;
  uint64_t seed;
} mk_qso_draw_params;

/* Draw quasars voxel by voxel from three quasar-density boxes delta_q,i at
   z_i (App. A).  At the voxel's centre redshift z (cosmological, from its
   distance to the observer) and growth G:
     a_i = b_q(z)(1 + z_i) / (b_q(z_i)(1 + z)),   p_i = exp(a_i delta_q,i);
     p12 interpolates p_1, p_2 linearly in z (t12 = (z - z_1)/(z_2 - z_1)),
     p23 extrapolates p_2, p_3 (t23 = (z - z_2)/(z_3 - z_2));
     p = lambda p12 + (1 - lambda) p23, lambda (clamped to [0, 1]) the weight
     at which the same combination of xi_i = (1 + xi0_i)^(a_i^2) - 1,
     xi0_i = b_q^2(z_i) G^2(z_i) xi_m5, equals b_q^2(z) G^2(z) xi_m5 (the
     paper matches them at r = 5 h^-1 Mpc);
     P = min(1, nbar(z) cell^3 max(p, 0) / E[p]), E[p] = sum of the weights
     times exp(a_i^2 sigma_i^2 / 2), sigma_i^2 = mean delta_q,i^2 of the box.
   Voxel v = (z n + y) n + x is drawn by Philox4x32-10, key (seed low, seed
   high), counter (v low, v high, 0x51534F, 0): accepted when
   (w0 + 1/2) 2^-32 < P, at origin + (x + u1, y + u2, z + u3) cell with
   u = (w + 1/2) 2^-32; id = v.  The catalogue lists accepted voxels in
   increasing v.  The coefficients are tabulated in r (host FP64, 8192
   points over the box's distance range, linear in between).
   d_box_q[i]: n^3 floats at stride box_stride (1 planar, 2 for the pairs
   of mk_synth_box's MK_BOX_INTERLEAVED output, which reads delta).
   d_qso: capacity records.  *h_count: quasars drawn (also beyond capacity,
   then MK_ERANGE and only the first capacity are written).  Synchronous. */
int mk_draw_qso(mk_ctx *ctx, const mk_qso_draw_params *params, const float *const d_box_q[3], int32_t box_stride,
                mk_qso *d_qso, int64_t capacity, int64_t *h_count);

/* ---------------------------------------------------------------- skewers */

/* Pre-FGPA skewers (Eq. gfield inputs).  Always computes the geometry of the
   n_qso quasars in d_qso: d_sk (n_qso records) and d_offsets (n_qso + 1).
   If h_total_px is not NULL the call synchronises and stores the total pixel
   count there (a size query).  If d_delta_out and d_eta_out are not NULL it
   also writes, per pixel, delta_tot = G delta_L + delta_S and eta = G eta_par
   (FP32, ragged, capacity_px entries available); otherwise they are ignored.
   delta_S of segment s (pixels s n_fft .. s n_fft + n_fft - 1 of a skewer) is
   the inverse real DFT (1/N normalisation) of modes
   X_m = A_m (e1 + i e2)/sqrt(2), 0 < m < N/2, X_{N/2} = A e1, X_0 = 0,
   A_m = sqrt(N P_S(k_m)/dr), with (e1, e2) the Box-Muller normals of
   Philox4x32-10 words: key (seed, id); for 0 < m < N/2 counter
   (m >> 1, s, id >> 32, 0), words (0,1) for even m and (2,3) for odd m; the
   Nyquist mode m = N/2 takes words (0,1) of counter 0, which no other mode
   uses. */
int mk_make_skewers(mk_ctx *ctx, const mk_box *box, const mk_qso *d_qso, int64_t n_qso,
                    const mk_skewer_params *params, mk_skewer *d_sk, int64_t *d_offsets,
                    float *d_delta_out, float *d_eta_out, int64_t capacity_px,
                    int64_t *h_total_px);

/* FGPA and rebin (Eq. FGPA): F = exp[-a exp(b (delta + c eta))] per fine
   pixel, then the mean of `rebin` consecutive pixels (incomplete tail
   dropped).  Writes d_offsets_out (n_sk + 1 entries, floor(n_i/rebin) per
   skewer) and d_flux (capacity_out entries).  Asynchronous; mk_sync reports
   MK_ERANGE for output past capacity_out or for a record whose pixels run
   past the redshift tables of params->dr (records made with another pixel
   length); such records are skipped. */
int mk_flux(mk_ctx *ctx, const mk_skewer_params *params, const mk_skewer *d_sk, int64_t n_sk,
            const float *d_delta, const float *d_eta, const mk_fgpa_nodes *nodes,
            int32_t rebin, float *d_flux, int64_t *d_offsets_out, int64_t capacity_out);

/* Statistics of ragged flux at output resolution `rebin` (d_offsets_out from
   mk_flux): per z bin the mean flux and sigma_F, P1D of delta_F over n_fft
   segments (Sec. 2.6, Sec. 4.1) and the pixel regression of F on (delta,
   eta) for b_F and beta_F (layout in mk_stats_out).  d_delta / d_eta are the fine-resolution fields (averaged over
   the same pixels) or NULL (their sums are then zero).  The z of an output
   pixel is the mean z of its fine pixels; a P1D segment's z is the mean over
   the segment.  Synchronous: fills *h_out.  MK_ERANGE (statistics not
   written) when a record's pixels run past the redshift tables of
   params->dr, as in mk_flux; mk_flux_stats and the tuning passes check the
   same. */
int mk_stats(mk_ctx *ctx, const mk_skewer_params *params, const mk_skewer *d_sk, int64_t n_sk,
             const int64_t *d_offsets_out, const float *d_flux, int32_t rebin,
             const float *d_delta, const float *d_eta, const mk_stat_bins *bins,
             mk_stats_out *h_out);

/* Statistics of a catalogue split into parts, e.g. one part per GPU of the
   paper's parallel runs (Sec. 3 splits the sky into slices processed apart):
   the raw sums (sums, p1d_sum, n_seg) of parts[0 .. n_parts-1], each the
   result of mk_stats / mk_flux_stats / mk_run over one part with the same
   bins, are added in index order, and the derived statistics (mean_flux,
   sigma_f, p1d_f, p1d_df, b_f, beta_f) are computed once from the totals, as
   the statistics calls do for a whole catalogue.  Only the raw sums of the
   parts are read: a caller that has already added them (an all-reduce over
   ranks) passes one part.  Host arithmetic; no context, no device.  *out may
   be one of the parts.  MK_EINVAL for NULL pointers, n_parts < 1 or bad bins. */
int mk_stats_merge(const mk_stats_out *parts, int32_t n_parts, const mk_stat_bins *bins, mk_stats_out *out);

/* Tuning pass over stored pre-FGPA skewers (the paper's post-production,
   Sec. 3, re-run for new FGPA parameters, Sec. 2.6): the FGPA of d_delta /
   d_eta with `nodes` (Eq. FGPA) and the statistics of that flux at full
   resolution (as mk_stats with rebin 1), without storing the flux.
   d_offsets are the skewer offsets (n_sk + 1).  Synchronous.  MK_EINVAL for
   bad parameters, nodes, bins or pointers; MK_ERANGE as mk_stats. */
int mk_flux_stats(mk_ctx *ctx, const mk_skewer_params *params, const mk_skewer *d_sk, int64_t n_sk,
                  const int64_t *d_offsets, const float *d_delta, const float *d_eta,
                  const mk_fgpa_nodes *nodes, const mk_stat_bins *bins, mk_stats_out *h_out);

/* The whole path in one pass (rebin 1): geometry, gather, growth, delta_S,
   FGPA and statistics (steps 1-7 above: Sec. 2.3, Sec. 2.4 and Eq. FGPA,
   Sec. 2.6) in one persistent kernel, skipping the stores that `flags` does
   not ask for.  MK_EINVAL for bad parameters, flags or pointers; MK_ERANGE
   (at the synchronisation) for stores past capacity_px or pixels outside
   the redshift tables.  P1D segments coincide with delta_S segments
   (bins->n_fft must equal params->n_fft).  d_delta_out / d_eta_out /
   d_flux_out may be NULL when not stored; they may also point to page-locked
   host memory (cudaHostAlloc; unified addressing makes it device-accessible),
   which the kernel then writes over the host link while it computes.  With MK_STATS the call
   synchronises and fills *h_out; otherwise it is asynchronous.
   MK_AUTOTUNE: the first call of a kernel variant (FFT length, box layout
   and size, store/statistics flags) times each admissible launch shape
   (CTA of 128 or 256 threads; register budget of 2, 3 or 4 256-thread CTAs per SM) on its
   own inputs and keeps the fastest for later calls.  MK_GRAPH: the step is
   captured into a CUDA graph on the context stream (which must not be the
   legacy default stream) and replayed while the arguments, tables and
   workspaces stay the same; with timing on, the timed region is then the
   whole graph. */
int mk_run(mk_ctx *ctx, const mk_box *box, const mk_qso *d_qso, int64_t n_qso,
           const mk_skewer_params *params, const mk_fgpa_nodes *nodes,
           const mk_stat_bins *bins, uint32_t flags, mk_skewer *d_sk, int64_t *d_offsets,
           float *d_delta_out, float *d_eta_out, float *d_flux_out, int64_t capacity_px,
           mk_stats_out *h_out);

/* The fused pass (as mk_run with MK_STORE_FLUX, plus MK_STATS if asked) with
   the catalogue and the flux in host memory, pipelined.  No counterpart in
   the paper (which writes skewers to disk after the run, Sec. 3): this is the
   library's way to bring a large flux array to the host at link speed.
   Steps: h_qso (n_qso records) is copied to the device; the geometry of all
   quasars runs once; the skewers are then processed in n_chunks consecutive
   slices of n_qso / n_chunks quasars, each slice's flux going to one of two
   device staging buffers and from there to h_flux_out (split over
   MK_HOST_COPY_STREAMS copy streams) while the next slice computes.
   h_qso and h_flux_out should be page-locked (cudaHostAlloc) so that the
   copies run asynchronously.  h_flux_out receives the flux at the skewer
   offsets of mk_make_skewers (n_qso + 1 offsets are not returned; *h_total_px
   receives their last value).  Statistics are those of mk_run over the whole
   catalogue (the slices' partial sums are reduced together once).
   flags: 0 or MK_STATS.  n_chunks in [1, MK_MAX_CHUNKS].  MK_ERANGE if the
   flux exceeds capacity_px floats (nothing is written to h_flux_out then).
   Uses the launch shape mk_run tuned for (MK_STORE_FLUX | flags).  The
   context's workspaces are reused by later calls.  Synchronous. */
int mk_run_host(mk_ctx *ctx, const mk_box *box, const mk_qso *h_qso, int64_t n_qso,
                const mk_skewer_params *params, const mk_fgpa_nodes *nodes,
                const mk_stat_bins *bins, uint32_t flags, int32_t n_chunks, float *h_flux_out,
                int64_t capacity_px, int64_t *h_total_px, mk_stats_out *h_out);

/* Launch shape the context uses for a fused-kernel variant: *threads per CTA
   and *occupancy target, the register budget of that many 256-thread CTAs
   per SM (2, 3 or 4).  layout: the box layout, plus 16 for MK_INTERP_GAUSS7,
   plus 32 for P_S tables at several redshifts (p_s_nodes >= 2; that
   instance has one register budget, 3).
   MK_OK when the autotuner chose it, MK_ERANGE when it is the default
   (still written). */
int mk_launch_config(mk_ctx *ctx, int32_t n_fft, int32_t layout, int32_t big_box, uint32_t flags,
                     int32_t *threads, int32_t *occupancy);

/* ---------------------------------------------------------------- statistics without allocation */

/* The paper has no counterpart to this call.  It is mk_stats for callers that
   cannot allocate device memory at the point where they need statistics:
   programs that hand all device memory to their own pool allocator at start-up,
   processes running under a hard device-memory cap, and latency-bound loops in
   which a cudaMalloc or cudaFree, which waits for the whole device, is not
   acceptable.  mk_stats keeps its scratch (segment counts and offsets, scan tile
   sums, per-CTA FP64 partial sums, the device copy of the result) in a
   workspace that it grows with cudaMalloc when a larger catalogue arrives.
   This call keeps the same scratch in one fixed array of
   MK_STATIC_SCRATCH_BYTES bytes in the library's own device memory, which every
   GPU that loads the library holds until the process exits, and it calls no
   allocating routine.
   Limits and conditions:
   - n_sk <= MK_STATIC_MAX_SKEWERS, otherwise MK_EINVAL and nothing runs.
   - The context must already hold the tables the call reads: the pixel tables
     of params->dr, the FFT twiddles of bins->n_fft and the z-bin tables.  An
     earlier allocating statistics call on this context with the same dr and
     bins->n_fft builds all three: mk_stats, mk_flux_stats, or mk_run /
     mk_run_host with MK_STATS (whose n_fft is bins->n_fft).  Without them the
     call returns MK_EINVAL and runs nothing.  For other bins of the same n_fft
     it rebuilds the z-bin tables with kernels into the memory that exists.
   - The first call on each context performs a set-up step (it looks up the
     device address of the array, with the context's device current); make
     that first call before any stream capture.
   - With mk_set_timing on, mk_last_kernel_ms reports the statistics kernel of
     this call.
   - All calls share the one array, which keeps the contents of the last call.
     Calls that overlap on the GPU (other threads, streams or contexts of the
     same process) race on it and corrupt each other's results.
   Arguments, results and synchronisation are those of mk_stats; the results
   equal mk_stats' up to the order in which FP64 partial sums are added. */
#define MK_STATIC_MAX_SKEWERS 131072
#define MK_STATIC_SCRATCH_BYTES (6u << 20)
int mk_stats_static(mk_ctx *ctx, const mk_skewer_params *params, const mk_skewer *d_sk, int64_t n_sk,
                    const int64_t *d_offsets_out, const float *d_flux, int32_t rebin,
                    const float *d_delta, const float *d_eta, const mk_stat_bins *bins,
                    mk_stats_out *h_out);

/* ---------------------------------------------------------------- surrogate MLP */

/* The paper has no counterpart to the surrogate: a learned map from FGPA
   parameters to the statistics the tuning of Sec. 2.6 matches, used to cut
   the number of full passes the tuning needs.  A multilayer perceptron
   4 -> 128 -> 128 -> 128 -> 35 with GELU hidden units (GELU(x) = x Phi(x)) and
   a linear output.  Parameters: MK_MLP_NPARAM floats in the order W0 [128x4],
   b0, W1 [128x128], b1, W2 [128x128], b2, W3 [35x128], b3, each W row-major
   [out][in].  The kernels use the weights in BF16, rounded from an FP32 master
   copy that Adam updates.  The tensor-core products take BF16 operands (the
   weights, the hidden activations, and in the backward pass the output
   gradient and each dz = dh GELU'(z)) and accumulate in FP32; biases, the
   4-wide first layer, the outputs and the loss are FP32.
   Device arrays are row-major: x n x 4, outputs n x 35.
   Errors: MK_EINVAL for NULL pointers or sizes outside the ranges stated
   below (max_batch in [1, 2^24]; n in [1, max_batch] for mk_mlp_loss_grad;
   1 <= batch <= max_batch and lr > 0 for mk_mlp_train and mk_surrogate_fit),
   MK_ENOMEM when the MLP's own device scratch cannot be allocated. */
#define MK_MLP_NPARAM 38179
#define MK_MLP_IN 4
#define MK_MLP_OUT 35
typedef struct mk_mlp mk_mlp; /* opaque, library-owned, bound to one context */

/* He-initialised weights (normal, variance 2/fan_in, seeded), zero biases.
   max_batch bounds the samples of one gradient evaluation (scratch size). */
int mk_mlp_create(mk_ctx *ctx, mk_mlp **out, int64_t max_batch, uint64_t seed);
void mk_mlp_destroy(mk_mlp *mlp);
/* Set the FP32 master parameters (the BF16 copy follows; Adam state resets). */
int mk_mlp_set_params(mk_mlp *mlp, const float *h_params);
/* FP32 master parameters and/or the BF16 copy the kernels use (either NULL). */
int mk_mlp_get_params(mk_mlp *mlp, float *h_params, uint16_t *h_bf16);
/* Inference: d_y = MLP(d_x) for n samples.  Asynchronous. */
int mk_mlp_forward(mk_mlp *mlp, const float *d_x, int64_t n, float *d_y);
/* Mean squared error over n x 35 outputs against d_t and its gradient with
   respect to every parameter (h_grad: MK_MLP_NPARAM floats), at the current
   weights, without an update.  n <= max_batch.  Synchronous. */
int mk_mlp_loss_grad(mk_mlp *mlp, const float *d_x, const float *d_t, int64_t n, double *h_loss,
                     float *h_grad);
/* One Adam step (Kingma & Ba 2015, Algorithm 1; beta 0.9, 0.999, eps 1e-8,
   bias-corrected with the MLP's step count, which it advances) on the FP32
   master parameters with the caller's gradient d_grad (MK_MLP_NPARAM floats,
   device); the BF16 copy follows.  The training kernels apply the same
   update after each minibatch.  Asynchronous.  MK_EINVAL for a NULL gradient
   or lr <= 0. */
int mk_mlp_adam_step(mk_mlp *mlp, const float *d_grad, float lr);
/* Adam (beta 0.9, 0.999, eps 1e-8) on shuffled minibatches of `batch` (<=
   max_batch) samples for `epochs` epochs, learning rate lr decayed on a cosine
   to lr/20; h_epoch_loss (epochs values) receives each epoch's mean training
   loss, or NULL.  Each epoch runs as one launch of a cluster of 8 CTAs (one
   GPC's worth of SMs): the minibatch gradient is summed in a fixed order, so
   training is deterministic for a given seed.  Synchronous. */
int mk_mlp_train(mk_mlp *mlp, const float *d_x, const float *d_t, int64_t n, int32_t batch,
                 int32_t epochs, float lr, uint64_t seed, double *h_epoch_loss);

/* ---------------------------------------------------------------- tuning of a, b, c */

/* Box of constant FGPA parameters from which surrogate training draws come. */
typedef struct mk_surrogate_space {
  double ln_a_min, ln_a_max, b_min, b_max, c_min, c_max;
  /* > 0: each draw is a linear profile in z through a point of the box above
     (at the middle of the z bins), slopes uniform in +-these maxima per unit z;
     every bin is then labelled with its effective parameters (the
     pixel-weighted mean of the node values over its pixels).  0: constant. */
  double dln_a_dz_max, db_dz_max, dc_dz_max;
} mk_surrogate_space;

/* Affine normalisation between physical surrogate inputs/outputs and the
   MLP's: x_mlp = (x - x_mean)/x_std, t = t_mlp t_std + t_mean.  Inputs are
   (z, ln a, b, c); outputs (Fbar, b_F, beta_F, ln P1D_dF of 32 k bins).
   calib_skewers: when > 0 (mk_surrogate_fit writes 0), mk_tune runs one pass
   over the first calib_skewers skewers of the catalogue being tuned at the
   surrogate's first fit and refits on the surrogate shifted by that pass's
   discrepancy before its first full pass.  When the surrogate was labelled on
   those very skewers the pass measures its own error free of sample
   variance; a surrogate labelled on another box also gets the offset between
   the boxes from it (up to the subset's sample variance). */
typedef struct mk_surrogate_norm {
  double x_mean[MK_MLP_IN], x_std[MK_MLP_IN];
  double t_mean[MK_MLP_OUT], t_std[MK_MLP_OUT];
  int64_t calib_skewers;
} mk_surrogate_norm;

/* Training set of the surrogate: n_draws parameter sets drawn uniformly in
   `space` (seeded), each applied at the z nodes (constant in z, or a linear
   profile when the space has slopes) in one
   tuning pass (mk_flux_stats) over the stored skewers; every z bin with
   pixel and P1D data and Fbar > 1e-3 gives one raw sample into h_x (4
   values) and h_t (35 values; bins->n_k must be 32).  *h_count receives the
   number of samples (at most n_draws * bins->n_z).  Synchronous. */
int mk_surrogate_labels(mk_ctx *ctx, const mk_skewer_params *params, const mk_skewer *d_sk,
                        int64_t n_sk, const int64_t *d_offsets, const float *d_delta,
                        const float *d_eta, const mk_stat_bins *bins,
                        const mk_surrogate_space *space, int32_t n_draws, uint64_t seed,
                        double *h_x, double *h_t, int64_t *h_count);

/* Fit the surrogate on n raw samples: computes *norm (means and standard
   deviations of the samples), uploads the normalised samples and runs
   mk_mlp_train.  Synchronous. */
int mk_surrogate_fit(mk_mlp *mlp, const double *h_x, const double *h_t, int64_t n, int32_t batch,
                     int32_t epochs, float lr, uint64_t seed, mk_surrogate_norm *norm,
                     double *h_epoch_loss);

#define MK_TUNE_PLAIN 0
#define MK_TUNE_SURROGATE 1

/* Tuning target (Sec. 2.6): mean flux, P1D_dF and optionally beta_F per z
   bin, with the tolerances that define convergence in every active bin:
   |Fbar - target| <= tol_mean_flux, |P1D/target - 1| <= tol_p1d in every k bin
   of [k_lo, k_hi), and |beta_F/target - 1| <= tol_beta when use_beta. */
typedef struct mk_tune_target {
  double mean_flux[MK_MAX_ZBINS];
  double p1d[MK_MAX_ZBINS][MK_MAX_KBINS];
  double beta[MK_MAX_ZBINS];
  int32_t use_beta;
  int32_t k_lo, k_hi;
  uint32_t active; /* bit i: tune z bin i */
  double tol_mean_flux, tol_p1d, tol_beta;
} mk_tune_target;

typedef struct mk_tune_report {
  int32_t converged;  /* 1 when every active bin met the tolerances on a full pass */
  int32_t passes;     /* full tuning passes over the skewers */
  int32_t iterations; /* parameter updates */
  double gpu_ms;      /* GPU time of all passes (calibration included) and of the surrogate inference */
  double wall_ms;
  double max_abs_dfbar, max_rel_p1d, max_rel_beta; /* of the last full pass */
  int32_t calib_passes; /* surrogate calibration passes over norm->calib_skewers skewers */
} mk_tune_report;

/* Solve for ln a, b, c at the z nodes in *inout (count = bins->n_z, nodes at
   the bin centres) so that the statistics of the stored skewers meet the
   target (Sec. 2.6 tunes a, b sigma_g and P_S by Minuit fits and ratio
   iterations; here a Levenberg-Marquardt step per node on
   r = [(Fbar - F*)/tol_F, ln(P1D/P*)/tol_P, (beta - b*)/(tol_b |b*|)]).
   MK_TUNE_PLAIN: each iteration is one pass at the current parameters plus
   three passes with ln a, b, c shifted (finite-difference Jacobian).
   MK_TUNE_SURROGATE: the parameters are first fitted to the target on the
   surrogate alone; every later iteration is one verifying pass, after which
   the fit is redone on the surrogate shifted by that pass's discrepancy
   (true minus predicted residual) plus a linear term in the parameter change
   whose slope is Broyden-updated from successive passes (when
   norm->calib_skewers > 0, a pass over that subset of the catalogue first
   corrects the surrogate's error at its fit).  Nodes of inactive
   bins follow the nearest active node (ties: the lower one).  Stops when a
   pass meets the tolerances or after max_passes passes.  Synchronous. */
int mk_tune(mk_ctx *ctx, const mk_skewer_params *params, const mk_skewer *d_sk, int64_t n_sk,
            const int64_t *d_offsets, const float *d_delta, const float *d_eta,
            const mk_stat_bins *bins, const mk_tune_target *target, int32_t method,
            mk_mlp *surrogate, const mk_surrogate_norm *norm, int32_t max_passes,
            mk_fgpa_nodes *inout, mk_tune_report *report);

/* ------------------------------------------- Sec. 2.6 tuning of a, b sigma_g and P_S */

/* Mean and dispersion of the FGPA flux of a Gaussian field (Sec. 2.6: with g
   Gaussian, F-bar and sigma_F depend only on a and b sigma_g):
   F = exp(-a exp(s xi)), xi ~ N(0, 1), s = b sigma_g.  Host only (composite
   8-point Gauss-Legendre over xi in [-10, 10]).  MK_EINVAL for a <= 0, s < 0
   or a NULL output. */
int mk_fgpa_gauss_moments(double a, double s, double *fbar, double *sigma_f);

/* The (a, s = b sigma_g) whose moments above are (fbar, sigma_f) (Sec. 2.6
   fits a and b sigma_g to the target F-bar and sigma_F): Newton iteration in
   (ln a, ln s).  MK_EINVAL unless 0 < fbar < 1 and
   0 < sigma_f < sqrt(fbar (1 - fbar)) (no (a, s) reaches it), or if the
   iteration does not converge. */
int mk_fit_a_bsigma(double fbar, double sigma_f, double *a, double *s);

#define MK_PS_TUNE_MAX_PASSES 128

typedef struct mk_ps_tune_report {
  int32_t passes;    /* fused passes run: n_outer (1 + n_inner) + 1 */
  double gpu_ms;     /* GPU time of the passes */
  double wall_ms;
  double sigma_f_target[MK_MAX_ZBINS]; /* from the integral of the target P1D */
  double bsigma[MK_MAX_ZBINS];         /* fitted b sigma_g per node */
  double sigma_g[MK_MAX_ZBINS];        /* measured on the last outer loop's first pass */
  /* of the last pass, over the active bins (P1D over k bins [k_lo, k_hi)) */
  double max_abs_dfbar, max_rel_p1d, max_rel_beta;
  double max_rel_p1d_pass[MK_PS_TUNE_MAX_PASSES]; /* the same P1D error after every pass */
} mk_ps_tune_report;

/* The tuning procedure of Sec. 2.6, each pass a fused synthesis of the whole
   catalogue (mk_run with MK_STATS; the paper re-generates its spectra for
   every P_S iteration).  Tuning redshifts are the z-bin centres of `bins`;
   bins outside target->active are not tuned and copy the nearest tuned node
   (ties: the lower).
     1. c = target beta (beta = f c, f = 1);
     2. per bin, a and s = b sigma_g are fitted (mk_fit_a_bsigma) to the target
        F-bar and to sigma_F = F-bar sqrt(sum over DFT modes m = 1..N-1 of
        P1D_dF(k_m) / (N dr)), N = bins->n_fft, the mode sum taken from the
        target's equal-count k-bin means (the Nyquist mode: the last bin's mean);
     3. n_outer times: one pass gives sigma_g^2 = var(delta_tot + c eta) over
        each bin's pixels (sigma_L^2 + sigma_S^2 + c^2 sigma_eta^2 + 2 c cov),
        then b = s / sigma_g, and from the second loop on one Newton step in
        ln a on that pass's F-bar (slope of the Gaussian-field moments, step
        capped at 0.5) keeps the mean flux; then n_inner passes, after each of which every
        P_S mode m of node i is multiplied by target P1D / measured P1D_dF of
        bin i in the k bin that holds P1D mode round(m bins->n_fft / n_fft)
        (clamped to 1 .. bins->n_fft/2);
     4. a last pass measures the result.
   box, d_qso, n_qso, params: as mk_run (params' own P_S fields are ignored).
   target: mean_flux in (0, 1), p1d > 0 in every one of the n_k bins and use_beta
   = 1 in every active bin; k_lo, k_hi and the tolerances only shape the report.
   d_sk (n_qso records), d_offsets (n_qso + 1): caller-owned device scratch.
   h_p_s: bins->n_z tables of n_fft/2 + 1 values (host, FP64), in: the start,
   out: the tuned tables.  out: bins->n_z nodes (z, ln a, b, c).
   n_outer >= 1, n_inner >= 0, passes <= MK_PS_TUNE_MAX_PASSES.  Synchronous.
   MK_EINVAL for arguments outside these ranges, a target that the (a, b
   sigma_g) fit cannot reach, or a tuned bin without pixels or P1D segments;
   the errors of mk_run otherwise. */
int mk_tune_ps(mk_ctx *ctx, const mk_box *box, const mk_qso *d_qso, int64_t n_qso,
               const mk_skewer_params *params, const mk_stat_bins *bins, const mk_tune_target *target,
               int32_t n_outer, int32_t n_inner, mk_skewer *d_sk, int64_t *d_offsets, double *h_p_s,
               mk_fgpa_nodes *out, mk_ps_tune_report *report);

/* ------------------------------------------- saved pre-production (Sec. 3) */

/* Write stored pre-FGPA skewers to a file, so that later post-production runs
   (FGPA and statistics with new a, b, c: mk_flux, mk_flux_stats, mk_tune)
   start from them instead of re-synthesising (the paper saves its
   pre-production the same way).  Little-endian file: the 8 bytes
   "MKSKEW01", int64 n_sk, int64 total pixels, n_sk mk_skewer records,
   n_sk + 1 int64 offsets, total FP32 delta_tot, total FP32 eta.  Device
   inputs as mk_make_skewers wrote them; copied through a pinned staging
   buffer of the context's stream.  Synchronous.  MK_EINVAL for NULL
   pointers or a file that cannot be written. */
int mk_save_skewers(mk_ctx *ctx, const char *path, const mk_skewer *d_sk, int64_t n_sk, const int64_t *d_offsets,
                    const float *d_delta, const float *d_eta);

/* Read a file of mk_save_skewers into caller-owned device buffers: up to
   cap_sk records (and cap_sk + 1 offsets) and cap_px pixels of delta_tot and
   eta.  *n_sk and *total_px receive the file's sizes; with NULL buffers (or
   too small capacities, then MK_ERANGE) nothing else is read, which makes
   the call a size query.  Synchronous.  MK_EINVAL for a missing, truncated
   or malformed file; malformed includes records and offsets that do not
   tile [0, total): record i must start where record i - 1 ends (offset 0
   for the first), have n >= 0 and j_lo >= 0, and offsets[i] must equal its
   start, offsets[n_sk] the total (checked on the host while staging, before
   anything is copied to the device). */
int mk_load_skewers(mk_ctx *ctx, const char *path, mk_skewer *d_sk, int64_t cap_sk, int64_t *d_offsets,
                    float *d_delta, float *d_eta, int64_t cap_px, int64_t *n_sk, int64_t *total_px);

/* ---------------------------------------------------------------- launch cap */

/* At most max_ctas CTAs for the persistent skewer and statistics kernels
   (mk_make_skewers, mk_run, mk_run_host, mk_stats, mk_flux_stats and the
   tuning passes); 0 (the default) lifts the cap, and the grids then hold as
   many CTAs as the SMs keep resident.  Results do not depend on the grid
   except through the order of floating-point additions.  With a small cap
   each team of threads runs many consecutive segments, keeping its pixel
   sums in registers across segments and z bins; it also leaves SMs free for
   other work on the GPU.  Takes effect at the next call.  MK_EINVAL for
   max_ctas < 0. */
int mk_set_grid_cap(mk_ctx *ctx, int32_t max_ctas);

/* Test hook for the one device wait of the library: the tuning pass
   (mk_flux_stats, the passes of mk_tune) waits for the bulk copies of each
   segment's fields on an mbarrier, for about a second at most, and then
   reports MK_ETIMEOUT (the context stays usable).  With on != 0 the pass
   issues no copies while still expecting their bytes and gives up after
   about 2^20 clock cycles, so that every such wait runs out; results are
   then invalid and the call returns MK_ETIMEOUT.  0 (the default) restores
   normal operation.  Takes effect at the next call. */
int mk_set_wait_test(mk_ctx *ctx, int32_t on);

/* Test hook for the host-side error paths: the next step of the given kind
   fails once, as if the CUDA call had failed, and the call that meets it
   returns the matching code with nothing half done that a later call would
   trust.  MK_FAULT_ALLOC: the next growth of a library workspace
   (MK_ENOMEM).  MK_FAULT_LAUNCH: the next fused run (mk_run) or statistics
   pass (mk_stats, mk_flux_stats) before its kernels are launched (MK_ECUDA).
   MK_FAULT_NONE clears a pending fault.  MK_EINVAL for other kinds. */
#define MK_FAULT_NONE 0
#define MK_FAULT_ALLOC 1
#define MK_FAULT_LAUNCH 2
int mk_inject_fault(mk_ctx *ctx, int32_t kind);

/* ---------------------------------------------------------------- timing */

/* When on (non-zero), the library records CUDA events on the context's
   stream around its main kernel: the skewer pass of mk_make_skewers and
   mk_run, the statistics pass of mk_stats. */
int mk_set_timing(mk_ctx *ctx, int on);

/* GPU time in milliseconds of the last timed main-kernel launch.  Waits for
   that launch to finish.  MK_EINVAL if nothing was timed. */
int mk_last_kernel_ms(mk_ctx *ctx, double *ms);

#ifdef __cplusplus
}
#endif
#endif
