/*
 * zeta.h -- C ABI of the GB300 (sm_103a) implementation of the in-situ multipole
 * algorithm for the isotropic three-point correlation function of
 * Ju et al. (2025), arXiv:2507.15209.
 *
 * The path, in the order of the paper's Fig. 1:
 *   zeta_assign          step (2)  B-spline (MRA) assignment of the catalogue and the
 *                                  contrast delta = eps/eps_bar - 1            (Sec. 2.1, Sec. 3)
 *   zeta_fft_r2c         step (2)  3-D real-to-complex DFT of delta            (Eq. trans-field-FT)
 *   zeta_reconstruct_alm steps (3)-(5)  multiply by sqrt(4 pi) i^l jbar_l(k;b) R_lm(k-hat) and
 *                                  C2R to the real fields a_lm(x; b)           (Eqs. 3PCF-multipole-window,
 *                                                                              SFC-3PCF-vertex)
 *   zeta_sum_grid        step (6)  grid summation: node form or the connection-coefficient
 *                                  (Gamma) form                               (Eqs. con-coeff, SFC-3PCF,
 *                                                                              3PCF-multipole-sum)
 *   zeta_sum_particles   step (6)  particle summation                         (Eq. DDD-sum-privertex)
 *   zeta_mass_term       step (6)  the uniform ("-1") term of the particle form, per l
 *   zeta_zeta_ell        steps (2)-(7)  the whole measurement of zeta_l(r1, r2), l <= lmax
 *   zeta_xi              the 2PCF from the l = 0 machinery           (Eq. pair-counting)
 *   zeta_host_legendre_sum, zeta_host_reduced_q  zeta(theta) and Q   (Eqs. triplet-counting, Q-factor)
 *
 * Conventions shared by every call
 *   - Grids are float32, indexed [z][y][x] with x fastest, side n, N_g = n^3, cell H = box/n.
 *   - A particle is four float32 (x, y, z, w) in box units; coordinates in [0, box).
 *   - delta_hat, the half spectrum, is complex64 (re, im interleaved) laid out [nz][ny][nx]
 *     with nx in [0, n/2): the x-Nyquist column is not stored, because every kernel of the
 *     method is zero on all Nyquist planes.  Its size is n^3/2 complex = n^3 floats.
 *     Forward DFT unnormalised, e^{-2 pi i n.l / n}; wavevector k = 2 pi n / box.
 *   - A field a_lm(x; b) is a float32 grid.  A stack of fields is bin-interleaved in groups of
 *     four: [group][z][y][x][4] with bin b in group b/4, lane b%4, the last group zero-padded,
 *     so a stack of nb fields holds 4*ceil(nb/4) * n^3 floats.
 *   - Real spherical harmonics without the Condon-Shortley phase:
 *     R_l0 = Y_l^0, R_lm = sqrt2 N_lm P_l^m(cos t) cos(m p) (m > 0), sin(|m| p) (m < 0).
 *   - Bins are [edges[b], edges[b+1]); the radial window of bin b is the r^2-weighted shell
 *     average jbar_l(k; b) of j_l(k r).
 *   - Gram outputs are float64 nbins x nbins row-major, ACCUMULATED into (+=), symmetric.
 *
 * Memory ownership
 *   - Every pointer argument named as device memory is owned by the caller; the library never
 *     frees it.  zeta_create allocates only small device tables (radial window table,
 *     twiddles, constants) that zeta_destroy frees.
 *   - Scratch memory comes from one caller-owned workspace (zeta_set_workspace); its size is
 *     given by zeta_workspace_bytes.  Calls on one context must not overlap in time (one
 *     stream per context, or external ordering), because they share the workspace.
 *
 * Errors
 *   - Every call returns ZETA_OK (0) or a negative code.  Arguments are validated on the host
 *     before anything is launched.  Launches are asynchronous on the given stream: a CUDA
 *     error is reported by the call that observes it; a data error detected on the device
 *     (non-finite particle) is latched in a device status word and returned by
 *     zeta_get_status, which synchronises the stream.
 *   - No call traps, asserts or spins without bound on the device.
 */
#ifndef ZETA_H
#define ZETA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t (NULL means the legacy default stream). */
typedef struct CUstream_st* zeta_stream;
typedef struct zeta_ctx zeta_ctx;

enum {
  ZETA_OK = 0,
  ZETA_EINVAL = -1,     /* invalid argument (host-side validation)                  */
  ZETA_ECUDA = -2,      /* a CUDA runtime call or kernel launch failed              */
  ZETA_ENOMEM = -3,     /* device allocation of the context's tables failed         */
  ZETA_ETIMEOUT = -4,   /* a bounded device wait gave up                            */
  ZETA_ENOTSUP = -5,    /* configuration not supported by this build                */
  ZETA_EWORKSPACE = -6, /* workspace missing or smaller than zeta_workspace_bytes   */
  ZETA_EDATA = -7       /* device found invalid input data (non-finite particle)    */
};

/* Summation forms (bit mask).  ZETA_WS_BACKWARD and ZETA_WS_SS only size the workspace for the
 * gradient calls and for zeta_zeta_ell_ss. */
enum { ZETA_SUM_NODE = 1, ZETA_SUM_GAMMA = 2, ZETA_SUM_PARTICLE = 4, ZETA_WS_BACKWARD = 8, ZETA_WS_SS = 16 };

/* Arithmetic of the node-form Gram contraction (Sec. 2.2 grid sum). */
enum {
  ZETA_GRAM_FP32 = 0,   /* plain float32 FMA, the reference path                    */
  ZETA_GRAM_TF32 = 1,   /* tensor cores, tf32 inputs, fp32 accumulation             */
  ZETA_GRAM_BF16 = 2,   /* tensor cores, bf16 inputs, fp32 accumulation             */
  ZETA_GRAM_BF16X3 = 3, /* tensor cores, split bf16 (hi*hi + hi*lo + lo*hi)          */
  ZETA_GRAM_BF16_FIELDS = 4 /* zeta_zeta_ell of the node form alone: the last inverse pass
                         stores the fields as bfloat16 (round to nearest even), half the
                         field bytes of the contraction; up to 20 bins the register-blocked
                         float32 Gram reads them, above 20 the tensor cores contract them
                         (A = the fields, B = delta a as a bf16 hi + lo pair, fp32
                         accumulation); other
                         forms are refused by zeta_zeta_ell (ZETA_EINVAL); zeta_sum_grid on
                         a caller's float32 fields runs the float32 Gram                   */
};

/* Radial part of the secondary-vertex windows (Sec. 3 binning, Eq. 3PCF-multipole-window). */
enum {
  ZETA_RADIAL_SHELL = 0, /* r^2-weighted average of j_l(k r) over the bin [edges[b], edges[b+1]) */
  ZETA_RADIAL_POINT = 1  /* the spherical shell of radius radii[b] itself: j_l(k r_b), the     */
                         /* paper's triangle sides R_A, R_B (one "bin" per radius)              */
};

typedef struct {
  int n;                /* grid side: power of two, 16 <= n <= 512                   */
  double box;           /* periodic box side, same unit as positions and edges       */
  int dsup;             /* basis support D: 2 (linear B-spline hat), 4 (cubic         */
                        /* B-spline), or 3: the genus-4 Daubechies scaling function   */
                        /* (Sec. 2.2, D_sup = D_g - 1 = 3; see "Daubechies basis")    */
  int lmax;             /* highest multipole l, 0 <= lmax <= 14                      */
  int nbins;            /* number of radial bins, 1 <= nbins <= 32                   */
  const double* edges;  /* host, nbins+1 strictly increasing, edges[0] > 0,          */
                        /* edges[nbins] < box/2; copied by zeta_create (SHELL only;  */
                        /* may be NULL with ZETA_RADIAL_POINT)                       */
  int gram;             /* ZETA_GRAM_*                                               */
  /* Vertex windows (Fig. 1 steps (3)-(4), Sec. 3); all zero keeps the defaults above.  Each
   * secondary vertex's kernel sqrt(4 pi) i^l W_l,b(|k|) R_lm(k-hat) may be multiplied by a
   * spherical tophat and by the basis power spectrum; the grid forms' primary vertex may be
   * smoothed by its own tophat.  W_TH(x) = 3 (sin x - x cos x) / x^3.                    */
  int radial;           /* ZETA_RADIAL_SHELL (0) or ZETA_RADIAL_POINT                 */
  const double* radii;  /* host, nbins radii in (0, box/2) for ZETA_RADIAL_POINT      */
  double tophat;        /* R >= 0: secondary vertices times W_TH(|k| R) (0: none)     */
  double tophat_primary;/* R >= 0: the node and Gamma forms' primary vertex delta is  */
                        /* replaced by IDFT[DFT(delta) W_TH(|k| R)] (0: none); the     */
                        /* particle form's primary vertex is the catalogue itself     */
  int phi_hat;          /* 1: secondary vertices times Phi-hat(n) = prod_d            */
                        /* |phi-hat(2 pi n_d / n)|^2 of the basis (no aliasing):       */
                        /* sinc^{2D}(pi n_d / n) for the B-splines                    */
} zeta_params;

/* Daubechies basis (dsup = 3).  phi is the scaling function of the genus-4 Daubechies filter
 * h = (1 + s, 3 + s, 3 - s, 1 - s) / (4 sqrt2), s = sqrt3, defined by the two-scale relation
 * phi(x) = sqrt2 sum_k h_k phi(2x - k), support [0, 3].  A particle at grid coordinate u = x / H
 * enters the three nodes l = floor(u) - 2 .. floor(u) with weight prod_d phi(u_d - l_d), where
 * phi(t) is read from the float32 table of its exact values at the dyadic points k / 2^10
 * (zeta_host_daub4_dyadic) joined linearly; the grid is laid out like the B-spline grids (node l
 * at index l).  The node form, the particle form (its uniform term with M(a) = [a == 0]: the
 * basis is orthonormal) and the Gamma form use the exact connection coefficients Gamma(a, b) =
 * int phi(x) phi(x - a) phi(x - b) dx of phi (zeta_host_daub4_gamma), applied per node through
 * their eigen-split (5 x 5 per axis, 125 terms per node).  The particle gradient
 * (zeta_backward_particles) and zeta_assign_noalloc take B-splines only (ZETA_ENOTSUP /
 * ZETA_EINVAL for dsup 3); the node gradient does not depend on the basis. */

/* Library version (major*10000 + minor*100 + patch). Host only. */
int zeta_version(void);

/* Human-readable text of an error code. Host only; never NULL. */
const char* zeta_strerror(int code);

/* Build the FP64 host tables (radial window jbar_l by integer |n|^2, spherical-harmonic
 * recurrence constants, twiddles, B-spline mass and connection values), upload them to the
 * current device, and return a context.  Needs a CUDA device.  *out is NULL on error. */
int zeta_create(const zeta_params* p, zeta_ctx** out);

/* Free the context and its device tables.  NULL is accepted. */
int zeta_destroy(zeta_ctx* ctx);

/* Bytes of workspace that zeta_zeta_ell needs for up to np_max particles and the given
 * summation forms; it also covers every single-step call.  0 on invalid arguments. */
size_t zeta_workspace_bytes(const zeta_ctx* ctx, int64_t np_max, int forms);

/* Hand the context a caller-owned device workspace (256-byte aligned, >= the size above).
 * The library keeps the pointer, never frees it. */
int zeta_set_workspace(zeta_ctx* ctx, void* dptr, size_t bytes);

/* Switch the arithmetic of the node-form Gram (ZETA_GRAM_*) of an existing context. */
int zeta_set_gram(zeta_ctx* ctx, int gram);

/* Number of 8x8x8-cell tiles that particle sorting uses: (n/8)^3. */
int64_t zeta_tile_count(const zeta_ctx* ctx);

/* Step (2): delta_l = eps_l / eps_bar - 1 with eps_l = sum_p w_p beta(u_p - l) (periodic)
 * and eps_bar = W / N_g.  particles: device float4[np]; delta: device float[n^3] (output);
 * wsum: device double[1] (output, W = sum_p w_p).  Deterministic: contributions are summed
 * as 64-bit fixed point.  Uses the workspace. */
int zeta_assign(zeta_ctx* ctx, const float* particles, int64_t np, float* delta, double* wsum,
                zeta_stream stream);

/* Step (2): delta_hat = DFT(delta), unnormalised, half spectrum without the x-Nyquist column.
 * delta: device float[n^3]; delta_hat: device complex64[n^3/2] (as float[n^3]). */
int zeta_fft_r2c(zeta_ctx* ctx, const float* delta, float* delta_hat, zeta_stream stream);

/* Steps (3)-(5): for bins b0 <= b < b1, a_lm(.; b) = IDFT[delta_hat * K_lm,b] with
 * K_lm,b(k) = sqrt(4 pi) i^l jbar_l(|k|; b) R_lm(k-hat), zero on every Nyquist plane and
 * IDFT normalised by 1/N_g.  b0 must be a multiple of 4.  alm: device float
 * [4*ceil((b1-b0)/4) * n^3] (output, bin-interleaved stack, bin b0 in lane 0 of group 0).
 * Uses the workspace for the intermediate half spectra. */
int zeta_reconstruct_alm(zeta_ctx* ctx, const float* delta_hat, int l, int m, int b0, int b1,
                         float* alm, zeta_stream stream);

/* Step (6), grid form, one (l, m): gram[b1][b2] += S for all bins, where
 *   form = ZETA_SUM_NODE:  S = (1/N_g) sum_l delta_l a_b1(l) a_b2(l)
 *   form = ZETA_SUM_GAMMA: S = (1/N_g) sum_l delta_l sum_{l1,l2} Gamma_{l1,l2} a_b1(l+l1) a_b2(l+l2)
 *                          (evaluated as the exact cell quadrature of (1/V) int n_rec f1 f2).
 * delta: device float[n^3]; alm: bin-interleaved stack of all nbins fields; gram: device
 * double[nbins^2]. */
int zeta_sum_grid(zeta_ctx* ctx, const float* delta, const float* alm, int form, double* gram,
                  zeta_stream stream);

/* Sort particles into 8x8x8-cell tiles (stable within a tile: original order).
 * particles: device float4[np]; sorted: device float4[np] (output);
 * tile_start: device int64[zeta_tile_count + 1] (output, exclusive prefix of tile counts). */
int zeta_sort_particles(zeta_ctx* ctx, const float* particles, int64_t np, float* sorted,
                        int64_t* tile_start, zeta_stream stream);

/* Step (6), particle form without the uniform term, one (l, m):
 * gram[b1][b2] += (1/W) sum_p w_p f_b1(x_p) f_b2(x_p), f_b(x) = sum_l beta(x/H - l) a_b(l).
 * sorted/tile_start: from zeta_sort_particles; wsum: device double[1] (W); alm as above.
 * Uses the workspace, which must be sized for np particles (zeta_workspace_bytes with
 * np_max >= np and ZETA_SUM_PARTICLE): the interpolated values f_b(x_p) are staged there. */
int zeta_sum_particles(zeta_ctx* ctx, const float* sorted, const int64_t* tile_start, int64_t np,
                       const double* wsum, const float* alm, double* gram, zeta_stream stream);

/* Step (6), the uniform term of the particle form summed over m for one l:
 * gram[b1][b2] += sign * U_l, U_l = sum_m (1/V) int f_b1 f_b2 dx
 *   = (2l+1)/N_g^2 sum_{k non-Nyquist} |delta_hat|^2 jbar_l(k;b1) jbar_l(k;b2) Mhat(k),
 * Mhat the DFT of the B-spline mass matrix.  sign is +1 or -1.  The mode weights are summed per
 * integer |n|^2 first (64-bit fixed point in units of their maximum x 2^-48, so the result does
 * not depend on the order of the modes); uses the workspace. */
int zeta_mass_term(zeta_ctx* ctx, const float* delta_hat, int l, double sign, double* gram,
                   zeta_stream stream);

/* Steps (2)-(7): zeta_l(b1, b2) for 0 <= l <= lmax and each requested form.
 * particles: device float4[np] (may be NULL only if delta is given and forms has no PARTICLE);
 * delta: device float[n^3] contrast to use instead of assigning the particles (or NULL);
 * zeta: device double[nforms * (lmax+1) * nbins * nbins] (output, overwritten), forms in
 * the order NODE, GAMMA, PARTICLE among those requested. */
int zeta_zeta_ell(zeta_ctx* ctx, const float* particles, int64_t np, const float* delta, int forms,
                  double* zeta, zeta_stream stream);

/* The Szapudi-Szalay estimator with a random catalogue, Eq. (SSestimator), in multipoles: with
 * delta_D and delta_R the contrasts of the data and of the randoms (each assigned like zeta_assign,
 * so D and R are normalised to unit mean density), the numerator is the measurement of
 * Delta = delta_D - delta_R (the SFC difference of Sec. 3) and the denominator that of
 * R~ = 1 + delta_R, each exactly as zeta_zeta_ell on a given delta (grid forms: ZETA_SUM_NODE
 * and/or ZETA_SUM_GAMMA).  The estimator is zeta(theta) = sum_l num_l P_l / sum_l den_l P_l
 * (zeta_host_legendre_sum).  data, randoms: device float4[nd], float4[nr]; num, den: device
 * double[nforms * (lmax+1) * nbins * nbins].  The workspace must be sized with ZETA_WS_SS. */
int zeta_zeta_ell_ss(zeta_ctx* ctx, const float* data, int64_t nd, const float* randoms, int64_t nr, int forms,
                     double* num, double* den, zeta_stream stream);

/* The 2PCF from the same machinery (Sec. 2.1, Eq. pair-counting with the translated field of
 * Eq. trans-field-FT; the isotropic shell filter of Eq. DD-windowfunction is the l = 0 window):
 *   node form      xi_b = (1/N_g) sum_l delta_p(l) a_00,b(l), evaluated in Fourier space as
 *                  (1/N_g^2) sum_n |delta_hat|^2 Phi-hat W_0,b W_p (Parseval; non-Nyquist modes)
 *                  from per-|n|^2 fixed-point sums of |delta_hat|^2 Phi-hat;
 *   particle form  xi_b = (1/W) sum_p w_p f_b(x_p), f_b the B-spline expansion of a_00,b at the
 *                  particles (the uniform term vanishes: the fields have zero mean).
 * particles / delta as for zeta_zeta_ell; forms: ZETA_SUM_NODE and/or ZETA_SUM_PARTICLE (the
 * Gamma form is not offered here); xi: device double[nforms * nbins] (forms in that order).
 * The context's vertex windows apply (radial, tophat, phi_hat; tophat_primary for the node form). */
int zeta_xi(zeta_ctx* ctx, const float* particles, int64_t np, const float* delta, int forms, double* xi,
            zeta_stream stream);

/* The node-form 2PCF at arbitrary radii (point shells j_0(k r), times the context's secondary
 * tophat, Phi-hat and primary tophat), from delta_hat (device, as zeta_fft_r2c writes it):
 * xi[i] = (1/N_g^2) sum_n |delta_hat|^2 Phi-hat j_0(|k| radii[i]) W_TH(|k| R) W_p(|k|); radii: host
 * double[nr] (0 < nr <= 4096, radii >= 0); xi: device double[nr].  This is the xi(r_3) the reduced
 * 3PCF needs at the third side of each triangle.  Synchronises the stream. */
int zeta_xi_radii(zeta_ctx* ctx, const float* delta_hat, int nr, const double* radii, double* xi,
                  zeta_stream stream);

/* The measurement split over (l, m) pairs, for running one catalogue on several GPUs.  The pairs
 * are independent (Eq. 3PCF-multipole-sum sums them; the paper's own code runs them in parallel,
 * Sec. 3.4), so P processes can each take the pairs of index i = l^2 + l + m with
 * i mod P == lm_rank (0 <= lm_rank < lm_size = P) and sum their results.
 * zeta_zeta_lm: the same steps as zeta_zeta_ell (every rank assigns, transforms and sorts the
 *   whole catalogue itself), but each (l, m) contribution is stored in its own slot instead of
 *   being accumulated: slots is device double[zeta_lm_slots(ctx, forms)], laid out
 *   [form][(lmax+1)^2 + lmax+1][nbins][nbins] with (l, m) at slot l^2 + l + m and the uniform
 *   term of l (particle form, subtracted) at slot (lmax+1)^2 + l, owned by the rank of (l, -l).
 *   Slots this rank does not own are written as zero, so an element-wise float64 sum of the P
 *   ranks' slot arrays (e.g. an all-reduce) is exact: every slot has one non-zero contributor.
 * zeta_reduce_lm: zeta[form][l][b1][b2] from the summed slots (device double in, device double
 *   [nforms * (lmax+1) * nbins * nbins] out), adding in the order zeta_zeta_ell adds them
 *   (0, the uniform term, then m = -l .. l), so the result is bit-identical to zeta_zeta_ell.
 * zeta_lm_slots: the number of doubles in a slot array (0 on invalid arguments). */
int zeta_zeta_lm(zeta_ctx* ctx, const float* particles, int64_t np, const float* delta, int forms, int lm_rank,
                 int lm_size, double* slots, zeta_stream stream);
int zeta_reduce_lm(zeta_ctx* ctx, const double* slots, int forms, double* zeta, zeta_stream stream);
size_t zeta_lm_slots(const zeta_ctx* ctx, int forms);

/* Gradients of L = sum_l sum_ij W_l[i][j] zeta_l[i][j] (weights: host double
 * [(lmax+1) * nbins * nbins]), by the transpose of every step with per-(l, m) recomputation of
 * the fields (nothing per (l, m) is stored).  With S_l = (W_l + W_l^T)/2, A_b the map delta ->
 * a_lm,b and A_b^T = (-1)^l IDFT diag(K_lm,b) DFT:
 *   zeta_backward_node:      grad = dL/d delta of the node form for the contrast grid delta
 *                            (device float[n^3] in and out);
 *   zeta_backward_particles: grad = dL/dx_p of the particle form with delta assigned from the
 *                            same particles (device float[np * 3] out, original order; the
 *                            weights w_p are held fixed).
 * The workspace must be sized with ZETA_WS_BACKWARD.  The particle scatter uses float atomics,
 * so that gradient is reproducible to float32 rounding only.  The secondary-vertex windows
 * (radial, tophat, phi_hat) enter the transposed kernels; a context with tophat_primary > 0
 * returns ZETA_ENOTSUP here. */
int zeta_backward_node(zeta_ctx* ctx, const float* delta, const double* weights, float* grad, zeta_stream stream);
int zeta_backward_particles(zeta_ctx* ctx, const float* particles, int64_t np, const double* weights, float* grad,
                            zeta_stream stream);

/* Many catalogues in one launch: catalogue i is particles[offsets[i] .. offsets[i+1]) (device
 * float4, concatenated; offsets is a host array of ncat+1 increasing values, each catalogue
 * non-empty).  The whole batch -- every catalogue's assignment, sorting, R2C and per-(l, m)
 * loop, in order -- is captured once into a CUDA graph that is instantiated and launched
 * with a single cudaGraphLaunch on `stream`; a later call with the same pointers, forms and
 * offsets relaunches the cached graph.  zeta: device double[ncat * nforms * (lmax+1) * nb * nb]
 * (each catalogue's block as zeta_zeta_ell writes it).  The workspace must cover the largest
 * catalogue; when it holds k >= 2 whole per-catalogue workspaces (k times
 * zeta_workspace_bytes(ctx, largest np, forms), k <= 4), k catalogues run concurrently: the
 * graph forks k streams, and catalogue i runs on stream i mod k in slice i mod k of the
 * workspace (the catalogues share no data, so their kernels overlap where the GPU has room).
 * Results do not depend on k.  Changing the workspace or the tuning drops the cached graph. */
int zeta_batch(zeta_ctx* ctx, const float* particles, const int64_t* offsets, int ncat, int forms, double* zeta,
               zeta_stream stream);

/* Autotuner: on this catalogue, times the Gram kernels that `forms` uses at persistent grid
 * sizes of 1, 2, 3, 4, 6 and 8 CTAs per SM and keeps the fastest for each kernel (used by all
 * later calls); with the particle form it then picks the staging threshold of
 * zeta_set_staging the same way; last it picks the tile shape of each field-reconstruction
 * pass (zeta_set_shapes).  Synchronises the stream; overwrites the workspace. */
int zeta_autotune(zeta_ctx* ctx, const float* particles, int64_t np, int forms, zeta_stream stream);

/* The tuned persistent grid sizes in CTAs per SM: [node fp32, particle, Gamma, mass,
 * node tensor-core].  Returns 5. */
int zeta_get_tuning(const zeta_ctx* ctx, int* ctas_per_sm, int n);

/* Set the first n (<= 5) persistent grid sizes, same order as zeta_get_tuning, e.g. to
 * restore a tuning saved from an earlier run.  Each value must be in [1, 16], else
 * ZETA_EINVAL and nothing changes.  Drops a cached batch graph. */
int zeta_set_tuning(zeta_ctx* ctx, const int* ctas_per_sm, int n);

/* Tile shapes of the three passes of the field reconstruction (zeta_reconstruct_alm and every
 * measurement): shape[0] z-pass (0: 8 columns per CTA, 1: 4), shape[1] y-pass (0: 16 columns,
 * 1: 8), shape[2] x-pass (0: 4 rows per CTA, 1: 2).  The shapes change only which threads
 * transform which columns, not the arithmetic of a transform.  zeta_autotune picks them by
 * timing each pass's two shapes on the caller's data.  Values other than 0 or 1, or n > 3:
 * ZETA_EINVAL and nothing changes.  Drops a cached batch graph.  zeta_get_shapes returns 3. */
int zeta_set_shapes(zeta_ctx* ctx, const int* shape, int n);
int zeta_get_shapes(const zeta_ctx* ctx, int* shape, int n);

/* Particle form: a batch of up to 128 particles of one 8x8x8-cell tile copies the tile's
 * halo of the fields into shared memory when it holds at least `min_particles` particles
 * (0: always; a value above 128: never) and otherwise reads each stencil through L1.
 * Both give the same sums up to float32 rounding order; the choice only moves time.
 * Default 0; zeta_autotune also picks it.  min_particles < 0 -> ZETA_EINVAL.  No counterpart
 * in the paper (an execution choice of this implementation). */
int zeta_set_staging(zeta_ctx* ctx, int min_particles);
/* The current threshold of zeta_set_staging (>= 0), or ZETA_EINVAL for a null context. */
int zeta_get_staging(const zeta_ctx* ctx);

/* Failure-detection self-test: launch one thread that waits, with the library's bounded
 * device wait of `spins` polls, on an mbarrier that nothing ever arrives on.  The wait runs
 * out, latches ZETA_ETIMEOUT in the device status word (read it with zeta_get_status) and the
 * kernel returns; the context stays usable.  No GPU fault, trap or hang is involved. */
int zeta_selftest_wait(zeta_ctx* ctx, int64_t spins, zeta_stream stream);

/* Synchronise the stream and return the latched device status (ZETA_OK or ZETA_EDATA /
 * ZETA_ETIMEOUT), clearing it. */
int zeta_get_status(zeta_ctx* ctx, zeta_stream stream);

/* Assignment that allocates nothing, for callers that cannot allocate device memory when
 * they call: code inside a host framework whose memory pool already owns the device,
 * latency-critical loops that cannot afford an allocation's implicit synchronisation, and
 * services that must not run out of memory once started.  The paper has no counterpart; it
 * computes exactly what zeta_assign computes (same kernels, same fixed-point sums), without
 * a context or workspace: n (16 <= n <= 128, power of two), box and dsup (2 or 4) are passed
 * directly.  particles: device float4[np]; delta: device float[n^3] (output); wsum: device
 * double[1] (output) or NULL.
 *   - Scratch is a fixed array of 16 MiB + 16 KiB inside the library; every GPU that loads
 *     the library holds it until the process exits.  n > 128 returns ZETA_EINVAL.
 *   - The first call on a device looks up that array's device address (cudaGetSymbolAddress)
 *     with the device current; make that first call before any stream capture begins.
 *   - Every call reuses the same array and clears it itself; calls that can overlap on the
 *     GPU (different streams, or different host threads on one device) race on it and must be
 *     ordered by the caller.
 *   - The looked-up address is kept for the life of the process: after cudaDeviceReset (or any
 *     other teardown of the device's primary context) this entry point must not be called again.
 *   - Non-finite input: zeta_assign reports a particle with a NaN or infinite component through
 *     zeta_get_status; this call has no context and does not synchronise, so it reports it in
 *     the result instead: if any particle is non-finite, every value of delta and *wsum is NaN.
 *   - Calls no cudaMalloc, cudaFree or allocating library routine. */
int zeta_assign_noalloc(int n, double box, int dsup, const float* particles, int64_t np, float* delta,
                        double* wsum, zeta_stream stream);

/* ---- stage timers (tracing) ----
 * When enabled, every kernel group the library issues is bracketed by a CUDA event pair on
 * its stream.  zeta_profile_enable resets the totals; zeta_profile_read synchronises the
 * recorded events and writes, for each stage i < nslots (see zeta_profile_stage_name), the
 * summed device milliseconds, the number of kernels launched and the number of calls.  It
 * returns the number of stages.  Launch and call counts are kept even when timing is off. */
int zeta_profile_enable(zeta_ctx* ctx, int enable);
int zeta_profile_read(zeta_ctx* ctx, double* ms, int64_t* launches, int64_t* calls, int nslots);
const char* zeta_profile_stage_name(int stage);

/* ---- host-only helpers (no device needed), for inspection and tests ---- */

/* jbar_l(k; [r_lo, r_hi)) in float64 for k = 2 pi sqrt(n2[i]) / box, as used in the tables. */
int zeta_host_jbar(int l, double box, double r_lo, double r_hi, const int64_t* n2, int64_t count,
                   double* out);

/* R_lm of the integer direction (vx, vy, vz) in float64 through the same recurrence the
 * device uses (host copy of the constants). */
double zeta_host_ylm(int l, int m, double vx, double vy, double vz);

/* The window table a context uploads (Eq. 3PCF-multipole-window averaged over each radial
 * bin, Fig. 1 step (3)): out[(l * N2 + n2) * nbp + b] = sqrt(4 pi) jbar_l(2 pi sqrt(n2) / box;
 * [edges[b], edges[b+1])) / n^3 in float32, for l <= lmax, n2 < N2 = 3 (n/2 - 1)^2 + 1 and
 * b < nbins, with nbp = 4 ceil(nbins / 4) and the padding bins zero.  out: caller-owned host
 * memory of (lmax + 1) N2 nbp floats.  n a power of two in [4, 512], box > 0, lmax <= 14,
 * 1 <= nbins <= 32, edges (nbins + 1 values) positive and increasing, else ZETA_EINVAL. */
int zeta_host_jbar_table(int n, double box, int lmax, int nbins, const double* edges, float* out);

/* The window table a context with these parameters uploads (the same layout as
 * zeta_host_jbar_table): out[(l * N2 + n2) * nbp + b] = sqrt(4 pi) W_l,b(2 pi sqrt(n2) / box) / n^3,
 * W_l,b the radial window of p->radial (bin average or point radius) times W_TH(k p->tophat) when
 * p->tophat > 0.  Host only; ZETA_EINVAL on invalid parameters. */
int zeta_host_window_table(const zeta_params* p, float* out);

/* Phi-hat per axis: out[i] = |phi-hat(2 pi f / n)|^2 for DFT index i < n, f its signed
 * frequency (Fig. 1 step (3), the basis power spectrum without aliasing): sinc^{2 dsup}(pi f / n)
 * for the B-splines (dsup 2, 4); for the Daubechies basis (dsup 3) the product
 * sinc^4(w/2) prod_{j>=1} (1 + 2 sin^2(w / 2^(j+1))), w = 2 pi f / n (the transform of the
 * two-scale relation).  Host only. */
int zeta_host_phi_hat(int n, int dsup, double* out);

/* The Daubechies scaling function's values at the dyadic points k / 2^level, k = 0 .. 3 * 2^level
 * (from its two-scale relation; the device table is the level-10 one rounded to float32).
 * out: caller-owned host memory of 3 * 2^level + 1 doubles; 0 <= level <= 20, else ZETA_EINVAL. */
int zeta_host_daub4_dyadic(int level, double* out);

/* The Daubechies basis's 1-D connection coefficients (Eq. con-coeff per axis):
 * gamma[(a + 2) * 5 + (b + 2)] = int phi(x) phi(x - a) phi(x - b) dx for |a|, |b| <= 2 (zero where
 * |a - b| >= 3), solved from the two-scale relation with sum_b Gamma(a, b) = [a == 0].  When lam and
 * u are not NULL they receive the eigen-split Gamma = U diag(lam) U^T the Gamma form applies:
 * lam[k] (5 doubles) and u[o * 5 + k] (25 doubles; row o is the offset o - 2).  Host only. */
int zeta_host_daub4_gamma(double* gamma, double* lam, double* u);

/* The 3PCF in angle from its multipoles, Eq. (triplet-counting): out[i][b1][b2] =
 * sum_{l <= lmax} zeta_l[l][b1][b2] P_l(mu[i]), P_l by the three-term recurrence, float64 host
 * arrays (zeta_l: (lmax+1) nb nb; mu: nmu values in [-1, 1]; out: nmu nb nb). */
int zeta_host_legendre_sum(int lmax, int nb, const double* zeta_l, int nmu, const double* mu, double* out);

/* The reduced 3PCF, Eq. (Q-factor): q[i] = zeta[i] / (xi1 xi2 + xi2 xi3 + xi3 xi1)[i], with xi1 =
 * xi(r_1), xi2 = xi(r_2), xi3 = xi(r_3) of each triangle.  Host arrays of count doubles. */
int zeta_host_reduced_q(int count, const double* zeta, const double* xi1, const double* xi2, const double* xi3,
                        double* q);

/* Mhat(k) = M(0) + 2 sum_{0<a<dsup} M(a) cos(2 pi k a / n) for 0 <= k < n, in float64: the 1-D
 * factor of the B-spline mass matrix's DFT in the uniform term of the particle form (Sec. 2.2,
 * Eq. DDD-sum-privertex); M(a) = int phi(u) phi(u - a) du (1 for every k with the orthonormal
 * Daubechies basis, dsup 3).  The context's device table is its float32 rounding.  out: n
 * doubles, caller-owned host memory.  2 <= n <= 2^20, dsup 2, 3 or 4, else ZETA_EINVAL. */
int zeta_host_mass_hat(int n, int dsup, double* out);

/* The per-cell quadrature of the connection-coefficient (Gamma) form (Eqs. con-coeff,
 * SFC-3PCF): q Gauss-Legendre nodes t[i] and weights wq[i] on [0, 1], and
 * beta[i * dsup + o] = beta_D(t[i] + dsup/2 - 1 - o), the stencil weights at node i.  Host
 * arrays of q, q and q * dsup doubles, caller-owned.  1 <= q <= 32, dsup 2 or 4, else
 * ZETA_EINVAL. */
int zeta_host_cell_quadrature(int q, int dsup, double* t, double* wq, double* beta);

#ifdef __cplusplus
}
#endif
#endif /* ZETA_H */
