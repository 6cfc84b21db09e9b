// Internal declarations shared by the translation units of libzeta.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/zeta.h"

namespace zk {

constexpr int kMaxL = 14;       // highest multipole supported by the tables
constexpr int kMaxBins = 32;    // highest number of radial bins
constexpr int kTile = 8;        // particle tiles are kTile^3 cells
constexpr int kMaxCtas = 4096;  // upper bound on persistent CTAs writing Gram partials

// ---- host tables (tables.cpp), all computed in float64 ----
// Number of integer |n|^2 values with every |n_d| <= n/2 - 1 (Nyquist planes excluded).
inline int64_t table_n2_count(int n) {
  const int64_t h = n / 2 - 1;
  return 3 * h * h + 1;
}
// The radial part of the secondary-vertex window: the r^2-weighted shell average over
// [edges[b], edges[b+1]) or the shell of radius radii[b] itself, times W_TH(k tophat) if tophat > 0.
struct VertexSpec {
  int radial = ZETA_RADIAL_SHELL;
  const double* edges = nullptr;
  const double* radii = nullptr;
  double tophat = 0.0;
};
// sqrt(4 pi) W_l,b(k) / N_g for l <= lmax, all n2 < table_n2_count(n), all bins, laid out
// [l][n2][b] with the bins padded to a multiple of 4 (one float4 gathers four bins); W_l,b the
// radial window of the spec (host_jbar_table: the plain shell average jbar_l(k; b)).
void host_jbar_table(int n, double box, int lmax, int nbins, const double* edges, std::vector<float>& out);
void host_window_table(int n, double box, int lmax, int nbins, const VertexSpec& v, std::vector<float>& out);
// Phi-hat per axis: sinc^{2 dsup}(pi f / n) at DFT index i (signed frequency f), float64.
void host_phi_hat_1d(int n, int dsup, std::vector<double>& out);
// W_TH(|k| radius) / N_g by integer |n|^2 < table_n2_count(n) (the primary-vertex tophat).
void host_tophat_table(int n, double box, double radius, std::vector<float>& out);
void host_jbar_values(int l, double box, double r_lo, double r_hi, const int64_t* n2, int64_t count,
                      double* out);
// W_n^e = exp(-2 pi i e / n), e < n, as (cos, sin) pairs rounded to float32.
void host_twiddles(int n, std::vector<float2>& out);
// Real-spherical-harmonic recurrence constants: mm[m], a[l][m], b[l][m] (l, m <= kMaxL).
void host_ylm_constants(double* mm, double* a, double* b);
// Gram values M(a) = int phi(u) phi(u - a) du for |a| < dsup, index a + dsup - 1 (B-splines;
// dsup 3, the orthonormal Daubechies function: [a == 0]).
void host_mass_1d(int dsup, double* out);
// The genus-4 Daubechies scaling function (dsup 3): its values at k / 2^level, k <= 3 * 2^level
// (two-scale relation); |phi-hat(omega)|^2; the 1-D connection coefficients Gamma(a, b),
// |a|, |b| <= 2, at [(a + 2) * 5 + b + 2]; and their eigen-split Gamma = U diag(lam) U^T with
// u[o * 5 + k] (offset o - 2, eigenvector k).
constexpr int kDaubLevel = 10;  // dyadic level of the point-value table the kernels interpolate
void host_daub4_dyadic(int level, std::vector<double>& out);
double host_daub4_power(double omega);
void host_daub4_gamma(double* g);
void host_daub4_gamma_split(std::vector<double>& lam, std::vector<double>& u);
// 1-D DFT of the mass sequence: Mhat(k) = sum_a M(a) cos(2 pi k a / n), k-index < n; with_phi
// multiplies by the square of the per-axis Phi-hat (the uniform term of Phi-hat-windowed fields).
void host_mass_hat(int n, int dsup, std::vector<float>& out, bool with_phi = false);
// Gauss-Legendre nodes/weights on [0, 1] (q points) and the stencil weights
// beta(t_q + dsup/2 - 1 - o) for o < dsup: wq[q], beta[q * dsup + o].
void host_cell_quadrature(int q, int dsup, std::vector<double>& t, std::vector<double>& wq,
                          std::vector<double>& beta);

// ---- stage timers (profile.cu): CUDA events around every kernel group ----
enum Stage {
  ST_ASSIGN = 0, ST_SORT, ST_R2C, ST_ALM_Z, ST_ALM_Y, ST_ALM_X, ST_GRAM_NODE, ST_GRAM_GAMMA, ST_GRAM_PART,
  ST_MASS, ST_REDUCE, ST_ADJ_POINT, ST_ADJ_FFT, ST_ADJ_OTHER, ST_COUNT
};
struct Profiler {
  bool on = false;
  struct Rec {
    int stage, nk;
    cudaEvent_t a, b;
  };
  std::vector<cudaEvent_t> pool;
  std::vector<Rec> pending;
  double ms[ST_COUNT] = {};
  long long launches[ST_COUNT] = {};
  long long calls[ST_COUNT] = {};
};

}  // namespace zk

struct zeta_ctx {
  zeta_params p{};
  std::vector<double> edges;
  int n = 0, nc = 0;
  int64_t ng = 0;
  int64_t nn2 = 0;
  int64_t ntiles = 0;
  int num_sms = 0;
  int device = 0;
  int gamma_q = 0;
  // device tables
  float* d_jtab = nullptr;    // [(l * nn2 + n2) * nbp + b], nbp = 4 * ceil(nbins / 4)
  float2* d_tw = nullptr;     // W_n^e, e < n
  float* d_mhat = nullptr;    // Mhat(k) for k-index < n
  float* d_gq = nullptr;      // cell quadrature: weights[q] then beta[q*dsup+o]
  float* d_phi = nullptr;     // Phi-hat per axis by DFT index (all ones without phi_hat)
  float* d_wprim = nullptr;   // primary-vertex tophat W_TH / N_g by |n|^2 (tophat_primary > 0)
  float* d_daub = nullptr;    // Daubechies basis (dsup 3): phi at k / 2^kDaubLevel, k <= 3 * 2^kDaubLevel
  std::vector<double> radii;
  int* d_status = nullptr;    // latched device status
  // workspace
  char* ws = nullptr;
  size_t ws_bytes = 0;
  mutable zk::Profiler prof;
  // persistent-grid size of each Gram kind, in CTAs per SM (set by zeta_autotune)
  int tune[5] = {3, 3, 4, 4, 1};
  // tile shape of each field-reconstruction pass (z, y, x), 0 = default (set by zeta_autotune)
  int alm_shape[3] = {0, 0, 0};
  // particle Gram: batches with at least this many particles stage their tile's halo in
  // shared memory; sparser ones gather from global memory
  int staged_min = 0;
  // CUDA graph of the last batch (zeta_batch); up to kMaxBatchStreams catalogues in flight, on
  // cap_stream and the auxiliary streams forked from it inside the capture
  static constexpr int kMaxBatchStreams = 4;
  bool capturing = false;
  cudaStream_t cap_stream = nullptr;
  cudaStream_t cap_aux[kMaxBatchStreams - 1] = {};
  cudaEvent_t cap_fork = nullptr;
  cudaEvent_t cap_join[kMaxBatchStreams - 1] = {};
  int batch_streams = 1;
  cudaGraphExec_t batch_exec = nullptr;
  std::vector<int64_t> batch_key;
};

namespace zk {

// The Daubechies basis (dsup 3) runs on the 4-node stencil of the cubic B-spline: every prepared
// particle's cell is one below floor(u) (cell_shift), so the stencil's nodes cell - 1 .. cell + 2
// are floor(u) - 2 .. floor(u) + 1, with weights phi(t + 2), phi(t + 1), phi(t) and 0.
inline int cell_shift(const zeta_ctx* c) { return c->p.dsup == 3 ? 1 : 0; }

#ifdef __CUDACC__
// phi(t + 2), phi(t + 1), phi(t), 0 for t in [0, 1), phi read from the table of its values at
// the dyadic points of level kDaubLevel joined linearly.
__device__ __forceinline__ void daub4_weights(float t, const float* __restrict__ tab, float* w) {
  constexpr int unit = 1 << kDaubLevel;
  const float sc = t * static_cast<float>(unit);  // exact: a power-of-two scale
  int i = static_cast<int>(sc);
  i = i < 0 ? 0 : (i > unit - 1 ? unit - 1 : i);
  const float f = sc - static_cast<float>(i);
#pragma unroll
  for (int o = 0; o < 3; ++o) {
    const float a = __ldg(tab + i + (2 - o) * unit), b = __ldg(tab + i + 1 + (2 - o) * unit);
    w[o] = fmaf(f, b - a, a);
  }
  w[3] = 0.f;
}
#endif

// Records an event pair around the kernels issued while it is alive (when profiling).
class StageScope {
 public:
  StageScope(const zeta_ctx* c, int stage, int nkernels, cudaStream_t s);
  ~StageScope();
  StageScope(const StageScope&) = delete;
  StageScope& operator=(const StageScope&) = delete;

 private:
  const zeta_ctx* c_;
  int stage_, nk_;
  cudaStream_t s_;
  cudaEvent_t a_ = nullptr;
};
void profile_release(const zeta_ctx* c);
// Raise a kernel's dynamic shared-memory limit to at least `bytes`, calling the runtime only the
// first time a kernel needs more (so later launches can be captured into a CUDA graph).
int ensure_smem(const void* kernel, size_t bytes);

// ---- launchers (fft.cu) ----
int set_ylm_constants();
int launch_r2c(const zeta_ctx* c, const float* delta, float2* dhat, cudaStream_t s);
// nf fields of bins b0.. : plain half spectra in spec (nf * n^3/2 complex, scratch), result in out as
// ceil(nf/4) bin-interleaved groups [g][z][y][x][4].
// bf16: the groups are written as four bfloat16 per point ([g][z][y][x][4], 8 bytes) instead of float4
int launch_alm(const zeta_ctx* c, const float2* dhat, int l, int m, int b0, int nf, float2* spec, float* out,
               cudaStream_t s, bool bf16 = false);
// Adjoint of the reconstruction for nf bin-interleaved real fields h_b (bins 0..nf-1):
// gk += sum_b (-1)^l K_lm,b DFT(h_b); spec is scratch for nf half spectra.
int launch_adj_spectral(const zeta_ctx* c, const float* fields, int nf, float2* spec, int l, int m, float2* gk,
                        cudaStream_t s);
// Inverse-only helpers reused by other stages: C2R of nf half spectra in place.
int launch_c2r_inplace(const zeta_ctx* c, float2* data, int nf, cudaStream_t s);
// The grid forms' primary vertex smoothed by the tophat: out (float[n^3]) = IDFT[dhat W_TH]
// (the workspace buffer out holds the intermediate half spectrum).
int launch_primary(const zeta_ctx* c, const float2* dhat, float* out, cudaStream_t s);

// ---- launchers (assign.cu) ----
int launch_assign(const zeta_ctx* c, const float4* parts, int64_t np, float* delta, double* wsum,
                  unsigned long long* acc, double* scratch2, cudaStream_t s);
int launch_wsum(const zeta_ctx* c, const float4* parts, int64_t np, double* wsum, double* scratch, cudaStream_t s);
constexpr int kAssignScratchDoubles = 2 * 1024 + 4;
// Per-particle data computed once per catalogue with the float64 cell arithmetic, so the kernels
// that run per (l, m) need none: the cell (linear index z n^2 + y n + x) and (t_x, t_y, t_z, w),
// the in-cell offsets and the weight (0 for a non-finite particle).  o_*: original order
// (scratch, with the tile of each particle), s_*: sorted order.
struct PartPrep {
  int* o_tile = nullptr;
  int* o_cell = nullptr;
  float4* o_tq = nullptr;
  int* s_cell = nullptr;
  float4* s_tq = nullptr;
};
// sorted_idx (optional): original index of each sorted particle; prep (optional): also write the
// prepared data of the sorted particles
int launch_sort(const zeta_ctx* c, const float4* parts, int64_t np, float4* sorted, int64_t* tile_start,
                int* counts, int* orig, cudaStream_t s, int* sorted_idx = nullptr, const PartPrep* prep = nullptr);
// Szapudi-Szalay fields: data_delta <- delta_D - delta_R, rand_delta <- 1 + delta_R
int launch_ss_fields(const zeta_ctx* c, float* data_delta, float* rand_delta, cudaStream_t s);
// prepared data of an already sorted catalogue
int launch_prep_sorted(const zeta_ctx* c, const float4* sorted, int64_t np, int* s_cell, float4* s_tq, cudaStream_t s);
// assignment from the sorted, prepared catalogue (weight sums, then one CTA per tile writes delta)
int launch_assign_tiles(const zeta_ctx* c, const float4* parts, int64_t np, const int64_t* tile_start,
                        const int* s_cell, const float4* s_tq, float* delta, double* wsum, double* scratch,
                        cudaStream_t s);

// ---- adjoint (adjoint.cu) ----
// S: symmetrised loss weights of one l, device float [nb][nb]
int launch_adj_node_point(const zeta_ctx* c, const float* delta, float* fields, const float* S, float* q,
                          cudaStream_t s);
int launch_adj_mass(const zeta_ctx* c, const float2* dhat, int l, const float* S, float2* gk, cudaStream_t s);
int launch_adj_points(const zeta_ctx* c, const float4* sorted, const int64_t* tile_start, const int* sorted_idx,
                      const float* fields, const float* S, const double* wsum, float* hfield, float* direct,
                      cudaStream_t s);
int launch_adj_finish_node(const zeta_ctx* c, const float* q, const float* g, float* grad, cudaStream_t s);
int launch_adj_finish_particles(const zeta_ctx* c, const float4* parts, int64_t np, const float* gdelta,
                                const double* wsum, const float* direct, float* grad, cudaStream_t s);

// ---- launchers (sums.cu) ----
enum GramKind { GK_NODE = 0, GK_PART = 1, GK_GAMMA = 2, GK_MASS = 3, GK_TC = 4 };
int gram_ctas(const zeta_ctx* c, int kind);
int launch_gram_node(const zeta_ctx* c, const float* delta, const float* alm, double* partials, cudaStream_t s,
                     bool bf16 = false);
int launch_gram_gamma(const zeta_ctx* c, const float* delta, const float* alm, double* partials,
                      cudaStream_t s);
int launch_gram_particles(const zeta_ctx* c, const int* s_cell, const float4* s_tq, const int64_t* tile_start,
                          int64_t np, const float* alm, float* pvals, double* partials, cudaStream_t s);
// Bytes of the interpolated particle rows [np][bins padded to 4] that launch_gram_particles uses.
size_t particle_rows_bytes(const zeta_ctx* c, int64_t np);
// tensor-core node Gram (gram_tc.cu), arithmetic chosen by c->p.gram
int launch_gram_node_tc(const zeta_ctx* c, const float* delta, const float* alm, double* partials, cudaStream_t s);
// Warp-specialised tensor-core node Gram (gram_ws.cu): ctas persistent CTAs, one partial each;
// raw 0: float32 fields (split: hi/lo bfloat16 operands), 1: bfloat16 fields.
int launch_gram_ws(const zeta_ctx* c, const float* delta, const void* fields, double* partials, int ctas, int raw,
                   bool split, cudaStream_t s);
int launch_wait_selftest(const zeta_ctx* c, long long spins, cudaStream_t s);
// Uniform term of the particle form: launch_mass_hist sums the mode weights of dhat per integer
// |n|^2 into hist (nn2 + 1 words: the sums, then the scale), once per catalogue; launch_mass
// writes the per-CTA partial Grams of one l from it.
int launch_mass_hist(const zeta_ctx* c, const float2* dhat, unsigned long long* hist, cudaStream_t s,
                     const float* table1d = nullptr);
// 2PCF from a histogram of (1 or 2) |delta_hat|^2 Phi-hat per |n|^2 (launch_mass_hist with c->d_phi):
// radii == nullptr: out[b] for the bins (nout = nbins); else out[i] at the point radii (device).
int launch_xi_hist(const zeta_ctx* c, const unsigned long long* hist, int nout, const double* radii, double* out,
                   cudaStream_t s);
// out[b] = sum_cta partials[cta][b] / *wdiv (fixed order)
int launch_reduce_vec(const zeta_ctx* c, const double* partials, int nparts, const double* wdiv, double* out,
                      cudaStream_t s);
// Particle form of the 2PCF: interpolated rows of the l = 0 fields, then per-CTA sums of w f_b.
int launch_particle_xi(const zeta_ctx* c, const int* s_cell, const float4* s_tq, const int64_t* tile_start,
                       int64_t np, const float* alm, float* pvals, double* partials, cudaStream_t s);
int launch_mass(const zeta_ctx* c, const unsigned long long* hist, int l, double* partials, cudaStream_t s);
// Weighted Gram of the interpolated particle rows ([np][bins padded to 4]) with the weights of the
// prepared records, register-blocked (<= 20 bins; ZETA_ENOTSUP above): grid CTAs, partials[grid].
int launch_gram_rows_rb(const zeta_ctx* c, const float* pvals, const float4* s_tq, int64_t np, double* partials,
                        int grid, cudaStream_t s);
// Number of per-CTA partial Grams launch_gram_particles writes.
int gram_particle_parts(const zeta_ctx* c);
// out[b1][b2] += scale * (1/ *wdiv if wdiv) * sum_cta partials[cta][b1][b2], symmetrised.
int launch_reduce(const zeta_ctx* c, const double* partials, int nparts, double scale, const double* wdiv,
                  double* out, cudaStream_t s, bool store = false);
// zeta[f][l] = per-(l, m) slots summed in the full measurement's order (see zeta_reduce_lm).
int launch_reduce_lm(const zeta_ctx* c, const double* slots, int nforms, int part_form, double* zeta, cudaStream_t s);

}  // namespace zk
