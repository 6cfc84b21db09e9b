// C ABI of libzeta: context, workspace, argument validation and the per-(l, m) hot loop
// of the measurement (Fig. 1 steps (2)-(7)).
#include <cmath>
#include <cstring>
#include <new>

#include "zeta_internal.h"

namespace {

using namespace zk;

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Layout {
  size_t delta = 0, dhat = 0, spectra = 0, fields = 0, partials = 0, small = 0, mhist = 0, sorted = 0, tstart = 0,
         counts = 0, orig = 0, pvals = 0, o_tile = 0, o_cell = 0, o_tq = 0, s_cell = 0, s_tq = 0, dprim = 0,
         xi_radii = 0, dss = 0;
  // backward (gradient) regions
  size_t gk = 0, q = 0, wts = 0, hfield = 0, direct = 0, sidx = 0;
  size_t total = 0;
};

// Workspace regions of the full measurement for np particles (np may be 0); with backward,
// also the regions of the gradient calls (placed after the forward ones).
Layout layout(const zeta_ctx* c, int64_t np, bool backward = false, bool ss = false) {
  Layout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align_up(off + bytes);
    return at;
  };
  const size_t g = static_cast<size_t>(c->ng) * sizeof(float);
  L.delta = take(g);
  L.dhat = take(g);
  L.spectra = take(g * c->p.nbins);                    // plain half spectra of the C2R passes
  L.fields = take(g * 4 * ((c->p.nbins + 3) / 4));     // bin-interleaved fields; also the assign accumulator
  L.partials = take(sizeof(double) * kMaxCtas * c->p.nbins * c->p.nbins);
  if (c->p.tophat_primary > 0) L.dprim = take(g);  // the grid forms' smoothed primary vertex
  L.xi_radii = take(sizeof(double) * 4096);          // radii of zeta_xi_radii
  L.small = take(sizeof(double) * (kAssignScratchDoubles + 8));
  L.mhist = take(sizeof(unsigned long long) * static_cast<size_t>(c->nn2 + 1));  // uniform-term sums per |n|^2
  L.sorted = take(sizeof(float4) * static_cast<size_t>(np));
  L.tstart = take(sizeof(int64_t) * static_cast<size_t>(c->ntiles + 1));
  L.counts = take(sizeof(int) * static_cast<size_t>(c->ntiles));
  L.orig = take(sizeof(int) * static_cast<size_t>(np));
  L.pvals = take(particle_rows_bytes(c, np));  // interpolated particle rows of one (l, m)
  // prepared particle data (cell, offsets, weight): original order (scratch) and sorted order
  L.o_tile = take(sizeof(int) * static_cast<size_t>(np));
  L.o_cell = take(sizeof(int) * static_cast<size_t>(np));
  L.o_tq = take(sizeof(float4) * static_cast<size_t>(np));
  L.s_cell = take(sizeof(int) * static_cast<size_t>(np));
  L.s_tq = take(sizeof(float4) * static_cast<size_t>(np));
  if (backward) {
    L.gk = take(g);
    L.q = take(g);
    L.wts = take(sizeof(float) * (kMaxL + 1) * kMaxBins * kMaxBins);
    L.hfield = take(g * 4 * ((c->p.nbins + 3) / 4));
    L.direct = take(sizeof(float) * 3 * static_cast<size_t>(np));
    L.sidx = take(sizeof(int) * static_cast<size_t>(np));
  }
  if (ss) L.dss = take(g);  // the random catalogue's grid of the Szapudi-Szalay estimator
  L.total = off;
  return L;
}

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// the node-form Gram runs on the tensor cores
bool tc_gram(const zeta_ctx* c) { return c->p.gram >= ZETA_GRAM_TF32 && c->p.gram <= ZETA_GRAM_BF16X3; }

int check_ctx(const zeta_ctx* c) { return c ? ZETA_OK : ZETA_EINVAL; }

int need_ws(const zeta_ctx* c, int64_t np, bool backward = false, bool ss = false) {
  if (!c->ws) return ZETA_EWORKSPACE;
  if (layout(c, np, backward, ss).total > c->ws_bytes) return ZETA_EWORKSPACE;
  return ZETA_OK;
}

template <typename T>
T* at(const zeta_ctx* c, size_t off) {
  return reinterpret_cast<T*>(c->ws + off);
}

PartPrep prep_of(const zeta_ctx* c, const Layout& L) {
  PartPrep q;
  q.o_tile = at<int>(c, L.o_tile);
  q.o_cell = at<int>(c, L.o_cell);
  q.o_tq = at<float4>(c, L.o_tq);
  q.s_cell = at<int>(c, L.s_cell);
  q.s_tq = at<float4>(c, L.s_tq);
  return q;
}

void drop_batch_graph(zeta_ctx* c) {
  if (c->batch_exec) cudaGraphExecDestroy(c->batch_exec);
  c->batch_exec = nullptr;
  c->batch_key.clear();
}

#define ZK_TRY(expr)             \
  do {                           \
    const int _rc = (expr);      \
    if (_rc != ZETA_OK) return _rc; \
  } while (0)

}  // namespace

extern "C" {

int zeta_version(void) { return 10000; }

const char* zeta_strerror(int code) {
  switch (code) {
    case ZETA_OK: return "ok";
    case ZETA_EINVAL: return "invalid argument";
    case ZETA_ECUDA: return "CUDA runtime error";
    case ZETA_ENOMEM: return "device allocation failed";
    case ZETA_ETIMEOUT: return "bounded device wait timed out";
    case ZETA_ENOTSUP: return "configuration not supported";
    case ZETA_EWORKSPACE: return "workspace missing or too small";
    case ZETA_EDATA: return "invalid input data (non-finite particle)";
    default: return "unknown error";
  }
}

int zeta_create(const zeta_params* p, zeta_ctx** out) {
  if (!out) return ZETA_EINVAL;
  *out = nullptr;
  if (!p || !is_pow2(p->n) || p->n < 16 || p->n > 512) return ZETA_EINVAL;
  if (!(p->box > 0) || !std::isfinite(p->box)) return ZETA_EINVAL;
  if (p->dsup < 2 || p->dsup > 4) return ZETA_EINVAL;  // 2, 4: B-splines; 3: Daubechies
  if (p->lmax < 0 || p->lmax > kMaxL) return ZETA_EINVAL;
  if (p->nbins < 1 || p->nbins > kMaxBins) return ZETA_EINVAL;
  if (p->gram < ZETA_GRAM_FP32 || p->gram > ZETA_GRAM_BF16_FIELDS) return ZETA_EINVAL;
  if (!(p->tophat >= 0) || !std::isfinite(p->tophat) || !(p->tophat_primary >= 0) ||
      !std::isfinite(p->tophat_primary) || (p->phi_hat != 0 && p->phi_hat != 1))
    return ZETA_EINVAL;
  if (p->radial == ZETA_RADIAL_SHELL) {
    if (!p->edges || !(p->edges[0] > 0)) return ZETA_EINVAL;
    for (int b = 0; b < p->nbins; ++b)
      if (!(p->edges[b + 1] > p->edges[b]) || !std::isfinite(p->edges[b + 1])) return ZETA_EINVAL;
    if (!(p->edges[p->nbins] < 0.5 * p->box)) return ZETA_EINVAL;
  } else if (p->radial == ZETA_RADIAL_POINT) {
    if (!p->radii) return ZETA_EINVAL;
    for (int b = 0; b < p->nbins; ++b)
      if (!(p->radii[b] > 0) || !(p->radii[b] < 0.5 * p->box)) return ZETA_EINVAL;
  } else {
    return ZETA_EINVAL;
  }

  zeta_ctx* c = new (std::nothrow) zeta_ctx();
  if (!c) return ZETA_ENOMEM;
  c->p = *p;
  if (p->radial == ZETA_RADIAL_SHELL) c->edges.assign(p->edges, p->edges + p->nbins + 1);
  else c->radii.assign(p->radii, p->radii + p->nbins);
  c->p.edges = c->edges.empty() ? nullptr : c->edges.data();
  c->p.radii = c->radii.empty() ? nullptr : c->radii.data();
  c->n = p->n;
  c->nc = p->n / 2;
  c->ng = static_cast<int64_t>(p->n) * p->n * p->n;
  c->nn2 = table_n2_count(p->n);
  c->ntiles = static_cast<int64_t>(p->n / kTile) * (p->n / kTile) * (p->n / kTile);
  c->gamma_q = p->dsup == 2 ? 2 : 5;
  if (p->nbins <= 20) c->tune[GK_NODE] = 1;  // the register-blocked node Gram holds one CTA per SM
  auto fail = [&](int rc) {
    zeta_destroy(c);
    return rc;
  };
  if (cudaGetDevice(&c->device) != cudaSuccess) return fail(ZETA_ECUDA);
  if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess)
    return fail(ZETA_ECUDA);

  std::vector<float> jtab;
  VertexSpec vs;
  vs.radial = p->radial;
  vs.edges = c->p.edges;
  vs.radii = c->p.radii;
  vs.tophat = p->tophat;
  host_window_table(p->n, p->box, p->lmax, p->nbins, vs, jtab);
  std::vector<float2> tw;
  host_twiddles(p->n, tw);
  std::vector<float> mhat;
  host_mass_hat(p->n, p->dsup, mhat, p->phi_hat != 0);
  std::vector<double> ph64;
  host_phi_hat_1d(p->n, p->dsup, ph64);
  std::vector<float> phi(p->n, 1.0f);
  if (p->phi_hat)
    for (int i = 0; i < p->n; ++i) phi[i] = static_cast<float>(ph64[i]);
  std::vector<float> wprim;
  if (p->tophat_primary > 0) host_tophat_table(p->n, p->box, p->tophat_primary, wprim);
  std::vector<float> gq;  // Gamma form: point weights [q], then stencil taps [q][taps]
  std::vector<float> daub;
  if (p->dsup == 3) {
    std::vector<double> lam, u, dy;
    host_daub4_gamma_split(lam, u);
    for (int k = 0; k < 5; ++k) gq.push_back(static_cast<float>(lam[k]));
    for (int k = 0; k < 5; ++k)
      for (int o = 0; o < 5; ++o) gq.push_back(static_cast<float>(u[o * 5 + k]));
    host_daub4_dyadic(kDaubLevel, dy);
    for (double v : dy) daub.push_back(static_cast<float>(v));
  } else {
    std::vector<double> qt, qw, qb;
    host_cell_quadrature(c->gamma_q, p->dsup, qt, qw, qb);
    for (double v : qw) gq.push_back(static_cast<float>(v));
    for (double v : qb) gq.push_back(static_cast<float>(v));
  }

  if (cudaMalloc(&c->d_jtab, jtab.size() * sizeof(float)) != cudaSuccess) return fail(ZETA_ENOMEM);
  if (cudaMalloc(&c->d_tw, tw.size() * sizeof(float2)) != cudaSuccess) return fail(ZETA_ENOMEM);
  if (cudaMalloc(&c->d_mhat, mhat.size() * sizeof(float)) != cudaSuccess) return fail(ZETA_ENOMEM);
  if (cudaMalloc(&c->d_gq, gq.size() * sizeof(float)) != cudaSuccess) return fail(ZETA_ENOMEM);
  if (cudaMalloc(&c->d_status, sizeof(int)) != cudaSuccess) return fail(ZETA_ENOMEM);
  if (cudaMalloc(&c->d_phi, phi.size() * sizeof(float)) != cudaSuccess) return fail(ZETA_ENOMEM);
  if (!daub.empty()) {
    if (cudaMalloc(&c->d_daub, daub.size() * sizeof(float)) != cudaSuccess) return fail(ZETA_ENOMEM);
    if (cudaMemcpy(c->d_daub, daub.data(), daub.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(ZETA_ECUDA);
  }
  if (cudaMemcpy(c->d_phi, phi.data(), phi.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(ZETA_ECUDA);
  if (!wprim.empty()) {
    if (cudaMalloc(&c->d_wprim, wprim.size() * sizeof(float)) != cudaSuccess) return fail(ZETA_ENOMEM);
    if (cudaMemcpy(c->d_wprim, wprim.data(), wprim.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(ZETA_ECUDA);
  }
  if (cudaMemcpy(c->d_jtab, jtab.data(), jtab.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->d_tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->d_mhat, mhat.data(), mhat.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->d_gq, gq.data(), gq.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(c->d_status, 0, sizeof(int)) != cudaSuccess)
    return fail(ZETA_ECUDA);
  if (set_ylm_constants() != ZETA_OK) return fail(ZETA_ECUDA);
  *out = c;
  return ZETA_OK;
}

int zeta_destroy(zeta_ctx* c) {
  if (!c) return ZETA_OK;
  profile_release(c);
  if (c->batch_exec) cudaGraphExecDestroy(c->batch_exec);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  for (int j = 0; j < zeta_ctx::kMaxBatchStreams - 1; ++j) {
    if (c->cap_aux[j]) cudaStreamDestroy(c->cap_aux[j]);
    if (c->cap_join[j]) cudaEventDestroy(c->cap_join[j]);
  }
  if (c->cap_fork) cudaEventDestroy(c->cap_fork);
  cudaFree(c->d_jtab);
  cudaFree(c->d_tw);
  cudaFree(c->d_mhat);
  cudaFree(c->d_gq);
  cudaFree(c->d_status);
  cudaFree(c->d_phi);
  cudaFree(c->d_wprim);
  cudaFree(c->d_daub);
  delete c;
  return ZETA_OK;
}

size_t zeta_workspace_bytes(const zeta_ctx* c, int64_t np_max, int forms) {
  if (!c || np_max < 0 || np_max > 0x7fffffffLL || forms < 0 || forms > 31) return 0;
  return layout(c, np_max, (forms & ZETA_WS_BACKWARD) != 0, (forms & ZETA_WS_SS) != 0).total;
}

int zeta_set_workspace(zeta_ctx* c, void* dptr, size_t bytes) {
  ZK_TRY(check_ctx(c));
  if (dptr && (reinterpret_cast<uintptr_t>(dptr) % kAlign)) return ZETA_EINVAL;
  c->ws = static_cast<char*>(dptr);
  c->ws_bytes = dptr ? bytes : 0;
  drop_batch_graph(c);  // a captured batch refers to the old workspace
  return ZETA_OK;
}

int64_t zeta_tile_count(const zeta_ctx* c) { return c ? c->ntiles : 0; }

int zeta_set_gram(zeta_ctx* c, int gram) {
  ZK_TRY(check_ctx(c));
  if (gram < ZETA_GRAM_FP32 || gram > ZETA_GRAM_BF16_FIELDS) return ZETA_EINVAL;
  c->p.gram = gram;
  drop_batch_graph(c);
  return ZETA_OK;
}

int zeta_assign(zeta_ctx* c, const float* particles, int64_t np, float* delta, double* wsum, zeta_stream stream) {
  ZK_TRY(check_ctx(c));
  if (!particles || np < 1 || np > 0x7fffffffLL || !delta) return ZETA_EINVAL;
  ZK_TRY(need_ws(c, 0));
  const Layout L = layout(c, 0);
  double* small = at<double>(c, L.small);
  double* w = wsum ? wsum : small + kAssignScratchDoubles + 4;
  return launch_assign(c, reinterpret_cast<const float4*>(particles), np, delta, w,
                       at<unsigned long long>(c, L.fields), small, stream);
}

int zeta_fft_r2c(zeta_ctx* c, const float* delta, float* delta_hat, zeta_stream stream) {
  ZK_TRY(check_ctx(c));
  if (!delta || !delta_hat) return ZETA_EINVAL;
  return launch_r2c(c, delta, reinterpret_cast<float2*>(delta_hat), stream);
}

int zeta_reconstruct_alm(zeta_ctx* c, const float* delta_hat, int l, int m, int b0, int b1, float* alm,
                         zeta_stream stream) {
  ZK_TRY(check_ctx(c));
  if (!delta_hat || !alm || l < 0 || l > c->p.lmax || m < -l || m > l || b0 < 0 || (b0 & 3) || b1 <= b0 ||
      b1 > c->p.nbins)
    return ZETA_EINVAL;
  ZK_TRY(need_ws(c, 0));
  const Layout L = layout(c, 0);
  return launch_alm(c, reinterpret_cast<const float2*>(delta_hat), l, m, b0, b1 - b0, at<float2>(c, L.spectra), alm,
                    stream);
}

int zeta_sum_grid(zeta_ctx* c, const float* delta, const float* alm, int form, double* gram, zeta_stream stream) {
  ZK_TRY(check_ctx(c));
  if (!delta || !alm || !gram || (form != ZETA_SUM_NODE && form != ZETA_SUM_GAMMA)) return ZETA_EINVAL;
  ZK_TRY(need_ws(c, 0));
  const Layout L = layout(c, 0);
  double* part = at<double>(c, L.partials);
  if (form == ZETA_SUM_NODE)
    ZK_TRY(!tc_gram(c) ? launch_gram_node(c, delta, alm, part, stream)
                       : launch_gram_node_tc(c, delta, alm, part, stream));
  else
    ZK_TRY(launch_gram_gamma(c, delta, alm, part, stream));
  return launch_reduce(c, part, gram_ctas(c, form == ZETA_SUM_NODE ? (tc_gram(c) ? GK_TC : GK_NODE) : GK_GAMMA),
                       1.0 / static_cast<double>(c->ng), nullptr, gram, stream);
}

int zeta_sort_particles(zeta_ctx* c, const float* particles, int64_t np, float* sorted, int64_t* tile_start,
                        zeta_stream stream) {
  ZK_TRY(check_ctx(c));
  if (!particles || np < 1 || np > 0x7fffffffLL || !sorted || !tile_start) return ZETA_EINVAL;
  ZK_TRY(need_ws(c, np));
  const Layout L = layout(c, np);
  return launch_sort(c, reinterpret_cast<const float4*>(particles), np, reinterpret_cast<float4*>(sorted),
                     tile_start, at<int>(c, L.counts), at<int>(c, L.orig), stream);
}

int zeta_sum_particles(zeta_ctx* c, const float* sorted, const int64_t* tile_start, int64_t np, const double* wsum,
                       const float* alm, double* gram, zeta_stream stream) {
  ZK_TRY(check_ctx(c));
  if (!sorted || !tile_start || np < 1 || !wsum || !alm || !gram) return ZETA_EINVAL;
  ZK_TRY(need_ws(c, np));
  const Layout L = layout(c, np);
  double* part = at<double>(c, L.partials);
  const PartPrep q = prep_of(c, L);
  ZK_TRY(launch_prep_sorted(c, reinterpret_cast<const float4*>(sorted), np, q.s_cell, q.s_tq, stream));
  ZK_TRY(launch_gram_particles(c, q.s_cell, q.s_tq, tile_start, np, alm, at<float>(c, L.pvals), part, stream));
  return launch_reduce(c, part, gram_particle_parts(c), 1.0, wsum, gram, stream);
}

int zeta_mass_term(zeta_ctx* c, const float* delta_hat, int l, double sign, double* gram, zeta_stream stream) {
  ZK_TRY(check_ctx(c));
  if (!delta_hat || !gram || l < 0 || l > c->p.lmax || !(sign == 1.0 || sign == -1.0)) return ZETA_EINVAL;
  ZK_TRY(need_ws(c, 0));
  const Layout L = layout(c, 0);
  double* part = at<double>(c, L.partials);
  unsigned long long* hist = at<unsigned long long>(c, L.mhist);
  ZK_TRY(launch_mass_hist(c, reinterpret_cast<const float2*>(delta_hat), hist, stream));
  ZK_TRY(launch_mass(c, hist, l, part, stream));
  const double scale = sign * (2.0 * l + 1.0) / (4.0 * 3.14159265358979323846);
  return launch_reduce(c, part, gram_ctas(c, GK_MASS), scale, nullptr, gram, stream);
}

}  // extern "C"

namespace {

// The measurement of Fig. 1 steps (2)-(7).  With lm_size > 1 only the (l, m) pairs of index
// i = l^2 + l + m with i mod lm_size == lm_rank run, and the uniform term of l runs on the owner
// of (l, -l).  slots == false: zeta is [form][l][nb][nb], accumulated in the order 0, uniform
// term, m = -l .. l.  slots == true: every contribution is stored in its own slot
// [form][(lmax+1)^2 + lmax+1][nb][nb] ((l, m) at l^2 + l + m, the uniform term of l at
// (lmax+1)^2 + l), the slots this call does not own set to zero.
int measure(zeta_ctx* c, const float* particles, int64_t np, const float* delta, int forms, int lm_rank, int lm_size,
            bool slots, double* zeta, cudaStream_t stream) {
  ZK_TRY(check_ctx(c));
  if (!zeta || forms < 1 || forms > 7 || lm_size < 1 || lm_rank < 0 || lm_rank >= lm_size) return ZETA_EINVAL;
  // bfloat16 fields serve the node form alone (the other forms interpolate or integrate them)
  const bool bf16f = c->p.gram == ZETA_GRAM_BF16_FIELDS;
  if (bf16f && forms != ZETA_SUM_NODE) return ZETA_EINVAL;
  const bool want_p = forms & ZETA_SUM_PARTICLE;
  if ((want_p || !delta) && (!particles || np < 1 || np > 0x7fffffffLL)) return ZETA_EINVAL;
  const int64_t npl = want_p ? np : 0;
  ZK_TRY(need_ws(c, npl));
  const Layout L = layout(c, npl);
  const int nb = c->p.nbins, lmax = c->p.lmax;
  const float4* parts = reinterpret_cast<const float4*>(particles);
  double* small = at<double>(c, L.small);
  double* wsum = small + kAssignScratchDoubles + 4;
  float* dl = delta ? const_cast<float*>(delta) : at<float>(c, L.delta);
  float2* dhat = at<float2>(c, L.dhat);
  float* fields = at<float>(c, L.fields);
  double* part = at<double>(c, L.partials);
  float4* sorted = at<float4>(c, L.sorted);
  int64_t* tstart = at<int64_t>(c, L.tstart);

  const PartPrep q = prep_of(c, L);
  if (want_p) {  // sort (and prepare) first; then the assignment is computed tile by tile
    ZK_TRY(launch_sort(c, parts, np, sorted, tstart, at<int>(c, L.counts), at<int>(c, L.orig), stream, nullptr, &q));
    if (!delta)
      ZK_TRY(launch_assign_tiles(c, parts, np, tstart, q.s_cell, q.s_tq, dl, wsum, small, stream));
    else
      ZK_TRY(launch_wsum(c, parts, np, wsum, small, stream));
  } else if (!delta) {
    ZK_TRY(launch_assign(c, parts, np, dl, wsum, reinterpret_cast<unsigned long long*>(fields), small, stream));
  }
  ZK_TRY(launch_r2c(c, dl, dhat, stream));
  unsigned long long* hist = at<unsigned long long>(c, L.mhist);
  if (want_p) ZK_TRY(launch_mass_hist(c, dhat, hist, stream));
  // the grid forms' primary vertex (smoothed by its tophat, if the context has one)
  const float* prim = dl;
  if (c->p.tophat_primary > 0 && (forms & (ZETA_SUM_NODE | ZETA_SUM_GAMMA))) {
    ZK_TRY(launch_primary(c, dhat, at<float>(c, L.dprim), stream));
    prim = at<float>(c, L.dprim);
  }

  int nforms = 0, idx_node = -1, idx_gamma = -1, idx_part = -1;
  if (forms & ZETA_SUM_NODE) idx_node = nforms++;
  if (forms & ZETA_SUM_GAMMA) idx_gamma = nforms++;
  if (want_p) idx_part = nforms++;
  const size_t nb2 = static_cast<size_t>(nb) * nb;
  const size_t nslot = slots ? static_cast<size_t>(lmax + 1) * (lmax + 1) + lmax + 1 : static_cast<size_t>(lmax + 1);
  const size_t per_form = nslot * nb2;
  if (cudaMemsetAsync(zeta, 0, sizeof(double) * per_form * nforms, stream) != cudaSuccess) return ZETA_ECUDA;
  // output block of form index f for (l, m) (m > l: the uniform term of l)
  auto out = [&](int f, int l, int m) {
    size_t slot = l;
    if (slots) slot = m > l ? static_cast<size_t>(lmax + 1) * (lmax + 1) + l : static_cast<size_t>(l) * l + l + m;
    return zeta + f * per_form + slot * nb2;
  };
  const double inv_ng = 1.0 / static_cast<double>(c->ng);
  for (int l = 0; l <= lmax; ++l) {
    if (want_p && (l * l) % lm_size == lm_rank) {
      ZK_TRY(launch_mass(c, hist, l, part, stream));
      ZK_TRY(launch_reduce(c, part, gram_ctas(c, GK_MASS), -(2.0 * l + 1.0) / (4.0 * 3.14159265358979323846), nullptr,
                           out(idx_part, l, l + 1), stream, slots));
    }
    for (int m = -l; m <= l; ++m) {
      if ((l * l + l + m) % lm_size != lm_rank) continue;
      ZK_TRY(launch_alm(c, dhat, l, m, 0, nb, at<float2>(c, L.spectra), fields, stream, bf16f));
      if (idx_node >= 0) {
        ZK_TRY(!tc_gram(c) ? launch_gram_node(c, prim, fields, part, stream, bf16f)
                           : launch_gram_node_tc(c, prim, fields, part, stream));
        ZK_TRY(launch_reduce(c, part, gram_ctas(c, tc_gram(c) ? GK_TC : GK_NODE), inv_ng, nullptr,
                             out(idx_node, l, m), stream, slots));
      }
      if (idx_gamma >= 0) {
        ZK_TRY(launch_gram_gamma(c, prim, fields, part, stream));
        ZK_TRY(launch_reduce(c, part, gram_ctas(c, GK_GAMMA), inv_ng, nullptr, out(idx_gamma, l, m), stream, slots));
      }
      if (idx_part >= 0) {
        ZK_TRY(launch_gram_particles(c, q.s_cell, q.s_tq, tstart, np, fields, at<float>(c, L.pvals), part, stream));
        ZK_TRY(launch_reduce(c, part, gram_particle_parts(c), 1.0, wsum, out(idx_part, l, m), stream, slots));
      }
    }
  }
  return ZETA_OK;
}

int nforms_of(int forms) { return ((forms & 1) ? 1 : 0) + ((forms & 2) ? 1 : 0) + ((forms & 4) ? 1 : 0); }

}  // namespace

extern "C" {

int zeta_zeta_ell(zeta_ctx* c, const float* particles, int64_t np, const float* delta, int forms, double* zeta,
                  zeta_stream stream) {
  return measure(c, particles, np, delta, forms, 0, 1, false, zeta, stream);
}

int zeta_xi(zeta_ctx* c, const float* particles, int64_t np, const float* delta, int forms, double* xi,
            zeta_stream stream) {
  ZK_TRY(check_ctx(c));
  if (!xi || forms < 1 || (forms & ~(ZETA_SUM_NODE | ZETA_SUM_PARTICLE))) return ZETA_EINVAL;
  const bool want_p = forms & ZETA_SUM_PARTICLE;
  if ((want_p || !delta) && (!particles || np < 1 || np > 0x7fffffffLL)) return ZETA_EINVAL;
  const int64_t npl = want_p ? np : 0;
  ZK_TRY(need_ws(c, npl));
  const Layout L = layout(c, npl);
  const int nb = c->p.nbins;
  const float4* parts = reinterpret_cast<const float4*>(particles);
  double* small = at<double>(c, L.small);
  double* wsum = small + kAssignScratchDoubles + 4;
  float* dl = delta ? const_cast<float*>(delta) : at<float>(c, L.delta);
  float2* dhat = at<float2>(c, L.dhat);
  float* fields = at<float>(c, L.fields);
  double* part = at<double>(c, L.partials);
  int64_t* tstart = at<int64_t>(c, L.tstart);
  const PartPrep q = prep_of(c, L);
  if (want_p) {
    ZK_TRY(launch_sort(c, parts, np, at<float4>(c, L.sorted), tstart, at<int>(c, L.counts), at<int>(c, L.orig),
                       stream, nullptr, &q));
    if (!delta)
      ZK_TRY(launch_assign_tiles(c, parts, np, tstart, q.s_cell, q.s_tq, dl, wsum, small, stream));
    else
      ZK_TRY(launch_wsum(c, parts, np, wsum, small, stream));
  } else if (!delta) {
    ZK_TRY(launch_assign(c, parts, np, dl, wsum, reinterpret_cast<unsigned long long*>(fields), small, stream));
  }
  ZK_TRY(launch_r2c(c, dl, dhat, stream));
  int f = 0;
  if (forms & ZETA_SUM_NODE) {
    unsigned long long* hist = at<unsigned long long>(c, L.mhist);
    ZK_TRY(launch_mass_hist(c, dhat, hist, stream, c->d_phi));
    ZK_TRY(launch_xi_hist(c, hist, nb, nullptr, xi + f * nb, stream));
    ++f;
  }
  if (want_p) {
    ZK_TRY(launch_alm(c, dhat, 0, 0, 0, nb, at<float2>(c, L.spectra), fields, stream));
    ZK_TRY(launch_particle_xi(c, q.s_cell, q.s_tq, tstart, np, fields, at<float>(c, L.pvals), part, stream));
    ZK_TRY(launch_reduce_vec(c, part, gram_particle_parts(c), wsum, xi + f * nb, stream));
  }
  return ZETA_OK;
}

int zeta_zeta_ell_ss(zeta_ctx* c, const float* data, int64_t nd, const float* randoms, int64_t nr, int forms,
                     double* num, double* den, zeta_stream stream) {
  ZK_TRY(check_ctx(c));
  if (!data || !randoms || nd < 1 || nr < 1 || nd > 0x7fffffffLL || nr > 0x7fffffffLL || !num || !den ||
      forms < 1 || (forms & ~(ZETA_SUM_NODE | ZETA_SUM_GAMMA)))
    return ZETA_EINVAL;
  ZK_TRY(need_ws(c, 0, false, true));
  const Layout L = layout(c, 0, false, true);
  double* small = at<double>(c, L.small);
  float* dd = at<float>(c, L.delta);
  float* dr = at<float>(c, L.dss);
  unsigned long long* acc = at<unsigned long long>(c, L.fields);
  double* w = small + kAssignScratchDoubles + 4;
  ZK_TRY(launch_assign(c, reinterpret_cast<const float4*>(data), nd, dd, w, acc, small, stream));
  ZK_TRY(launch_assign(c, reinterpret_cast<const float4*>(randoms), nr, dr, w, acc, small, stream));
  ZK_TRY(launch_ss_fields(c, dd, dr, stream));
  ZK_TRY(measure(c, nullptr, 0, dd, forms, 0, 1, false, num, stream));
  return measure(c, nullptr, 0, dr, forms, 0, 1, false, den, stream);
}

int zeta_xi_radii(zeta_ctx* c, const float* delta_hat, int nr, const double* radii, double* xi, zeta_stream stream) {
  ZK_TRY(check_ctx(c));
  if (!delta_hat || !radii || !xi || nr < 1 || nr > 4096) return ZETA_EINVAL;
  for (int i = 0; i < nr; ++i)
    if (!(radii[i] >= 0) || !std::isfinite(radii[i])) return ZETA_EINVAL;
  ZK_TRY(need_ws(c, 0));
  const Layout L = layout(c, 0);
  // the radii go to the device through the workspace's small scratch (after the weight sums)
  double* dr = at<double>(c, L.xi_radii);
  if (cudaMemcpyAsync(dr, radii, sizeof(double) * nr, cudaMemcpyHostToDevice, stream) != cudaSuccess)
    return ZETA_ECUDA;
  unsigned long long* hist = at<unsigned long long>(c, L.mhist);
  ZK_TRY(launch_mass_hist(c, reinterpret_cast<const float2*>(delta_hat), hist, stream, c->d_phi));
  ZK_TRY(launch_xi_hist(c, hist, nr, dr, xi, stream));
  // the host array must stay valid until the copy has been read
  return cudaStreamSynchronize(stream) == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
}

int zeta_zeta_lm(zeta_ctx* c, const float* particles, int64_t np, const float* delta, int forms, int lm_rank,
                 int lm_size, double* slots, zeta_stream stream) {
  return measure(c, particles, np, delta, forms, lm_rank, lm_size, true, slots, stream);
}

int zeta_reduce_lm(zeta_ctx* c, const double* slots, int forms, double* zeta, zeta_stream stream) {
  ZK_TRY(check_ctx(c));
  if (!slots || !zeta || forms < 1 || forms > 7) return ZETA_EINVAL;
  const int nforms = nforms_of(forms);
  return launch_reduce_lm(c, slots, nforms, (forms & ZETA_SUM_PARTICLE) ? nforms - 1 : -1, zeta, stream);
}

size_t zeta_lm_slots(const zeta_ctx* c, int forms) {
  if (!c || forms < 1 || forms > 7) return 0;
  const size_t L1 = static_cast<size_t>(c->p.lmax) + 1;
  return nforms_of(forms) * (L1 * L1 + L1) * c->p.nbins * c->p.nbins;
}

int zeta_batch(zeta_ctx* c, const float* particles, const int64_t* offsets, int ncat, int forms, double* zeta,
               zeta_stream stream) {
  ZK_TRY(check_ctx(c));
  if (!particles || !offsets || ncat < 1 || !zeta || forms < 1 || forms > 7 || offsets[0] < 0) return ZETA_EINVAL;
  int64_t np_max = 0;
  for (int i = 0; i < ncat; ++i) {
    const int64_t np = offsets[i + 1] - offsets[i];
    if (np < 1 || np > 0x7fffffffLL) return ZETA_EINVAL;
    if (np > np_max) np_max = np;
  }
  const int64_t npl = (forms & ZETA_SUM_PARTICLE) ? np_max : 0;
  ZK_TRY(need_ws(c, npl));
  // catalogues in flight: as many whole per-catalogue workspaces as the caller's holds (<= 4)
  const size_t per_ws = layout(c, npl).total;
  int k = static_cast<int>(c->ws_bytes / per_ws);
  if (k > zeta_ctx::kMaxBatchStreams) k = zeta_ctx::kMaxBatchStreams;
  if (k > ncat) k = ncat;
  if (k < 1) k = 1;
  std::vector<int64_t> key = {static_cast<int64_t>(reinterpret_cast<uintptr_t>(particles)),
                              static_cast<int64_t>(reinterpret_cast<uintptr_t>(zeta)), forms, ncat, k};
  key.insert(key.end(), offsets, offsets + ncat + 1);
  if (!c->batch_exec || key != c->batch_key) {
    drop_batch_graph(c);
    if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
      return ZETA_ECUDA;
    if (!c->cap_fork && cudaEventCreateWithFlags(&c->cap_fork, cudaEventDisableTiming) != cudaSuccess)
      return ZETA_ECUDA;
    for (int j = 0; j < k - 1; ++j) {
      if (!c->cap_aux[j] && cudaStreamCreateWithFlags(&c->cap_aux[j], cudaStreamNonBlocking) != cudaSuccess)
        return ZETA_ECUDA;
      if (!c->cap_join[j] && cudaEventCreateWithFlags(&c->cap_join[j], cudaEventDisableTiming) != cudaSuccess)
        return ZETA_ECUDA;
    }
    int nforms = ((forms & 1) ? 1 : 0) + ((forms & 2) ? 1 : 0) + ((forms & 4) ? 1 : 0);
    const size_t per_cat = static_cast<size_t>(nforms) * (c->p.lmax + 1) * c->p.nbins * c->p.nbins;
    c->capturing = true;
    if (cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      c->capturing = false;
      return ZETA_ECUDA;
    }
    int rc = ZETA_OK;
    // fork: the auxiliary streams join the capture behind an event of the capturing stream
    if (k > 1 && cudaEventRecord(c->cap_fork, c->cap_stream) != cudaSuccess) rc = ZETA_ECUDA;
    for (int j = 0; j < k - 1 && rc == ZETA_OK; ++j)
      if (cudaStreamWaitEvent(c->cap_aux[j], c->cap_fork, 0) != cudaSuccess) rc = ZETA_ECUDA;
    // catalogue i runs on stream i mod k in workspace slice i mod k (the launches record the
    // slice's addresses, so the context's workspace is switched only while capturing)
    char* const ws0 = c->ws;
    const size_t ws_bytes0 = c->ws_bytes;
    for (int i = 0; i < ncat && rc == ZETA_OK; ++i) {
      const int j = i % k;
      c->ws = ws0 + j * per_ws;
      c->ws_bytes = per_ws;
      rc = zeta_zeta_ell(c, particles + 4 * offsets[i], offsets[i + 1] - offsets[i], nullptr, forms,
                         zeta + i * per_cat, j == 0 ? c->cap_stream : c->cap_aux[j - 1]);
    }
    c->ws = ws0;
    c->ws_bytes = ws_bytes0;
    // join every auxiliary stream back into the capturing stream
    for (int j = 0; j < k - 1; ++j) {
      if (cudaEventRecord(c->cap_join[j], c->cap_aux[j]) != cudaSuccess ||
          cudaStreamWaitEvent(c->cap_stream, c->cap_join[j], 0) != cudaSuccess)
        rc = rc ? rc : ZETA_ECUDA;
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(c->cap_stream, &g);
    c->capturing = false;
    c->batch_streams = k;
    if (rc != ZETA_OK || ec != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return rc != ZETA_OK ? rc : ZETA_ECUDA;
    }
    const cudaError_t ei = cudaGraphInstantiate(&c->batch_exec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      c->batch_exec = nullptr;
      return ZETA_ECUDA;
    }
    c->batch_key = key;
  }
  return cudaGraphLaunch(c->batch_exec, stream) == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
}

int zeta_autotune(zeta_ctx* c, const float* particles, int64_t np, int forms, zeta_stream stream) {
  ZK_TRY(check_ctx(c));
  if (!particles || np < 1 || np > 0x7fffffffLL || forms < 1 || forms > 7) return ZETA_EINVAL;
  const bool want_p = forms & ZETA_SUM_PARTICLE;
  ZK_TRY(need_ws(c, want_p ? np : 0));
  const Layout L = layout(c, want_p ? np : 0);
  const float4* parts = reinterpret_cast<const float4*>(particles);
  double* small = at<double>(c, L.small);
  double* wsum = small + kAssignScratchDoubles + 4;
  float* dl = at<float>(c, L.delta);
  float2* dhat = at<float2>(c, L.dhat);
  float* fields = at<float>(c, L.fields);
  double* part = at<double>(c, L.partials);
  float4* sorted = at<float4>(c, L.sorted);
  int64_t* tstart = at<int64_t>(c, L.tstart);
  // representative data: this catalogue's fields for one (l, m)
  const PartPrep q = prep_of(c, L);
  ZK_TRY(launch_assign(c, parts, np, dl, wsum, reinterpret_cast<unsigned long long*>(fields), small, stream));
  ZK_TRY(launch_r2c(c, dl, dhat, stream));
  unsigned long long* hist = at<unsigned long long>(c, L.mhist);
  if (want_p) {
    ZK_TRY(launch_sort(c, parts, np, sorted, tstart, at<int>(c, L.counts), at<int>(c, L.orig), stream, nullptr, &q));
    ZK_TRY(launch_mass_hist(c, dhat, hist, stream));
  }
  const int l = c->p.lmax < 2 ? c->p.lmax : 2;
  ZK_TRY(launch_alm(c, dhat, l, 0, 0, c->p.nbins, at<float2>(c, L.spectra), fields, stream));
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return ZETA_ECUDA;
  auto run = [&](int kind) -> int {
    switch (kind) {
      case GK_NODE: return launch_gram_node(c, dl, fields, part, stream);
      case GK_TC: return launch_gram_node_tc(c, dl, fields, part, stream);
      case GK_GAMMA: return launch_gram_gamma(c, dl, fields, part, stream);
      case GK_PART:
        return launch_gram_particles(c, q.s_cell, q.s_tq, tstart, np, fields, at<float>(c, L.pvals), part, stream);
      default: return launch_mass(c, hist, l, part, stream);
    }
  };
  std::vector<int> kinds;
  if (forms & ZETA_SUM_NODE) kinds.push_back(tc_gram(c) ? GK_TC : GK_NODE);
  if (forms & ZETA_SUM_GAMMA) kinds.push_back(GK_GAMMA);
  if (want_p) {
    kinds.push_back(GK_PART);
    kinds.push_back(GK_MASS);
  }
  int rc = ZETA_OK;
  // one warm-up call, then the faster of two timed blocks of three calls (-1 on error)
  auto time_ms = [&](int kind) -> float {
    if ((rc = run(kind)) != ZETA_OK) return -1.f;
    float best_ms = 1e30f;
    for (int rep = 0; rep < 2; ++rep) {
      cudaEventRecord(e0, stream);
      for (int r = 0; r < 3 && rc == ZETA_OK; ++r) rc = run(kind);
      cudaEventRecord(e1, stream);
      if (rc != ZETA_OK || cudaEventSynchronize(e1) != cudaSuccess) {
        rc = rc ? rc : ZETA_ECUDA;
        return -1.f;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) best_ms = ms;
    }
    return best_ms;
  };
  const int cand[] = {1, 2, 3, 4, 6, 8};
  for (int kind : kinds) {
    float best = 1e30f;
    int best_c = c->tune[kind];
    for (int cc : cand) {
      c->tune[kind] = cc;
      const float ms = time_ms(kind);
      if (ms < 0.f) break;
      if (ms < best) {
        best = ms;
        best_c = cc;
      }
    }
    c->tune[kind] = best_c;
    if (rc != ZETA_OK) break;
    if (kind == GK_PART) {  // then the halo-staging threshold at that grid size
      const int thr[] = {0, 8, 16, 32, 64, 257};
      float best_t = 1e30f;
      int best_m = c->staged_min;
      for (int m : thr) {
        c->staged_min = m;
        const float ms = time_ms(kind);
        if (ms < 0.f) break;
        if (ms < best_t) {
          best_t = ms;
          best_m = m;
        }
      }
      c->staged_min = best_m;
      if (rc != ZETA_OK) break;
    }
  }
  // tile shapes of the three field-reconstruction passes, one pass at a time (the other two
  // passes cost the same under either shape of the pass being chosen)
  float2* spec = at<float2>(c, L.spectra);
  auto time_alm = [&]() -> float {
    if ((rc = launch_alm(c, dhat, l, 0, 0, c->p.nbins, spec, fields, stream)) != ZETA_OK) return -1.f;
    float best_ms = 1e30f;
    for (int rep = 0; rep < 2; ++rep) {
      cudaEventRecord(e0, stream);
      for (int r = 0; r < 2 && rc == ZETA_OK; ++r) rc = launch_alm(c, dhat, l, 0, 0, c->p.nbins, spec, fields, stream);
      cudaEventRecord(e1, stream);
      if (rc != ZETA_OK || cudaEventSynchronize(e1) != cudaSuccess) {
        rc = rc ? rc : ZETA_ECUDA;
        return -1.f;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) best_ms = ms;
    }
    return best_ms;
  };
  for (int pass = 0; pass < 3 && rc == ZETA_OK; ++pass) {
    float best = 1e30f;
    int best_s = 0;
    for (int sh = 0; sh < 2; ++sh) {
      c->alm_shape[pass] = sh;
      const float ms = time_alm();
      if (ms < 0.f) break;
      if (ms < best) {
        best = ms;
        best_s = sh;
      }
    }
    c->alm_shape[pass] = best_s;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  drop_batch_graph(c);
  return rc;
}

int zeta_set_staging(zeta_ctx* c, int min_particles) {
  ZK_TRY(check_ctx(c));
  if (min_particles < 0) return ZETA_EINVAL;
  c->staged_min = min_particles;
  drop_batch_graph(c);
  return ZETA_OK;
}

int zeta_get_staging(const zeta_ctx* c) {
  if (!c) return ZETA_EINVAL;
  return c->staged_min;
}

int zeta_set_tuning(zeta_ctx* c, const int* ctas_per_sm, int n) {
  ZK_TRY(check_ctx(c));
  if (!ctas_per_sm || n < 0 || n > 5) return ZETA_EINVAL;
  for (int i = 0; i < n; ++i)
    if (ctas_per_sm[i] < 1 || ctas_per_sm[i] > 16) return ZETA_EINVAL;
  for (int i = 0; i < n; ++i) c->tune[i] = ctas_per_sm[i];
  drop_batch_graph(c);
  return ZETA_OK;
}

int zeta_get_tuning(const zeta_ctx* c, int* ctas_per_sm, int n) {
  if (!c || !ctas_per_sm || n < 0) return ZETA_EINVAL;
  for (int i = 0; i < n && i < 5; ++i) ctas_per_sm[i] = c->tune[i];
  return 5;
}

int zeta_set_shapes(zeta_ctx* c, const int* shape, int n) {
  ZK_TRY(check_ctx(c));
  if (!shape || n < 0 || n > 3) return ZETA_EINVAL;
  for (int i = 0; i < n; ++i)
    if (shape[i] != 0 && shape[i] != 1) return ZETA_EINVAL;
  for (int i = 0; i < n; ++i) c->alm_shape[i] = shape[i];
  drop_batch_graph(c);
  return ZETA_OK;
}

int zeta_get_shapes(const zeta_ctx* c, int* shape, int n) {
  if (!c || !shape || n < 0) return ZETA_EINVAL;
  for (int i = 0; i < n && i < 3; ++i) shape[i] = c->alm_shape[i];
  return 3;
}

}  // extern "C"

namespace {
// S_l = (W_l + W_l^T) / 2 as float, uploaded to the workspace
int upload_weights(zeta_ctx* c, const double* w, float* dst, cudaStream_t s) {
  const int nb = c->p.nbins, L1 = c->p.lmax + 1;
  std::vector<float> h(static_cast<size_t>(L1) * nb * nb);
  for (int l = 0; l < L1; ++l)
    for (int i = 0; i < nb; ++i)
      for (int j = 0; j < nb; ++j) {
        const double a = w[(static_cast<size_t>(l) * nb + i) * nb + j], b = w[(static_cast<size_t>(l) * nb + j) * nb + i];
        if (!std::isfinite(a)) return ZETA_EINVAL;
        h[(static_cast<size_t>(l) * nb + i) * nb + j] = static_cast<float>(0.5 * (a + b));
      }
  if (cudaMemcpyAsync(dst, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice, s) != cudaSuccess) return ZETA_ECUDA;
  return cudaStreamSynchronize(s) == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
}
}  // namespace

extern "C" {

int zeta_backward_node(zeta_ctx* c, const float* delta, const double* weights, float* grad, zeta_stream stream) {
  ZK_TRY(check_ctx(c));
  if (!delta || !weights || !grad) return ZETA_EINVAL;
  if (c->p.tophat_primary > 0) return ZETA_ENOTSUP;
  ZK_TRY(need_ws(c, 0, true));
  const Layout L = layout(c, 0, true);
  const int nb = c->p.nbins;
  float* S = at<float>(c, L.wts);
  ZK_TRY(upload_weights(c, weights, S, stream));
  float2* dhat = at<float2>(c, L.dhat);
  float2* gk = at<float2>(c, L.gk);
  float* q = at<float>(c, L.q);
  float* fields = at<float>(c, L.fields);
  float2* spec = at<float2>(c, L.spectra);
  ZK_TRY(launch_r2c(c, delta, dhat, stream));
  if (cudaMemsetAsync(q, 0, sizeof(float) * c->ng, stream) != cudaSuccess ||
      cudaMemsetAsync(gk, 0, sizeof(float) * c->ng, stream) != cudaSuccess)
    return ZETA_ECUDA;
  for (int l = 0; l <= c->p.lmax; ++l) {
    const float* Sl = S + static_cast<size_t>(l) * nb * nb;
    for (int m = -l; m <= l; ++m) {
      ZK_TRY(launch_alm(c, dhat, l, m, 0, nb, spec, fields, stream));
      ZK_TRY(launch_adj_node_point(c, delta, fields, Sl, q, stream));
      ZK_TRY(launch_adj_spectral(c, fields, nb, spec, l, m, gk, stream));
    }
  }
  ZK_TRY(launch_c2r_inplace(c, gk, 1, stream));
  return launch_adj_finish_node(c, q, reinterpret_cast<float*>(gk), grad, stream);
}

int zeta_backward_particles(zeta_ctx* c, const float* particles, int64_t np, const double* weights, float* grad,
                            zeta_stream stream) {
  ZK_TRY(check_ctx(c));
  if (!particles || np < 1 || np > 0x7fffffffLL || !weights || !grad) return ZETA_EINVAL;
  if (c->p.tophat_primary > 0) return ZETA_ENOTSUP;
  if (c->p.dsup == 3) return ZETA_ENOTSUP;  // the Daubechies function has no derivative to move points with
  ZK_TRY(need_ws(c, np, true));
  const Layout L = layout(c, np, true);
  const int nb = c->p.nbins;
  float* S = at<float>(c, L.wts);
  ZK_TRY(upload_weights(c, weights, S, stream));
  const float4* parts = reinterpret_cast<const float4*>(particles);
  double* small = at<double>(c, L.small);
  double* wsum = small + kAssignScratchDoubles + 4;
  float* dl = at<float>(c, L.delta);
  float2* dhat = at<float2>(c, L.dhat);
  float* fields = at<float>(c, L.fields);
  float2* spec = at<float2>(c, L.spectra);
  float4* sorted = at<float4>(c, L.sorted);
  int64_t* tstart = at<int64_t>(c, L.tstart);
  int* sidx = at<int>(c, L.sidx);
  float2* gk = at<float2>(c, L.gk);
  float* hfield = at<float>(c, L.hfield);
  float* direct = at<float>(c, L.direct);
  const size_t hbytes = sizeof(float) * c->ng * 4 * ((nb + 3) / 4);
  ZK_TRY(launch_assign(c, parts, np, dl, wsum, reinterpret_cast<unsigned long long*>(fields), small, stream));
  ZK_TRY(launch_r2c(c, dl, dhat, stream));
  ZK_TRY(launch_sort(c, parts, np, sorted, tstart, at<int>(c, L.counts), at<int>(c, L.orig), stream, sidx));
  if (cudaMemsetAsync(gk, 0, sizeof(float) * c->ng, stream) != cudaSuccess ||
      cudaMemsetAsync(direct, 0, sizeof(float) * 3 * np, stream) != cudaSuccess)
    return ZETA_ECUDA;
  for (int l = 0; l <= c->p.lmax; ++l) {
    const float* Sl = S + static_cast<size_t>(l) * nb * nb;
    ZK_TRY(launch_adj_mass(c, dhat, l, Sl, gk, stream));
    for (int m = -l; m <= l; ++m) {
      ZK_TRY(launch_alm(c, dhat, l, m, 0, nb, spec, fields, stream));
      if (cudaMemsetAsync(hfield, 0, hbytes, stream) != cudaSuccess) return ZETA_ECUDA;
      ZK_TRY(launch_adj_points(c, sorted, tstart, sidx, fields, Sl, wsum, hfield, direct, stream));
      ZK_TRY(launch_adj_spectral(c, hfield, nb, spec, l, m, gk, stream));
    }
  }
  ZK_TRY(launch_c2r_inplace(c, gk, 1, stream));
  return launch_adj_finish_particles(c, parts, np, reinterpret_cast<float*>(gk), wsum, direct, grad, stream);
}

int zeta_selftest_wait(zeta_ctx* c, int64_t spins, zeta_stream stream) {
  ZK_TRY(check_ctx(c));
  if (spins < 0) return ZETA_EINVAL;
  return launch_wait_selftest(c, spins, stream);
}

int zeta_get_status(zeta_ctx* c, zeta_stream stream) {
  ZK_TRY(check_ctx(c));
  if (cudaStreamSynchronize(stream) != cudaSuccess) return ZETA_ECUDA;
  int h = 0;
  if (cudaMemcpy(&h, c->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return ZETA_ECUDA;
  if (cudaMemset(c->d_status, 0, sizeof(int)) != cudaSuccess) return ZETA_ECUDA;
  if (h & 2) return ZETA_ETIMEOUT;
  if (h & 1) return ZETA_EDATA;
  return ZETA_OK;
}

}  // extern "C"
