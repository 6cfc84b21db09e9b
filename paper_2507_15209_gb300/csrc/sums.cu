// Summation stages of the method on sm_103a (Fig. 1 step (6)) in plain float32 arithmetic.
//
// Every form is a weighted Gram over radial bins, sum_points w * v_b1 * v_b2:
//   node form      points = grid nodes,  v = a_lm(node; b), w = delta(node)
//                  (the grid sum of Eq. 3PCF-multipole-sum with the fields at nodes)
//   Gamma form     points = Gauss-Legendre nodes of every cell (Q = 2 for D = 2, 5 for D = 4),
//                  v = f_b = sum_l beta a_b(l), w = q-weight * n_rec(node); exact for the
//                  piecewise-polynomial integrand, hence equal to the connection-coefficient
//                  double sum of Eqs. (con-coeff) and (SFC-3PCF)
//   particle form  points = particles, v = f_b(x_p), w = w_p   (Eq. DDD-sum-privertex)
//   mass term      points = half-spectrum modes, v = jbar_b(|k|), w = |delta_hat|^2 Mhat(k)
// A CTA stages a batch of points' weights and values in shared memory; each thread owns a
// 4x4 block of the upper triangle of the bin Gram and a slice of the batch, accumulating in
// float32 and flushing to float64 every 16 points.  Partials per CTA are reduced in a fixed
// order by k_reduce, so results are bit-reproducible.
#include "fft.cuh"
#include "zeta_internal.h"

namespace zk {
namespace {

constexpr int kThreads = 256;
constexpr int kPB = 256;  // points per batch (one per thread in the interpolation phase)

template <int NBP>
struct Gram {
  static constexpr int NBLK = NBP / 4;
  static constexpr int NPAIR = NBLK * (NBLK + 1) / 2;
  static constexpr int NGRP = kThreads / NPAIR;
  static constexpr int NBS = NBP + 4;  // shared-memory row stride of the value table
};

__device__ __forceinline__ void pair_blocks(int p, int nblk, int& b1, int& b2) {
  int r = 0;
  while (p >= nblk - r) {
    p -= nblk - r;
    ++r;
  }
  b1 = r;
  b2 = r + p;
}

template <int NBP>
struct GramAcc {
  float acc[4][4];
  double dacc[4][4];
  int pending;
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        acc[i][j] = 0.f;
        dacc[i][j] = 0.0;
      }
    pending = 0;
  }
  __device__ __forceinline__ void flush() {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        dacc[i][j] += acc[i][j];
        acc[i][j] = 0.f;
      }
    pending = 0;
  }
  // vals: [npts][NBS] shared, wts: [npts] shared
  __device__ __forceinline__ void add(const float* vals, const float* wts, int npts, int b1, int b2, int grp) {
    for (int pt = grp; pt < npts; pt += Gram<NBP>::NGRP) {
      const float w = wts[pt];
      const float4 x = *reinterpret_cast<const float4*>(vals + pt * Gram<NBP>::NBS + 4 * b1);
      const float4 y = *reinterpret_cast<const float4*>(vals + pt * Gram<NBP>::NBS + 4 * b2);
      const float xs[4] = {x.x * w, x.y * w, x.z * w, x.w * w};
      const float ys[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(xs[i], ys[j], acc[i][j]);
      if (++pending == 16) flush();
    }
  }
};

// Reduce the per-thread accumulators of a CTA (fixed order) and write its partial
// [NB][NB] (upper triangle valid) to part.  red: shared double buffer NGRP*NPAIR*16.
template <int NBP>
__device__ void cta_store(GramAcc<NBP>& g, double* red, int nb, double* part) {
  using G = Gram<NBP>;
  g.flush();
  const int tid = threadIdx.x;
  const int pr = tid % G::NPAIR, grp = tid / G::NPAIR;
  __syncthreads();
  if (grp < G::NGRP) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) red[(grp * G::NPAIR + pr) * 16 + i * 4 + j] = g.dacc[i][j];
  }
  __syncthreads();
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int r = e / nb, cidx = e % nb;
    const int lo = r < cidx ? r : cidx, hi = r < cidx ? cidx : r;
    const int B1 = lo / 4, B2 = hi / 4;
    // pair index of (B1, B2) in the upper-triangle enumeration
    int p = 0;
    for (int q = 0; q < B1; ++q) p += G::NBLK - q;
    p += B2 - B1;
    double sum = 0.0;
    for (int k = 0; k < G::NGRP; ++k) sum += red[(k * G::NPAIR + p) * 16 + (lo % 4) * 4 + (hi % 4)];
    part[e] = sum;
  }
}

// ---------------------------------------------------------------------------------------
// Node form: persistent CTAs over chunks of kPB grid points.
template <int NBP>
__global__ void __launch_bounds__(kThreads) k_gram_node(const float* __restrict__ delta, const float* __restrict__ alm,
                                                        long long ng, int nb, double* __restrict__ partials) {
  using G = Gram<NBP>;
  extern __shared__ __align__(16) unsigned char smraw[];
  float* vals = reinterpret_cast<float*>(smraw);
  float* wts = vals + kPB * G::NBS;
  double* red = reinterpret_cast<double*>(wts + kPB);
  const int pr = threadIdx.x % G::NPAIR, grp = threadIdx.x / G::NPAIR;
  int b1 = 0, b2 = 0;
  pair_blocks(pr, G::NBLK, b1, b2);
  GramAcc<NBP> g;
  g.init();
  const long long nchunk = ng / kPB;
  for (long long ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {
    const long long p0 = ch * kPB;
    __syncthreads();
    wts[threadIdx.x] = delta[p0 + threadIdx.x];
    for (int b = 0; b < NBP; ++b) vals[threadIdx.x * G::NBS + b] = (b < nb) ? alm[b * ng + p0 + threadIdx.x] : 0.f;
    __syncthreads();
    if (grp < G::NGRP) g.add(vals, wts, kPB, b1, b2, grp);
  }
  cta_store<NBP>(g, red, nb, partials + static_cast<long long>(blockIdx.x) * nb * nb);
}

// ---------------------------------------------------------------------------------------
// Particle and Gamma forms: persistent CTAs over 8x8x8-cell tiles; per tile the fields'
// halo block (tile + stencil reach) is staged in shared memory, kBC bins at a time, laid
// out [z][y][x][bin] so each stencil point is read as float4s.
constexpr int kBC = 8;

template <int D>
__device__ __forceinline__ void bsw(float t, float* w) {
  if (D == 2) {
    w[0] = 1.f - t;
    w[1] = t;
  } else {
    const float t2 = t * t, t3 = t2 * t, s = 1.f - t;
    w[0] = s * s * s * (1.f / 6.f);
    w[1] = (3.f * t3 - 6.f * t2 + 4.f) * (1.f / 6.f);
    w[2] = (-3.f * t3 + 3.f * t2 + 3.f * t + 1.f) * (1.f / 6.f);
    w[3] = t3 * (1.f / 6.f);
  }
}

// Load fields [b0, b0+cnt) of the halo block starting at cell (x0, y0, z0) (periodic).
template <int HS>
__device__ __forceinline__ void load_halo(float* halo, const float* __restrict__ f, long long ng, int n, int x0, int y0,
                                          int z0, int b0, int cnt) {
  constexpr int H3 = HS * HS * HS;
  for (int idx = threadIdx.x; idx < H3 * kBC; idx += blockDim.x) {
    const int b = idx / H3, r = idx % H3;
    const int hx = r % HS, hy = (r / HS) % HS, hz = r / (HS * HS);
    float v = 0.f;
    if (b < cnt) {
      const int gx = (x0 + hx) & (n - 1), gy = (y0 + hy) & (n - 1), gz = (z0 + hz) & (n - 1);
      v = f[(b0 + b) * ng + (static_cast<long long>(gz) * n + gy) * n + gx];
    }
    halo[r * kBC + b] = v;
  }
}

// Interpolate kBC fields at one point from the halo (local stencil origin lx, ly, lz).
template <int D, int HS>
__device__ __forceinline__ void interp_point(const float* halo, int lx, int ly, int lz, const float* wx,
                                             const float* wy, const float* wz, float* out) {
  float a[kBC];
#pragma unroll
  for (int b = 0; b < kBC; ++b) a[b] = 0.f;
#pragma unroll
  for (int oz = 0; oz < D; ++oz) {
#pragma unroll
    for (int oy = 0; oy < D; ++oy) {
      const float wyz = wz[oz] * wy[oy];
      const float* row = halo + (((lz + oz) * HS + ly + oy) * HS + lx) * kBC;
#pragma unroll
      for (int ox = 0; ox < D; ++ox) {
        const float w = wyz * wx[ox];
        const float4 v0 = *reinterpret_cast<const float4*>(row + ox * kBC);
        const float4 v1 = *reinterpret_cast<const float4*>(row + ox * kBC + 4);
        a[0] = fmaf(w, v0.x, a[0]);
        a[1] = fmaf(w, v0.y, a[1]);
        a[2] = fmaf(w, v0.z, a[2]);
        a[3] = fmaf(w, v0.w, a[3]);
        a[4] = fmaf(w, v1.x, a[4]);
        a[5] = fmaf(w, v1.y, a[5]);
        a[6] = fmaf(w, v1.z, a[6]);
        a[7] = fmaf(w, v1.w, a[7]);
      }
    }
  }
#pragma unroll
  for (int b = 0; b < kBC; ++b) out[b] = a[b];
}

// MODE 0: particles (sorted, tile_start).  MODE 1: Gamma-form cell quadrature.
template <int NBP, int D, int MODE>
__global__ void __launch_bounds__(kThreads)
    k_gram_points(const float4* __restrict__ sorted, const long long* __restrict__ tile_start,
                  const float* __restrict__ delta, const float* __restrict__ alm, long long ng, int n, int nb,
                  double inv_h, const float* __restrict__ gq, int q, double* __restrict__ partials) {
  using G = Gram<NBP>;
  constexpr int HS = kTile + D - 1;
  constexpr int H3 = HS * HS * HS;
  extern __shared__ __align__(16) unsigned char smraw[];
  float* halo = reinterpret_cast<float*>(smraw);            // [H3][kBC]
  float* vals = halo + H3 * kBC;                             // [kPB][NBS]
  float* wts = vals + kPB * G::NBS;                          // [kPB]
  double* red = reinterpret_cast<double*>(wts + kPB);        // NGRP*NPAIR*16
  const int pr = threadIdx.x % G::NPAIR, grp = threadIdx.x / G::NPAIR;
  int b1 = 0, b2 = 0;
  pair_blocks(pr, G::NBLK, b1, b2);
  GramAcc<NBP> g;
  g.init();
  const int nt = n / kTile;
  const long long ntiles = static_cast<long long>(nt) * nt * nt;
  constexpr int OFF = D / 2 - 1;
  const int q3 = q * q * q;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int tx = static_cast<int>(t % nt), ty = static_cast<int>((t / nt) % nt), tz = static_cast<int>(t / (static_cast<long long>(nt) * nt));
    const int x0 = tx * kTile - OFF, y0 = ty * kTile - OFF, z0 = tz * kTile - OFF;
    long long s0, s1;
    if (MODE == 0) {
      s0 = tile_start[t];
      s1 = tile_start[t + 1];
    } else {
      s0 = 0;
      s1 = static_cast<long long>(kTile * kTile * kTile) * q3;
    }
    if (s1 == s0) continue;
    for (long long bs = s0; bs < s1; bs += kPB) {
      const int cnt = static_cast<int>((s1 - bs) < kPB ? (s1 - bs) : kPB);
      // this thread's point: local stencil origin and weights
      const int me = threadIdx.x;
      int lx = 0, ly = 0, lz = 0;
      float wx[D], wy[D], wz[D];
      float pw = 0.f;
      if (me < cnt) {
        if (MODE == 0) {
          const float4 pp = sorted[bs + me];
          double u[3] = {static_cast<double>(pp.x) * inv_h, static_cast<double>(pp.y) * inv_h,
                         static_cast<double>(pp.z) * inv_h};
          int ci[3];
          float tt[3];
          for (int d = 0; d < 3; ++d) {
            double v = u[d] - floor(u[d] / n) * n;
            int c = static_cast<int>(floor(v));
            double fr = v - c;
            if (c >= n) c -= n;
            ci[d] = c;
            tt[d] = static_cast<float>(fr);
            if (tt[d] >= 1.f) tt[d] = 0.99999994f;
          }
          lx = ci[0] - tx * kTile;
          ly = ci[1] - ty * kTile;
          lz = ci[2] - tz * kTile;
          bsw<D>(tt[0], wx);
          bsw<D>(tt[1], wy);
          bsw<D>(tt[2], wz);
          pw = isfinite(pp.w) ? pp.w : 0.f;
          if (lx < 0 || lx >= kTile || ly < 0 || ly >= kTile || lz < 0 || lz >= kTile) {  // not of this tile
            lx = ly = lz = 0;
            pw = 0.f;
          }
        } else {
          const long long id = bs + me;
          const int cell = static_cast<int>(id / q3), qq = static_cast<int>(id % q3);
          lx = cell % kTile;
          ly = (cell / kTile) % kTile;
          lz = cell / (kTile * kTile);
          const int qx = qq % q, qy = (qq / q) % q, qz = qq / (q * q);
          const float* beta = gq + q;
          for (int o = 0; o < D; ++o) {
            wx[o] = beta[qx * D + o];
            wy[o] = beta[qy * D + o];
            wz[o] = beta[qz * D + o];
          }
          pw = gq[qx] * gq[qy] * gq[qz];
        }
      }
      if (MODE == 1) {  // weight includes n_rec(node) = interpolated delta
        __syncthreads();
        load_halo<HS>(halo, delta, ng, n, x0, y0, z0, 0, 1);
        __syncthreads();
        if (me < cnt) {
          float tmp[kBC];
          interp_point<D, HS>(halo, lx, ly, lz, wx, wy, wz, tmp);
          pw *= tmp[0];
        }
      }
      for (int bc = 0; bc < nb; bc += kBC) {
        __syncthreads();
        load_halo<HS>(halo, alm, ng, n, x0, y0, z0, bc, (nb - bc) < kBC ? (nb - bc) : kBC);
        __syncthreads();
        if (me < cnt) {
          float tmp[kBC];
          interp_point<D, HS>(halo, lx, ly, lz, wx, wy, wz, tmp);
#pragma unroll
          for (int b = 0; b < kBC; ++b)
            if (bc + b < NBP) vals[me * G::NBS + bc + b] = tmp[b];
        }
      }
      __syncthreads();
      if (me < cnt) {
        wts[me] = pw;
        for (int b = nb; b < NBP; ++b) vals[me * G::NBS + b] = 0.f;
      }
      __syncthreads();
      if (grp < G::NGRP) g.add(vals, wts, cnt, b1, b2, grp);
    }
  }
  cta_store<NBP>(g, red, nb, partials + static_cast<long long>(blockIdx.x) * nb * nb);
}

// ---------------------------------------------------------------------------------------
// Mass (uniform) term: points = stored half-spectrum modes.
template <int NBP>
__global__ void __launch_bounds__(kThreads) k_gram_mass(const float2* __restrict__ dhat, const float* __restrict__ jt,
                                                        long long nn2, const float* __restrict__ mhat, int n, int nb,
                                                        double* __restrict__ partials) {
  using G = Gram<NBP>;
  extern __shared__ __align__(16) unsigned char smraw[];
  float* vals = reinterpret_cast<float*>(smraw);
  float* wts = vals + kPB * G::NBS;
  double* red = reinterpret_cast<double*>(wts + kPB);
  const int pr = threadIdx.x % G::NPAIR, grp = threadIdx.x / G::NPAIR;
  int b1 = 0, b2 = 0;
  pair_blocks(pr, G::NBLK, b1, b2);
  GramAcc<NBP> g;
  g.init();
  const int nc = n / 2;
  const long long total = static_cast<long long>(n) * n * nc;
  const long long nchunk = total / kPB;
  for (long long ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {
    const long long i = ch * kPB + threadIdx.x;
    const int ix = static_cast<int>(i % nc), iy = static_cast<int>((i / nc) % n), iz = static_cast<int>(i / (static_cast<long long>(nc) * n));
    const bool nyq = (iy == n / 2) || (iz == n / 2);
    const int fy = iy < n / 2 ? iy : iy - n, fz = iz < n / 2 ? iz : iz - n;
    const long long n2 = static_cast<long long>(ix) * ix + fy * fy + fz * fz;
    __syncthreads();
    float w = 0.f;
    if (!nyq) {
      const float2 d = dhat[i];
      w = (ix == 0 ? 1.f : 2.f) * (d.x * d.x + d.y * d.y) * mhat[ix] * mhat[iy] * mhat[iz];
    }
    wts[threadIdx.x] = w;
    for (int b = 0; b < NBP; ++b) vals[threadIdx.x * G::NBS + b] = (b < nb && !nyq) ? __ldg(jt + b * nn2 + n2) : 0.f;
    __syncthreads();
    if (grp < G::NGRP) g.add(vals, wts, kPB, b1, b2, grp);
  }
  cta_store<NBP>(g, red, nb, partials + static_cast<long long>(blockIdx.x) * nb * nb);
}

__global__ void k_reduce(const double* __restrict__ part, int nparts, int nb, double scale,
                         const double* __restrict__ wdiv, double* __restrict__ out) {
  const int e = threadIdx.x;
  if (e >= nb * nb) return;
  const int r = e / nb, c = e % nb;
  const int lo = r < c ? r : c, hi = r < c ? c : r;
  double sum = 0.0;
  for (int k = 0; k < nparts; ++k) sum += part[static_cast<long long>(k) * nb * nb + lo * nb + hi];
  double sc = scale;
  if (wdiv) sc /= *wdiv;
  out[e] += sc * sum;
}

template <int NBP>
size_t smem_node() {
  using G = Gram<NBP>;
  return (kPB * G::NBS + kPB) * sizeof(float) + G::NGRP * G::NPAIR * 16 * sizeof(double);
}
template <int NBP, int D>
size_t smem_points() {
  using G = Gram<NBP>;
  constexpr int HS = kTile + D - 1;
  return (HS * HS * HS * kBC + kPB * G::NBS + kPB) * sizeof(float) + G::NGRP * G::NPAIR * 16 * sizeof(double);
}

template <typename K>
int prep(K kernel, size_t bytes) {
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes)) != cudaSuccess)
    return ZETA_ECUDA;
  return ZETA_OK;
}

template <int NBP>
int node_impl(const zeta_ctx* c, const float* delta, const float* alm, double* partials, cudaStream_t s) {
  StageScope prof(c, ST_GRAM_NODE, 1, s);
  const size_t sm = smem_node<NBP>();
  if (prep(k_gram_node<NBP>, sm)) return ZETA_ECUDA;
  k_gram_node<NBP><<<gram_ctas(c), kThreads, sm, s>>>(delta, alm, c->ng, c->p.nbins, partials);
  return cudaGetLastError() == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
}

template <int NBP, int D, int MODE>
int points_impl(const zeta_ctx* c, const float4* sorted, const int64_t* tile_start, const float* delta,
                const float* alm, double* partials, cudaStream_t s) {
  StageScope prof(c, MODE == 0 ? ST_GRAM_PART : ST_GRAM_GAMMA, 1, s);
  const size_t sm = smem_points<NBP, D>();
  if (prep(k_gram_points<NBP, D, MODE>, sm)) return ZETA_ECUDA;
  k_gram_points<NBP, D, MODE><<<gram_ctas(c), kThreads, sm, s>>>(
      sorted, reinterpret_cast<const long long*>(tile_start), delta, alm, c->ng, c->n, c->p.nbins, c->n / c->p.box,
      c->d_gq, c->gamma_q, partials);
  return cudaGetLastError() == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
}

template <int NBP>
int mass_impl(const zeta_ctx* c, const float2* dhat, int l, double* partials, cudaStream_t s) {
  StageScope prof(c, ST_MASS, 1, s);
  const size_t sm = smem_node<NBP>();
  if (prep(k_gram_mass<NBP>, sm)) return ZETA_ECUDA;
  const float* jt = c->d_jtab + static_cast<long long>(l) * c->p.nbins * c->nn2;
  k_gram_mass<NBP><<<gram_ctas(c), kThreads, sm, s>>>(dhat, jt, c->nn2, c->d_mhat, c->n, c->p.nbins, partials);
  return cudaGetLastError() == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
}

inline int nbp_of(int nb) { return nb <= 8 ? 8 : nb <= 16 ? 16 : nb <= 24 ? 24 : 32; }

}  // namespace

int gram_ctas(const zeta_ctx* c) {
  int g = c->num_sms * 2;
  return g > kMaxCtas ? kMaxCtas : g;
}

#define ZK_NBP_SWITCH(nb, CALL)       \
  switch (nbp_of(nb)) {               \
    case 8: return CALL(8);           \
    case 16: return CALL(16);         \
    case 24: return CALL(24);         \
    default: return CALL(32);         \
  }

int launch_gram_node(const zeta_ctx* c, const float* delta, const float* alm, double* partials, cudaStream_t s) {
#define ZK_CALL(P) node_impl<P>(c, delta, alm, partials, s)
  ZK_NBP_SWITCH(c->p.nbins, ZK_CALL)
#undef ZK_CALL
}

int launch_gram_gamma(const zeta_ctx* c, const float* delta, const float* alm, double* partials, cudaStream_t s) {
  if (c->p.dsup == 2) {
#define ZK_CALL(P) points_impl<P, 2, 1>(c, nullptr, nullptr, delta, alm, partials, s)
    ZK_NBP_SWITCH(c->p.nbins, ZK_CALL)
#undef ZK_CALL
  } else {
#define ZK_CALL(P) points_impl<P, 4, 1>(c, nullptr, nullptr, delta, alm, partials, s)
    ZK_NBP_SWITCH(c->p.nbins, ZK_CALL)
#undef ZK_CALL
  }
}

int launch_gram_particles(const zeta_ctx* c, const float4* sorted, const int64_t* tile_start, const float* alm,
                          double* partials, cudaStream_t s) {
  if (c->p.dsup == 2) {
#define ZK_CALL(P) points_impl<P, 2, 0>(c, sorted, tile_start, nullptr, alm, partials, s)
    ZK_NBP_SWITCH(c->p.nbins, ZK_CALL)
#undef ZK_CALL
  } else {
#define ZK_CALL(P) points_impl<P, 4, 0>(c, sorted, tile_start, nullptr, alm, partials, s)
    ZK_NBP_SWITCH(c->p.nbins, ZK_CALL)
#undef ZK_CALL
  }
}

int launch_mass(const zeta_ctx* c, const float2* dhat, int l, double* partials, cudaStream_t s) {
#define ZK_CALL(P) mass_impl<P>(c, dhat, l, partials, s)
  ZK_NBP_SWITCH(c->p.nbins, ZK_CALL)
#undef ZK_CALL
}

int launch_reduce(const zeta_ctx* c, const double* partials, int nparts, double scale, const double* wdiv,
                  double* out, cudaStream_t s) {
  StageScope prof(c, ST_REDUCE, 1, s);
  const int nb = c->p.nbins;
  k_reduce<<<1, 1024, 0, s>>>(partials, nparts, nb, scale, wdiv, out);
  return cudaGetLastError() == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
}

}  // namespace zk
