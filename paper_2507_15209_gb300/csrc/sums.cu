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
// float32 and flushing to float64 every kFlush points.  Partials per CTA are reduced in a fixed
// order by k_reduce, so results are bit-reproducible.
#include "fft.cuh"
#include "zeta_internal.h"

namespace zk {
namespace {

constexpr int kThreads = 256;
constexpr int kPB = 256;  // points per batch (one per thread in the interpolation phase)
// float32 partial sums are moved into float64 every kFlush points per thread (float64
// arithmetic is a small fraction of float32 throughput on this part, so flushes are rare)
constexpr int kFlush = 128;

template <int NBP, int NT = kThreads>
struct Gram {
  static constexpr int NBLK = NBP / 4;
  static constexpr int NPAIR = NBLK * (NBLK + 1) / 2;
  static constexpr int NGRP = NT / NPAIR;
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

// Asynchronous global -> shared copies (completion tracked per thread in commit groups).
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
template <int NPEND>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(NPEND) : "memory");
}

template <int NBP, int NT = kThreads>
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
  // vals: [npts][NBS] shared, wts: [npts] shared.  This thread takes points grp, grp + NGRP,
  // ...; the float32 partials are flushed before a call that would take them past kFlush
  // points (a call brings at most kPB / NGRP <= kFlush points), so the loop itself is
  // flush-free and U points are in flight at a time.
  template <int U = 2>
  __device__ __forceinline__ void add(const float* vals, const float* wts, int npts, int b1, int b2, int grp) {
    constexpr int NG = Gram<NBP, NT>::NGRP;
    constexpr int NBS = Gram<NBP, NT>::NBS;
    const int count = grp < npts ? (npts - grp + NG - 1) / NG : 0;
    if (pending + count > kFlush) flush();
    pending += count;
    int pt = grp;
    for (; pt + (U - 1) * NG < npts; pt += U * NG) {
      float w[U];
      float4 x[U], y[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        w[u] = wts[pt + u * NG];
        x[u] = *reinterpret_cast<const float4*>(vals + (pt + u * NG) * NBS + 4 * b1);
        y[u] = *reinterpret_cast<const float4*>(vals + (pt + u * NG) * NBS + 4 * b2);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) accum(x[u], y[u], w[u]);
    }
    for (; pt < npts; pt += NG) {
      const float4 x = *reinterpret_cast<const float4*>(vals + pt * NBS + 4 * b1);
      const float4 y = *reinterpret_cast<const float4*>(vals + pt * NBS + 4 * b2);
      accum(x, y, wts[pt]);
    }
  }
  __device__ __forceinline__ void accum(float4 x, float4 y, float w) {
    const float xs[4] = {x.x * w, x.y * w, x.z * w, x.w * w};
    const float ys[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(xs[i], ys[j], acc[i][j]);
  }
};

// Reduce the per-thread accumulators of a CTA (fixed order) and write its partial
// [NB][NB] (upper triangle valid) to part.  red: shared double buffer NGRP*NPAIR*16.
template <int NBP, int NT = kThreads>
__device__ void cta_store(GramAcc<NBP, NT>& g, double* red, int nb, double* part) {
  using G = Gram<NBP, NT>;
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
// Node form: persistent CTAs over chunks of kPB grid points of the bin-interleaved fields;
// the next chunk is loaded into registers while the current one is contracted.
template <int NBP>
__global__ void __launch_bounds__(kThreads) k_gram_node(const float* __restrict__ delta, const float4* __restrict__ f4,
                                                        long long ng, int nb, double* __restrict__ partials) {
  using G = Gram<NBP>;
  constexpr int GMAX = NBP / 4;
  extern __shared__ __align__(16) unsigned char smraw[];
  float* vals = reinterpret_cast<float*>(smraw);
  float* wts = vals + kPB * G::NBS;
  double* red = reinterpret_cast<double*>(smraw);  // reused after the main loop
  const int pr = threadIdx.x % G::NPAIR, grp = threadIdx.x / G::NPAIR;
  int b1 = 0, b2 = 0;
  pair_blocks(pr, G::NBLK, b1, b2);
  const int ngrp = (nb + 3) / 4;
  GramAcc<NBP> g;
  g.init();
  const long long nchunk = ng / kPB;
  float dnext = 0.f;
  float4 vnext[GMAX];
  long long ch = blockIdx.x;
  auto fetch = [&](long long c) {
    const long long p = c * kPB + threadIdx.x;
    dnext = __ldg(delta + p);
#pragma unroll
    for (int q = 0; q < GMAX; ++q)
      vnext[q] = (q < ngrp) ? __ldg(f4 + q * ng + p) : make_float4(0.f, 0.f, 0.f, 0.f);
  };
  if (ch < nchunk) fetch(ch);
  for (; ch < nchunk; ch += gridDim.x) {
    __syncthreads();
    wts[threadIdx.x] = dnext;
#pragma unroll
    for (int q = 0; q < GMAX; ++q) *reinterpret_cast<float4*>(vals + threadIdx.x * G::NBS + 4 * q) = vnext[q];
    __syncthreads();
    if (ch + gridDim.x < nchunk) fetch(ch + gridDim.x);
    if (grp < G::NGRP) g.add(vals, wts, kPB, b1, b2, grp);
  }
  __syncthreads();
  cta_store<NBP>(g, red, nb, partials + static_cast<long long>(blockIdx.x) * nb * nb);
}

// ---------------------------------------------------------------------------------------
// Particle and Gamma forms: persistent CTAs over 8x8x8-cell tiles, kPB points per batch.
// Phase 1 puts each point's stencil origin and B-spline weights in shared memory; phase 2
// spreads (point, bin group) tasks over the CTA, each gathering its D^3 stencil of float4
// bin groups straight from the L1-cached fields (the tile's halo stays resident in L1);
// phase 3 contracts the batch.
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

// MODE 0: particles (sorted, tile_start).  MODE 1: Gamma-form cell quadrature.
template <int NBP, int D, int MODE>
__global__ void __launch_bounds__(kThreads)
    k_gram_points(const float4* __restrict__ sorted, const long long* __restrict__ tile_start,
                  const float* __restrict__ delta, const float4* __restrict__ f4, long long ng, int n, int nb,
                  double inv_h, const float* __restrict__ gq, int q, double* __restrict__ partials) {
  using G = Gram<NBP>;
  extern __shared__ __align__(16) unsigned char smraw[];
  float* vals = reinterpret_cast<float*>(smraw);    // [kPB][NBS]
  float* wts = vals + kPB * G::NBS;                  // [kPB]
  int4* org = reinterpret_cast<int4*>(wts + kPB);    // [kPB] stencil origin (unwrapped cells)
  float* bw = reinterpret_cast<float*>(org + kPB);   // [kPB][3*D] weights x, y, z
  double* red = reinterpret_cast<double*>(smraw);    // reused after the main loop
  const int pr = threadIdx.x % G::NPAIR, grp = threadIdx.x / G::NPAIR;
  int b1 = 0, b2 = 0;
  pair_blocks(pr, G::NBLK, b1, b2);
  GramAcc<NBP> g;
  g.init();
  const int ngrp = (nb + 3) / 4;
  const int nt = n / kTile;
  const long long ntiles = static_cast<long long>(nt) * nt * nt;
  constexpr int OFF = D / 2 - 1;
  const int q3 = q * q * q;
  const int mask = n - 1;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int tx = static_cast<int>(t % nt), ty = static_cast<int>((t / nt) % nt),
              tz = static_cast<int>(t / (static_cast<long long>(nt) * nt));
    long long s0, s1;
    if (MODE == 0) {
      s0 = tile_start[t];
      s1 = tile_start[t + 1];
    } else {
      s0 = 0;
      s1 = static_cast<long long>(kTile * kTile * kTile) * q3;
    }
    for (long long bs = s0; bs < s1; bs += kPB) {
      const int cnt = static_cast<int>((s1 - bs) < kPB ? (s1 - bs) : kPB);
      __syncthreads();
      // phase 1: per point
      const int me = threadIdx.x;
      if (me < cnt) {
        float wx[D], wy[D], wz[D];
        int cx, cy, cz;
        float pw;
        if (MODE == 0) {
          const float4 pp = sorted[bs + me];
          const double u[3] = {static_cast<double>(pp.x) * inv_h, static_cast<double>(pp.y) * inv_h,
                               static_cast<double>(pp.z) * inv_h};
          int ci[3];
          float tt[3];
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const double v = u[d] - floor(u[d] / n) * n;
            int c = static_cast<int>(floor(v));
            const double fr = v - c;
            if (c >= n) c -= n;
            ci[d] = c;
            tt[d] = static_cast<float>(fr);
            if (tt[d] >= 1.f) tt[d] = 0.99999994f;
          }
          cx = ci[0];
          cy = ci[1];
          cz = ci[2];
          bsw<D>(tt[0], wx);
          bsw<D>(tt[1], wy);
          bsw<D>(tt[2], wz);
          pw = (isfinite(pp.x) && isfinite(pp.y) && isfinite(pp.z) && isfinite(pp.w)) ? pp.w : 0.f;
        } else {
          const long long id = bs + me;
          const int cell = static_cast<int>(id / q3), qq = static_cast<int>(id % q3);
          cx = tx * kTile + cell % kTile;
          cy = ty * kTile + (cell / kTile) % kTile;
          cz = tz * kTile + cell / (kTile * kTile);
          const int qx = qq % q, qy = (qq / q) % q, qz = qq / (q * q);
          const float* beta = gq + q;
#pragma unroll
          for (int o = 0; o < D; ++o) {
            wx[o] = beta[qx * D + o];
            wy[o] = beta[qy * D + o];
            wz[o] = beta[qz * D + o];
          }
          // n_rec at the node: the B-spline expansion of delta
          float nr = 0.f;
#pragma unroll
          for (int oz = 0; oz < D; ++oz)
#pragma unroll
            for (int oy = 0; oy < D; ++oy) {
              const long long row = (static_cast<long long>((cz - OFF + oz) & mask) * n + ((cy - OFF + oy) & mask)) * n;
              float a = 0.f;
#pragma unroll
              for (int ox = 0; ox < D; ++ox) a = fmaf(wx[ox], __ldg(delta + row + ((cx - OFF + ox) & mask)), a);
              nr = fmaf(wz[oz] * wy[oy], a, nr);
            }
          pw = gq[qx] * gq[qy] * gq[qz] * nr;
        }
        org[me] = make_int4(cx - OFF, cy - OFF, cz - OFF, 0);
#pragma unroll
        for (int o = 0; o < D; ++o) {
          bw[me * 3 * D + o] = wx[o];
          bw[me * 3 * D + D + o] = wy[o];
          bw[me * 3 * D + 2 * D + o] = wz[o];
        }
        wts[me] = pw;
#pragma unroll
        for (int b = 4 * ngrp; b < NBP; ++b) vals[me * G::NBS + b] = 0.f;
      }
      __syncthreads();
      // phase 2: (point, group) gathers, D lanes per task (one per x offset of the stencil) so
      // that a warp load covers 32/D tasks with D consecutive float4 (one row segment) each
      // (the loop runs in whole warps so every lane reaches the shuffles; D divides 32)
      const int total = cnt * ngrp * D;
      const int lane = threadIdx.x & 31;
      for (int tb = threadIdx.x - lane; tb < total; tb += blockDim.x) {
        const int task = tb + lane;
        const bool act = task < total;
        const int ox = task % D, pg = task / D;
        const int p = act ? pg % cnt : 0, q4 = act ? pg / cnt : 0;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        if (act) {
          const int4 o = org[p];
          const float* w = bw + p * 3 * D;
          const float4* base = f4 + q4 * ng;
          const int xo = (o.x + ox) & mask;
          const float wx = w[ox];
#pragma unroll
          for (int oz = 0; oz < D; ++oz) {
            const long long zrow = static_cast<long long>((o.z + oz) & mask) * n;
#pragma unroll
            for (int oy = 0; oy < D; ++oy) {
              const float ww = w[2 * D + oz] * w[D + oy] * wx;
              const float4 v = __ldg(base + (zrow + ((o.y + oy) & mask)) * n + xo);
              acc.x = fmaf(ww, v.x, acc.x);
              acc.y = fmaf(ww, v.y, acc.y);
              acc.z = fmaf(ww, v.z, acc.z);
              acc.w = fmaf(ww, v.w, acc.w);
            }
          }
        }
#pragma unroll
        for (int off = 1; off < D; off <<= 1) {
          acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off, D);
          acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off, D);
          acc.z += __shfl_xor_sync(0xffffffffu, acc.z, off, D);
          acc.w += __shfl_xor_sync(0xffffffffu, acc.w, off, D);
        }
        if (act && ox == 0) *reinterpret_cast<float4*>(vals + p * G::NBS + 4 * q4) = acc;
      }
      __syncthreads();
      if (grp < G::NGRP) g.add(vals, wts, cnt, b1, b2, grp);
    }
  }
  __syncthreads();
  cta_store<NBP>(g, red, nb, partials + static_cast<long long>(blockIdx.x) * nb * nb);
}

// ---------------------------------------------------------------------------------------
// Particle form with the tile's halo staged in shared memory.
//
// Tiles are visited in Morton order (neighbouring CTAs work on neighbouring tiles, so halo
// re-reads hit L2), in batches of up to kPBP particles.  A batch with at least `staged_min`
// particles interpolates from shared-memory copies of its tile's halo -- the
// (8 + D - 1)^3 nodes around the tile, one bin group (float4) at a time.  The halo copies are
// the items of a KST-slot cp.async ring that runs KST - 1 items ahead of the interpolation,
// across batch and tile boundaries, so the copy latency hides behind the work of earlier
// items.  Each particle's D^3 stencil is read by 8 lanes; rows are padded so that the 8 lanes
// of one shared-memory phase hit distinct banks.  Sparser batches are left to
// k_gram_part_l1; a particle whose cell is not inside its tile (only possible for
// inconsistent or non-finite input) reads its stencil from global memory.
constexpr int kPBP = 128;  // particles per batch
constexpr int kKST = 3;    // halo ring slots

template <int D>
struct Halo {
  static constexpr int HD = kTile + D - 1;          // nodes per side
  static constexpr int XP = D == 4 ? 12 : 10;       // row pitch (float4)
  static constexpr int PP = D == 4 ? HD * XP : 92;  // plane pitch (float4)
  static constexpr int SIZE = HD * PP;              // float4 per slot
};


// Morton index -> one tile coordinate: keeps bits 0, 3, 6, ... of v, packed (nt a power of
// two, at most 2^21)
__device__ __forceinline__ int morton_compact(unsigned long long v) {
  v &= 0x1249249249249249ULL;
  v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ULL;
  v = (v ^ (v >> 4)) & 0x100f00f00f00f00fULL;
  v = (v ^ (v >> 8)) & 0x001f0000ff0000ffULL;
  v = (v ^ (v >> 16)) & 0x001f00000000ffffULL;
  v = (v ^ (v >> 32)) & 0x00000000001fffffULL;
  return static_cast<int>(v);
}

template <int NBP, int D>
struct PartSmem {
  using G = Gram<NBP>;
  static constexpr size_t HALO = static_cast<size_t>(kKST) * Halo<D>::SIZE * sizeof(float4);
  static constexpr size_t VALS = static_cast<size_t>(kPBP) * G::NBS * sizeof(float);
  // per-particle weights: D = 4: the 16 products wz * wy in lane order, then wx[4];
  // D = 2: the 8 node weights
  static constexpr int PW = D == 4 ? 20 : 8;
  static constexpr size_t MAIN =
      HALO + VALS + kPBP * sizeof(float) + kPBP * sizeof(int4) + static_cast<size_t>(kPBP) * PW * sizeof(float);
};

// Sum a float4 over the 8 lanes of an aligned lane group (reduce-scatter): afterwards lanes
// with bit 0 clear hold component 2*bit2 + bit1 of the total in the return value.
__device__ __forceinline__ float sum8_scatter(float4 a, int l8) {
  const bool b2 = l8 & 4, b1 = l8 & 2;
  const float s0 = b2 ? a.x : a.z, s1 = b2 ? a.y : a.w;
  float k0 = b2 ? a.z : a.x, k1 = b2 ? a.w : a.y;
  k0 += __shfl_xor_sync(0xffffffffu, s0, 4);
  k1 += __shfl_xor_sync(0xffffffffu, s1, 4);
  const float s = b1 ? k0 : k1;
  float k = b1 ? k1 : k0;
  k += __shfl_xor_sync(0xffffffffu, s, 2);
  k += __shfl_xor_sync(0xffffffffu, k, 1);
  return k;
}

// Cell of a coordinate and the offset in it, wrapped into [0, n): u = x / H in float64, the
// cell floor(u) and t = u - floor(u) in [0, 1).  The periodic reduction of u is applied only
// when u is outside [0, n) -- for u inside it is the identity -- and 1/n is exact for n a
// power of two, so the result equals that of the assignment kernel's u - floor(u / n) n.
__device__ __forceinline__ int cell_frac(float x, double inv_h, int n, double inv_n, float& t) {
  double u = static_cast<double>(x) * inv_h;
  if (!(u >= 0.0 && u < n)) u -= floor(u * inv_n) * n;
  const double fl = floor(u);
  int c = static_cast<int>(fl);
  t = static_cast<float>(u - fl);
  if (c >= n) c -= n;
  if (c < 0) c += n;
  if (t >= 1.f) t = 0.99999994f;
  return c;
}

// The tiles of one CTA in order: tile k is Morton index blockIdx.x + k * gridDim.x.
struct TileWalk {
  const long long* ts;
  long long ntiles;
  int nt;
  __device__ __forceinline__ bool tile(long long k, long long& s0, long long& s1, int& tx, int& ty, int& tz) const {
    const long long i = blockIdx.x + k * gridDim.x;
    if (i >= ntiles) return false;
    const unsigned long long u = static_cast<unsigned long long>(i);
    tx = morton_compact(u);
    ty = morton_compact(u >> 1);
    tz = morton_compact(u >> 2);
    const long long t = (static_cast<long long>(tz) * nt + ty) * nt + tx;
    s0 = ts[t];
    s1 = ts[t + 1];
    return true;
  }
};

template <int NBP, int D>
__global__ void __launch_bounds__(kThreads, 2)
    k_gram_part(const float4* __restrict__ sorted, const long long* __restrict__ tile_start,
                const float4* __restrict__ f4, long long ng, int n, int nb, double inv_h, int staged_min,
                double* __restrict__ partials) {
  using G = Gram<NBP>;
  using H = Halo<D>;
  extern __shared__ __align__(16) unsigned char smraw[];
  float4* halo = reinterpret_cast<float4*>(smraw);                                   // [KST][SIZE]
  float* vals = reinterpret_cast<float*>(smraw + kKST * H::SIZE * sizeof(float4));  // [kPBP][NBS]
  float* wts = vals + kPBP * G::NBS;                                                  // [kPBP]
  int4* org = reinterpret_cast<int4*>(wts + kPBP);  // [kPBP] global stencil origin; w = halo index or -1
  constexpr int PW = PartSmem<NBP, D>::PW;
  float* bw = reinterpret_cast<float*>(org + kPBP);  // [kPBP][PW] stencil weights
  double* red = reinterpret_cast<double*>(smraw);    // reused after the main loop
  const int pr = threadIdx.x % G::NPAIR, grp = threadIdx.x / G::NPAIR;
  int b1 = 0, b2 = 0;
  pair_blocks(pr, G::NBLK, b1, b2);
  GramAcc<NBP> g;
  g.init();
  const int ngrp = (nb + 3) / 4;
  const int nt = n / kTile;
  const long long ntiles = static_cast<long long>(nt) * nt * nt;
  constexpr int OFF = D / 2 - 1;
  const int mask = n - 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int l8 = lane & 7;
  const double inv_n = 1.0 / n;

  // ---- producer: the next staged (tile, batch, group) item, identical in every thread
  const TileWalk walk{tile_start, ntiles, nt};
  long long pk = 0, ps0 = 0, ps1 = 0;
  int ptx = 0, pty = 0, ptz = 0;
  bool pvalid = walk.tile(0, ps0, ps1, ptx, pty, ptz);
  long long pbs = ps0;  // batch start
  int pq = -1;          // group of the last item issued
  auto p_advance = [&]() {
    ++pq;
    while (pvalid) {
      if (pbs < ps1) {
        const long long c = ps1 - pbs;
        if ((c < kPBP ? c : kPBP) >= staged_min && pq < ngrp) return;
        pbs += kPBP;  // batch done (or not staged)
        pq = 0;
      } else {
        pvalid = walk.tile(++pk, ps0, ps1, ptx, pty, ptz);
        pbs = ps0;
        pq = 0;
      }
    }
  };
  long long pi = 0;  // items issued
  // this thread's particle of the next batch, loaded when that batch's first item is issued
  // (at least kKST - 1 items before the batch starts when every batch has >= 2 groups)
  const bool pf = ngrp >= kKST - 1;
  float4 ppn = make_float4(0.f, 0.f, 0.f, 0.f);
  // copy lanes: thread = (plane offset hz0, row y, node x) of an HD x HD plane; planes step by
  // kPlanes (node indices fit in 32 bits: n^3 <= 2^27)
  constexpr int kPlane = H::HD * H::HD;
  constexpr int kPlanes = kThreads / kPlane;
  const int cz0 = threadIdx.x / kPlane, cy = (threadIdx.x % kPlane) / H::HD, cx = threadIdx.x % H::HD;
  const int n2 = n * n;
  auto issue_next = [&]() {  // one commit group per call (empty once the sequence ends)
    p_advance();
    if (pf && pvalid && pq == 0 && threadIdx.x < ps1 - pbs) ppn = __ldg(sorted + pbs + threadIdx.x);
    if (pvalid && cz0 < kPlanes) {
      const float4* src = f4 + pq * ng + (((pty * kTile - OFF + cy) & mask) * n + ((ptx * kTile - OFF + cx) & mask));
      float4* dst = halo + (pi % kKST) * H::SIZE + cy * H::XP + cx;
      const int hz = ptz * kTile - OFF;
#pragma unroll 2
      for (int z = cz0; z < H::HD; z += kPlanes) cp_async16(dst + z * H::PP, src + ((hz + z) & mask) * n2);
    }
    ++pi;
    cp_async_commit();
  };
#pragma unroll
  for (int j = 0; j < kKST - 1; ++j) issue_next();

  // ---- consumer
  long long ci = 0;  // staged items consumed
  long long s0, s1;
  int tx, ty, tz;
  for (long long k = 0; walk.tile(k, s0, s1, tx, ty, tz); ++k) {
    for (long long bs = s0; bs < s1; bs += kPBP) {
      const int cnt = static_cast<int>((s1 - bs) < kPBP ? (s1 - bs) : kPBP);
      if (cnt < staged_min) continue;  // k_gram_part_l1 takes this batch
      constexpr bool staged = true;
      __syncthreads();  // previous batch's readers of vals and the per-point arrays are done
      // phase 1: per particle
      const int me = threadIdx.x;
      if (me < cnt) {
        float wx[D], wy[D], wz[D];
        const float4 pp = pf ? ppn : sorted[bs + me];
        const bool fin = isfinite(pp.x) && isfinite(pp.y) && isfinite(pp.z) && isfinite(pp.w);
        const float pc[3] = {pp.x, pp.y, pp.z};
        int cix[3];
        float tt[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) cix[d] = cell_frac(fin ? pc[d] : 0.f, inv_h, n, inv_n, tt[d]);
        bsw<D>(tt[0], wx);
        bsw<D>(tt[1], wy);
        bsw<D>(tt[2], wz);
        const int lx = cix[0] - tx * kTile, ly = cix[1] - ty * kTile, lz = cix[2] - tz * kTile;
        const bool inside = lx >= 0 && lx < kTile && ly >= 0 && ly < kTile && lz >= 0 && lz < kTile;
        org[me] = make_int4(cix[0] - OFF, cix[1] - OFF, cix[2] - OFF,
                            (staged && inside) ? lz * H::PP + ly * H::XP + lx : -1);
        float* pw = bw + me * PW;
        if (D == 4) {  // lane (ox, oy0) takes nodes (oz, oy0 + 2 j): products [oy0][oz][j]
#pragma unroll
          for (int oy0 = 0; oy0 < 2; ++oy0)
#pragma unroll
            for (int oz = 0; oz < 4; ++oz)
#pragma unroll
              for (int j = 0; j < 2; ++j) pw[oy0 * 8 + oz * 2 + j] = wz[oz] * wy[oy0 + 2 * j];
#pragma unroll
          for (int o = 0; o < 4; ++o) pw[16 + o] = wx[o];
        } else {  // lane (ox, oy, oz) = bits (0, 1, 2)
#pragma unroll
          for (int e = 0; e < 8; ++e) pw[e] = wz[(e >> 2) & 1] * wy[(e >> 1) & 1] * wx[e & 1];
        }
        wts[me] = fin ? pp.w : 0.f;
#pragma unroll
        for (int b = 4 * ngrp; b < NBP; ++b) vals[me * G::NBS + b] = 0.f;
      }
      // phase 2: one bin group at a time, 8 lanes per particle
      for (int q = 0; q < ngrp; ++q) {
        if (staged) cp_async_wait<kKST - 2>();  // this item's copies (this thread's) are done
        __syncthreads();  // ... and everyone's; phase 1 visible; the previous item's readers done
        const float4* hb = halo + (ci % kKST) * H::SIZE;
        if (staged) {
          issue_next();  // into the slot read by the previous item
          ++ci;
        }
        const float4* gsrc = f4 + q * ng;
        for (int pb = warp * 4; pb < cnt; pb += (kThreads / 32) * 4) {  // warp-uniform
          const int p = pb + (lane >> 3);
          float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
          if (p < cnt) {
            const int4 o = org[p];
            const float* w = bw + p * PW;
            if (D == 4) {
              const int ox = l8 & 3, oy0 = l8 >> 2;
              const float4 ya = *reinterpret_cast<const float4*>(w + oy0 * 8);
              const float4 yb = *reinterpret_cast<const float4*>(w + oy0 * 8 + 4);
              const float wx = w[16 + ox];
              const float ww[8] = {ya.x * wx, ya.y * wx, ya.z * wx, ya.w * wx,
                                   yb.x * wx, yb.y * wx, yb.z * wx, yb.w * wx};  // [oz][j]
              if (o.w >= 0) {
                const float4* hp = hb + o.w + oy0 * H::XP + ox;
#pragma unroll
                for (int oz = 0; oz < 4; ++oz)
#pragma unroll
                  for (int j = 0; j < 2; ++j) {
                    const float4 v = hp[oz * H::PP + 2 * j * H::XP];
                    const float c = ww[oz * 2 + j];
                    acc.x = fmaf(c, v.x, acc.x);
                    acc.y = fmaf(c, v.y, acc.y);
                    acc.z = fmaf(c, v.z, acc.z);
                    acc.w = fmaf(c, v.w, acc.w);
                  }
              } else {
                const int xo = (o.x + ox) & mask;
#pragma unroll
                for (int oz = 0; oz < 4; ++oz)
#pragma unroll
                  for (int j = 0; j < 2; ++j) {
                    const int oy = oy0 + 2 * j;
                    const long long gi =
                        (static_cast<long long>((o.z + oz) & mask) * n + ((o.y + oy) & mask)) * n + xo;
                    const float4 v = __ldg(gsrc + gi);
                    const float c = ww[oz * 2 + j];
                    acc.x = fmaf(c, v.x, acc.x);
                    acc.y = fmaf(c, v.y, acc.y);
                    acc.z = fmaf(c, v.z, acc.z);
                    acc.w = fmaf(c, v.w, acc.w);
                  }
              }
            } else {  // D == 2: one node per lane
              const int ox = l8 & 1, oy = (l8 >> 1) & 1, oz = l8 >> 2;
              const float c = w[l8];
              float4 v;
              if (o.w >= 0) {
                v = hb[o.w + oz * H::PP + oy * H::XP + ox];
              } else {
                const long long gi = (static_cast<long long>((o.z + oz) & mask) * n + ((o.y + oy) & mask)) * n +
                                     ((o.x + ox) & mask);
                v = __ldg(gsrc + gi);
              }
              acc = make_float4(c * v.x, c * v.y, c * v.z, c * v.w);
            }
          }
          const float tot = sum8_scatter(acc, l8);
          if (p < cnt && !(l8 & 1)) vals[p * G::NBS + 4 * q + (l8 >> 1)] = tot;
        }
      }
      __syncthreads();
      if (grp < G::NGRP) g.add(vals, wts, cnt, b1, b2, grp);
    }
  }
  cp_async_wait<0>();  // only empty groups can remain; drain before the buffer is reused
  __syncthreads();
  cta_store<NBP>(g, red, nb, partials + static_cast<long long>(blockIdx.x) * nb * nb);
}

// ---------------------------------------------------------------------------------------
// Particle form from L1-cached global loads, for batches the staged kernel leaves out.
//
// One CTA of 512 threads works on one tile batch at a time, so the tile's halo of every
// bin group (about 100 KB for 20 bins) stays resident in L1 while all warps read it.  A
// particle's stencil is read by D * ngrp lanes at once -- lane (q, ox) accumulates the D^2
// rows of bin group q at x offset ox, 16-byte loads, D^2 of them independent -- and the D
// partial sums of a group are combined by a reduce-scatter over the x lanes, so no barrier
// separates the bin groups.
constexpr int kThreadsL1 = 512;
constexpr int kPBL = 128;  // particles per batch

template <int NBP, int D>
struct PartL1Smem {
  using G = Gram<NBP, kThreadsL1>;
  static constexpr int PW = PartSmem<NBP, D>::PW;
  static constexpr size_t MAIN = static_cast<size_t>(kPBL) * G::NBS * sizeof(float) + kPBL * sizeof(float) +
                                 kPBL * sizeof(int4) + static_cast<size_t>(kPBL) * PW * sizeof(float);
  static constexpr size_t RED = static_cast<size_t>(G::NGRP) * G::NPAIR * 16 * sizeof(double);
  static constexpr size_t BYTES = MAIN > RED ? MAIN : RED;
};

template <int NBP, int D>
__global__ void __launch_bounds__(kThreadsL1, 1)
    k_gram_part_l1(const float4* __restrict__ sorted, const long long* __restrict__ tile_start,
                   const float4* __restrict__ f4, long long ng, int n, int nb, double inv_h, int staged_min,
                   double* __restrict__ partials) {
  using G = Gram<NBP, kThreadsL1>;
  constexpr int PW = PartL1Smem<NBP, D>::PW;
  extern __shared__ __align__(16) unsigned char smraw[];
  float* vals = reinterpret_cast<float*>(smraw);  // [kPBL][NBS]
  float* wts = vals + kPBL * G::NBS;              // [kPBL]
  int4* org = reinterpret_cast<int4*>(wts + kPBL);  // [kPBL] stencil origin (cells, wrapped later)
  float* bw = reinterpret_cast<float*>(org + kPBL);  // [kPBL][PW]
  double* red = reinterpret_cast<double*>(smraw);    // reused after the main loop
  const int pr = threadIdx.x % G::NPAIR, grp = threadIdx.x / G::NPAIR;
  int b1 = 0, b2 = 0;
  pair_blocks(pr, G::NBLK, b1, b2);
  GramAcc<NBP, kThreadsL1> g;
  g.init();
  const int ngrp = (nb + 3) / 4;
  const int nt = n / kTile;
  const TileWalk walk{tile_start, static_cast<long long>(nt) * nt * nt, nt};
  constexpr int OFF = D / 2 - 1;
  const int mask = n - 1, n2 = n * n;
  const double inv_n = 1.0 / n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = kThreadsL1 / 32;
  // lane -> (particle slot, bin group, x offset)
  const int LP = D * ngrp, PPW = 32 / LP;
  const int ps = lane / LP, q = (lane % LP) / D, ox = lane % D;
  const bool lane_on = ps < PPW;
  const float4* gq4 = f4 + q * ng;
  long long s0, s1;
  int tx, ty, tz;
  for (long long k = 0; walk.tile(k, s0, s1, tx, ty, tz); ++k) {
    for (long long bs = s0; bs < s1; bs += kPBL) {
      const int cnt = static_cast<int>((s1 - bs) < kPBL ? (s1 - bs) : kPBL);
      if (cnt >= staged_min) continue;  // the staged kernel takes this batch
      __syncthreads();  // previous batch's readers are done
      const int me = threadIdx.x;
      if (me < cnt) {
        float wx[D], wy[D], wz[D];
        const float4 pp = sorted[bs + me];
        const bool fin = isfinite(pp.x) && isfinite(pp.y) && isfinite(pp.z) && isfinite(pp.w);
        const float pc[3] = {pp.x, pp.y, pp.z};
        int cix[3];
        float tt[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) cix[d] = cell_frac(fin ? pc[d] : 0.f, inv_h, n, inv_n, tt[d]);
        bsw<D>(tt[0], wx);
        bsw<D>(tt[1], wy);
        bsw<D>(tt[2], wz);
        org[me] = make_int4(cix[0] - OFF, cix[1] - OFF, cix[2] - OFF, 0);
        float* pw = bw + me * PW;
        if (D == 4) {  // [oz][oy] products wz * wy, then wx[4]
#pragma unroll
          for (int oz = 0; oz < 4; ++oz)
#pragma unroll
            for (int oy = 0; oy < 4; ++oy) pw[oz * 4 + oy] = wz[oz] * wy[oy];
#pragma unroll
          for (int o = 0; o < 4; ++o) pw[16 + o] = wx[o];
        } else {  // [oz][oy][ox] node weights
#pragma unroll
          for (int e = 0; e < 8; ++e) pw[e] = wz[(e >> 2) & 1] * wy[(e >> 1) & 1] * wx[e & 1];
        }
        wts[me] = fin ? pp.w : 0.f;
#pragma unroll
        for (int b = 4 * ngrp; b < NBP; ++b) vals[me * G::NBS + b] = 0.f;
      }
      __syncthreads();
      for (int pb = warp * PPW; pb < cnt; pb += NW * PPW) {  // warp-uniform
        const int p = pb + ps;
        const bool act = lane_on && p < cnt;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        if (act) {
          const int4 o = org[p];
          const float* w = bw + p * PW;
          const int xo = (o.x + ox) & mask;
          int yr[D], zr[D];
#pragma unroll
          for (int j = 0; j < D; ++j) {
            yr[j] = ((o.y + j) & mask) * n;
            zr[j] = ((o.z + j) & mask) * n2;
          }
          if (D == 4) {
            const float wxo = w[16 + ox];
#pragma unroll
            for (int oz = 0; oz < 4; ++oz) {
              const float4 wyz = *reinterpret_cast<const float4*>(w + oz * 4);
              const float wr[4] = {wyz.x * wxo, wyz.y * wxo, wyz.z * wxo, wyz.w * wxo};
#pragma unroll
              for (int oy = 0; oy < 4; ++oy) {
                const float4 v = __ldg(gq4 + (zr[oz] + yr[oy] + xo));
                acc.x = fmaf(wr[oy], v.x, acc.x);
                acc.y = fmaf(wr[oy], v.y, acc.y);
                acc.z = fmaf(wr[oy], v.z, acc.z);
                acc.w = fmaf(wr[oy], v.w, acc.w);
              }
            }
          } else {
#pragma unroll
            for (int oz = 0; oz < 2; ++oz)
#pragma unroll
              for (int oy = 0; oy < 2; ++oy) {
                const float c = w[oz * 4 + oy * 2 + ox];
                const float4 v = __ldg(gq4 + (zr[oz] + yr[oy] + xo));
                acc.x = fmaf(c, v.x, acc.x);
                acc.y = fmaf(c, v.y, acc.y);
                acc.z = fmaf(c, v.z, acc.z);
                acc.w = fmaf(c, v.w, acc.w);
              }
          }
        }
        // reduce-scatter over the D x lanes of (p, q): afterwards lane ox holds the total of
        // component(s) ox (D = 4) or 2 ox, 2 ox + 1 (D = 2)
        float* dst = vals + p * G::NBS + 4 * q;
        if (D == 4) {
          const bool hi = ox & 2;
          const float sa = hi ? acc.x : acc.z, sb = hi ? acc.y : acc.w;
          float ka = hi ? acc.z : acc.x, kb = hi ? acc.w : acc.y;
          ka += __shfl_xor_sync(0xffffffffu, sa, 2);
          kb += __shfl_xor_sync(0xffffffffu, sb, 2);
          const bool odd = ox & 1;
          const float s = odd ? ka : kb;
          float kk = odd ? kb : ka;
          kk += __shfl_xor_sync(0xffffffffu, s, 1);
          if (act) dst[ox] = kk;
        } else {
          const bool odd = ox & 1;
          const float sa = odd ? acc.x : acc.z, sb = odd ? acc.y : acc.w;
          float ka = odd ? acc.z : acc.x, kb = odd ? acc.w : acc.y;
          ka += __shfl_xor_sync(0xffffffffu, sa, 1);
          kb += __shfl_xor_sync(0xffffffffu, sb, 1);
          if (act) {
            dst[2 * ox] = ka;
            dst[2 * ox + 1] = kb;
          }
        }
      }
      __syncthreads();
      if (grp < G::NGRP) g.add(vals, wts, cnt, b1, b2, grp);
    }
  }
  __syncthreads();
  cta_store<NBP, kThreadsL1>(g, red, nb, partials + static_cast<long long>(blockIdx.x) * nb * nb);
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
    const int nbp = 4 * ((nb + 3) / 4);
    for (int b = 0; b < NBP; ++b) vals[threadIdx.x * G::NBS + b] = (b < nb && !nyq) ? __ldg(jt + n2 * nbp + b) : 0.f;
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
size_t red_bytes() {
  using G = Gram<NBP>;
  return G::NGRP * G::NPAIR * 16 * sizeof(double);
}
template <int NBP>
size_t smem_node() {
  using G = Gram<NBP>;
  const size_t main = (kPB * G::NBS + kPB) * sizeof(float);
  return main > red_bytes<NBP>() ? main : red_bytes<NBP>();
}
template <int NBP>
size_t smem_mass() {
  using G = Gram<NBP>;
  return (kPB * G::NBS + kPB) * sizeof(float) + red_bytes<NBP>();
}
template <int NBP, int D>
size_t smem_points() {
  using G = Gram<NBP>;
  const size_t main = (kPB * G::NBS + kPB) * sizeof(float) + kPB * sizeof(int4) + kPB * 3 * D * sizeof(float);
  return main > red_bytes<NBP>() ? main : red_bytes<NBP>();
}

template <int NBP, int D>
size_t smem_part() {
  const size_t main = PartSmem<NBP, D>::MAIN;
  return main > red_bytes<NBP>() ? main : red_bytes<NBP>();
}

template <typename K>
int prep(K kernel, size_t bytes) {
  return ensure_smem(reinterpret_cast<const void*>(kernel), bytes);
}

template <int NBP>
int node_impl(const zeta_ctx* c, const float* delta, const float* alm, double* partials, cudaStream_t s) {
  StageScope prof(c, ST_GRAM_NODE, 1, s);
  const size_t sm = smem_node<NBP>();
  if (prep(k_gram_node<NBP>, sm)) return ZETA_ECUDA;
  k_gram_node<NBP><<<gram_ctas(c, GK_NODE), kThreads, sm, s>>>(delta, reinterpret_cast<const float4*>(alm), c->ng,
                                                     c->p.nbins, partials);
  return cudaGetLastError() == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
}

template <int NBP, int D, int MODE>
int points_impl(const zeta_ctx* c, const float4* sorted, const int64_t* tile_start, const float* delta,
                const float* alm, double* partials, cudaStream_t s) {
  StageScope prof(c, MODE == 0 ? ST_GRAM_PART : ST_GRAM_GAMMA, 1, s);
  const size_t sm = smem_points<NBP, D>();
  if (prep(k_gram_points<NBP, D, MODE>, sm)) return ZETA_ECUDA;
  k_gram_points<NBP, D, MODE><<<gram_ctas(c, MODE == 0 ? GK_PART : GK_GAMMA), kThreads, sm, s>>>(
      sorted, reinterpret_cast<const long long*>(tile_start), delta, reinterpret_cast<const float4*>(alm), c->ng,
      c->n, c->p.nbins, c->n / c->p.box,
      c->d_gq, c->gamma_q, partials);
  return cudaGetLastError() == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
}

// Which particle kernels run for the staging threshold: the staged one if some batch can
// reach the threshold, the L1 one if some batch can fall below it.
inline bool part_staged_on(const zeta_ctx* c) { return c->staged_min <= kPBP; }
inline bool part_l1_on(const zeta_ctx* c) { return c->staged_min > 1; }

template <int NBP, int D>
int part_impl(const zeta_ctx* c, const float4* sorted, const int64_t* tile_start, const float* alm, double* partials,
              cudaStream_t s) {
  StageScope prof(c, ST_GRAM_PART, part_staged_on(c) + part_l1_on(c), s);
  const long long* ts = reinterpret_cast<const long long*>(tile_start);
  const float4* f4 = reinterpret_cast<const float4*>(alm);
  const double inv_h = c->n / c->p.box;
  int off = 0;
  if (part_staged_on(c)) {
    const size_t sm = smem_part<NBP, D>();
    if (prep(k_gram_part<NBP, D>, sm)) return ZETA_ECUDA;
    const int g = gram_ctas(c, GK_PART);
    k_gram_part<NBP, D><<<g, kThreads, sm, s>>>(sorted, ts, f4, c->ng, c->n, c->p.nbins, inv_h, c->staged_min,
                                                partials);
    off = g;
  }
  if (part_l1_on(c)) {
    const size_t sm = PartL1Smem<NBP, D>::BYTES;
    if (prep(k_gram_part_l1<NBP, D>, sm)) return ZETA_ECUDA;
    k_gram_part_l1<NBP, D><<<c->num_sms, kThreadsL1, sm, s>>>(
        sorted, ts, f4, c->ng, c->n, c->p.nbins, inv_h, c->staged_min,
        partials + static_cast<long long>(off) * c->p.nbins * c->p.nbins);
  }
  return cudaGetLastError() == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
}

template <int NBP>
int mass_impl(const zeta_ctx* c, const float2* dhat, int l, double* partials, cudaStream_t s) {
  StageScope prof(c, ST_MASS, 1, s);
  const size_t sm = smem_mass<NBP>();
  if (prep(k_gram_mass<NBP>, sm)) return ZETA_ECUDA;
  const float* jt = c->d_jtab + static_cast<long long>(l) * c->nn2 * (4 * ((c->p.nbins + 3) / 4));
  k_gram_mass<NBP><<<gram_ctas(c, GK_MASS), kThreads, sm, s>>>(dhat, jt, c->nn2, c->d_mhat, c->n, c->p.nbins, partials);
  return cudaGetLastError() == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
}

// bins padded to whole groups of four: the Gram blocks cover no more than the next multiple of 4
inline int nbp_of(int nb) { return 4 * ((nb + 3) / 4); }

}  // namespace

int gram_particle_parts(const zeta_ctx* c) {
  return (part_staged_on(c) ? gram_ctas(c, GK_PART) : 0) + (part_l1_on(c) ? c->num_sms : 0);
}

int gram_ctas(const zeta_ctx* c, int kind) {
  int per = c->tune[kind];
  if (per < 1) per = 1;
  int g = c->num_sms * per;
  return g > kMaxCtas ? kMaxCtas : g;
}

#define ZK_NBP_SWITCH(nb, CALL)       \
  switch (nbp_of(nb)) {               \
    case 4: return CALL(4);           \
    case 8: return CALL(8);           \
    case 12: return CALL(12);         \
    case 16: return CALL(16);         \
    case 20: return CALL(20);         \
    case 24: return CALL(24);         \
    case 28: return CALL(28);         \
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
#define ZK_CALL(P) part_impl<P, 2>(c, sorted, tile_start, alm, partials, s)
    ZK_NBP_SWITCH(c->p.nbins, ZK_CALL)
#undef ZK_CALL
  } else {
#define ZK_CALL(P) part_impl<P, 4>(c, sorted, tile_start, alm, partials, s)
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
