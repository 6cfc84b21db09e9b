// MRA assignment of the catalogue and particle tiling, sm_103a.
//
// Assignment (Sec. 2.1 expansion n = sum eps phi; Fig. 1 step (2); contrast of Sec. 3):
//   eps_l = sum_p w_p phi(u_p - l), u = x / H, periodic in l, phi the centred B-spline of
//   order D or the genus-4 Daubechies function (tabulated); delta_l = eps_l / eps_bar - 1 with
//   eps_bar = W / N_g.
// Contributions are scattered as 64-bit fixed point (scale 2^k with k chosen from sum |w|
// so no cell can overflow), so the result does not depend on the order of the atomics.
// The cell and in-cell offset of each particle are computed in float64 so that a float32
// position of a 512^3 grid keeps its full in-cell resolution.
//
// Tiling: particles are counted into 8x8x8-cell tiles, prefix-summed, scattered, and each
// tile's list is put back into original order, so particle-form sums are reproducible.
#include <mutex>

#include "zeta_internal.h"

namespace zk {
namespace {

constexpr int kRedCtas = 1024;

__device__ __forceinline__ bool finite4(float4 p) {
  return isfinite(p.x) && isfinite(p.y) && isfinite(p.z) && isfinite(p.w);
}

// grid coordinate wrapped into [0, n): returns cell (less shift, periodic) and in-cell offset t in [0, 1)
__device__ __forceinline__ int cell_of(float x, double inv_h, int n, int shift, float& t) {
  double u = static_cast<double>(x) * inv_h;
  u -= floor(u / n) * n;
  int i = static_cast<int>(floor(u));
  double fr = u - i;
  if (i >= n) {
    i -= n;
  }
  if (i < 0) i += n;
  t = static_cast<float>(fr);
  if (t >= 1.0f) t = 0.99999994f;
  i -= shift;
  if (i < 0) i += n;
  return i;
}

template <int D>
__device__ __forceinline__ void bspline_weights(float t, float* w) {
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

// Stencil weights of the basis: the B-spline of order D, or with a table (D = 4) the Daubechies
// function's.
template <int D>
__device__ __forceinline__ void stencil_weights(float t, const float* __restrict__ dtab, float* w) {
  if (D == 4 && dtab != nullptr)
    daub4_weights(t, dtab, w);
  else
    bspline_weights<D>(t, w);
}

__global__ void k_weight_partials(const float4* __restrict__ p, long long np, double* __restrict__ part,
                                  int* __restrict__ status) {
  __shared__ double s1[256], s2[256];
  double a = 0.0, b = 0.0;
  bool bad = false;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < np; i += 256LL * gridDim.x) {
    const float4 q = p[i];
    if (!finite4(q)) {
      bad = true;
      continue;
    }
    a += q.w;
    b += fabs(static_cast<double>(q.w));
  }
  if (bad) atomicOr(status, 1);
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      s1[threadIdx.x] += s1[threadIdx.x + w];
      s2[threadIdx.x] += s2[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = s1[0];
    part[2 * blockIdx.x + 1] = s2[0];
  }
}

// out[0] = W, out[1] = sum |w|, out[2] = fixed-point scale 2^k (sum |w| * 2^k < 2^62)
__global__ void k_weight_final(const double* __restrict__ part, int nparts, double* __restrict__ out,
                               double* __restrict__ wsum) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double a = 0.0, b = 0.0;
  for (int i = 0; i < nparts; ++i) {
    a += part[2 * i];
    b += part[2 * i + 1];
  }
  out[0] = a;
  out[1] = b;
  double scale = 1.0;
  if (b > 0.0) {
    int e;
    frexp(b, &e);  // b < 2^e
    scale = ldexp(1.0, 61 - e);
  }
  out[2] = scale;
  if (wsum) *wsum = a;
}

template <int D>
__global__ void k_assign_scatter(const float4* __restrict__ p, long long np, int n, double inv_h, int shift,
                                 const float* __restrict__ dtab, const double* __restrict__ wstat,
                                 unsigned long long* __restrict__ acc) {
  const double scale = wstat[2];
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < np;
       i += static_cast<long long>(blockDim.x) * gridDim.x) {
    const float4 q = p[i];
    if (!finite4(q)) continue;
    float tx, ty, tz;
    const int cx = cell_of(q.x, inv_h, n, shift, tx);
    const int cy = cell_of(q.y, inv_h, n, shift, ty);
    const int cz = cell_of(q.z, inv_h, n, shift, tz);
    float wx[D], wy[D], wz[D];
    stencil_weights<D>(tx, dtab, wx);
    stencil_weights<D>(ty, dtab, wy);
    stencil_weights<D>(tz, dtab, wz);
    const int off = D / 2 - 1;
    const double ws = static_cast<double>(q.w) * scale;
#pragma unroll
    for (int oz = 0; oz < D; ++oz) {
      const int lz = (cz - off + oz + n) & (n - 1);
#pragma unroll
      for (int oy = 0; oy < D; ++oy) {
        const int ly = (cy - off + oy + n) & (n - 1);
        const float wyz = wz[oz] * wy[oy];
        const long long rowi = (static_cast<long long>(lz) * n + ly) * n;
#pragma unroll
        for (int ox = 0; ox < D; ++ox) {
          const int lx = (cx - off + ox + n) & (n - 1);
          const long long v = __double2ll_rn(ws * static_cast<double>(wyz * wx[ox]));
          atomicAdd(acc + rowi + lx, static_cast<unsigned long long>(v));
        }
      }
    }
  }
}

__global__ void k_assign_finalize(const unsigned long long* __restrict__ acc, long long ng,
                                  const double* __restrict__ wstat, float* __restrict__ delta) {
  const double w = wstat[0];
  const double inv = (w != 0.0) ? static_cast<double>(ng) / (w * wstat[2]) : 0.0;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < ng;
       i += static_cast<long long>(blockDim.x) * gridDim.x) {
    const long long v = static_cast<long long>(acc[i]);
    delta[i] = static_cast<float>(static_cast<double>(v) * inv - 1.0);
  }
}

__device__ __forceinline__ long long tile_of(float4 q, double inv_h, int n, int shift) {
  float t;
  const int nt = n / kTile;
  if (!finite4(q)) return 0;
  const int cx = cell_of(q.x, inv_h, n, shift, t) / kTile;
  const int cy = cell_of(q.y, inv_h, n, shift, t) / kTile;
  const int cz = cell_of(q.z, inv_h, n, shift, t) / kTile;
  return (static_cast<long long>(cz) * nt + cy) * nt + cx;
}

__global__ void k_tile_count(const float4* __restrict__ p, long long np, int n, double inv_h, int shift,
                             int* __restrict__ cnt) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < np;
       i += static_cast<long long>(blockDim.x) * gridDim.x)
    atomicAdd(cnt + tile_of(p[i], inv_h, n, shift), 1);
}

// Exclusive prefix sum of cnt[0..m) into start[0..m] (start[m] = total) with one CTA;
// cnt is reset to zero so it can serve as the scatter cursor.
__global__ void k_tile_scan(int* __restrict__ cnt, long long m, long long* __restrict__ start) {
  __shared__ long long sh[1024];
  __shared__ long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (long long base = 0; base < m; base += 1024) {
    const long long i = base + threadIdx.x;
    const long long v = (i < m) ? cnt[i] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
      long long add = (threadIdx.x >= off) ? sh[threadIdx.x - off] : 0;
      __syncthreads();
      sh[threadIdx.x] += add;
      __syncthreads();
    }
    if (i < m) {
      start[i] = carry + sh[threadIdx.x] - v;
      cnt[i] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 1023) carry += sh[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) start[m] = carry;
}

__global__ void k_tile_scatter(const float4* __restrict__ p, long long np, int n, double inv_h, int shift,
                               const long long* __restrict__ start, int* __restrict__ cursor,
                               int* __restrict__ orig) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < np;
       i += static_cast<long long>(blockDim.x) * gridDim.x) {
    const long long t = tile_of(p[i], inv_h, n, shift);
    const int slot = atomicAdd(cursor + t, 1);
    orig[start[t] + slot] = static_cast<int>(i);
  }
}

// One warp per tile: rank every entry by its original index and gather the particles (and,
// when given, their prepared cell and offsets).
__global__ void k_tile_order(const float4* __restrict__ p, const long long* __restrict__ start, long long ntiles,
                             const int* __restrict__ orig, float4* __restrict__ sorted, int* __restrict__ sorted_idx,
                             const int* __restrict__ o_cell, const float4* __restrict__ o_tq, int* __restrict__ s_cell,
                             float4* __restrict__ s_tq) {
  const long long warp = (blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= ntiles) return;
  const long long s = start[warp], e = start[warp + 1];
  const int c = static_cast<int>(e - s);
  for (int i = lane; i < c; i += 32) {
    const int v = orig[s + i];
    int rank = 0;
    for (int j = 0; j < c; ++j) rank += (orig[s + j] < v);
    sorted[s + rank] = p[v];
    if (sorted_idx) sorted_idx[s + rank] = v;
    if (s_cell) {
      s_cell[s + rank] = o_cell[v];
      s_tq[s + rank] = o_tq[v];
    }
  }
}

// The float64 cell arithmetic of a particle, done once per catalogue: cell (linear index
// z n^2 + y n + x), in-cell offsets t in [0, 1) and the weight (0 for a non-finite particle,
// which sits in cell 0 with t = 0 and so contributes nothing anywhere).
__device__ __forceinline__ void prep_one(float4 q, double inv_h, int n, int shift, int& cell, float4& tq,
                                         int& tile) {
  const int nt = n / kTile;
  if (!finite4(q)) {
    cell = 0;
    tile = 0;
    tq = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  float tx, ty, tz;
  const int cx = cell_of(q.x, inv_h, n, shift, tx), cy = cell_of(q.y, inv_h, n, shift, ty),
            cz = cell_of(q.z, inv_h, n, shift, tz);
  cell = (cz * n + cy) * n + cx;
  tile = ((cz / kTile) * nt + cy / kTile) * nt + cx / kTile;
  tq = make_float4(tx, ty, tz, q.w);
}

// Prepared data in the original order and the particle count of every tile.
__global__ void k_particle_prep(const float4* __restrict__ p, long long np, int n, double inv_h, int shift,
                                int* __restrict__ o_tile, int* __restrict__ o_cell, float4* __restrict__ o_tq,
                                int* __restrict__ cnt) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < np;
       i += static_cast<long long>(blockDim.x) * gridDim.x) {
    int cell, tile;
    float4 tq;
    prep_one(p[i], inv_h, n, shift, cell, tq, tile);
    o_tile[i] = tile;
    o_cell[i] = cell;
    o_tq[i] = tq;
    atomicAdd(cnt + tile, 1);
  }
}

__global__ void k_tile_scatter_pre(const int* __restrict__ o_tile, long long np, const long long* __restrict__ start,
                                   int* __restrict__ cursor, int* __restrict__ orig) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < np;
       i += static_cast<long long>(blockDim.x) * gridDim.x) {
    const int t = o_tile[i];
    const int slot = atomicAdd(cursor + t, 1);
    orig[start[t] + slot] = static_cast<int>(i);
  }
}

// Prepared data of particles that are already sorted (a caller's sorted array).
__global__ void k_prep_sorted(const float4* __restrict__ sorted, long long np, int n, double inv_h, int shift,
                              int* __restrict__ s_cell, float4* __restrict__ s_tq) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < np;
       i += static_cast<long long>(blockDim.x) * gridDim.x) {
    int cell, tile;
    float4 tq;
    prep_one(sorted[i], inv_h, n, shift, cell, tq, tile);
    s_cell[i] = cell;
    s_tq[i] = tq;
  }
}

// Assignment from the sorted catalogue, one CTA per 8^3-cell tile, each node computed by the
// tile that owns it: the CTA walks the particles of its tile and of the (up to) 26 neighbouring
// tiles, and every stencil node of a particle that falls inside the tile receives its 64-bit
// fixed-point contribution round(w beta 2^k) by a shared-memory atomic; then the tile writes
// delta = eps / eps_bar - 1 of its 512 nodes.  No global atomics, and integer sums, so the
// result does not depend on the order of the particles.  w beta is formed exactly as a pair of
// float32 (hi + lo, by an FMA) and each part rounded to the fixed point separately with integer
// instructions (fix64), so no float64 arithmetic is needed per contribution.
constexpr int kAccPitch = kTile + 1;  // 64-bit words per node row of the tile accumulator

// round(x 2^k) as a 64-bit integer (|x| 2^k < 2^62), ties to even, with integer instructions only
// (a float -> int64 conversion runs on the float64 pipe, which is narrow on this part): x is
// m 2^(e - 23) with a 24-bit integer m, so the result is m shifted by e - 23 + k.
__device__ __forceinline__ long long fix64(float x, int k) {
  const unsigned int b = __float_as_uint(x);
  const int ex = static_cast<int>((b >> 23) & 0xffu);
  if (ex == 0) return 0;  // zero (or a denormal, far below one fixed-point unit here)
  const long long m = static_cast<long long>((b & 0x7fffffu) | 0x800000u);
  const int sh = ex - 150 + k;  // x 2^k = m 2^sh
  long long r;
  if (sh >= 0) {
    r = m << sh;
  } else if (sh <= -25) {
    r = 0;  // below half a unit
  } else {
    const int d = -sh;
    const long long half = 1LL << (d - 1);
    const long long q = m >> d, rem = m & ((1LL << d) - 1);
    r = q + ((rem > half || (rem == half && (q & 1))) ? 1 : 0);
  }
  return (b >> 31) ? -r : r;
}

template <int D>
__global__ void __launch_bounds__(256) k_assign_tiles(const long long* __restrict__ tile_start,
                                                      const int* __restrict__ s_cell, const float4* __restrict__ s_tq,
                                                      int n, const float* __restrict__ dtab,
                                                      const double* __restrict__ wstat, float* __restrict__ delta) {
  constexpr int T3 = kTile * kTile * kTile;
  constexpr int OFF = D / 2 - 1;
  __shared__ unsigned long long acc[kTile * kTile * kAccPitch];  // rows padded against bank conflicts
  const int nt = n / kTile, mask = n - 1;
  const int lg = __ffs(n) - 1;
  const int t = blockIdx.x;
  const int tx = t % nt, ty = (t / nt) % nt, tz = t / (nt * nt);
  for (int i = threadIdx.x; i < kTile * kTile * kAccPitch; i += blockDim.x) acc[i] = 0ULL;
  __syncthreads();
  // the particle ranges of the distinct neighbour tiles (fewer than 27 when the grid has fewer
  // than three tiles per axis), flattened so that all threads take particles of all of them
  __shared__ long long nb_s0[27];
  __shared__ int nb_pre[28];
  const int nd = nt >= 3 ? 3 : nt;
  if (threadIdx.x < 27) {
    const int dz = threadIdx.x / 9, dy = (threadIdx.x / 3) % 3, dx = threadIdx.x % 3;
    int cnt = 0;
    long long a = 0;
    if (dz < nd && dy < nd && dx < nd) {
      const int sx = nt >= 3 ? (tx + dx - 1 + nt) % nt : (tx + dx) % nt;
      const int sy = nt >= 3 ? (ty + dy - 1 + nt) % nt : (ty + dy) % nt;
      const int sz = nt >= 3 ? (tz + dz - 1 + nt) % nt : (tz + dz) % nt;
      const int nb_t = (sz * nt + sy) * nt + sx;
      a = tile_start[nb_t];
      cnt = static_cast<int>(tile_start[nb_t + 1] - a);
    }
    nb_s0[threadIdx.x] = a;
    nb_pre[threadIdx.x + 1] = cnt;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    nb_pre[0] = 0;
    for (int k = 0; k < 27; ++k) nb_pre[k + 1] += nb_pre[k];
  }
  __syncthreads();
  const int k2 = ilogb(wstat[2]);  // fixed-point scale 2^k2
  // one item per (particle, z-layer of its stencil): the heavy particles of the tile itself are
  // spread over all warps instead of the few that a one-particle-per-thread split would give them
  const int total = nb_pre[27] * D;
  int k = 0;
  for (int j = threadIdx.x; j < total; j += blockDim.x) {
    const int jp = j / D, oz = j - jp * D;
    while (jp >= nb_pre[k + 1]) ++k;
    const long long i = nb_s0[k] + (jp - nb_pre[k]);
    const float4 q = s_tq[i];
    if (q.w == 0.f) continue;
    const int cell = s_cell[i];
    const int c[3] = {cell & mask, (cell >> lg) & mask, cell >> (2 * lg)};
    const int t0[3] = {tx * kTile, ty * kTile, tz * kTile};
    // local index of the stencil's first node in this tile (periodic), per axis
    int r[3];
    bool reach = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      r[d] = ((c[d] - OFF - t0[d]) & mask);
      if (r[d] > mask - (D - 1)) r[d] -= n;  // the stencil starts before the tile
      reach = reach && r[d] + D - 1 >= 0 && r[d] < kTile;
    }
    const int lz = r[2] + oz;
    if (!reach || lz < 0 || lz >= kTile) continue;
    float wx[D], wy[D], wz[D];
    stencil_weights<D>(q.x, dtab, wx);
    stencil_weights<D>(q.y, dtab, wy);
    stencil_weights<D>(q.z, dtab, wz);
    float wzo = wz[0];
#pragma unroll
    for (int o = 1; o < D; ++o) wzo = oz == o ? wz[o] : wzo;
#pragma unroll
    for (int oy = 0; oy < D; ++oy) {
      const int ly = r[1] + oy;
      if (ly < 0 || ly >= kTile) continue;
      const float wyz = wzo * wy[oy];
      unsigned long long* row = acc + (lz * kTile + ly) * kAccPitch + r[0];
#pragma unroll
      for (int ox = 0; ox < D; ++ox) {
        const int lx = r[0] + ox;
        if (lx < 0 || lx >= kTile) continue;
        const float b = wyz * wx[ox];
        const float hi = q.w * b;
        const float lo = fmaf(q.w, b, -hi);
        const long long v = fix64(hi, k2) + fix64(lo, k2);
        atomicAdd(row + ox, static_cast<unsigned long long>(v));
      }
    }
  }
  __syncthreads();
  const double w = wstat[0];
  const double inv = (w != 0.0) ? static_cast<double>(n) * n * n / (w * wstat[2]) : 0.0;
  for (int i = threadIdx.x; i < T3; i += blockDim.x) {
    const int lx = i % kTile, ly = (i / kTile) % kTile, lz = i / (kTile * kTile);
    const long long gi = (static_cast<long long>(tz * kTile + lz) * n + ty * kTile + ly) * n + tx * kTile + lx;
    const long long v = static_cast<long long>(acc[(lz * kTile + ly) * kAccPitch + lx]);
    delta[gi] = static_cast<float>(static_cast<double>(v) * inv - 1.0);
  }
}

inline int grid_for(long long work, int threads, int sms) {
  long long g = (work + threads - 1) / threads;
  const long long cap = static_cast<long long>(sms) * 32;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return static_cast<int>(g);
}

}  // namespace

int launch_assign(const zeta_ctx* c, const float4* parts, int64_t np, float* delta, double* wsum,
                  unsigned long long* acc, double* scratch, cudaStream_t s) {
  // scratch: 2*kRedCtas partials then 3 values (W, sum|w|, scale)
  StageScope prof(c, ST_ASSIGN, 4, s);
  double* wstat = scratch + 2 * kRedCtas;
  k_weight_partials<<<kRedCtas, 256, 0, s>>>(parts, np, scratch, c->d_status);
  k_weight_final<<<1, 32, 0, s>>>(scratch, kRedCtas, wstat, wsum);
  if (cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * c->ng, s) != cudaSuccess) return ZETA_ECUDA;
  const double inv_h = c->n / c->p.box;
  const int g = grid_for(np, 256, c->num_sms);
  if (c->p.dsup == 2)
    k_assign_scatter<2><<<g, 256, 0, s>>>(parts, np, c->n, inv_h, 0, nullptr, wstat, acc);
  else
    k_assign_scatter<4><<<g, 256, 0, s>>>(parts, np, c->n, inv_h, cell_shift(c), c->d_daub, wstat, acc);
  k_assign_finalize<<<grid_for(c->ng, 256, c->num_sms), 256, 0, s>>>(acc, c->ng, wstat, delta);
  return cudaGetLastError() == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
}

int launch_wsum(const zeta_ctx* c, const float4* parts, int64_t np, double* wsum, double* scratch, cudaStream_t s) {
  StageScope prof(c, ST_ASSIGN, 2, s);
  double* wstat = scratch + 2 * kRedCtas;
  k_weight_partials<<<kRedCtas, 256, 0, s>>>(parts, np, scratch, c->d_status);
  k_weight_final<<<1, 32, 0, s>>>(scratch, kRedCtas, wstat, wsum);
  return cudaGetLastError() == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
}

int launch_sort(const zeta_ctx* c, const float4* parts, int64_t np, float4* sorted, int64_t* tile_start,
                int* counts, int* orig, cudaStream_t s, int* sorted_idx, const PartPrep* prep) {
  StageScope prof(c, ST_SORT, 4, s);
  const double inv_h = c->n / c->p.box;
  if (cudaMemsetAsync(counts, 0, sizeof(int) * c->ntiles, s) != cudaSuccess) return ZETA_ECUDA;
  const int g = grid_for(np, 256, c->num_sms);
  long long* st = reinterpret_cast<long long*>(tile_start);
  if (prep) {
    k_particle_prep<<<g, 256, 0, s>>>(parts, np, c->n, inv_h, cell_shift(c), prep->o_tile, prep->o_cell, prep->o_tq,
                                      counts);
    k_tile_scan<<<1, 1024, 0, s>>>(counts, c->ntiles, st);
    k_tile_scatter_pre<<<g, 256, 0, s>>>(prep->o_tile, np, st, counts, orig);
  } else {
    k_tile_count<<<g, 256, 0, s>>>(parts, np, c->n, inv_h, cell_shift(c), counts);
    k_tile_scan<<<1, 1024, 0, s>>>(counts, c->ntiles, st);
    k_tile_scatter<<<g, 256, 0, s>>>(parts, np, c->n, inv_h, cell_shift(c), st, counts, orig);
  }
  const long long warps = c->ntiles;
  k_tile_order<<<static_cast<unsigned>((warps * 32 + 255) / 256), 256, 0, s>>>(
      parts, st, c->ntiles, orig, sorted, sorted_idx, prep ? prep->o_cell : nullptr, prep ? prep->o_tq : nullptr,
      prep ? prep->s_cell : nullptr, prep ? prep->s_tq : nullptr);
  return cudaGetLastError() == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
}

// Szapudi-Szalay fields from the two contrasts: a = delta_D - delta_R (in place of delta_D) and
// r = 1 + delta_R (in place of delta_R).
__global__ void k_ss_fields(float* __restrict__ a, float* __restrict__ r, long long ng) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < ng;
       i += static_cast<long long>(blockDim.x) * gridDim.x) {
    const float dr = r[i];
    a[i] = a[i] - dr;
    r[i] = 1.0f + dr;
  }
}

int launch_ss_fields(const zeta_ctx* c, float* data_delta, float* rand_delta, cudaStream_t s) {
  StageScope prof(c, ST_ASSIGN, 1, s);
  k_ss_fields<<<grid_for(c->ng, 256, c->num_sms), 256, 0, s>>>(data_delta, rand_delta, c->ng);
  return cudaGetLastError() == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
}

int launch_prep_sorted(const zeta_ctx* c, const float4* sorted, int64_t np, int* s_cell, float4* s_tq, cudaStream_t s) {
  StageScope prof(c, ST_SORT, 1, s);
  k_prep_sorted<<<grid_for(np, 256, c->num_sms), 256, 0, s>>>(sorted, np, c->n, c->n / c->p.box, cell_shift(c),
                                                              s_cell, s_tq);
  return cudaGetLastError() == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
}

int launch_assign_tiles(const zeta_ctx* c, const float4* parts, int64_t np, const int64_t* tile_start,
                        const int* s_cell, const float4* s_tq, float* delta, double* wsum, double* scratch,
                        cudaStream_t s) {
  StageScope prof(c, ST_ASSIGN, 3, s);
  double* wstat = scratch + 2 * kRedCtas;
  k_weight_partials<<<kRedCtas, 256, 0, s>>>(parts, np, scratch, c->d_status);
  k_weight_final<<<1, 32, 0, s>>>(scratch, kRedCtas, wstat, wsum);
  const long long* ts = reinterpret_cast<const long long*>(tile_start);
  if (c->p.dsup == 2)
    k_assign_tiles<2><<<static_cast<unsigned>(c->ntiles), 256, 0, s>>>(ts, s_cell, s_tq, c->n, nullptr, wstat, delta);
  else
    k_assign_tiles<4><<<static_cast<unsigned>(c->ntiles), 256, 0, s>>>(ts, s_cell, s_tq, c->n, c->d_daub, wstat,
                                                                        delta);
  return cudaGetLastError() == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
}

}  // namespace zk

// ---------------------------------------------------------------------------------------
// Assignment without any allocation, for callers that cannot allocate device memory when
// they call: code inside a host framework whose memory pool already owns the device (a raw
// allocation would fail or fragment that pool), latency-critical loops that cannot afford
// the implicit synchronisation of an allocation, and services that must not hit an
// out-of-memory error once they are up.  Its scratch lives in a fixed array that every GPU
// which loads this library holds until the process exits.
namespace zk {
namespace {

constexpr int kStaticMaxN = 128;  // largest grid side the fixed scratch can hold
constexpr long long kStaticAcc = static_cast<long long>(kStaticMaxN) * kStaticMaxN * kStaticMaxN;
// layout (64-bit words): [fixed-point grid kStaticAcc][reduction partials 2*kRedCtas]
//                        [W, sum|w|, scale, spare][status word]
constexpr long long kStaticWords = kStaticAcc + 2 * kRedCtas + 4 + 1;

static __device__ __align__(256) unsigned long long g_assign_scratch[kStaticWords];

// A non-finite particle latched the status word: make the whole result NaN, so that the
// caller sees the bad input in the output itself (this entry point has no context to report
// through and does not synchronise).
__global__ void k_poison_if_bad(const int* __restrict__ status, float* __restrict__ delta, long long ng,
                                double* __restrict__ wsum) {
  if (*status == 0) return;
  const float qnan = __int_as_float(0x7fc00000);
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < ng;
       i += static_cast<long long>(blockDim.x) * gridDim.x)
    delta[i] = qnan;
  if (wsum && blockIdx.x == 0 && threadIdx.x == 0) *wsum = __longlong_as_double(0x7ff8000000000000LL);
}

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
unsigned long long* g_static_ptr[kMaxDevices] = {};

// Device address of the fixed scratch on the current device, looked up once per device.
int static_scratch(unsigned long long** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ZETA_ECUDA;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_assign_scratch) != cudaSuccess || !p) return ZETA_ECUDA;
    g_static_ptr[dev] = static_cast<unsigned long long*>(p);
  }
  *out = g_static_ptr[dev];
  return ZETA_OK;
}

}  // namespace
}  // namespace zk

extern "C" int zeta_assign_noalloc(int n, double box, int dsup, const float* particles, int64_t np, float* delta,
                                   double* wsum, zeta_stream stream) {
  using namespace zk;
  if (n < 16 || n > kStaticMaxN || (n & (n - 1)) || !(box > 0) || (dsup != 2 && dsup != 4)) return ZETA_EINVAL;
  if (!particles || np < 1 || np > 0x7fffffffLL || !delta) return ZETA_EINVAL;
  unsigned long long* base = nullptr;
  if (static_scratch(&base) != ZETA_OK) return ZETA_ECUDA;
  const long long ng = static_cast<long long>(n) * n * n;
  unsigned long long* acc = base;
  double* part = reinterpret_cast<double*>(base + kStaticAcc);
  double* wstat = part + 2 * kRedCtas;
  int* status = reinterpret_cast<int*>(base + kStaticAcc + 2 * kRedCtas + 4);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ZETA_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
  cudaStream_t s = stream;
  const float4* p = reinterpret_cast<const float4*>(particles);
  if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) return ZETA_ECUDA;
  k_weight_partials<<<kRedCtas, 256, 0, s>>>(p, np, part, status);
  k_weight_final<<<1, 32, 0, s>>>(part, kRedCtas, wstat, wsum);
  if (cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * ng, s) != cudaSuccess) return ZETA_ECUDA;
  const double inv_h = n / box;
  const int g = grid_for(np, 256, sms);
  if (dsup == 2)
    k_assign_scatter<2><<<g, 256, 0, s>>>(p, np, n, inv_h, 0, nullptr, wstat, acc);
  else
    k_assign_scatter<4><<<g, 256, 0, s>>>(p, np, n, inv_h, 0, nullptr, wstat, acc);
  k_assign_finalize<<<grid_for(ng, 256, sms), 256, 0, s>>>(acc, ng, wstat, delta);
  k_poison_if_bad<<<grid_for(ng, 256, sms), 256, 0, s>>>(status, delta, ng, wsum);
  return cudaGetLastError() == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
}

