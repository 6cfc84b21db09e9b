// B-spline (MRA) assignment of the catalogue and particle tiling, sm_103a.
//
// Assignment (Sec. 2.1 expansion n = sum eps phi; Fig. 1 step (2); contrast of Sec. 3):
//   eps_l = sum_p w_p beta(u_p - l), u = x / H, periodic in l, beta the centred B-spline of
//   order D; delta_l = eps_l / eps_bar - 1 with eps_bar = W / N_g.
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

// grid coordinate wrapped into [0, n): returns cell and in-cell offset t in [0, 1)
__device__ __forceinline__ int cell_of(float x, double inv_h, int n, float& t) {
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
__global__ void k_assign_scatter(const float4* __restrict__ p, long long np, int n, double inv_h,
                                 const double* __restrict__ wstat, unsigned long long* __restrict__ acc) {
  const double scale = wstat[2];
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < np;
       i += static_cast<long long>(blockDim.x) * gridDim.x) {
    const float4 q = p[i];
    if (!finite4(q)) continue;
    float tx, ty, tz;
    const int cx = cell_of(q.x, inv_h, n, tx);
    const int cy = cell_of(q.y, inv_h, n, ty);
    const int cz = cell_of(q.z, inv_h, n, tz);
    float wx[D], wy[D], wz[D];
    bspline_weights<D>(tx, wx);
    bspline_weights<D>(ty, wy);
    bspline_weights<D>(tz, wz);
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

__device__ __forceinline__ long long tile_of(float4 q, double inv_h, int n) {
  float t;
  const int nt = n / kTile;
  if (!finite4(q)) return 0;
  const int cx = cell_of(q.x, inv_h, n, t) / kTile;
  const int cy = cell_of(q.y, inv_h, n, t) / kTile;
  const int cz = cell_of(q.z, inv_h, n, t) / kTile;
  return (static_cast<long long>(cz) * nt + cy) * nt + cx;
}

__global__ void k_tile_count(const float4* __restrict__ p, long long np, int n, double inv_h, int* __restrict__ cnt) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < np;
       i += static_cast<long long>(blockDim.x) * gridDim.x)
    atomicAdd(cnt + tile_of(p[i], inv_h, n), 1);
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

__global__ void k_tile_scatter(const float4* __restrict__ p, long long np, int n, double inv_h,
                               const long long* __restrict__ start, int* __restrict__ cursor,
                               int* __restrict__ orig) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < np;
       i += static_cast<long long>(blockDim.x) * gridDim.x) {
    const long long t = tile_of(p[i], inv_h, n);
    const int slot = atomicAdd(cursor + t, 1);
    orig[start[t] + slot] = static_cast<int>(i);
  }
}

// One warp per tile: rank every entry by its original index and gather the particles.
__global__ void k_tile_order(const float4* __restrict__ p, const long long* __restrict__ start, long long ntiles,
                             const int* __restrict__ orig, float4* __restrict__ sorted, int* __restrict__ sorted_idx) {
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
    k_assign_scatter<2><<<g, 256, 0, s>>>(parts, np, c->n, inv_h, wstat, acc);
  else
    k_assign_scatter<4><<<g, 256, 0, s>>>(parts, np, c->n, inv_h, wstat, acc);
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
                int* counts, int* orig, cudaStream_t s, int* sorted_idx) {
  StageScope prof(c, ST_SORT, 4, s);
  const double inv_h = c->n / c->p.box;
  if (cudaMemsetAsync(counts, 0, sizeof(int) * c->ntiles, s) != cudaSuccess) return ZETA_ECUDA;
  const int g = grid_for(np, 256, c->num_sms);
  long long* st = reinterpret_cast<long long*>(tile_start);
  k_tile_count<<<g, 256, 0, s>>>(parts, np, c->n, inv_h, counts);
  k_tile_scan<<<1, 1024, 0, s>>>(counts, c->ntiles, st);
  k_tile_scatter<<<g, 256, 0, s>>>(parts, np, c->n, inv_h, st, counts, orig);
  const long long warps = c->ntiles;
  k_tile_order<<<static_cast<unsigned>((warps * 32 + 255) / 256), 256, 0, s>>>(parts, st, c->ntiles, orig, sorted,
                                                                             sorted_idx);
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
    k_assign_scatter<2><<<g, 256, 0, s>>>(p, np, n, inv_h, wstat, acc);
  else
    k_assign_scatter<4><<<g, 256, 0, s>>>(p, np, n, inv_h, wstat, acc);
  k_assign_finalize<<<grid_for(ng, 256, sms), 256, 0, s>>>(acc, ng, wstat, delta);
  k_poison_if_bad<<<grid_for(ng, 256, sms), 256, 0, s>>>(status, delta, ng, wsum);
  return cudaGetLastError() == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
}

