// Weighted-Gram machinery shared by the summation kernels (Fig. 1 step (6)).
//
// Every summation form is a weighted Gram over radial bins, sum_points w * v_b1 * v_b2.  A CTA
// stages a batch of points' weights and values in shared memory; each thread owns a 4x4 block
// of the upper triangle of the bin Gram and a slice of the batch, accumulating in float32 and
// flushing to float64 every kFlush points.  Partials per CTA are reduced in a fixed order by
// k_reduce, so results are bit-reproducible.
#pragma once
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

constexpr long long kSpin = 1LL << 22;      // polls of a bounded mbarrier wait (about 4 s in all)
constexpr uint32_t kSuspendNs = 1000;         // a waiting thread sleeps in the poll up to this long

// ---- mbarriers --------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// bounded wait for the completion of the phase with the given parity; false on timeout
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, uint32_t parity) {
  const uint32_t a = smem_addr(bar);
  for (long long it = 0; it < kSpin; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P;\n\tmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2, %3;\n\t"
        "selp.b32 %0, 1, 0, P;\n\t}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity), "r"(kSuspendNs)
        : "memory");
    if (ok) return true;
  }
  return false;
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

// Reduce the per-thread accumulators of the NT threads that hold them (fixed order) and write
// their partial [NB][NB] (upper triangle valid) to part.  red: shared double buffer
// NGRP*NPAIR*16.  BAR = 0: the whole CTA takes part (tid = threadIdx.x); otherwise the NT
// threads synchronise on named barrier BAR and pass their index among themselves.
template <int NBP, int NT = kThreads, int BAR = 0>
__device__ void cta_store(GramAcc<NBP, NT>& g, double* red, int nb, double* part, int tid = -1) {
  using G = Gram<NBP, NT>;
  auto sync = [] {
    if (BAR == 0)
      __syncthreads();
    else
      asm volatile("bar.sync %0, %1;" ::"n"(BAR), "n"(NT) : "memory");
  };
  g.flush();
  if (tid < 0) tid = threadIdx.x;
  const int pr = tid % G::NPAIR, grp = tid / G::NPAIR;
  sync();
  if (grp < G::NGRP) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) red[(grp * G::NPAIR + pr) * 16 + i * 4 + j] = g.dacc[i][j];
  }
  sync();
  for (int e = tid; e < nb * nb; e += NT) {
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

// bins padded to whole groups of four: the Gram blocks cover no more than the next multiple of 4
inline int nbp_of(int nb) { return 4 * ((nb + 3) / 4); }

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

template <int NBP, int NT = kThreads>
size_t red_bytes() {
  using G = Gram<NBP, NT>;
  return static_cast<size_t>(G::NGRP) * G::NPAIR * 16 * sizeof(double);
}

template <typename K>
int prep(K kernel, size_t bytes) {
  return ensure_smem(reinterpret_cast<const void*>(kernel), bytes);
}

}  // namespace
}  // namespace zk
