// Node-form Gram contraction on the fifth-generation tensor cores (tcgen05, sm_103a).
//
// G[b1][b2] = sum_x a_b1(x) * (delta(x) a_b2(x)) (the grid sum of Eq. 3PCF-multipole-sum at one
// (l, m)) is a dense contraction over the grid points: D = A B^T with A[b][x] = a_b(x) and
// B[b][x] = delta(x) a_b(x), K = the points.  A CTA streams chunks of kKT points:
//   * 256 threads load the bin-interleaved fields (float4 = four bins) and delta for the next
//     chunk into registers while the tensor core works on the current one, convert them to
//     the MMA operand type and store them into shared memory in the canonical no-swizzle
//     K-major layout (8-row x 16-byte core matrices; LBO = 128 B along K, SBO along rows);
//   * one thread issues tcgen05.mma (M = 128 bin rows, zero-padded; N = 32; D in TMEM, fp32)
//     and tcgen05.commit to the buffer's mbarrier; two buffers alternate;
//   * every kFlushStages chunks (and at the end) warp 0 reads D with tcgen05.ld and adds it
//     to float64 registers, so long sums do not accumulate in float32.
// Operand arithmetic: TF32 (kind::tf32), BF16 (kind::f16), or split BF16 with three products
// hi*hi + hi*lo + lo*hi (the lo*lo term is below float32 resolution of the result).
// Waits on an mbarrier are bounded: on timeout the CTA latches ZETA_ETIMEOUT in the status
// word, stops issuing, and still frees its TMEM.
#include <cuda_bf16.h>

#include <cstdint>

#include "zeta_internal.h"

namespace zk {
namespace {

constexpr int kTcThreads = 256;
constexpr int kKT = 64;           // points per chunk (K of one stage)
constexpr int kM = 128;           // MMA M: bin rows of A, zero-padded
constexpr int kN = 32;            // MMA N: bin rows of B, zero-padded
constexpr int kFlushStages = 64;  // chunks between float64 flushes
constexpr uint32_t kTmemCols = 32;
constexpr long long kSpinLimit = 1LL << 26;

template <int MODE>
struct TcT;
template <>
struct TcT<ZETA_GRAM_TF32> {
  static constexpr int ES = 4, KI = 8, SPLIT = 1;
  static constexpr uint32_t FMT = 2;
};
template <>
struct TcT<ZETA_GRAM_BF16> {
  static constexpr int ES = 2, KI = 16, SPLIT = 1;
  static constexpr uint32_t FMT = 1;
};
template <>
struct TcT<ZETA_GRAM_BF16X3> {
  static constexpr int ES = 2, KI = 16, SPLIT = 2;
  static constexpr uint32_t FMT = 1;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: no swizzle, K-major
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
  d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
  d |= static_cast<uint64_t>(1) << 46;  // descriptor version of this architecture
  return d;
}

// instruction descriptor: D f32, A/B format FMT, both K-major, N = kN, M = kM
template <uint32_t FMT>
__device__ __forceinline__ uint32_t make_idesc() {
  return (1u << 4) | (FMT << 7) | (FMT << 10) | (static_cast<uint32_t>(kN >> 3) << 17) |
         (static_cast<uint32_t>(kM >> 4) << 24);
}

template <int MODE>
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  if (MODE == ZETA_GRAM_TF32) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc));
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc));
  }
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// bounded wait for the phase of the given parity; returns false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (long long it = 0; it < kSpinLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P;\n\tmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, P;\n\t}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_load32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// byte offset of element (row, e) in an operand tile of kKT elements per row
template <int ES>
__device__ __forceinline__ uint32_t tile_off(int row, int e) {
  constexpr uint32_t SBO = kKT * ES * 8;
  return (row >> 3) * SBO + ((e * ES) >> 4) * 128 + (row & 7) * 16 + ((e * ES) & 15);
}

template <int MODE>
__device__ __forceinline__ void put_elem(unsigned char* hi, unsigned char* lo, uint32_t off, float x) {
  using T = TcT<MODE>;
  if (T::ES == 4) {
    *reinterpret_cast<uint32_t*>(hi + off) = to_tf32(x);
  } else {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    *reinterpret_cast<__nv_bfloat16*>(hi + off) = h;
    if (T::SPLIT == 2) *reinterpret_cast<__nv_bfloat16*>(lo + off) = __float2bfloat16_rn(x - __bfloat162float(h));
  }
}

template <int MODE>
__global__ void __launch_bounds__(kTcThreads) k_gram_node_tc(const float* __restrict__ delta, const float4* __restrict__ f4,
                                                             long long ng, int nb, double* __restrict__ partials,
                                                             int* __restrict__ status) {
  using T = TcT<MODE>;
  constexpr uint32_t ABYTES = kM * kKT * T::ES;  // one operand tile of A
  constexpr uint32_t BBYTES = kN * kKT * T::ES;
  constexpr uint32_t SBO = kKT * T::ES * 8;
  constexpr uint32_t STAGE = T::SPLIT * (ABYTES + BBYTES);
  extern __shared__ __align__(1024) unsigned char smraw[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ngrp = (nb + 3) >> 2;
  for (uint32_t i = tid; i < 2 * STAGE / 16; i += kTcThreads) reinterpret_cast<uint4*>(smraw)[i] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = make_idesc<T::FMT>();

  double acc[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) acc[i] = 0.0;

  const long long nchunk = ng / kKT;
  const int p = tid % kKT, qt = tid / kKT;  // point in chunk, group quarter
  // register prefetch of one chunk: delta and up to two float4 groups (groups qt, qt + 4)
  float dn = 0.f;
  float4 vn0 = make_float4(0.f, 0.f, 0.f, 0.f), vn1 = vn0;
  auto fetch = [&](long long ch) {
    const long long gp = ch * kKT + p;
    dn = __ldg(delta + gp);
    vn0 = (qt < ngrp) ? __ldg(f4 + qt * ng + gp) : make_float4(0.f, 0.f, 0.f, 0.f);
    vn1 = (qt + 4 < ngrp) ? __ldg(f4 + (qt + 4) * ng + gp) : make_float4(0.f, 0.f, 0.f, 0.f);
  };
  long long ch = blockIdx.x;
  if (ch < nchunk) fetch(ch);
  int stage = 0;
  bool started = false;
  bool ok = true;
  for (; ch < nchunk; ch += gridDim.x, ++stage) {
    const int b = stage & 1;
    unsigned char* base = smraw + b * STAGE;
    unsigned char* Ahi = base;
    unsigned char* Bhi = base + ABYTES;
    unsigned char* Alo = base + ABYTES + BBYTES;
    unsigned char* Blo = Alo + ABYTES;
    if (stage >= 2 && ok) {
      if (!mbar_wait(&bar[b], ((stage - 2) >> 1) & 1)) ok = false;
    }
    const float d = dn;
    const float4 v0 = vn0, v1 = vn1;
    if (ch + gridDim.x < nchunk) fetch(ch + gridDim.x);
    const float a0[4] = {v0.x, v0.y, v0.z, v0.w};
    const float a1[4] = {v1.x, v1.y, v1.z, v1.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (qt < ngrp) {
        const int r = 4 * qt + j;
        put_elem<MODE>(Ahi, Alo, tile_off<T::ES>(r, p), a0[j]);
        put_elem<MODE>(Bhi, Blo, tile_off<T::ES>(r, p), d * a0[j]);
      }
      if (qt + 4 < ngrp) {
        const int r = 4 * (qt + 4) + j;
        put_elem<MODE>(Ahi, Alo, tile_off<T::ES>(r, p), a1[j]);
        put_elem<MODE>(Bhi, Blo, tile_off<T::ES>(r, p), d * a1[j]);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (!ok) abort_flag = 1;
    __syncthreads();
    if (abort_flag) break;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t aa = smem_u32(Ahi), ab = smem_u32(Bhi), la = smem_u32(Alo), lb = smem_u32(Blo);
#pragma unroll
      for (int k = 0; k < kKT / T::KI; ++k) {
        const uint32_t koff = k * 2 * 128;  // two core matrices along K per instruction
        const uint64_t dA = make_desc(aa + koff, 128, SBO), dB = make_desc(ab + koff, 128, SBO);
        mma<MODE>(tmem, dA, dB, idesc, (started || k > 0) ? 1u : 0u);
        if (T::SPLIT == 2) {
          mma<MODE>(tmem, dA, make_desc(lb + koff, 128, SBO), idesc, 1u);
          mma<MODE>(tmem, make_desc(la + koff, 128, SBO), dB, idesc, 1u);
        }
      }
      commit(&bar[b]);
    }
    started = true;
    if ((stage + 1) % kFlushStages == 0) {
      // drain: wait for this chunk's products, move D into float64, restart accumulation
      if (!mbar_wait(&bar[b], (stage >> 1) & 1)) ok = false;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (warp == 0 && ok) {
        float v[32];
        tmem_load32(tmem, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) acc[i] += static_cast<double>(v[i]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      started = false;
    }
  }
  if (started && ok) {
    const int last = stage - 1;
    if (!mbar_wait(&bar[last & 1], (last >> 1) & 1)) ok = false;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0 && ok) {
      float v[32];
      tmem_load32(tmem, v);
#pragma unroll
      for (int i = 0; i < 32; ++i) acc[i] += static_cast<double>(v[i]);
    }
  }
  if (!ok || abort_flag) atomicOr(status, 2);
  if (warp == 0 && lane < nb) {
    double* part = partials + static_cast<long long>(blockIdx.x) * nb * nb + lane * nb;
#pragma unroll
    for (int c = 0; c < 32; ++c)
      if (c < nb) part[c] = acc[c];
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// Diagnostic: wait on an mbarrier that nothing ever arrives on, with the same bounded wait
// the tensor-core kernel uses; the timeout must latch ZETA_ETIMEOUT and return.
__global__ void k_wait_selftest(long long spins, int* __restrict__ status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  const uint32_t a = smem_u32(&bar);
  bool done = false;
  for (long long it = 0; it < spins && !done; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P;\n\tmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, P;\n\t}\n"
        : "=r"(ok)
        : "r"(a), "r"(0u)
        : "memory");
    done = ok != 0;
  }
  if (!done) atomicOr(status, 2);
}

template <int MODE>
int tc_impl(const zeta_ctx* c, const float* delta, const float* alm, double* partials, cudaStream_t s) {
  using T = TcT<MODE>;
  const size_t sm = 2 * T::SPLIT * static_cast<size_t>(kM + kN) * kKT * T::ES;
  if (ensure_smem(reinterpret_cast<const void*>(k_gram_node_tc<MODE>), sm) != ZETA_OK) return ZETA_ECUDA;
  k_gram_node_tc<MODE><<<gram_ctas(c, GK_TC), kTcThreads, sm, s>>>(delta, reinterpret_cast<const float4*>(alm), c->ng,
                                                            c->p.nbins, partials, c->d_status);
  return cudaGetLastError() == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
}

}  // namespace

int launch_wait_selftest(const zeta_ctx* c, long long spins, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(spins, c->d_status);
  return cudaGetLastError() == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
}

int launch_gram_node_tc(const zeta_ctx* c, const float* delta, const float* alm, double* partials, cudaStream_t s) {
  StageScope prof(c, ST_GRAM_NODE, 1, s);
  switch (c->p.gram) {
    case ZETA_GRAM_TF32: return tc_impl<ZETA_GRAM_TF32>(c, delta, alm, partials, s);
    case ZETA_GRAM_BF16: return tc_impl<ZETA_GRAM_BF16>(c, delta, alm, partials, s);
    case ZETA_GRAM_BF16X3: return tc_impl<ZETA_GRAM_BF16X3>(c, delta, alm, partials, s);
    default: return ZETA_ENOTSUP;
  }
}

}  // namespace zk
