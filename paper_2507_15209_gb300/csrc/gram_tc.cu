// Node-form Gram contraction on the fifth-generation tensor cores (tcgen05, sm_103a), TF32
// operands.  (The BF16 and split-BF16 contractions run in the warp-specialised kernel of
// gram_ws.cu.)
//
// G[b1][b2] = sum_x a_b1(x) * (delta(x) a_b2(x)) (the grid sum of Eq. 3PCF-multipole-sum at one
// (l, m)) is a dense contraction over the grid points: D = A B^T with A[b][x] = a_b(x) and
// B[b][x] = delta(x) a_b(x), K = the points.  A CTA streams chunks of kKT points:
//   * 256 threads load the bin-interleaved fields (float4 = four bins) and delta of one stage,
//     convert them to the MMA operand type and store them into shared memory in the canonical
//     no-swizzle K-major layout (8-row x 16-byte core matrices; LBO = 128 B along K, SBO along
//     rows) while the tensor core works on the previous stage (two buffers, mbarriers);
//   * block-diagonal packing fills all 128 rows: 128 / nb slots of nb bins, each slot a
//     different run of points; one thread issues tcgen05.mma (M = N = 128, D fp32 in TMEM,
//     128 columns) and tcgen05.commit;
//   * every kFlushStages stages (and at the end) warps 0-3 read D with tcgen05.ld and add the
//     diagonal blocks into float64 registers, so long sums do not accumulate in float32.
// Operand arithmetic: TF32 (kind::tf32).
// Waits on an mbarrier are bounded: on timeout the CTA latches ZETA_ETIMEOUT in the status
// word, stops issuing, and still frees its TMEM.
#include <cstdint>

#include "zeta_internal.h"

namespace zk {
namespace {

constexpr int kTcThreads = 256;
constexpr int kM = 128;           // MMA M
constexpr int kN = 128;           // MMA N
constexpr int kFlushStages = 8;   // stages between float64 flushes of the accumulator
constexpr uint32_t kTmemCols = 128;
constexpr long long kSpinLimit = 1LL << 26;

template <int MODE>
struct TcT;
// ES: operand bytes; KT: points per slot and stage (32 bytes of K per
// instruction -> KT * ES / 32 instructions per stage)
template <>
struct TcT<ZETA_GRAM_TF32> {
  static constexpr int ES = 4, KT = 32;
  static constexpr uint32_t FMT = 2;
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

__device__ __forceinline__ void mma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
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

// byte offset of element (row, e) in an operand tile of KT elements per row
template <int ES, int KT>
__device__ __forceinline__ uint32_t tile_off(int row, int e) {
  constexpr uint32_t SBO = KT * ES * 8;
  return (row >> 3) * SBO + ((e * ES) >> 4) * 128 + (row & 7) * 16 + ((e * ES) & 15);
}

// Pack four consecutive values (rounded to tf32) into one 16-byte core-matrix row segment.
__device__ __forceinline__ uint4 pack16(const float* x) {
  return make_uint4(to_tf32(x[0]), to_tf32(x[1]), to_tf32(x[2]), to_tf32(x[3]));
}

// Block-diagonal packing: NS = min(128 / nb, 32 / groups) slots, each a different run of KT points.  Row
// s*nb + b of A holds bin b of slot s, row s*nb + b of B holds delta * bin b of slot s, so the
// diagonal nb x nb blocks of D = A B^T are the Gram contributions of the NS runs (the other
// blocks are discarded); no operand row is padding unless 128 % nb != 0.
template <int MODE>
__global__ void __launch_bounds__(kTcThreads, 2) k_gram_node_tc(const float* __restrict__ delta, const float4* __restrict__ f4,
                                                             long long ng, int nb, double* __restrict__ partials,
                                                             int* __restrict__ status) {
  using T = TcT<MODE>;
  constexpr int KT = T::KT;
  constexpr uint32_t TILE = kM * KT * T::ES;  // one operand tile (A and B have 128 rows each)
  constexpr uint32_t SBO = KT * T::ES * 8;
  constexpr uint32_t STAGE = 2 * TILE;
  extern __shared__ __align__(1024) unsigned char smraw[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;

  const int tid = threadIdx.x, warp = tid >> 5;
  const int ngrp = (nb + 3) >> 2;
  // slots: as many runs of KT points as fit in 128 rows and in one 16-byte task per thread
  const int ns = (kM / nb) < (32 / ngrp) ? (kM / nb) : (32 / ngrp);
  const int pts = ns * KT;            // points per stage
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

  // float64 accumulators of the nb x nb result: entry e = tid + 256 i
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  // flush: D (128 x 128 fp32) -> shared memory (the idle operand buffers) -> the diagonal
  // blocks summed over the slots into the float64 accumulators
  auto flush = [&]() {
    float* dsm = reinterpret_cast<float*>(smraw);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp < 4) {
#pragma unroll
      for (int q = 0; q < kN / 32; ++q) {
        float v[32];
        tmem_load32(tmem + (static_cast<uint32_t>(32 * warp) << 16) + 32 * q, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) dsm[tid * (kN + 1) + 32 * q + i] = v[i];
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int e = tid + kTcThreads * i;
      if (e < nb * nb) {
        const int b1 = e / nb, b2 = e % nb;
        float sum = 0.f;
        for (int sl = 0; sl < ns; ++sl) sum += dsm[(sl * nb + b1) * (kN + 1) + sl * nb + b2];
        acc[i] += static_cast<double>(sum);
      }
    }
    __syncthreads();
  };

  // This CTA's stages: full chunks ch = blockIdx.x + i * gridDim.x; the last CTA also takes the
  // ragged tail (ng not a multiple of the stage size) as one more, partial stage.
  const long long nchunk = ng / pts;
  const long long tail = ng - nchunk * pts;
  const long long nfull = (nchunk > blockIdx.x) ? (nchunk - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const long long nmine = nfull + ((tail > 0 && blockIdx.x == gridDim.x - 1) ? 1 : 0);
  auto stage_at = [&](long long i, long long& p0, int& npts) {
    if (i < nfull) {
      p0 = (blockIdx.x + i * gridDim.x) * static_cast<long long>(pts);
      npts = pts;
    } else {
      p0 = nchunk * static_cast<long long>(pts);
      npts = static_cast<int>(tail);
    }
  };
  // register prefetch of one stage: this thread's task (CP consecutive points of one slot and
  // one bin group); one task per thread covers every configuration with nb <= 32
  constexpr int CP = 16 / T::ES;
  const int ntask = (pts / CP) * ngrp;
  float4 pv[CP];
  float pd[CP];
  auto fetch = [&](long long p0, int npts) {
    const int pc = tid % (pts / CP), g = tid / (pts / CP);
#pragma unroll
    for (int i = 0; i < CP; ++i) {
      const int pt = pc * CP + i;
      const bool in = tid < ntask && pt < npts;
      pv[i] = in ? __ldg(f4 + g * ng + p0 + pt) : make_float4(0.f, 0.f, 0.f, 0.f);
      pd[i] = in ? __ldg(delta + p0 + pt) : 0.f;
    }
  };
  int stage = 0;
  bool started = false, ok = true;
  if (nmine > 0) {
    long long p0;
    int np0;
    stage_at(0, p0, np0);
    fetch(p0, np0);
  }
  for (long long it = 0; it < nmine; ++it) {
    const int b = stage & 1;
    unsigned char* base = smraw + b * STAGE;
    unsigned char* Ahi = base;
    unsigned char* Bhi = base + TILE;
    if (stage >= 2 && ok) {
      if (!mbar_wait(&bar[b], ((stage - 2) >> 1) & 1)) ok = false;
    }
    if (tid < ntask) {
      const int pc = tid % (pts / CP), g = tid / (pts / CP);
      const int pt0 = pc * CP;
      const int sl = pt0 / KT, k0 = pt0 % KT;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int bin = 4 * g + j;
        if (bin >= nb) break;
        float av[CP], bv[CP];
#pragma unroll
        for (int i = 0; i < CP; ++i) {
          const float x = j == 0 ? pv[i].x : j == 1 ? pv[i].y : j == 2 ? pv[i].z : pv[i].w;
          av[i] = x;
          bv[i] = pd[i] * x;
        }
        const uint32_t off = tile_off<T::ES, KT>(sl * nb + bin, k0);
        *reinterpret_cast<uint4*>(Ahi + off) = pack16(av);
        *reinterpret_cast<uint4*>(Bhi + off) = pack16(bv);
      }
    }
    if (it + 1 < nmine) {  // next stage's loads are in flight while this one is contracted
      long long p1;
      int np1;
      stage_at(it + 1, p1, np1);
      fetch(p1, np1);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (!ok) abort_flag = 1;
    __syncthreads();
    if (abort_flag) break;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t aa = smem_u32(Ahi), ab = smem_u32(Bhi);
#pragma unroll
      for (int k = 0; k < KT * T::ES / 32; ++k) {
        const uint32_t koff = k * 2 * 128;  // two core matrices along K per instruction
        const uint64_t dA = make_desc(aa + koff, 128, SBO), dB = make_desc(ab + koff, 128, SBO);
        mma(tmem, dA, dB, idesc, (started || k > 0) ? 1u : 0u);
      }
      commit(&bar[b]);
    }
    started = true;
    if ((stage + 1) % kFlushStages == 0) {
      if (!mbar_wait(&bar[b], (stage >> 1) & 1)) ok = false;
      if (ok) flush();
      started = false;
    }
    ++stage;
  }
  if (started && ok && !abort_flag) {
    const int last = stage - 1;
    if (!mbar_wait(&bar[last & 1], (last >> 1) & 1)) ok = false;
    if (ok) flush();
  }
  if (!ok || abort_flag) atomicOr(status, 2);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int e = tid + kTcThreads * i;
    if (e < nb * nb) partials[static_cast<long long>(blockIdx.x) * nb * nb + e] = acc[i];
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
  // two stages of operands; the flush also stages the 128 x 129 float D tile in the same bytes
  const size_t ops = 2 * 2 * static_cast<size_t>(kM) * T::KT * T::ES;
  const size_t dtile = static_cast<size_t>(kM) * (kN + 1) * sizeof(float);
  const size_t sm = ops > dtile ? ops : dtile;
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
    case ZETA_GRAM_BF16: return launch_gram_ws(c, delta, alm, partials, gram_ctas(c, GK_TC), 0, false, s);
    case ZETA_GRAM_BF16X3: return launch_gram_ws(c, delta, alm, partials, gram_ctas(c, GK_TC), 0, true, s);
    default: return ZETA_ENOTSUP;
  }
}

}  // namespace zk
