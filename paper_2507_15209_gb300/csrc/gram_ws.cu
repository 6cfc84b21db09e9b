// Warp-specialised node-form Gram on the fifth-generation tensor cores (tcgen05, kind::f16).
//
// G[b1][b2] = sum_x a_b1(x) delta(x) a_b2(x) (the grid sum of Eq. 3PCF-multipole-sum at one
// (l, m)) is a dense contraction over the grid points x: D = A B^T with A[b][x] = a_b(x) and
// B[b][x] = delta(x) a_b(x).  A stage is 256 consecutive points split into four slots of 64;
// slot s fills operand rows 32 s .. 32 s + nbp - 1 (nbp = nb rounded up to 4; the fields of the
// padding bins are zero, and rows up to 32 s + 31 stay zero), so the
// diagonal 32 x 32 blocks of one M = N = 128 product are the Gram contributions of the four
// slots.  Roles of the 512 threads:
//   warp 0, one lane   bulk-copies the stage's raw data (delta and the bin groups of the
//                      fields, float32 or bfloat16) into a ring of shared-memory slots,
//                      counted on the slot's mbarrier in bytes;
//   warps 2-11         convert a raw slot into the K-major bfloat16 operand tiles (8-row x
//                      16-byte core matrices) of an operand slot: A = a (hi and, split, lo
//                      parts), B = delta a (hi and, split, lo);
//   warp 1, one lane   issues tcgen05.mma for every operand slot into one of two TMEM
//                      accumulators (128 columns each) and commits to the slot's `empty`
//                      barrier; after kWsPeriod stages it commits the accumulator to the
//                      epilogue and switches to the other one;
//   warps 12-15        (one per TMEM lane quadrant = slot) read their slot's diagonal block
//                      with tcgen05.ld and add it to float64 registers, so float32 sums run
//                      over at most kWsPeriod x 64 products.
// Operand arithmetic: BF16 (A hi, B hi), split BF16 (hi*hi + hi*lo + lo*hi), and bfloat16
// fields (A exact, B = delta a split into hi + lo: two products, so delta a keeps 16 bits and
// the fields' own rounding is the only one left).  Every wait is bounded; a timeout latches ZETA_ETIMEOUT,
// stops the CTA's roles and still frees its TMEM after the MMAs it issued have completed.
#include <cuda_bf16.h>

#include <cstdint>
#include <type_traits>

#include "gram.cuh"

namespace zk {
namespace {

constexpr int kWsThreads = 512;
constexpr int kWsPts = 256;          // points per stage (4 slots of 64)
constexpr int kWsKT = 64;            // points per slot and stage (K of the stage)
constexpr int kWsPeriod = 8;         // stages per float32 accumulation period
constexpr int kWsConvFirst = 2;      // first converter warp
constexpr int kWsConv = 10;          // converter warps
constexpr int kWsEpiFirst = 12;      // first epilogue warp (quadrant = warp % 4)
constexpr uint32_t kWsTile = 128 * kWsKT * 2;  // one bf16 operand tile, 128 rows: 16 KB
constexpr uint32_t kWsSbo = kWsKT * 2 * 8;     // 8-row group stride of a tile
constexpr uint32_t kWsTmemCols = 256;          // two 128-column accumulators
constexpr long long kWsSpin = 1LL << 22;   // waits of at most kWsSuspendNs each: about 4 s in all
constexpr uint32_t kWsSuspendNs = 1000;     // a waiting thread sleeps until the phase completes or this

__device__ __forceinline__ uint32_t ws_smem(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void ws_bar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(ws_smem(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void ws_arrive(uint64_t* bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}\n" ::"r"(ws_smem(bar))
               : "memory");
}

__device__ __forceinline__ void ws_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}\n" ::"r"(
                   ws_smem(bar)),
               "r"(bytes)
               : "memory");
}

// bounded wait for the phase of the given parity; false on timeout.  The thread sleeps in the
// try_wait (up to kWsSuspendNs) instead of polling shared memory.
__device__ __forceinline__ bool ws_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = ws_smem(bar);
  for (long long it = 0; it < kWsSpin; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P;\n\tmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2, %3;\n\t"
        "selp.b32 %0, 1, 0, P;\n\t}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity), "r"(kWsSuspendNs)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// global -> shared bulk copy completing on an mbarrier (16-byte aligned, size a multiple of 16)
__device__ __forceinline__ void ws_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(ws_smem(dst)),
      "l"(src), "r"(bytes), "r"(ws_smem(bar))
      : "memory");
}

// shared-memory matrix descriptor: no swizzle, K-major (LBO along K, SBO between 8-row groups)
__device__ __forceinline__ uint64_t ws_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
  d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  return d;
}

// instruction descriptor: D f32, A and B bf16, both K-major, N = 128, M = 128
__device__ __forceinline__ uint32_t ws_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(128 >> 3) << 17) |
         (static_cast<uint32_t>(128 >> 4) << 24);
}

__device__ __forceinline__ void ws_mma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void ws_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(ws_smem(bar))
               : "memory");
}

__device__ __forceinline__ void ws_tmem_load32(uint32_t taddr, float* v) {
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

// byte offset of element (row, k) in a K-major bf16 tile of kWsKT elements per row
__device__ __forceinline__ uint32_t ws_off(int row, int k) {
  return (row >> 3) * kWsSbo + ((k * 2) >> 4) * 128 + (row & 7) * 16 + ((k * 2) & 15);
}

__device__ __forceinline__ uint32_t ws_pack(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ __forceinline__ float ws_bf(uint32_t bits16) { return __uint_as_float(bits16 << 16); }

// Shared-memory plan: RR raw slots, OR operand slots, the barriers.  RAW 0: float32 fields (16 bytes
// per point and bin group), 1: bfloat16 fields (8 bytes).
template <int NBP, int RAW, int NA, int NB>
struct WsPlan {
  static constexpr int G = NBP / 4;
  static constexpr uint32_t GB = RAW == 0 ? 16 : 8;  // bytes per point and group
  // a group's run of points, skewed by 32 bytes so that the groups start in different banks
  static constexpr uint32_t GST = kWsPts * GB + 32;
  static constexpr uint32_t RAWSLOT = kWsPts * 4 + G * GST;  // delta, then the groups
  static constexpr uint32_t OPSLOT = (NA + NB) * kWsTile;
  // operand slots: 4 of 32 KB, 3 of 48 KB, 2 of 64 KB (the converters run that many stages ahead)
  static constexpr int ORF = static_cast<int>((144u * 1024u) / OPSLOT);
  static constexpr int OR = ORF < 2 ? 2 : ORF;
  // as many raw slots as fit (the bulk copies of several stages in flight cover the DRAM latency)
  static constexpr int RRF = static_cast<int>((200u * 1024u - OR * OPSLOT) / RAWSLOT);
  static constexpr int RR = RRF > 12 ? 12 : (RRF < 2 ? 2 : RRF);
  static constexpr uint32_t RAW_OFF = OR * OPSLOT;  // operand ring first (1024-aligned tiles)
  static constexpr uint32_t BAR_OFF = RAW_OFF + RR * RAWSLOT;
  static constexpr uint32_t BYTES = BAR_OFF + 2 * (RR + OR + 2) * 8 + 16;
  static_assert(4 * 32 * NBP * 8 <= OR * OPSLOT, "the final reduction reuses the operand ring");
  static_assert(BYTES <= 227 * 1024, "shared memory");
};

template <int NBP, int RAW, int NA, int NB>
__global__ void __launch_bounds__(kWsThreads, 1)
    k_gram_ws(const float* __restrict__ delta, const unsigned char* __restrict__ fields, long long ng, int nb,
              double* __restrict__ partials, int* __restrict__ status) {
  using P = WsPlan<NBP, RAW, NA, NB>;
  extern __shared__ __align__(1024) unsigned char smws[];
  uint64_t* raw_full = reinterpret_cast<uint64_t*>(smws + P::BAR_OFF);
  uint64_t* raw_empty = raw_full + P::RR;
  uint64_t* op_full = raw_empty + P::RR;
  uint64_t* op_empty = op_full + P::OR;
  uint64_t* acc_full = op_empty + P::OR;
  uint64_t* acc_empty = acc_full + 2;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // the operand ring starts zero: rows 32 s + nbp .. 32 s + 31 are never written
  for (uint32_t i = tid; i < P::OR * P::OPSLOT / 16; i += kWsThreads)
    reinterpret_cast<uint4*>(smws)[i] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    for (int s = 0; s < P::RR; ++s) {
      ws_bar_init(&raw_full[s], 1);
      ws_bar_init(&raw_empty[s], kWsConv);
    }
    for (int s = 0; s < P::OR; ++s) {
      ws_bar_init(&op_full[s], kWsConv);
      ws_bar_init(&op_empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      ws_bar_init(&acc_full[s], 1);
      ws_bar_init(&acc_empty[s], 4);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(ws_smem(&tmem_slot)),
                 "r"(kWsTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the zeroed tiles, for the MMA
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  const long long nstage = ng / kWsPts;  // ng is a multiple of 4096
  const long long nmine = nstage > blockIdx.x ? (nstage - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const long long nper = (nmine + kWsPeriod - 1) / kWsPeriod;
  double acc[NBP];
#pragma unroll
  for (int j = 0; j < NBP; ++j) acc[j] = 0.0;

  if (warp == 0) {  // ---- producer
    if (lane == 0) {
      long long i = 0;
      for (; i < nmine && !abort_flag; ++i) {
        const int s = static_cast<int>(i % P::RR);
        if (i >= P::RR && !ws_wait(&raw_empty[s], static_cast<uint32_t>(((i / P::RR) - 1) & 1))) {
          abort_flag = 1;
          break;
        }
        const long long p0 = (blockIdx.x + i * gridDim.x) * static_cast<long long>(kWsPts);
        unsigned char* slot = smws + P::RAW_OFF + s * P::RAWSLOT;
        ws_expect_tx(&raw_full[s], kWsPts * 4 + P::G * kWsPts * P::GB);
        ws_copy(slot, delta + p0, kWsPts * 4, &raw_full[s]);
#pragma unroll 1
        for (int g = 0; g < P::G; ++g)
          ws_copy(slot + kWsPts * 4 + g * P::GST, fields + (g * ng + p0) * P::GB, kWsPts * P::GB, &raw_full[s]);
      }
      // copies of the last slots may still be landing if the converters stopped early
      for (long long j = (i > P::RR ? i - P::RR : 0); j < i; ++j)
        ws_wait(&raw_full[j % P::RR], static_cast<uint32_t>((j / P::RR) & 1));
    }
  } else if (warp == 1) {  // ---- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = ws_idesc();
      long long issued = 0;  // stages whose MMAs were issued
      for (long long i = 0; i < nmine && !abort_flag; ++i) {
        const int o = static_cast<int>(i % P::OR);
        if (!ws_wait(&op_full[o], static_cast<uint32_t>((i / P::OR) & 1))) {
          abort_flag = 1;
          break;
        }
        const long long per = i / kWsPeriod;
        const int buf = static_cast<int>(per & 1);
        const bool first = (i % kWsPeriod) == 0;
        if (first && per >= 2 && !ws_wait(&acc_empty[buf], static_cast<uint32_t>(((per / 2) - 1) & 1))) {
          abort_flag = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t base = ws_smem(smws + o * P::OPSLOT);
        const uint32_t d = tmem + buf * 128;
#pragma unroll
        for (int k = 0; k < kWsKT / 16; ++k) {
          const uint32_t koff = k * 256;  // 16 bf16 = two core matrices along K per instruction
          const uint64_t da = ws_desc(base + koff, 128, kWsSbo);
          const uint64_t db = ws_desc(base + NA * kWsTile + koff, 128, kWsSbo);
          ws_mma(d, da, db, idesc, (first && k == 0) ? 0u : 1u);
          if (NB == 2) ws_mma(d, da, ws_desc(base + (NA + 1) * kWsTile + koff, 128, kWsSbo), idesc, 1u);
          if (NA == 2) ws_mma(d, ws_desc(base + kWsTile + koff, 128, kWsSbo), db, idesc, 1u);
        }
        ws_commit(&op_empty[o]);
        if ((i % kWsPeriod) == kWsPeriod - 1 || i == nmine - 1) ws_commit(&acc_full[buf]);
        issued = i + 1;
      }
      // nothing may be in flight when the accumulators are freed
      if (issued > 0) {
        const long long j = issued - 1;
        if (!ws_wait(&op_empty[j % P::OR], static_cast<uint32_t>((j / P::OR) & 1))) abort_flag = 1;
      }
    }
  } else if (warp < kWsEpiFirst) {  // ---- converters
    // task (slot, octet of points, bin pair j): the rows 2j and 2j + 1 of the slot for 8 points.
    // Bins past nb (padding of the last group) hold zeros, so every pair is written.  The two
    // rows are stored in an order that gives the 8 lanes of a shared-memory phase 8 different
    // rows mod 8 (one 16-byte segment per bank group).
    const int ct = tid - 32 * kWsConvFirst;
    constexpr int NP2 = NBP / 2;
    constexpr int NTASK = 4 * 8 * NP2;
    for (long long i = 0; i < nmine; ++i) {
      if (__shfl_sync(0xffffffffu, abort_flag, 0)) break;  // warp-uniform
      const int s = static_cast<int>(i % P::RR), o = static_cast<int>(i % P::OR);
      // one lane per warp polls the barriers (fewer shared-memory polls), the warp follows it
      bool ok = true;
      if (lane == 0) {
        ok = ws_wait(&raw_full[s], static_cast<uint32_t>((i / P::RR) & 1));
        if (ok && i >= P::OR) ok = ws_wait(&op_empty[o], static_cast<uint32_t>(((i / P::OR) - 1) & 1));
      }
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) {
        abort_flag = 1;
        break;
      }
      const unsigned char* raw = smws + P::RAW_OFF + s * P::RAWSLOT;
      const float* rd = reinterpret_cast<const float*>(raw);
      unsigned char* op = smws + o * P::OPSLOT;
      for (int t = ct; t < NTASK; t += 32 * kWsConv) {
        const int j = t % NP2, so = t / NP2;
        const int sl = so / 8, oc = so % 8;
        const int p0 = sl * kWsKT + 8 * oc;  // first point of the octet in the stage
        const float4 d0 = *reinterpret_cast<const float4*>(rd + p0);
        const float4 d1 = *reinterpret_cast<const float4*>(rd + p0 + 4);
        const float dv[8] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w};
        const unsigned char* gsrc = raw + kWsPts * 4 + (j >> 1) * P::GST;
        float x0[8], x1[8];  // bins 2j and 2j + 1 of the 8 points
        uint32_t w[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          if (RAW == 0) {
            const float2 f = *reinterpret_cast<const float2*>(gsrc + (p0 + e) * 16 + (j & 1) * 8);
            x0[e] = f.x;
            x1[e] = f.y;
          } else {
            w[e] = *reinterpret_cast<const uint32_t*>(gsrc + (p0 + e) * 8 + (j & 1) * 4);
            x0[e] = __uint_as_float(w[e] << 16);
            x1[e] = __uint_as_float(w[e] & 0xffff0000u);
          }
        }
        uint4 ah[2], al[2], bh[2], bl[2];  // [row 2j, row 2j + 1]
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const float* x = r == 0 ? x0 : x1;
          uint32_t* pah = &ah[r].x;
          uint32_t* pal = &al[r].x;
          uint32_t* pbh = &bh[r].x;
          uint32_t* pbl = &bl[r].x;
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            if (RAW == 1) {
              pah[e] = __byte_perm(w[2 * e], w[2 * e + 1], r == 0 ? 0x5410 : 0x7632);
            } else {
              pah[e] = ws_pack(x[2 * e], x[2 * e + 1]);
              if (NA == 2) pal[e] = ws_pack(x[2 * e] - ws_bf(pah[e] & 0xffffu), x[2 * e + 1] - ws_bf(pah[e] >> 16));
            }
            const float y0 = dv[2 * e] * x[2 * e], y1 = dv[2 * e + 1] * x[2 * e + 1];
            pbh[e] = ws_pack(y0, y1);
            if (NB == 2) pbl[e] = ws_pack(y0 - ws_bf(pbh[e] & 0xffffu), y1 - ws_bf(pbh[e] >> 16));
          }
        }
        auto store_row = [&](auto rc) {
          constexpr int r = decltype(rc)::value;
          const uint32_t off = ws_off(32 * sl + 2 * j + r, 8 * oc);
          *reinterpret_cast<uint4*>(op + off) = ah[r];
          if (NA == 2) *reinterpret_cast<uint4*>(op + kWsTile + off) = al[r];
          *reinterpret_cast<uint4*>(op + NA * kWsTile + off) = bh[r];
          if (NB == 2) *reinterpret_cast<uint4*>(op + (NA + 1) * kWsTile + off) = bl[r];
        };
        if ((j >> 2) & 1) {  // which of the two rows this lane stores first
          store_row(std::integral_constant<int, 1>{});
          store_row(std::integral_constant<int, 0>{});
        } else {
          store_row(std::integral_constant<int, 0>{});
          store_row(std::integral_constant<int, 1>{});
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // operand tiles, for the MMA
      __syncwarp();
      if (lane == 0) {
        ws_arrive(&raw_empty[s]);
        ws_arrive(&op_full[o]);
      }
    }
  } else {  // ---- epilogue: quadrant q = slot q, lane = bin b1
    const int q = warp & 3;
    for (long long per = 0; per < nper; ++per) {
      if (__shfl_sync(0xffffffffu, abort_flag, 0)) break;  // warp-uniform
      const int buf = static_cast<int>(per & 1);
      bool ok = true;
      if (lane == 0) ok = ws_wait(&acc_full[buf], static_cast<uint32_t>((per / 2) & 1));
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) {
        abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      float v[32];
      ws_tmem_load32(tmem + (static_cast<uint32_t>(32 * q) << 16) + buf * 128 + 32 * q, v);
#pragma unroll
      for (int j = 0; j < NBP; ++j) acc[j] += static_cast<double>(v[j]);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) ws_arrive(&acc_empty[buf]);
    }
  }
  if (abort_flag && tid == 0) atomicOr(status, 2);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  // the four slots' blocks summed in a fixed order: red[q][b1][b2] in the (idle) operand ring
  double* red = reinterpret_cast<double*>(smws);
  if (warp >= kWsEpiFirst) {
    const int q = warp & 3;
#pragma unroll
    for (int j = 0; j < NBP; ++j) red[(q * 32 + lane) * NBP + j] = acc[j];
  }
  __syncthreads();
  double* out = partials + static_cast<long long>(blockIdx.x) * nb * nb;
  for (int e = tid; e < nb * nb; e += kWsThreads) {
    const int b1 = e / nb, b2 = e % nb;
    double sum = 0.0;
    for (int q = 0; q < 4; ++q) sum += red[(q * 32 + b1) * NBP + b2];
    out[e] = abort_flag ? 0.0 : sum;
  }
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kWsTmemCols) : "memory");
  }
}

template <int NBP, int RAW, int NA, int NB>
int ws_impl(const zeta_ctx* c, const float* delta, const void* fields, double* partials, int ctas, cudaStream_t s) {
  if constexpr (NBP > 32) {
    return ZETA_ENOTSUP;
  } else {
    using P = WsPlan<NBP, RAW, NA, NB>;
    if (prep(k_gram_ws<NBP, RAW, NA, NB>, P::BYTES)) return ZETA_ECUDA;
    k_gram_ws<NBP, RAW, NA, NB><<<ctas, kWsThreads, P::BYTES, s>>>(
        delta, reinterpret_cast<const unsigned char*>(fields), c->ng, c->p.nbins, partials, c->d_status);
    return cudaGetLastError() == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
  }
}

}  // namespace

// raw: 0 float32 fields (modes ZETA_GRAM_BF16 / ZETA_GRAM_BF16X3), 1 bfloat16 fields (B split)
int launch_gram_ws(const zeta_ctx* c, const float* delta, const void* fields, double* partials, int ctas, int raw,
                   bool split, cudaStream_t s) {
  if (c->ng % kWsPts) return ZETA_ENOTSUP;
  // bulk copies start on 16-byte boundaries
  if ((reinterpret_cast<uintptr_t>(delta) | reinterpret_cast<uintptr_t>(fields)) & 15) return ZETA_EINVAL;
  if (raw == 1) {
#define ZK_CALL(P) ws_impl<P, 1, 1, 2>(c, delta, fields, partials, ctas, s)
    ZK_NBP_SWITCH(c->p.nbins, ZK_CALL)
#undef ZK_CALL
  }
  if (split) {
#define ZK_CALL(P) ws_impl<P, 0, 2, 2>(c, delta, fields, partials, ctas, s)
    ZK_NBP_SWITCH(c->p.nbins, ZK_CALL)
#undef ZK_CALL
  }
#define ZK_CALL(P) ws_impl<P, 0, 1, 1>(c, delta, fields, partials, ctas, s)
  ZK_NBP_SWITCH(c->p.nbins, ZK_CALL)
#undef ZK_CALL
}

}  // namespace zk
