// Grid summation stages of the method on sm_103a (Fig. 1 step (6)) in plain float32 arithmetic,
// the uniform term of the particle form and the final reduction.
//
//   node form      points = grid nodes,  v = a_lm(node; b), w = delta(node)
//                  (the grid sum of Eq. 3PCF-multipole-sum with the fields at nodes)
//   Gamma form     points = Gauss-Legendre nodes of every cell (Q = 2 for D = 2, 5 for D = 4),
//                  v = f_b = sum_l beta a_b(l), w = q-weight * n_rec(node); exact for the
//                  piecewise-polynomial integrand, hence equal to the connection-coefficient
//                  double sum of Eqs. (con-coeff) and (SFC-3PCF)
//   mass term      points = the integer values of |n|^2, v = jbar_b(|k|), w = the sum of
//                  (1 or 2) |delta_hat|^2 Mhat over the half-spectrum modes of that |n|^2
// The particle form (Eq. DDD-sum-privertex) is in particles.cu.  The weighted-Gram machinery
// shared by all of them is in gram.cuh.
#include <utility>

#include "gram.cuh"

namespace zk {
namespace {

// ---------------------------------------------------------------------------------------
// Node form: persistent CTAs over chunks of kPB grid points of the bin-interleaved fields.
// Warp 0 copies each chunk (delta and the float4 bin groups of every point) with cp.async into
// the next slot of a kNKS-slot ring and arrives on the slot's `full` mbarrier when its copies
// have landed; the other seven warps contract the chunk and arrive on the slot's `empty`
// mbarrier, so the copies run up to kNKS chunks ahead and no CTA-wide barrier separates the
// chunks.  Every wait is bounded and latches ZETA_ETIMEOUT in the status word.
constexpr int kNodeCons = 224;  // consumer threads
constexpr int kNKS = 2;         // chunk ring slots

template <int NBP>
struct NodeRing {
  using G = Gram<NBP, kNodeCons>;
  static constexpr int SLOTF = kPB * G::NBS + kPB;  // floats per slot: values, then weights
  static constexpr size_t MAIN = static_cast<size_t>(kNKS) * SLOTF * sizeof(float) + 2 * kNKS * sizeof(unsigned long long);
  static constexpr size_t RED = static_cast<size_t>(G::NGRP) * G::NPAIR * 16 * sizeof(double);
  static constexpr size_t BYTES = MAIN > RED ? MAIN : RED;
};

template <int NBP>
__global__ void __launch_bounds__(kThreads) k_gram_node(const float* __restrict__ delta, const float4* __restrict__ f4,
                                                        long long ng, int nb, double* __restrict__ partials,
                                                        int* __restrict__ status) {
  using G = Gram<NBP, kNodeCons>;
  using R = NodeRing<NBP>;
  extern __shared__ __align__(16) unsigned char smraw[];
  float* ring = reinterpret_cast<float*>(smraw);
  unsigned long long* full = reinterpret_cast<unsigned long long*>(smraw + kNKS * R::SLOTF * sizeof(float));
  unsigned long long* empty = full + kNKS;
  double* red = reinterpret_cast<double*>(smraw);  // reused after the main loop
  const int ngrp = (nb + 3) / 4;
  const long long nchunk = ng / kPB;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kNKS; ++s) {
      mbar_init(&full[s], 32);
      mbar_init(&empty[s], kNodeCons / 32);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (warp == 0) {  // ---- producer
    long long i = 0;
    bool ok = true;
    for (long long ch = blockIdx.x; ch < nchunk; ch += gridDim.x, ++i) {
      const int s = static_cast<int>(i % kNKS);
      const long long u = i / kNKS;
      if (u > 0 && !mbar_wait(&empty[s], static_cast<uint32_t>((u - 1) & 1))) {
        ok = false;
        break;
      }
      float* v = ring + s * R::SLOTF;
      const long long p0 = ch * kPB;
      for (int j = lane; j < kPB; j += 32) {
        cp_async4(v + kPB * G::NBS + j, delta + p0 + j);
        for (int q = 0; q < ngrp; ++q) cp_async16(v + j * G::NBS + 4 * q, f4 + q * ng + p0 + j);
      }
      asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(&full[s])) : "memory");
    }
    if (!ok && lane == 0) atomicOr(status, 2);
    for (long long j = (i > kNKS ? i - kNKS : 0); j < i; ++j)
      mbar_wait(&full[j % kNKS], static_cast<uint32_t>((j / kNKS) & 1));
    return;
  }
  // ---- consumers
  const int ct = threadIdx.x - 32;
  const int pr = ct % G::NPAIR, grp = ct / G::NPAIR;
  int b1 = 0, b2 = 0;
  pair_blocks(pr, G::NBLK, b1, b2);
  GramAcc<NBP, kNodeCons> g;
  g.init();
  long long i = 0;
  bool ok = true;
  for (long long ch = blockIdx.x; ch < nchunk; ch += gridDim.x, ++i) {
    const int s = static_cast<int>(i % kNKS);
    if (ok && !mbar_wait(&full[s], static_cast<uint32_t>((i / kNKS) & 1))) ok = false;
    const float* v = ring + s * R::SLOTF;
    if (ok && grp < G::NGRP) g.add(v, v + kPB * G::NBS, kPB, b1, b2, grp);
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
  if (!ok && ct == 0) atomicOr(status, 2);
  cta_store<NBP, kNodeCons, 1>(g, red, nb, partials + static_cast<long long>(blockIdx.x) * nb * nb, ct);
}

// ---------------------------------------------------------------------------------------
// Node form, register-blocked (nbins <= 20).  Persistent CTAs over chunks of kRbChunk grid
// points.  Warp 0 streams each chunk (delta, then the float4 bin groups: 1 + NBP/4 contiguous
// runs of global memory) into the next slot of a kRbSlots-slot ring with bulk asynchronous
// copies whose completion the slot's `full` mbarrier counts in bytes; eight consumer warps wait
// on `full`, each takes 32-point sub-chunks (one point per lane) and accumulates, in float32
// registers, its share of the whole upper triangle of the bin Gram -- the NP = NBP (NBP + 1) / 2
// pairs are split into PARTS halves taken by different warps -- and arrives on the slot's
// `empty` mbarrier, which the producer waits on before refilling it.  A point costs a lane
// NBP / 4 + 1 shared-memory loads and NBP + NP / PARTS multiplies and FMAs, so the contraction
// runs at the pace of the copies.  Every kRbFlush points per lane the warp sums each accumulator
// over its lanes with a fixed butterfly into its float64 row in shared memory; at the end the
// warps of a part are summed in warp order.  Deterministic; every wait is bounded and latches
// ZETA_ETIMEOUT in the status word.
constexpr int kRbCons = 8;                       // consumer warps
constexpr int kRbThreads = 32 * (kRbCons + 1);   // plus one producer warp
constexpr int kRbChunk = 256;                    // points per ring slot
constexpr int kRbSlots = 8;
constexpr int kRbFlush = 128;                    // points per lane between float64 flushes

template <int NBP>
struct Tri {
  static constexpr int NP = NBP * (NBP + 1) / 2;
  static constexpr int PARTS = NP > 120 ? 2 : 1;
  static constexpr int NPH = (NP + PARTS - 1) / PARTS;
  static constexpr int G4 = NBP / 4;
  // pair index k (row-major over b1 <= b2) -> b1, b2
  __host__ __device__ static constexpr int b1_of(int k) {
    int r = 0;
    while (k >= NBP - r) {
      k -= NBP - r;
      ++r;
    }
    return r;
  }
  __host__ __device__ static constexpr int b2_of(int k) {
    int r = 0;
    while (k >= NBP - r) {
      k -= NBP - r;
      ++r;
    }
    return r + k;
  }
};

// acc[k] += (w v[b1]) v[b2] for the pairs K0 + k of half H; the pair indices are template
// arguments, so every register index is a compile-time constant.
template <int NBP, int H, int... K>
__device__ __forceinline__ void rb_accum_seq(float (&acc)[Tri<NBP>::NPH], const float (&v)[NBP], float w,
                                             std::integer_sequence<int, K...>) {
  using T = Tri<NBP>;
  constexpr int K0 = H * T::NPH;
  float xs[NBP];
#pragma unroll
  for (int b = 0; b < NBP; ++b) xs[b] = v[b] * w;  // unused rows are dead code
  ((K0 + K < T::NP ? (acc[K] = fmaf(xs[T::b1_of(K0 + K < T::NP ? K0 + K : 0)],
                                    v[T::b2_of(K0 + K < T::NP ? K0 + K : 0)], acc[K]))
                   : 0.f),
   ...);
}

// Sum each accumulator over the warp's lanes (fixed butterfly); lane j keeps the totals of the
// pairs k = j, j + 32, ... and adds them to its own float64 accumulators, so a flush costs
// NPH / 32 float64 additions per lane instead of NPH predicated ones per warp.
template <int NBP>
__device__ __forceinline__ void rb_flush(float (&acc)[Tri<NBP>::NPH], double (&dacc)[(Tri<NBP>::NPH + 31) / 32],
                                         int lane) {
  constexpr int NR = (Tri<NBP>::NPH + 31) / 32;
  float mine[NR];
#pragma unroll
  for (int i = 0; i < NR; ++i) mine[i] = 0.f;
#pragma unroll
  for (int k = 0; k < Tri<NBP>::NPH; ++k) {
    float x = acc[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    mine[k >> 5] = lane == (k & 31) ? x : mine[k >> 5];
    acc[k] = 0.f;
  }
#pragma unroll
  for (int i = 0; i < NR; ++i) dacc[i] += static_cast<double>(mine[i]);
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
// one contiguous global -> shared copy (16-byte aligned, size a multiple of 16) whose bytes the
// mbarrier counts on completion
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

// Slot layouts of the register-blocked Gram: MODE 0 node form (delta, then the float4 bin
// groups), 1 node form on bfloat16 fields (delta, then bfloat16 x 4 groups), 2 particle rows
// (the float4 (t, w) records, then the rows [particle][NBP]); cnt points in the last chunk.
template <int NBP, int MODE>
struct RbLayout {
  static constexpr int G4 = NBP / 4;
  static constexpr int SLOT = MODE == 2 ? kRbChunk * (16 + 4 * NBP) : kRbChunk * (4 + (MODE == 1 ? 8 : 16) * G4);
};

template <int NBP, int H, int MODE>
__device__ __forceinline__ bool rb_consume(const unsigned char* ring, unsigned long long* full,
                                           unsigned long long* empty, long long nmine, int sub, int nsub,
                                           double* drow, int lane, long long ntot, long long c0, long long cstride) {
  using T = Tri<NBP>;
  using Lo = RbLayout<NBP, MODE>;
  constexpr int NR = (T::NPH + 31) / 32;
  float acc[T::NPH];
  double dacc[NR];
#pragma unroll
  for (int k = 0; k < T::NPH; ++k) acc[k] = 0.f;
#pragma unroll
  for (int i = 0; i < NR; ++i) dacc[i] = 0.0;
  int pending = 0;
  bool ok = true;
  for (long long i = 0; i < nmine; ++i) {
    const int s = static_cast<int>(i % kRbSlots);
    if (!mbar_wait(&full[s], static_cast<uint32_t>((i / kRbSlots) & 1))) {
      ok = false;
      break;
    }
    const unsigned char* slot = ring + s * Lo::SLOT;
    const long long left = ntot - (c0 + i * cstride) * kRbChunk;
    const int cnt = left < kRbChunk ? static_cast<int>(left) : kRbChunk;
    for (int j = sub; j < kRbChunk / 32; j += nsub) {
      const int p = j * 32 + lane;
      if (j * 32 >= cnt) break;  // warp-uniform
      float v[NBP];
      float w;
      if constexpr (MODE == 2) {
        w = reinterpret_cast<const float4*>(slot)[p].w;
        const float4* row = reinterpret_cast<const float4*>(slot + kRbChunk * 16) + p * T::G4;
#pragma unroll
        for (int q = 0; q < T::G4; ++q) {
          const float4 x = row[q];
          v[4 * q] = x.x;
          v[4 * q + 1] = x.y;
          v[4 * q + 2] = x.z;
          v[4 * q + 3] = x.w;
        }
      } else {
        w = reinterpret_cast<const float*>(slot)[p];
#pragma unroll
        for (int q = 0; q < T::G4; ++q) {
          if constexpr (MODE == 1) {  // bfloat16 -> float is a 16-bit shift
            const uint2 x = reinterpret_cast<const uint2*>(slot + kRbChunk * 4)[q * kRbChunk + p];
            v[4 * q] = __uint_as_float(x.x << 16);
            v[4 * q + 1] = __uint_as_float(x.x & 0xffff0000u);
            v[4 * q + 2] = __uint_as_float(x.y << 16);
            v[4 * q + 3] = __uint_as_float(x.y & 0xffff0000u);
          } else {
            const float4 x = reinterpret_cast<const float4*>(slot + kRbChunk * 4)[q * kRbChunk + p];
            v[4 * q] = x.x;
            v[4 * q + 1] = x.y;
            v[4 * q + 2] = x.z;
            v[4 * q + 3] = x.w;
          }
        }
      }
      if (p >= cnt) {  // a ragged last chunk (particle rows only): the slot's tail was not written by
        w = 0.f;       // this chunk's copy and may hold anything, NaN included, so zero the values too
#pragma unroll
        for (int q = 0; q < NBP; ++q) v[q] = 0.f;
      }
      rb_accum_seq<NBP, H>(acc, v, w, std::make_integer_sequence<int, T::NPH>{});
      if (++pending == kRbFlush) {
        rb_flush<NBP>(acc, dacc, lane);
        pending = 0;
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
  rb_flush<NBP>(acc, dacc, lane);
#pragma unroll
  for (int i = 0; i < NR; ++i)
    if (32 * i + lane < T::NPH) drow[32 * i + lane] = dacc[i];
  return ok;
}

// MODE 0/1: node form over ng grid points (delta, fields); MODE 2: weighted Gram of the particle
// rows over ng = np particles (delta = the prepared float4 records as floats, fields = the rows).
template <int NBP, int MODE>
__global__ void __launch_bounds__(kRbThreads, 1)
    k_gram_node_rb(const float* __restrict__ delta, const unsigned char* __restrict__ fields, long long ng, int nb,
                   double* __restrict__ partials, int* __restrict__ status) {
  using T = Tri<NBP>;
  using Lo = RbLayout<NBP, MODE>;
  extern __shared__ __align__(128) unsigned char smq[];
  unsigned char* ring = smq;                                                               // [kRbSlots][SLOT]
  unsigned long long* full = reinterpret_cast<unsigned long long*>(smq + kRbSlots * Lo::SLOT);
  unsigned long long* empty = full + kRbSlots;
  double* dsum = reinterpret_cast<double*>(empty + kRbSlots);                             // [kRbCons][NPH]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < kRbCons * T::NPH; i += blockDim.x) dsum[i] = 0.0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kRbSlots; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kRbCons);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const long long nchunk = (ng + kRbChunk - 1) / kRbChunk;
  const long long nmine = nchunk > blockIdx.x ? (nchunk - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  if (warp == 0) {  // ---- producer
    bool ok = true;
    if (lane == 0) {
      for (long long i = 0; i < nmine; ++i) {
        const int s = static_cast<int>(i % kRbSlots);
        if (i >= kRbSlots && !mbar_wait(&empty[s], static_cast<uint32_t>(((i / kRbSlots) - 1) & 1))) {
          ok = false;
          break;
        }
        const long long p0 = (blockIdx.x + i * gridDim.x) * static_cast<long long>(kRbChunk);
        unsigned char* slot = ring + s * Lo::SLOT;
        if constexpr (MODE == 2) {  // a ragged last chunk copies only its particles
          const long long left = ng - p0;
          const uint32_t cnt = static_cast<uint32_t>(left < kRbChunk ? left : kRbChunk);
          mbar_expect_tx(&full[s], cnt * (16 + 4 * NBP));
          bulk_copy(slot, delta + 4 * p0, cnt * 16, &full[s]);
          bulk_copy(slot + kRbChunk * 16, fields + p0 * 4 * NBP, cnt * 4 * NBP, &full[s]);
        } else {
          constexpr int GB = MODE == 1 ? 8 : 16;
          mbar_expect_tx(&full[s], Lo::SLOT);
          bulk_copy(slot, delta + p0, kRbChunk * 4, &full[s]);
#pragma unroll
          for (int q = 0; q < T::G4; ++q)
            bulk_copy(slot + kRbChunk * 4 + q * kRbChunk * GB, fields + (q * ng + p0) * GB, kRbChunk * GB, &full[s]);
        }
      }
      if (!ok) atomicOr(status, 2);
      // copies of the last slots may still be landing if the consumers stopped early
      for (long long j = (nmine > kRbSlots ? nmine - kRbSlots : 0); j < nmine; ++j)
        mbar_wait(&full[j % kRbSlots], static_cast<uint32_t>((j / kRbSlots) & 1));
    }
    __syncwarp();
  } else {  // ---- consumers
    const int cw = warp - 1;
    const int part = cw % T::PARTS, sub = cw / T::PARTS, nsub = kRbCons / T::PARTS;
    bool ok;
    if (part == 0)
      ok = rb_consume<NBP, 0, MODE>(ring, full, empty, nmine, sub, nsub, dsum + cw * T::NPH, lane, ng, blockIdx.x,
                                    gridDim.x);
    else
      ok = rb_consume<NBP, (T::PARTS > 1 ? 1 : 0), MODE>(ring, full, empty, nmine, sub, nsub, dsum + cw * T::NPH,
                                                         lane, ng, blockIdx.x, gridDim.x);
    if (!ok && lane == 0) atomicOr(status, 2);
  }
  __syncthreads();
  double* out = partials + static_cast<long long>(blockIdx.x) * nb * nb;
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int r = e / nb, c = e % nb;
    const int lo = r < c ? r : c, hi = r < c ? c : r;
    const int k = lo * NBP - lo * (lo - 1) / 2 + (hi - lo);  // row-major pair index
    const int pt = k / T::NPH, kk = k % T::NPH;
    double sum = 0.0;
    for (int w = pt; w < kRbCons; w += T::PARTS) sum += dsum[w * T::NPH + kk];
    out[e] = sum;
  }
}

template <int NBP, int MODE>
constexpr size_t smem_node_rb() {
  return static_cast<size_t>(kRbSlots) * RbLayout<NBP, MODE>::SLOT + 2 * kRbSlots * sizeof(unsigned long long) +
         static_cast<size_t>(kRbCons) * Tri<NBP>::NPH * sizeof(double);
}

// ---------------------------------------------------------------------------------------
// Gamma form: persistent CTAs over 8x8x8-cell tiles, NC cells of K^3 points each per batch.
// B-splines (D = 2, 4): the points are the K^3 Gauss-Legendre nodes of each cell (K = 2, 5), so
// the sum is the exact integral of n_rec f_b1 f_b2 over the cell.  Daubechies (D = 5): the
// per-axis connection coefficients split as gamma = U diag(lam) U^T (5 x 5), so
// sum_l delta_l sum_{o1,o2} Gamma(o1, o2) a_b1(l + o1) a_b2(l + o2)
//   = sum_l sum_k (lam_kx lam_ky lam_kz delta_l) A_k,b1(l) A_k,b2(l),
// A_k(l) = sum_o U[ox][kx] U[oy][ky] U[oz][kz] a(l + o - 2): the "points" of node l are the 5^3
// eigen-indices k and the point weight is the product of lam times delta at the node itself.
// Either way a point's value is a tensor-product filter of the cell's D^3 stencil with the
// per-axis D x K matrix F(o, k) = gq[K + k D + o], and the kernel applies it one axis at a time:
// x (D^2 rows -> D^2 K values), y (-> D K^2), z (-> K^3), D taps each, per cell and channel
// (the bin groups as float4, and for the B-splines delta as a fourth, whose filtered value is
// n_rec at the point).  That is D^2 K + D K^2 + K^3 outputs of D taps instead of K^3 outputs
// of D^3 taps.  The x pass reads the L1-cached fields, each stencil row once for a run of CX
// cells along x ((CX + D - 1) D^2 loads per run and channel instead of K^3 D^3 per cell), and
// writes into the space of the value table (dead until the z pass), the y
// pass into its own buffer, the z pass into the value table and the point weights; phase 4
// contracts the batch.
template <int NBP, int D>
struct GammaShape {
  static constexpr bool DB = D == 5;
  static constexpr int K = D == 2 ? 2 : 5;   // points per axis
  static constexpr int K3 = K * K * K;
  static constexpr int NC = kPB / K3;        // cells per batch (2 or 32)
  static constexpr int CX = NC < kTile ? NC : kTile;  // cells per run along x (2 or 8)
  static constexpr int CR = NC / CX;                  // runs per batch
  static constexpr int OFF = DB ? 2 : D / 2 - 1;
  static constexpr int NCH = NBP / 4 + (DB ? 0 : 1);
  // row pitches (float4) of the x- and y-pass outputs per (channel, cell, oz): padded for K = 5
  // to 5 mod 8, so that the y and z passes (lanes along kx, then the next row) hit distinct
  // banks
  static constexpr int XR = K == 5 ? (D * K + 7 - 5) / 8 * 8 + 5 : D * K;
  static constexpr int YR = K == 5 ? (K * K + 7 - 5) / 8 * 8 + 5 : K * K;
  static constexpr int XF = NCH * NC * D * XR * 4;      // floats of the x-pass output
  static constexpr int VF = kPB * Gram<NBP>::NBS + kPB;  // floats of the value table and weights
  static constexpr int AF = XF > VF ? XF : VF;
  static constexpr int YF = NCH * NC * D * YR * 4;      // floats of the y-pass output
  static_assert((kTile * kTile * kTile) % NC == 0 && kTile % CX == 0, "a tile holds whole batches and runs");
  static_assert(XR >= D * K && YR >= K * K, "pitches hold a row");
  static_assert(AF % 4 == 0, "the y buffer starts on a 16-byte boundary");
};

template <int NBP, int D>
__global__ void __launch_bounds__(kThreads)
    k_gram_gamma(const float* __restrict__ delta, const float4* __restrict__ f4, long long ng, int n, int nb,
                 const float* __restrict__ gq, double* __restrict__ partials) {
  using G = Gram<NBP>;
  using S = GammaShape<NBP, D>;
  constexpr int K = S::K, NC = S::NC, OFF = S::OFF;
  extern __shared__ __align__(16) unsigned char smraw[];
  float* vals = reinterpret_cast<float*>(smraw);             // [kPB][NBS]
  float* wts = vals + kPB * G::NBS;                           // [kPB]
  float4* xbuf = reinterpret_cast<float4*>(smraw);           // [ch][cell][oz][oy][kx], aliases vals
  float4* ybuf = reinterpret_cast<float4*>(vals + S::AF);    // [ch][cell][oz][ky][kx]
  double* red = reinterpret_cast<double*>(smraw);            // reused after the main loop
  const int pr = threadIdx.x % G::NPAIR, grp = threadIdx.x / G::NPAIR;
  int b1 = 0, b2 = 0;
  pair_blocks(pr, G::NBLK, b1, b2);
  GramAcc<NBP> g;
  g.init();
  float fm[D][K], qw[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    qw[k] = __ldg(gq + k);
#pragma unroll
    for (int o = 0; o < D; ++o) fm[o][k] = __ldg(gq + K + k * D + o);
  }
  const int ngrp = (nb + 3) / 4;
  const int nch = ngrp + (S::DB ? 0 : 1);
  const int nt = n / kTile;
  const long long ntiles = static_cast<long long>(nt) * nt * nt;
  const int mask = n - 1;
  constexpr int NBATCH = kTile * kTile * kTile / NC;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int tx = static_cast<int>(t % nt), ty = static_cast<int>((t / nt) % nt),
              tz = static_cast<int>(t / (static_cast<long long>(nt) * nt));
    for (int bt = 0; bt < NBATCH; ++bt) {
      auto cell = [&](int j, int& cx, int& cy, int& cz) {
        const int ci = bt * NC + j;
        cx = tx * kTile + ci % kTile;
        cy = ty * kTile + (ci / kTile) % kTile;
        cz = tz * kTile + ci / (kTile * kTile);
      };
      __syncthreads();  // the previous batch's contraction is done with the value table
      // x pass: task (channel, run, oz, oy) loads the CX + D - 1 nodes of one stencil row that
      // the run's CX cells share and filters them into K values per cell
      for (int i = threadIdx.x; i < nch * S::CR * D * D; i += kThreads) {
        constexpr int CX = S::CX, NE = CX + D - 1;
        const int oy = i % D, oz = (i / D) % D, cr = (i / (D * D)) % S::CR, ch = i / (D * D * S::CR);
        int cx, cy, cz;
        cell(cr * CX, cx, cy, cz);
        const long long row = (static_cast<long long>((cz - OFF + oz) & mask) * n + ((cy - OFF + oy) & mask)) * n;
        float4 in[NE];
        if (ch < ngrp) {
          const float4* base = f4 + ch * ng + row;
#pragma unroll
          for (int e = 0; e < NE; ++e) in[e] = __ldg(base + ((cx - OFF + e) & mask));
        } else {
#pragma unroll
          for (int e = 0; e < NE; ++e) in[e] = make_float4(__ldg(delta + row + ((cx - OFF + e) & mask)), 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int c = 0; c < CX; ++c) {
          float4* out = xbuf + ((ch * NC + cr * CX + c) * D + oz) * S::XR + oy * K;
#pragma unroll
          for (int k = 0; k < K; ++k) {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int o = 0; o < D; ++o) {
              v.x = fmaf(fm[o][k], in[c + o].x, v.x);
              v.y = fmaf(fm[o][k], in[c + o].y, v.y);
              v.z = fmaf(fm[o][k], in[c + o].z, v.z);
              v.w = fmaf(fm[o][k], in[c + o].w, v.w);
            }
            out[k] = v;
          }
        }
      }
      __syncthreads();
      // y pass: task (channel, cell, oz, kx) filters D x-pass values into K
      for (int i = threadIdx.x; i < nch * NC * D * K; i += kThreads) {
        const int kx = i % K, r = i / K;
        const float4* src = xbuf + r * S::XR + kx;
        float4 in[D];
#pragma unroll
        for (int o = 0; o < D; ++o) in[o] = src[o * K];
        float4* out = ybuf + r * S::YR + kx;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int o = 0; o < D; ++o) {
            v.x = fmaf(fm[o][k], in[o].x, v.x);
            v.y = fmaf(fm[o][k], in[o].y, v.y);
            v.z = fmaf(fm[o][k], in[o].z, v.z);
            v.w = fmaf(fm[o][k], in[o].w, v.w);
          }
          out[k * K] = v;
        }
      }
      __syncthreads();
      // z pass: task (channel, cell, ky, kx) filters D y-pass values into the K points along z
      for (int i = threadIdx.x; i < nch * NC * K * K; i += kThreads) {
        const int kk = i % (K * K), r = i / (K * K);
        const int j = r % NC, ch = r / NC;
        const int kx = kk % K, ky = kk / K;
        const float4* src = ybuf + r * D * S::YR + kk;
        float4 in[D];
#pragma unroll
        for (int o = 0; o < D; ++o) in[o] = src[o * S::YR];
        const float wxy = __ldg(gq + kx) * __ldg(gq + ky);
        float dn = 0.f;
        if (S::DB && ch == 0) {  // delta at the node itself
          int cx, cy, cz;
          cell(j, cx, cy, cz);
          dn = __ldg(delta + (static_cast<long long>(cz) * n + cy) * n + cx);
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
          float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int o = 0; o < D; ++o) {
            v.x = fmaf(fm[o][k], in[o].x, v.x);
            v.y = fmaf(fm[o][k], in[o].y, v.y);
            v.z = fmaf(fm[o][k], in[o].z, v.z);
            v.w = fmaf(fm[o][k], in[o].w, v.w);
          }
          const int p = j * S::K3 + k * K * K + kk;
          const float w = wxy * qw[k];
          if (ch < ngrp) *reinterpret_cast<float4*>(vals + p * G::NBS + 4 * ch) = v;
          else wts[p] = w * v.x;  // n_rec at the point
          if (S::DB && ch == 0) wts[p] = w * dn;
        }
      }
      __syncthreads();
      if (grp < G::NGRP) g.add(vals, wts, NC * S::K3, b1, b2, grp);
    }
  }
  __syncthreads();
  cta_store<NBP>(g, red, nb, partials + static_cast<long long>(blockIdx.x) * nb * nb);
}

// ---------------------------------------------------------------------------------------
// Uniform term of the particle form: U_l[b1][b2] = (2l+1)/(4 pi) sum_k w(k) J_l,b1(|n|^2)
// J_l,b2(|n|^2), w = (1, or 2 off the ix = 0 plane) |delta_hat|^2 Mhat over the stored half
// spectrum without its Nyquist planes.  The window depends on the mode only through the
// integer |n|^2, so w is summed per |n|^2 once per catalogue and each l is then a Gram over
// the 3 (n/2 - 1)^2 + 1 values of |n|^2 (Nyquist planes excluded).  The per-|n|^2 sums are
// 64-bit fixed point in units of max(w) 2^-48: integer atomics, so the sums do not depend on
// the order of the modes, and a value of |n|^2 holds far fewer than 2^16 modes, so no sum can
// overflow.
constexpr double kMassUnit = 281474976710656.0;  // 2^48

__device__ __forceinline__ bool mass_mode(long long i, int n, const float2* __restrict__ dhat,
                                          const float* __restrict__ mhat, double& w, long long& n2) {
  const int nc = n / 2;
  const int ix = static_cast<int>(i % nc), iy = static_cast<int>((i / nc) % n),
            iz = static_cast<int>(i / (static_cast<long long>(nc) * n));
  if (iy == n / 2 || iz == n / 2) return false;
  const int fy = iy < n / 2 ? iy : iy - n, fz = iz < n / 2 ? iz : iz - n;
  n2 = static_cast<long long>(ix) * ix + fy * fy + fz * fz;
  const float2 d = dhat[i];
  w = (ix == 0 ? 1.0 : 2.0) * (static_cast<double>(d.x) * d.x + static_cast<double>(d.y) * d.y) *
      (static_cast<double>(mhat[ix]) * mhat[iy] * mhat[iz]);
  return true;
}

// max_k w(k) as the bits of a non-negative double (their unsigned order is the numeric order)
__global__ void k_mass_max(const float2* __restrict__ dhat, const float* __restrict__ mhat, int n,
                           unsigned long long* __restrict__ wmax_bits) {
  const long long total = static_cast<long long>(n) * n * (n / 2);
  unsigned long long m = 0;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long long>(blockDim.x) * gridDim.x) {
    double w;
    long long n2;
    if (mass_mode(i, n, dhat, mhat, w, n2)) {
      const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(w));
      m = b > m ? b : m;
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, m, off);
    m = o > m ? o : m;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(wmax_bits, m);
}

__global__ void k_mass_hist(const float2* __restrict__ dhat, const float* __restrict__ mhat, int n,
                            const unsigned long long* __restrict__ wmax_bits, unsigned long long* __restrict__ hist) {
  const double wmax = __longlong_as_double(static_cast<long long>(*wmax_bits));
  if (!(wmax > 0.0)) return;
  const double scale = kMassUnit / wmax;
  const long long total = static_cast<long long>(n) * n * (n / 2);
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long long>(blockDim.x) * gridDim.x) {
    double w;
    long long n2;
    if (mass_mode(i, n, dhat, mhat, w, n2)) {
      const unsigned long long q = __double2ull_rn(w * scale);
      if (q) atomicAdd(hist + n2, q);
    }
  }
}

// Gram of one l over the values of |n|^2: weight S(|n|^2), values J_l,b(|n|^2)
template <int NBP>
__global__ void __launch_bounds__(kThreads) k_gram_mass(const unsigned long long* __restrict__ hist,
                                                        const unsigned long long* __restrict__ wmax_bits,
                                                        const float* __restrict__ jt, long long nn2, int nb,
                                                        double* __restrict__ partials) {
  using G = Gram<NBP>;
  extern __shared__ __align__(16) unsigned char smraw[];
  float* vals = reinterpret_cast<float*>(smraw);
  float* wts = vals + kPB * G::NBS;
  double* red = reinterpret_cast<double*>(smraw);  // reused after the main loop
  const int pr = threadIdx.x % G::NPAIR, grp = threadIdx.x / G::NPAIR;
  int b1 = 0, b2 = 0;
  pair_blocks(pr, G::NBLK, b1, b2);
  GramAcc<NBP> g;
  g.init();
  const double unit = __longlong_as_double(static_cast<long long>(*wmax_bits)) / kMassUnit;
  const int nbp = 4 * ((nb + 3) / 4);
  const long long nchunk = (nn2 + kPB - 1) / kPB;
  for (long long ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {
    const long long p = ch * kPB + threadIdx.x;
    const long long left = nn2 - ch * kPB;
    const int cnt = left < kPB ? static_cast<int>(left) : kPB;
    __syncthreads();
    if (threadIdx.x < cnt) {
      wts[threadIdx.x] = static_cast<float>(static_cast<double>(hist[p]) * unit);
      for (int b = 0; b < NBP; ++b) vals[threadIdx.x * G::NBS + b] = (b < nb) ? __ldg(jt + p * nbp + b) : 0.f;
    }
    __syncthreads();
    if (grp < G::NGRP) g.add(vals, wts, cnt, b1, b2, grp);
  }
  __syncthreads();
  cta_store<NBP>(g, red, nb, partials + static_cast<long long>(blockIdx.x) * nb * nb);
}

// One warp per output entry: lane j sums the partials j, j + 32, ... in order, then a fixed
// butterfly combines the lanes, so the result does not depend on scheduling.
__global__ void k_reduce(const double* __restrict__ part, int nparts, int nb, double scale,
                         const double* __restrict__ wdiv, double* __restrict__ out, int store) {
  const int e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (e >= nb * nb) return;  // whole warps leave together
  const int r = e / nb, c = e % nb;
  const int lo = r < c ? r : c, hi = r < c ? c : r;
  double sum = 0.0;
  for (int k = lane; k < nparts; k += 32) sum += part[static_cast<long long>(k) * nb * nb + lo * nb + hi];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
  if (lane == 0) {
    double sc = scale;
    if (wdiv) sc /= *wdiv;
    // the product is rounded before the add (no fused multiply-add), so a contribution stored
    // in a slot and added later (zeta_reduce_lm) rounds exactly as one added here
    const double c = __dmul_rn(sc, sum);
    out[e] = store ? c : __dadd_rn(out[e], c);
  }
}

// zeta_l of every form from per-(l, m) contribution slots, in the order the full measurement
// adds them: 0, then the uniform term of l (particle form), then m = -l .. l.  One thread per
// output entry.  slots: [form][(lmax+1)^2 + lmax+1][nb][nb], (l, m) at l^2 + l + m, the
// uniform term of l at (lmax+1)^2 + l.
__global__ void k_reduce_lm(const double* __restrict__ slots, int nforms, int part_form, int lmax, int nb,
                            double* __restrict__ zeta) {
  const int nb2 = nb * nb;
  const int total = nforms * (lmax + 1) * nb2;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int e = i % nb2, l = (i / nb2) % (lmax + 1), f = i / (nb2 * (lmax + 1));
  const int nslot = (lmax + 1) * (lmax + 1) + lmax + 1;
  const double* sf = slots + static_cast<long long>(f) * nslot * nb2;
  double acc = 0.0;
  if (f == part_form) acc = __dadd_rn(acc, sf[static_cast<long long>((lmax + 1) * (lmax + 1) + l) * nb2 + e]);
  for (int m = -l; m <= l; ++m) acc = __dadd_rn(acc, sf[static_cast<long long>(l * l + l + m) * nb2 + e]);
  zeta[i] = acc;
}

// ---------------------------------------------------------------------------------------
// 2PCF (Eq. pair-counting with Eq. trans-field-FT; Sec. 3 for the windows).  By Parseval the node
// form (1/N_g) sum_l delta_p(l) a_00,b(l) equals (1/N_g^2) sum_n |delta_hat|^2 Phi-hat(n) W_0,b(k)
// W_p(k) over the non-Nyquist modes, which depends on the mode only through |n|^2 apart from
// Phi-hat: so the per-|n|^2 sums H of (1 or 2) |delta_hat|^2 Phi-hat (the fixed-point histogram of
// the uniform term, with Phi-hat as its per-axis table) give every bin, and any radius, as one
// sum over the 3 (n/2 - 1)^2 + 1 values of |n|^2.  One CTA per output value; each thread sums
// a fixed stride of |n|^2 in float64 and the CTA reduces in a fixed order.
// mode 0: out[b] for the bins, radial factor from the window table (l = 0 row);
// mode 1: out[i] for radii[i], radial factor j_0(k r_i) W_TH(k rsec).
__global__ void __launch_bounds__(256) k_xi_hist(const unsigned long long* __restrict__ hist,
                                                 const unsigned long long* __restrict__ wmax_bits, long long nn2,
                                                 const float* __restrict__ jt0, int nbp, const float* __restrict__ wprim,
                                                 double ng, double kunit, const double* __restrict__ radii,
                                                 double rsec, int mode, double* __restrict__ out) {
  __shared__ double red[256];
  const double unit = __longlong_as_double(static_cast<long long>(*wmax_bits)) / kMassUnit;
  const int o = blockIdx.x;
  double acc = 0.0;
  for (long long i = threadIdx.x; i < nn2; i += blockDim.x) {
    const unsigned long long h = hist[i];
    if (!h) continue;
    double f;
    if (mode == 0) {
      f = static_cast<double>(__ldg(jt0 + i * nbp + o)) * ng * 0.28209479177387814;  // / sqrt(4 pi)
    } else {
      const double k = kunit * sqrt(static_cast<double>(i));
      const double x = k * radii[o];
      f = x > 0.0 ? sin(x) / x : 1.0;
      if (rsec > 0.0) {
        const double y = k * rsec;
        f *= y > 1e-2 ? 3.0 * (sin(y) - y * cos(y)) / (y * y * y) : 1.0 - y * y / 10.0;
      }
    }
    if (wprim) f *= static_cast<double>(__ldg(wprim + i)) * ng;
    acc += static_cast<double>(h) * f;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[o] = red[0] * unit / (ng * ng);
}

template <int NBP>
size_t smem_node() {
  return NodeRing<NBP>::BYTES;
}
template <int NBP>
size_t smem_mass() {
  using G = Gram<NBP>;
  const size_t main = (kPB * G::NBS + kPB) * sizeof(float);
  return main > red_bytes<NBP>() ? main : red_bytes<NBP>();
}
template <int NBP, int D>
size_t smem_gamma() {
  using S = GammaShape<NBP, D>;
  const size_t main = static_cast<size_t>(S::AF + S::YF) * sizeof(float);
  return main > red_bytes<NBP>() ? main : red_bytes<NBP>();
}

template <int NBP>
int node_impl(const zeta_ctx* c, const float* delta, const float* alm, double* partials, cudaStream_t s,
              bool bf16) {
  StageScope prof(c, ST_GRAM_NODE, 1, s);
  if constexpr (NBP <= 20) {
    const unsigned char* f = reinterpret_cast<const unsigned char*>(alm);
    // the ring's bulk copies start on 16-byte boundaries
    if ((reinterpret_cast<uintptr_t>(delta) | reinterpret_cast<uintptr_t>(alm)) & 15) return ZETA_EINVAL;
    if (bf16) {  // bfloat16 fields, register-blocked float32 Gram (faster here than the tensor cores)
      const size_t smr = smem_node_rb<NBP, 1>();
      if (prep(k_gram_node_rb<NBP, 1>, smr)) return ZETA_ECUDA;
      k_gram_node_rb<NBP, 1><<<gram_ctas(c, GK_NODE), kRbThreads, smr, s>>>(delta, f, c->ng, c->p.nbins, partials,
                                                                           c->d_status);
    } else {
      const size_t smr = smem_node_rb<NBP, 0>();
      if (prep(k_gram_node_rb<NBP, 0>, smr)) return ZETA_ECUDA;
      k_gram_node_rb<NBP, 0><<<gram_ctas(c, GK_NODE), kRbThreads, smr, s>>>(delta, f, c->ng, c->p.nbins, partials,
                                                                           c->d_status);
    }
    return cudaGetLastError() == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
  }
  if (bf16)  // bfloat16 fields with more than 20 bins: the tensor-core Gram (gram_ws.cu)
    return launch_gram_ws(c, delta, alm, partials, gram_ctas(c, GK_NODE), 1, false, s);
  const size_t sm = smem_node<NBP>();
  if (prep(k_gram_node<NBP>, sm)) return ZETA_ECUDA;
  k_gram_node<NBP><<<gram_ctas(c, GK_NODE), kThreads, sm, s>>>(delta, reinterpret_cast<const float4*>(alm), c->ng,
                                                                 c->p.nbins, partials, c->d_status);
  return cudaGetLastError() == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
}

template <int NBP, int D>
int gamma_impl(const zeta_ctx* c, const float* delta, const float* alm, double* partials, cudaStream_t s) {
  StageScope prof(c, ST_GRAM_GAMMA, 1, s);
  const size_t sm = smem_gamma<NBP, D>();
  if (prep(k_gram_gamma<NBP, D>, sm)) return ZETA_ECUDA;
  if (c->gamma_q != GammaShape<NBP, D>::K) return ZETA_EINVAL;
  k_gram_gamma<NBP, D><<<gram_ctas(c, GK_GAMMA), kThreads, sm, s>>>(
      delta, reinterpret_cast<const float4*>(alm), c->ng, c->n, c->p.nbins, c->d_gq, partials);
  return cudaGetLastError() == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
}

template <int NBP>
int mass_impl(const zeta_ctx* c, const unsigned long long* hist, int l, double* partials, cudaStream_t s) {
  StageScope prof(c, ST_MASS, 1, s);
  const size_t sm = smem_mass<NBP>();
  if (prep(k_gram_mass<NBP>, sm)) return ZETA_ECUDA;
  const float* jt = c->d_jtab + static_cast<long long>(l) * c->nn2 * (4 * ((c->p.nbins + 3) / 4));
  k_gram_mass<NBP><<<gram_ctas(c, GK_MASS), kThreads, sm, s>>>(hist, hist + c->nn2, jt, c->nn2, c->p.nbins, partials);
  return cudaGetLastError() == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
}

template <int NBP>
int rows_rb_impl(const zeta_ctx* c, const float* pvals, const float4* s_tq, int64_t np, double* partials, int grid,
                 cudaStream_t s) {
  if constexpr (NBP <= 20) {
    const size_t smr = smem_node_rb<NBP, 2>();
    if (prep(k_gram_node_rb<NBP, 2>, smr)) return ZETA_ECUDA;
    k_gram_node_rb<NBP, 2><<<grid, kRbThreads, smr, s>>>(reinterpret_cast<const float*>(s_tq),
                                                         reinterpret_cast<const unsigned char*>(pvals), np,
                                                         c->p.nbins, partials, c->d_status);
    return cudaGetLastError() == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
  }
  return ZETA_ENOTSUP;
}

}  // namespace

int launch_gram_rows_rb(const zeta_ctx* c, const float* pvals, const float4* s_tq, int64_t np, double* partials,
                        int grid, cudaStream_t s) {
#define ZK_CALL(P) rows_rb_impl<P>(c, pvals, s_tq, np, partials, grid, s)
  ZK_NBP_SWITCH(c->p.nbins, ZK_CALL)
#undef ZK_CALL
}

int gram_ctas(const zeta_ctx* c, int kind) {
  int per = c->tune[kind];
  if (per < 1) per = 1;
  if (kind == GK_TC && c->p.gram == ZETA_GRAM_TF32) per *= 2;  // the TF32 kernel holds two CTAs per SM
  int g = c->num_sms * per;
  return g > kMaxCtas ? kMaxCtas : g;
}

int launch_gram_node(const zeta_ctx* c, const float* delta, const float* alm, double* partials, cudaStream_t s,
                     bool bf16) {
#define ZK_CALL(P) node_impl<P>(c, delta, alm, partials, s, bf16)
  ZK_NBP_SWITCH(c->p.nbins, ZK_CALL)
#undef ZK_CALL
}

int launch_gram_gamma(const zeta_ctx* c, const float* delta, const float* alm, double* partials, cudaStream_t s) {
  if (c->p.dsup == 2) {
#define ZK_CALL(P) gamma_impl<P, 2>(c, delta, alm, partials, s)
    ZK_NBP_SWITCH(c->p.nbins, ZK_CALL)
#undef ZK_CALL
  } else if (c->p.dsup == 3) {
#define ZK_CALL(P) gamma_impl<P, 5>(c, delta, alm, partials, s)
    ZK_NBP_SWITCH(c->p.nbins, ZK_CALL)
#undef ZK_CALL
  } else {
#define ZK_CALL(P) gamma_impl<P, 4>(c, delta, alm, partials, s)
    ZK_NBP_SWITCH(c->p.nbins, ZK_CALL)
#undef ZK_CALL
  }
}

int launch_mass_hist(const zeta_ctx* c, const float2* dhat, unsigned long long* hist, cudaStream_t s,
                     const float* table1d) {
  StageScope prof(c, ST_MASS, 2, s);
  // hist[0 .. nn2) the fixed-point sums, hist[nn2] the bits of max w
  if (cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * (c->nn2 + 1), s) != cudaSuccess) return ZETA_ECUDA;
  const int grid = c->num_sms * 8;
  const float* t = table1d ? table1d : c->d_mhat;
  k_mass_max<<<grid, kThreads, 0, s>>>(dhat, t, c->n, hist + c->nn2);
  k_mass_hist<<<grid, kThreads, 0, s>>>(dhat, t, c->n, hist + c->nn2, hist);
  return cudaGetLastError() == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
}

// out[b] = (1 / *wdiv) sum_cta partials[cta][b], the CTAs in order (one thread per b).
__global__ void k_reduce_vec(const double* __restrict__ part, int nparts, int nb, const double* __restrict__ wdiv,
                             double* __restrict__ out) {
  const int b = threadIdx.x;
  if (b >= nb) return;
  double sum = 0.0;
  for (int k = 0; k < nparts; ++k) sum += part[static_cast<long long>(k) * nb + b];
  out[b] = sum / *wdiv;
}

int launch_reduce_vec(const zeta_ctx* c, const double* partials, int nparts, const double* wdiv, double* out,
                      cudaStream_t s) {
  StageScope prof(c, ST_REDUCE, 1, s);
  k_reduce_vec<<<1, 32, 0, s>>>(partials, nparts, c->p.nbins, wdiv, out);
  return cudaGetLastError() == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
}

int launch_xi_hist(const zeta_ctx* c, const unsigned long long* hist, int nout, const double* radii, double* out,
                   cudaStream_t s) {
  StageScope prof(c, ST_MASS, 1, s);
  const int nbp = 4 * ((c->p.nbins + 3) / 4);
  const double kunit = 2.0 * 3.14159265358979323846 / c->p.box;
  k_xi_hist<<<nout, 256, 0, s>>>(hist, hist + c->nn2, c->nn2, c->d_jtab, nbp, c->d_wprim, static_cast<double>(c->ng),
                                 kunit, radii, c->p.tophat, radii ? 1 : 0, out);
  return cudaGetLastError() == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
}

int launch_mass(const zeta_ctx* c, const unsigned long long* hist, int l, double* partials, cudaStream_t s) {
#define ZK_CALL(P) mass_impl<P>(c, hist, l, partials, s)
  ZK_NBP_SWITCH(c->p.nbins, ZK_CALL)
#undef ZK_CALL
}

int launch_reduce(const zeta_ctx* c, const double* partials, int nparts, double scale, const double* wdiv,
                  double* out, cudaStream_t s, bool store) {
  StageScope prof(c, ST_REDUCE, 1, s);
  const int nb = c->p.nbins;
  k_reduce<<<(nb * nb + 7) / 8, 256, 0, s>>>(partials, nparts, nb, scale, wdiv, out, store ? 1 : 0);
  return cudaGetLastError() == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
}

int launch_reduce_lm(const zeta_ctx* c, const double* slots, int nforms, int part_form, double* zeta, cudaStream_t s) {
  StageScope prof(c, ST_REDUCE, 1, s);
  const int total = nforms * (c->p.lmax + 1) * c->p.nbins * c->p.nbins;
  k_reduce_lm<<<(total + 255) / 256, 256, 0, s>>>(slots, nforms, part_form, c->p.lmax, c->p.nbins, zeta);
  return cudaGetLastError() == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
}

}  // namespace zk
