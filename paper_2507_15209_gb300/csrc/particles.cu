// Particle form of the method on sm_103a (Fig. 1 step (6), Eq. DDD-sum-privertex):
// P_lm[b1][b2] = (1/W) sum_p w_p f_b1(x_p) f_b2(x_p), f_b(x) = sum_l beta_D(x/H - l) a_lm(l; b).
//
// Two phases per (l, m):
//   interpolation  f_b(x_p) for every sorted particle, written as rows [particle][bins]
//                  (k_interp_part from a shared-memory copy of the tile halo; k_interp_part_l1
//                  for tile batches below the staging threshold);
//   Gram           the weighted Gram of those rows (k_gram_rows, the machinery of gram.cuh).
// Splitting them keeps the Gram's float64 accumulators out of the interpolation kernel, which
// then runs three CTAs per SM.
#include "gram.cuh"

namespace zk {
namespace {

constexpr int kPBP = 128;  // particles per tile batch

template <int D>
struct Halo {
  static constexpr int HD = kTile + D - 1;          // nodes per side
  static constexpr int XP = D == 4 ? 12 : 10;       // row pitch (float4)
  static constexpr int PP = D == 4 ? HD * XP : 92;  // plane pitch (float4)
  static constexpr int SIZE = HD * PP;              // float4 per slot
  static constexpr int SLOT = (SIZE * 16 + 127) / 128 * 128 / 16;  // ring slot stride, 128-byte multiple
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

// ---------------------------------------------------------------------------------------
// Interpolation from the tile halo in shared memory.
//
// Tiles of 8^3 cells in Morton order (neighbouring CTAs on neighbouring tiles, so halo re-reads
// hit L2), batches of up to kPBP particles of a tile; a batch with at least `staged_min`
// particles is handled here.  Warps 0 and 1 are producers: for every (batch, bin group) item
// they copy the (8 + D - 1)^3 halo nodes of that group (float4) into the next slot of a
// kKS-slot ring with 16-byte cp.async (periodic wrap in the address; one linear offset for a
// tile away from the box faces), and each producer thread arrives on the slot's `full`
// mbarrier once its copies have landed.  The other warps consume the items in the same order:
// wait on `full`, interpolate, and arrive on the slot's `empty` mbarrier, which the producers
// wait on before refilling the slot; so the consumer warps never wait for each other between
// bin groups.  (Tiled tensor copies of the halo box were measured too: they left the L2 hit
// rate at 39 % against 63 % for these copies and tripled the DRAM reads.)  Each particle's D^3 stencil is read by 8 lanes (rows padded so
// that the 8 lanes of one shared-memory phase hit distinct banks); the weight products are
// formed once per particle and the 8-lane sum is a reduce-scatter.  A particle whose cell is
// not inside its tile (only for inconsistent or non-finite input) reads global memory.  Every
// wait is bounded and latches ZETA_ETIMEOUT in the status word.
constexpr int kIThreads = 256;          // two producer warps and six consumer warps
constexpr int kPW = 2;                  // producer warps
constexpr int kCons = kIThreads - 32 * kPW;  // consumer threads
constexpr int kCW = kCons / 32;         // consumer warps
constexpr int kKS = 2;                  // halo ring slots

template <int NBP, int D>
struct InterpSmem {
  static constexpr int NBS = NBP + 4;          // shared row stride of the values
  static constexpr int PW = D == 4 ? 20 : 8;   // weights per particle
  static constexpr size_t HALO = static_cast<size_t>(kKS) * Halo<D>::SLOT * sizeof(float4);
  static constexpr size_t VALS = static_cast<size_t>(kPBP) * NBS * sizeof(float);
  static constexpr size_t ORG = kPBP * sizeof(int4);
  static constexpr size_t BW = static_cast<size_t>(kPBP) * PW * sizeof(float);
  static constexpr size_t BYTES = HALO + VALS + ORG + BW + 2 * kKS * sizeof(unsigned long long);
};

__device__ __forceinline__ void consumer_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kCons) : "memory"); }

// Per-particle setup shared by both interpolation kernels: stencil origin, the in-tile halo
// index (or -1), and the weights in the order the gather lanes read them.  From the prepared
// cell (linear index, n = 2^lg) and in-cell offsets of the particle: integer and float32
// arithmetic only.
template <int D, int PW>
__device__ __forceinline__ void particle_setup(int cell, float4 tq, int n, int lg, int tx, int ty, int tz,
                                               bool staged, const float* __restrict__ dtab, int4& org, float* pw) {
  using H = Halo<D>;
  constexpr int OFF = D / 2 - 1;
  float wx[D], wy[D], wz[D];
  const int cix[3] = {cell & (n - 1), (cell >> lg) & (n - 1), cell >> (2 * lg)};
  if (D == 4 && dtab != nullptr) {  // Daubechies basis (the cell is one below floor(u))
    daub4_weights(tq.x, dtab, wx);
    daub4_weights(tq.y, dtab, wy);
    daub4_weights(tq.z, dtab, wz);
  } else {
    bsw<D>(tq.x, wx);
    bsw<D>(tq.y, wy);
    bsw<D>(tq.z, wz);
  }
  const int lx = cix[0] - tx * kTile, ly = cix[1] - ty * kTile, lz = cix[2] - tz * kTile;
  const bool inside = lx >= 0 && lx < kTile && ly >= 0 && ly < kTile && lz >= 0 && lz < kTile;
  org = make_int4(cix[0] - OFF, cix[1] - OFF, cix[2] - OFF, (staged && inside) ? lz * H::PP + ly * H::XP + lx : -1);
  if (D == 4) {  // lane (ox, oy0) takes nodes (oz, oy0 + 2 j): products [oy0][oz][j], then wx
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
}

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

// The producer's walk over staged (tile, batch, group) items, identical to the consumers'; the
// next tile's particle range is loaded one tile ahead.
struct ItemWalk {
  TileWalk walk;
  int ngrp, staged_min;
  long long pk = 0, s0 = 0, s1 = 0, bs = 0, n0 = 0, n1 = 0;
  int tx = 0, ty = 0, tz = 0, q = -1, nx = 0, ny = 0, nz = 0;
  bool valid = false, have_next = false;
  __device__ __forceinline__ void start() {
    valid = walk.tile(0, s0, s1, tx, ty, tz);
    have_next = walk.tile(1, n0, n1, nx, ny, nz);
    bs = s0;
  }
  __device__ __forceinline__ void next() {
    ++q;
    while (valid) {
      if (bs < s1) {
        const long long c = s1 - bs;
        if ((c < kPBP ? c : kPBP) >= staged_min && q < ngrp) return;
        bs += kPBP;  // batch done (or not staged)
        q = 0;
      } else {
        ++pk;
        valid = have_next;
        s0 = n0;
        s1 = n1;
        tx = nx;
        ty = ny;
        tz = nz;
        have_next = walk.tile(pk + 1, n0, n1, nx, ny, nz);
        bs = s0;
        q = 0;
      }
    }
  }
};

template <int NBP, int D>
__global__ void __launch_bounds__(kIThreads, 3)
    k_interp_part(const int* __restrict__ s_cell, const float4* __restrict__ s_tq,
                  const long long* __restrict__ tile_start, const float4* __restrict__ f4, long long ng, int n, int nb,
                  int staged_min, const float* __restrict__ dtab, float* __restrict__ pvals, int* __restrict__ status) {
  using H = Halo<D>;
  using S = InterpSmem<NBP, D>;
  constexpr int PW = S::PW;
  constexpr int SLOT = Halo<D>::SLOT;
  extern __shared__ __align__(128) unsigned char smq[];
  float4* halo = reinterpret_cast<float4*>(smq);                                    // [kKS][SIZE]
  float* vals = reinterpret_cast<float*>(smq + S::HALO);                            // [kPBP][NBS]
  int4* org = reinterpret_cast<int4*>(smq + S::HALO + S::VALS);                     // [kPBP]
  float* bw = reinterpret_cast<float*>(smq + S::HALO + S::VALS + S::ORG);           // [kPBP][PW]
  unsigned long long* full = reinterpret_cast<unsigned long long*>(smq + S::HALO + S::VALS + S::ORG + S::BW);
  unsigned long long* empty = full + kKS;
  const int ngrp = (nb + 3) / 4;
  const int nt = n / kTile;
  const TileWalk walk{tile_start, static_cast<long long>(nt) * nt * nt, nt};
  constexpr int OFF = D / 2 - 1;
  const int mask = n - 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kKS; ++s) {
      mbar_init(&full[s], 32 * kPW);
      mbar_init(&empty[s], kCW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp < kPW) {  // ---- producers
    const int pt = threadIdx.x;
    const int n2 = n * n;
    ItemWalk it{walk, ngrp, staged_min};
    it.start();
    long long i = 0;
    bool ok = true;
    for (;;) {
      it.next();
      if (!it.valid) break;
      const int s = static_cast<int>(i % kKS);
      const long long u = i / kKS;
      if (u > 0 && !mbar_wait(&empty[s], static_cast<uint32_t>((u - 1) & 1))) {
        ok = false;
        break;
      }
      float4* dst = halo + s * SLOT;
      const float4* src = f4 + it.q * ng;
      const int hx = it.tx * kTile - OFF, hy = it.ty * kTile - OFF, hz = it.tz * kTile - OFF;
      // this thread's nodes e = pt + k * NP of the halo, (x, y, z) stepped with carries
      constexpr int NP = 32 * kPW, HD = H::HD;
      constexpr int SX = NP % HD, SY = (NP / HD) % HD, SZ = NP / (HD * HD);
      int x = pt % HD, y = (pt / HD) % HD, z = pt / (HD * HD);
      const bool inner = it.tx >= 1 && it.tx <= nt - 2 && it.ty >= 1 && it.ty <= nt - 2 && it.tz >= 1 &&
                         it.tz <= nt - 2;
      if (inner) {  // no periodic wrap: one linear offset
        const float4* base = src + (hz * n2 + hy * n + hx);
        for (; z < HD;) {
          cp_async16(dst + z * H::PP + y * H::XP + x, base + (z * n2 + y * n + x));
          x += SX;
          y += SY;
          z += SZ;
          if (x >= HD) { x -= HD; ++y; }
          if (y >= HD) { y -= HD; ++z; }
        }
      } else {
        for (; z < HD;) {
          cp_async16(dst + z * H::PP + y * H::XP + x,
                     src + (((hz + z) & mask) * n2 + ((hy + y) & mask) * n + ((hx + x) & mask)));
          x += SX;
          y += SY;
          z += SZ;
          if (x >= HD) { x -= HD; ++y; }
          if (y >= HD) { y -= HD; ++z; }
        }
      }
      // arrives on `full` once this thread's copies have landed
      asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(&full[s])) : "memory");
      ++i;
    }
    if (!ok && pt == 0) atomicOr(status, 2);
    // copies of the last items may still be landing if the consumers stopped early
    for (long long j = (i > kKS ? i - kKS : 0); j < i; ++j)
      mbar_wait(&full[j % kKS], static_cast<uint32_t>((j / kKS) & 1));
    return;
  }

  // ---- consumers
  const int ct = threadIdx.x - 32 * kPW, cw = warp - kPW;
  const int l8 = lane & 7;
  const int lg = __ffs(n) - 1;
  long long ci = 0;
  bool ok = true;
  long long s0 = 0, s1 = 0;
  int tx = 0, ty = 0, tz = 0;
  // the next tile's particle range and this thread's particle of the next batch are loaded one
  // step ahead, so their global-memory latency is not on the consumers' critical path
  long long n0 = 0, n1 = 0;
  int nx = 0, ny = 0, nz = 0;
  bool have_next = walk.tile(0, n0, n1, nx, ny, nz);
  long long pf_bs = -1;
  int pf_cell = 0;
  float4 pf_tq = make_float4(0.f, 0.f, 0.f, 0.f);
  for (long long k = 0; have_next; ++k) {
    s0 = n0;
    s1 = n1;
    tx = nx;
    ty = ny;
    tz = nz;
    have_next = walk.tile(k + 1, n0, n1, nx, ny, nz);
    for (long long bs = s0; bs < s1; bs += kPBP) {
      const int cnt = static_cast<int>((s1 - bs) < kPBP ? (s1 - bs) : kPBP);
      if (cnt < staged_min) continue;  // k_interp_part_l1 takes this batch
      if (ct < cnt) {
        const bool pre = pf_bs == bs;
        particle_setup<D, PW>(pre ? pf_cell : s_cell[bs + ct], pre ? pf_tq : s_tq[bs + ct], n, lg, tx, ty, tz,
                              true, dtab, org[ct], bw + ct * PW);
      }
      {  // prefetch the next batch (this tile's next one, or the first of the next tile)
        const bool same = bs + kPBP < s1;
        const long long nb0 = same ? bs + kPBP : (have_next ? n0 : -1);
        const long long nend = same ? s1 : n1;
        pf_bs = nb0;
        if (nb0 >= 0 && nb0 + ct < nend && ct < kPBP) {
          pf_cell = s_cell[nb0 + ct];
          pf_tq = s_tq[nb0 + ct];
        }
      }
      consumer_sync();  // setup visible; the previous batch's value rows are written out
      for (int q = 0; q < ngrp; ++q, ++ci) {
        const int s = static_cast<int>(ci % kKS);
        if (ok && !mbar_wait(&full[s], static_cast<uint32_t>((ci / kKS) & 1))) ok = false;
        const float4* hb = halo + s * SLOT;
        const float4* gsrc = f4 + q * ng;
        for (int pb = cw * 4; pb < cnt; pb += kCW * 4) {  // warp-uniform
          const int p = pb + (lane >> 3);
          float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
          if (p < cnt && ok) {
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
          if (p < cnt && !(l8 & 1)) vals[p * S::NBS + 4 * q + (l8 >> 1)] = tot;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);  // this warp is done with the slot
      }
      consumer_sync();  // the batch's value rows are complete
      float4* dst = reinterpret_cast<float4*>(pvals + bs * NBP);
      for (int e = ct; e < cnt * (NBP / 4); e += kCons) {
        const int p = e / (NBP / 4), j = e % (NBP / 4);
        dst[e] = *reinterpret_cast<const float4*>(vals + p * S::NBS + 4 * j);
      }
    }
  }
  if (!ok && ct == 0) atomicOr(status, 2);
}

// ---------------------------------------------------------------------------------------
// Interpolation through L1, for tile batches below the staging threshold.  One CTA of 512
// threads works on one tile batch at a time, so the tile's halo of every bin group (about
// 100 KB for 20 bins) stays resident in L1 while all warps read it.  A particle's stencil is
// read by D * ngrp lanes at once -- lane (q, ox) accumulates the D^2 rows of bin group q at x
// offset ox with independent 16-byte loads -- and the D partial sums of a group are combined
// by a reduce-scatter over the x lanes.
constexpr int kThreadsL1 = 512;

template <int NBP, int D>
struct InterpL1Smem {
  static constexpr int NBS = NBP + 4;
  static constexpr int PW = InterpSmem<NBP, D>::PW;
  static constexpr size_t BYTES = static_cast<size_t>(kPBP) * NBS * sizeof(float) + kPBP * sizeof(int4) +
                                  static_cast<size_t>(kPBP) * PW * sizeof(float);
};

template <int NBP, int D>
__global__ void __launch_bounds__(kThreadsL1, 1)
    k_interp_part_l1(const int* __restrict__ s_cell, const float4* __restrict__ s_tq,
                     const long long* __restrict__ tile_start, const float4* __restrict__ f4, long long ng, int n,
                     int nb, int staged_min, const float* __restrict__ dtab, float* __restrict__ pvals) {
  using S = InterpL1Smem<NBP, D>;
  constexpr int PW = S::PW;
  extern __shared__ __align__(16) unsigned char smraw[];
  float* vals = reinterpret_cast<float*>(smraw);        // [kPBP][NBS]
  int4* org = reinterpret_cast<int4*>(vals + kPBP * S::NBS);  // [kPBP]
  float* bw = reinterpret_cast<float*>(org + kPBP);     // [kPBP][PW]
  const int ngrp = (nb + 3) / 4;
  const int nt = n / kTile;
  const TileWalk walk{tile_start, static_cast<long long>(nt) * nt * nt, nt};
  const int mask = n - 1, n2 = n * n;
  const int lg = __ffs(n) - 1;
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
    for (long long bs = s0; bs < s1; bs += kPBP) {
      const int cnt = static_cast<int>((s1 - bs) < kPBP ? (s1 - bs) : kPBP);
      if (cnt >= staged_min) continue;  // the staged kernel takes this batch
      __syncthreads();  // the previous batch's value rows are written out
      if (threadIdx.x < cnt)
        particle_setup<D, PW>(s_cell[bs + threadIdx.x], s_tq[bs + threadIdx.x], n, lg, tx, ty, tz, false, dtab,
                              org[threadIdx.x], bw + threadIdx.x * PW);
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
          if (D == 4) {  // weights [oy0][oz][j] (node oy = oy0 + 2 j), then wx
            const float wxo = w[16 + ox];
#pragma unroll
            for (int oz = 0; oz < 4; ++oz)
#pragma unroll
              for (int oy = 0; oy < 4; ++oy) {
                const float c = w[(oy & 1) * 8 + oz * 2 + (oy >> 1)] * wxo;
                const float4 v = __ldg(gq4 + (zr[oz] + yr[oy] + xo));
                acc.x = fmaf(c, v.x, acc.x);
                acc.y = fmaf(c, v.y, acc.y);
                acc.z = fmaf(c, v.z, acc.z);
                acc.w = fmaf(c, v.w, acc.w);
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
        float* dst = vals + p * S::NBS + 4 * q;
        if (D == 4) {
          const bool hi = ox & 2;
          const float sa = hi ? acc.x : acc.z, sb = hi ? acc.y : acc.w;
          float ka = hi ? acc.z : acc.x, kb = hi ? acc.w : acc.y;
          ka += __shfl_xor_sync(0xffffffffu, sa, 2);
          kb += __shfl_xor_sync(0xffffffffu, sb, 2);
          const bool odd = ox & 1;
          const float sv = odd ? ka : kb;
          float kk = odd ? kb : ka;
          kk += __shfl_xor_sync(0xffffffffu, sv, 1);
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
      float4* out = reinterpret_cast<float4*>(pvals + bs * NBP);
      for (int e = threadIdx.x; e < cnt * (NBP / 4); e += blockDim.x) {
        const int p = e / (NBP / 4), j = e % (NBP / 4);
        out[e] = *reinterpret_cast<const float4*>(vals + p * S::NBS + 4 * j);
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// Weighted Gram of the interpolated rows: points = sorted particles, v = f_b(x_p) (rows of
// NBP floats), w = w_p (0 for a non-finite particle).  Persistent CTAs over chunks of kPB
// rows; the next chunk is loaded into registers while the current one is contracted.
template <int NBP>
__global__ void __launch_bounds__(kThreads) k_gram_rows(const float* __restrict__ pvals,
                                                        const float4* __restrict__ s_tq, long long np, int nb,
                                                        double* __restrict__ partials) {
  using G = Gram<NBP>;
  constexpr int GV = NBP / 4;
  extern __shared__ __align__(16) unsigned char smraw[];
  float* vals = reinterpret_cast<float*>(smraw);
  float* wts = vals + kPB * G::NBS;
  double* red = reinterpret_cast<double*>(smraw);  // reused after the main loop
  const int pr = threadIdx.x % G::NPAIR, grp = threadIdx.x / G::NPAIR;
  int b1 = 0, b2 = 0;
  pair_blocks(pr, G::NBLK, b1, b2);
  GramAcc<NBP> g;
  g.init();
  const long long nchunk = (np + kPB - 1) / kPB;
  float wnext = 0.f;
  float4 vnext[GV];
  auto fetch = [&](long long c) {
    const long long p = c * kPB + threadIdx.x;
    if (p < np) {
      wnext = __ldg(s_tq + p).w;  // 0 for a non-finite particle
      const float4* row = reinterpret_cast<const float4*>(pvals + p * NBP);
#pragma unroll
      for (int j = 0; j < GV; ++j) vnext[j] = __ldg(row + j);
    } else {
      wnext = 0.f;
#pragma unroll
      for (int j = 0; j < GV; ++j) vnext[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  long long ch = blockIdx.x;
  if (ch < nchunk) fetch(ch);
  for (; ch < nchunk; ch += gridDim.x) {
    const long long left = np - ch * kPB;
    const int cnt = left < kPB ? static_cast<int>(left) : kPB;
    __syncthreads();
    wts[threadIdx.x] = wnext;
#pragma unroll
    for (int j = 0; j < GV; ++j) *reinterpret_cast<float4*>(vals + threadIdx.x * G::NBS + 4 * j) = vnext[j];
    __syncthreads();
    if (ch + gridDim.x < nchunk) fetch(ch + gridDim.x);
    if (grp < G::NGRP) g.add(vals, wts, cnt, b1, b2, grp);
  }
  __syncthreads();
  cta_store<NBP>(g, red, nb, partials + static_cast<long long>(blockIdx.x) * nb * nb);
}

template <int NBP>
size_t smem_rows() {
  using G = Gram<NBP>;
  const size_t main = (kPB * G::NBS + kPB) * sizeof(float);
  return main > red_bytes<NBP>() ? main : red_bytes<NBP>();
}

// Which interpolation kernels run for the staging threshold: the staged one if some batch
// can reach it, the L1 one if some batch can fall below it.
inline bool part_staged_on(const zeta_ctx* c) { return c->staged_min <= kPBP; }
inline bool part_l1_on(const zeta_ctx* c) { return c->staged_min > 1; }
constexpr int kRowsCtasPerSm = 2;

template <int NBP, int D>
int part_impl(const zeta_ctx* c, const int* s_cell, const float4* s_tq, const int64_t* tile_start, int64_t np,
              const float* alm, float* pvals, double* partials, cudaStream_t s) {
  StageScope prof(c, ST_GRAM_PART, part_staged_on(c) + part_l1_on(c) + 1, s);
  const long long* ts = reinterpret_cast<const long long*>(tile_start);
  const float4* f4 = reinterpret_cast<const float4*>(alm);
  if (part_staged_on(c)) {
    const size_t sm = InterpSmem<NBP, D>::BYTES;
    if (prep(k_interp_part<NBP, D>, sm)) return ZETA_ECUDA;
    k_interp_part<NBP, D><<<gram_ctas(c, GK_PART), kIThreads, sm, s>>>(s_cell, s_tq, ts, f4, c->ng, c->n,
                                                                       c->p.nbins, c->staged_min, c->d_daub, pvals,
                                                                       c->d_status);
  }
  if (part_l1_on(c)) {
    const size_t sm = InterpL1Smem<NBP, D>::BYTES;
    if (prep(k_interp_part_l1<NBP, D>, sm)) return ZETA_ECUDA;
    k_interp_part_l1<NBP, D><<<c->num_sms, kThreadsL1, sm, s>>>(s_cell, s_tq, ts, f4, c->ng, c->n, c->p.nbins,
                                                                c->staged_min, c->d_daub, pvals);
  }
  if constexpr (NBP <= 20) {  // register-blocked Gram of the rows (sums.cu), one CTA per SM
    return launch_gram_rows_rb(c, pvals, s_tq, np, partials, gram_particle_parts(c), s);
  }
  const size_t sm = smem_rows<NBP>();
  if (prep(k_gram_rows<NBP>, sm)) return ZETA_ECUDA;
  k_gram_rows<NBP><<<gram_particle_parts(c), kThreads, sm, s>>>(pvals, s_tq, np, c->p.nbins, partials);
  return cudaGetLastError() == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
}

// Per-CTA sums of w_p f_b(x_p) over the interpolated rows (the particle form of the 2PCF): each
// thread sums a fixed stride of particles in float32 runs of at most kFlush particles, flushed to
// float64; the CTA adds its threads in a fixed order.  partials[cta][nb].
template <int NBP>
__global__ void __launch_bounds__(kThreads) k_row_sums(const float* __restrict__ pvals, const float4* __restrict__ s_tq,
                                                       long long np, int nb, double* __restrict__ partials) {
  __shared__ double red[kThreads];
  double dacc[NBP];
  float acc[NBP];
#pragma unroll
  for (int b = 0; b < NBP; ++b) {
    dacc[b] = 0.0;
    acc[b] = 0.f;
  }
  int pending = 0;
  for (long long p = blockIdx.x * static_cast<long long>(kThreads) + threadIdx.x; p < np;
       p += static_cast<long long>(kThreads) * gridDim.x) {
    const float w = __ldg(s_tq + p).w;
    const float4* row = reinterpret_cast<const float4*>(pvals + p * NBP);
#pragma unroll
    for (int j = 0; j < NBP / 4; ++j) {
      const float4 v = __ldg(row + j);
      acc[4 * j] = fmaf(w, v.x, acc[4 * j]);
      acc[4 * j + 1] = fmaf(w, v.y, acc[4 * j + 1]);
      acc[4 * j + 2] = fmaf(w, v.z, acc[4 * j + 2]);
      acc[4 * j + 3] = fmaf(w, v.w, acc[4 * j + 3]);
    }
    if (++pending == kFlush) {
#pragma unroll
      for (int b = 0; b < NBP; ++b) {
        dacc[b] += acc[b];
        acc[b] = 0.f;
      }
      pending = 0;
    }
  }
#pragma unroll
  for (int b = 0; b < NBP; ++b) {
    if (b >= nb) break;  // uniform across the CTA
    red[threadIdx.x] = dacc[b] + static_cast<double>(acc[b]);
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) partials[static_cast<long long>(blockIdx.x) * nb + b] = red[0];
    __syncthreads();
  }
}

template <int NBP, int D>
int xi_impl(const zeta_ctx* c, const int* s_cell, const float4* s_tq, const int64_t* tile_start, int64_t np,
            const float* alm, float* pvals, double* partials, cudaStream_t s) {
  StageScope prof(c, ST_GRAM_PART, part_staged_on(c) + part_l1_on(c) + 1, s);
  const long long* ts = reinterpret_cast<const long long*>(tile_start);
  const float4* f4 = reinterpret_cast<const float4*>(alm);
  if (part_staged_on(c)) {
    const size_t sm = InterpSmem<NBP, D>::BYTES;
    if (prep(k_interp_part<NBP, D>, sm)) return ZETA_ECUDA;
    k_interp_part<NBP, D><<<gram_ctas(c, GK_PART), kIThreads, sm, s>>>(s_cell, s_tq, ts, f4, c->ng, c->n,
                                                                       c->p.nbins, c->staged_min, c->d_daub, pvals,
                                                                       c->d_status);
  }
  if (part_l1_on(c)) {
    const size_t sm = InterpL1Smem<NBP, D>::BYTES;
    if (prep(k_interp_part_l1<NBP, D>, sm)) return ZETA_ECUDA;
    k_interp_part_l1<NBP, D><<<c->num_sms, kThreadsL1, sm, s>>>(s_cell, s_tq, ts, f4, c->ng, c->n, c->p.nbins,
                                                                c->staged_min, c->d_daub, pvals);
  }
  k_row_sums<NBP><<<gram_particle_parts(c), kThreads, 0, s>>>(pvals, s_tq, np, c->p.nbins, partials);
  return cudaGetLastError() == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
}

}  // namespace

int gram_particle_parts(const zeta_ctx* c) { return c->p.nbins <= 20 ? c->num_sms : c->num_sms * kRowsCtasPerSm; }

int launch_particle_xi(const zeta_ctx* c, const int* s_cell, const float4* s_tq, const int64_t* tile_start,
                       int64_t np, const float* alm, float* pvals, double* partials, cudaStream_t s) {
  if (c->p.dsup == 2) {
#define ZK_CALL(P) xi_impl<P, 2>(c, s_cell, s_tq, tile_start, np, alm, pvals, partials, s)
    ZK_NBP_SWITCH(c->p.nbins, ZK_CALL)
#undef ZK_CALL
  } else {
#define ZK_CALL(P) xi_impl<P, 4>(c, s_cell, s_tq, tile_start, np, alm, pvals, partials, s)
    ZK_NBP_SWITCH(c->p.nbins, ZK_CALL)
#undef ZK_CALL
  }
}

size_t particle_rows_bytes(const zeta_ctx* c, int64_t np) {
  return sizeof(float) * static_cast<size_t>(np) * nbp_of(c->p.nbins);
}

int launch_gram_particles(const zeta_ctx* c, const int* s_cell, const float4* s_tq, const int64_t* tile_start,
                          int64_t np, const float* alm, float* pvals, double* partials, cudaStream_t s) {
  if (c->p.dsup == 2) {
#define ZK_CALL(P) part_impl<P, 2>(c, s_cell, s_tq, tile_start, np, alm, pvals, partials, s)
    ZK_NBP_SWITCH(c->p.nbins, ZK_CALL)
#undef ZK_CALL
  } else {
#define ZK_CALL(P) part_impl<P, 4>(c, s_cell, s_tq, tile_start, np, alm, pvals, partials, s)
    ZK_NBP_SWITCH(c->p.nbins, ZK_CALL)
#undef ZK_CALL
  }
}

}  // namespace zk
