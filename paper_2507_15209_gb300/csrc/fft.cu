// 3-D DFT stages of the method on sm_103a (Fig. 1 steps (2) and (5)).
//
// Forward (once per catalogue):  delta (real [z][y][x]) -> x-pass R2C -> y-pass -> z-pass
//   gives delta_hat[z][y][nx < n/2]; the x-Nyquist column is dropped because every kernel
//   of the method vanishes on Nyquist planes.
// Inverse (per (l, m) and radial bin; the hot loop):  z-pass that reads delta_hat once
//   per CTA tile and, for every bin of the launch, multiplies by the multipole window
//   K_lm,b(n) = i^l [sqrt(4 pi) jbar_l(|k|; b) / N_g] R_lm(n-hat) (Eqs. 3PCF-multipole-window
//   and SFC-3PCF-vertex) before transforming -> y-pass in place -> x-pass C2R of four
//   fields at a time, written bin-interleaved ([group][z][y][x][4]) so that every
//   consumer reads four bins of a point with one 16-byte load.
//
// Every pass moves a tile of T contiguous complex columns (or RB rows) between HBM and
// shared memory with coalesced accesses and transforms it with the radix-8 shared-memory
// FFT of fft.cuh.
#include <cuda_bf16.h>

#include "fft.cuh"
#include "fftreg.cuh"
#include "zeta_internal.h"

namespace zk {

__constant__ float c_ylm_mm[kMaxL + 1];
__constant__ float c_ylm_a[(kMaxL + 1) * (kMaxL + 1)];
__constant__ float c_ylm_b[(kMaxL + 1) * (kMaxL + 1)];

int set_ylm_constants() {
  double mm[kMaxL + 1], a[(kMaxL + 1) * (kMaxL + 1)], b[(kMaxL + 1) * (kMaxL + 1)];
  host_ylm_constants(mm, a, b);
  float fm[kMaxL + 1], fa[(kMaxL + 1) * (kMaxL + 1)], fb[(kMaxL + 1) * (kMaxL + 1)];
  for (int i = 0; i <= kMaxL; ++i) fm[i] = static_cast<float>(mm[i]);
  for (int i = 0; i < (kMaxL + 1) * (kMaxL + 1); ++i) {
    fa[i] = static_cast<float>(a[i]);
    fb[i] = static_cast<float>(b[i]);
  }
  if (cudaMemcpyToSymbol(c_ylm_mm, fm, sizeof(fm)) != cudaSuccess) return ZETA_ECUDA;
  if (cudaMemcpyToSymbol(c_ylm_a, fa, sizeof(fa)) != cudaSuccess) return ZETA_ECUDA;
  if (cudaMemcpyToSymbol(c_ylm_b, fb, sizeof(fb)) != cudaSuccess) return ZETA_ECUDA;
  return ZETA_OK;
}

// R_lm of the integer wavevector (nx, ny, nz) != 0: fully normalised associated-Legendre
// recurrence in cos(theta) times Re/Im of (sin(theta) e^{i phi})^|m|.
__device__ __forceinline__ float ylm_dev(int l, int m, float nx, float ny, float nz) {
  const float r2 = nx * nx + ny * ny + nz * nz;
  if (r2 == 0.f) return l == 0 ? 0.28209479177387814f : 0.f;
  const float rinv = 1.0f / sqrtf(r2);
  const float ct = nz * rinv, sx = nx * rinv, sy = ny * rinv;
  const int am = m < 0 ? -m : m;
  float cr = 1.f, ci = 0.f;
  for (int k = 0; k < am; ++k) {
    const float t = cr * sx - ci * sy;
    ci = cr * sy + ci * sx;
    cr = t;
  }
  float qm1 = 0.f, qc = c_ylm_mm[am];
  for (int ll = am + 1; ll <= l; ++ll) {
    const float qn = c_ylm_a[ll * (kMaxL + 1) + am] * ct * qc - c_ylm_b[ll * (kMaxL + 1) + am] * qm1;
    qm1 = qc;
    qc = qn;
  }
  const float ang = (m == 0) ? 1.f : 1.41421356237309505f * (m > 0 ? cr : ci);
  return qc * ang;
}

__device__ __forceinline__ int signed_freq(int i, int n) { return i < n / 2 ? i : i - n; }

// two floats as a pair of bfloat16 (round to nearest even), the first in the low half
__device__ __forceinline__ uint32_t bf16x2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// ---------------------------------------------------------------------------------------
// Threads per CTA of a register-staged transform: eight points per thread, at most MAXT.
template <int L, int C, int MAXT>
struct RegThreads {
  static constexpr int V = L * C / 8;
  static constexpr int NT = V < MAXT ? V : MAXT;
};

// Complex pencils along y (AXIS 1) or z (AXIS 2), in place; grid (nc/T, n, nfields).
template <int N, int T, bool INV, int AXIS>
__global__ void __launch_bounds__(RegThreads<N, T, 512>::NT) k_fft_axis(float2* __restrict__ data, long long fstride,
                                                                      const float2* __restrict__ twg) {
  constexpr int NC = N / 2;
  constexpr int NT = RegThreads<N, T, 512>::NT;
  extern __shared__ float2 sm[];
  float2* tw = sm;                     // per-stage twiddles
  float2* ex = sm + StageTw<N>::SIZE;  // [N][T]
  const int x0 = blockIdx.x * T;
  const long long o = blockIdx.y;
  float2* d = data + blockIdx.z * fstride;
  const long long stride = (AXIS == 1) ? NC : static_cast<long long>(N) * NC;
  const long long base = (AXIS == 1) ? o * N * NC + x0 : o * NC + x0;
  stage_tw_fill<N>(tw, twg, 1);
  auto load = [&](int col, int k) { return d[base + k * stride + col]; };
  auto store = [&](int col, int k, float2 v) { d[base + k * stride + col] = v; };
  __syncthreads();
  fft_reg<N, T, NT, INV, false>(ex, T, tw, load, store);
}

// Real rows -> half spectrum without Nyquist; grid (n*n/RB).
template <int N, int RB>
__global__ void __launch_bounds__(256) k_r2c_x(const float* __restrict__ in, float2* __restrict__ out,
                                               const float2* __restrict__ twg) {
  constexpr int NC = N / 2, PS = RB + 1;
  extern __shared__ float2 sm[];
  float2* tw = sm;          // W_N^e, e < N
  float2* tw2 = sm + N;     // W_NC^e = W_N^{2e}, e < NC
  float2* buf = tw2 + NC;   // [NC][PS]
  const long long r0 = static_cast<long long>(blockIdx.x) * RB;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = twg[i];
  for (int i = threadIdx.x; i < NC; i += blockDim.x) tw2[i] = twg[2 * i];
  const float2* rin = reinterpret_cast<const float2*>(in);
  for (int idx = threadIdx.x; idx < NC * RB; idx += blockDim.x) {
    const int r = idx / NC, j = idx % NC;
    buf[j * PS + r] = rin[(r0 + r) * NC + j];
  }
  fft_smem<NC, false>(buf, PS, RB, tw2);
  for (int idx = threadIdx.x; idx < NC * RB; idx += blockDim.x) {
    const int r = idx / NC, k = idx % NC;
    const float2 zk = buf[fft_pos_of<NC>(k) * PS + r];
    const float2 zm = cconj(buf[fft_pos_of<NC>((NC - k) & (NC - 1)) * PS + r]);
    const float2 e = cscale(cadd(zk, zm), 0.5f);
    const float2 dd = csub(zk, zm);
    const float2 od = make_float2(0.5f * dd.y, -0.5f * dd.x);  // (zk - conj zm) / (2i)
    out[(r0 + r) * NC + k] = cadd(e, cmul(tw[k], od));
  }
}

// Half spectrum (x-Nyquist implicitly zero) -> real rows, in place; grid (n*n/RB, nfields).
template <int N, int RB>
__global__ void __launch_bounds__(256) k_c2r_x(float2* __restrict__ data, long long fstride,
                                               const float2* __restrict__ twg) {
  constexpr int NC = N / 2, PS = RB + 1;
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* tw2 = sm + N;
  float2* buf = tw2 + NC;
  float2* d = data + blockIdx.y * fstride;
  const long long r0 = static_cast<long long>(blockIdx.x) * RB;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = twg[i];
  for (int i = threadIdx.x; i < NC; i += blockDim.x) tw2[i] = twg[2 * i];
  for (int idx = threadIdx.x; idx < NC * RB; idx += blockDim.x) {
    const int r = idx / NC, k = idx % NC;
    buf[k * PS + r] = d[(r0 + r) * NC + k];
  }
  __syncthreads();
  // Z[k] = (X[k] + conj X[NC-k]) + i e^{+2 pi i k/N} (X[k] - conj X[NC-k]), X[NC] = 0
  constexpr int NP = NC / 2 + 1;
  for (int idx = threadIdx.x; idx < NP * RB; idx += blockDim.x) {
    const int r = idx / NP, k = idx % NP;
    const int kp = NC - k;  // partner (== NC for k == 0, which is the zero Nyquist)
    const float2 xk = buf[k * PS + r];
    const float2 xp = (k == 0) ? make_float2(0.f, 0.f) : buf[kp * PS + r];
    const float2 wk = cconj(tw[k]);
    const float2 zk = cadd(cadd(xk, cconj(xp)), mul_i(cmul(wk, csub(xk, cconj(xp)))));
    if (k != 0 && kp != k) {
      const float2 wp = cconj(tw[kp]);
      const float2 zp = cadd(cadd(xp, cconj(xk)), mul_i(cmul(wp, csub(xp, cconj(xk)))));
      buf[kp * PS + r] = zp;
    }
    buf[k * PS + r] = zk;
  }
  fft_smem<NC, true>(buf, PS, RB, tw2);
  for (int idx = threadIdx.x; idx < NC * RB; idx += blockDim.x) {
    const int r = idx / NC, j = idx % NC;
    d[(r0 + r) * NC + j] = buf[fft_pos_of<NC>(j) * PS + r];
  }
}

// e^{i pi j / 16} (j mod 16), from cos(a pi / 16), a = 0..8, written out; with j a compile-time
// constant the factors become instruction operands.
__device__ __forceinline__ float2 root32(int j) {
  constexpr float c[9] = {1.0f,
                          0.980785280403230449f,
                          0.923879532511286756f,
                          0.831469612302545237f,
                          0.707106781186547524f,
                          0.555570233019602225f,
                          0.382683432365089772f,
                          0.195090322016128268f,
                          0.0f};
  const int a = j & 15;
  return make_float2(a <= 8 ? c[a] : -c[16 - a], a <= 8 ? c[8 - a] : c[a - 8]);
}

// x-pass of the field reconstruction: C2R of the rows of four fields at once, written as
// one bin-interleaved group [z][y][x][4] (lane j = field 4g + j; missing fields give 0).
// The half-length complex transform takes Z[k] = (X[k] + conj X[NC-k]) + i e^{2 pi i k/N}
// (X[k] - conj X[NC-k]) (X[NC] = 0) straight from global memory; its outputs z[j] =
// (x[2j], x[2j+1]) are gathered in shared memory and leave as float4 bin groups.
// grid (n*n/RB, ngroups); spec holds nf plain half spectra, fstride complex apart.
template <int N, int RB, bool BF16 = false>
__global__ void __launch_bounds__(RegThreads<N / 2, 4 * RB, 256>::NT)
    k_c2r_x4(const float2* __restrict__ spec, long long fstride, int nf, float4* __restrict__ out,
             const float2* __restrict__ twg) {
  constexpr int NC = N / 2, C = 4 * RB, PS = C + 1;
  constexpr int NT = RegThreads<NC, C, 256>::NT;
  extern __shared__ float2 sm[];
  float2* tw = sm;                      // W_N^e, e < N
  float2* tw2 = sm + N;                 // per-stage twiddles of the length-NC transform
  float2* ex = tw2 + StageTw<NC>::SIZE;  // [NC][PS] exchange, then the outputs in natural order
  float2* res = ex;
  const int g = blockIdx.y;
  const long long r0 = static_cast<long long>(blockIdx.x) * RB;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = twg[i];
  stage_tw_fill<NC>(tw2, twg, 2);
  __syncthreads();
  auto store = [&](int c, int j, float2 v) { res[j * PS + c] = v; };
  // z_k = (X_k + conj X_{NC-k}) + i conj(W_N^k) (X_k - conj X_{NC-k}), X_{NC} = 0
  auto packw = [](float2 wk, float2 xk, float2 xp) -> float2 {  // wk = conj(W_N^k)
    return cadd(cadd(xk, cconj(xp)), mul_i(cmul(wk, csub(xk, cconj(xp)))));
  };
  auto pack = [&](int k, float2 xk, float2 xp) -> float2 { return packw(cconj(tw[k]), xk, xp); };
  constexpr int R0 = plan_radix<NC>(0);
  constexpr int PPT = NC * C / NT;
  constexpr int NTASK0 = PPT / R0;
  constexpr int H = NC / R0 / 2;
  constexpr int HS = H >= 1 ? H : 1;  // H = 0 (tiny rows) rules the pairing out below
  constexpr bool MIRROR = (NTASK0 % 2 == 0) && H >= 1 && (NT % HS == 0) && (NTASK0 / 2) * (NT / HS) == C;
  if constexpr (MIRROR) {
    // each thread holds both points of every (k, NC - k) pair: one load per point
    float2 xv[PPT];
    int pts[PPT];
#pragma unroll
    for (int sl = 0; sl < PPT; ++sl) {
      int c, p;
      reg_slot<NC, C, NT, 2>(sl, c, p);
      pts[sl] = p;
      const int f = 4 * g + c / RB;
      xv[sl] = (f < nf) ? spec[f * fstride + (r0 + c % RB) * NC + p] : make_float2(0.f, 0.f);
    }
    const bool u0 = (threadIdx.x % H) == 0;
    float2 v[PPT];
    static_assert(16 % R0 == 0, "stage-0 radix divides 16");
#pragma unroll
    for (int i = 0; i < NTASK0; ++i) {
      // the task's points are k + q NC / R0, and conj(W_N^{k + q NC/R0}) = conj(W_N^k) e^{i pi q / R0}:
      // one table read per task instead of R0
      const float2 w0 = cconj(tw[pts[i * R0]]);
#pragma unroll
      for (int q = 0; q < R0; ++q) {
        const int sl = i * R0 + q;
        const float2 other = xv[((i & 1) == 0 ? i + 1 : i - 1) * R0 + (R0 - 1 - q)];
        float2 self_pair;  // k = 0 (even task) or k = NC / R0 / 2 (odd task) pairs within the task
        if ((i & 1) == 0)
          self_pair = (q == 0) ? make_float2(0.f, 0.f) : xv[i * R0 + (R0 - q)];
        else
          self_pair = xv[i * R0 + (R0 - 1 - q)];
        const float2 wq = q == 0 ? w0 : cmul(w0, root32(q * (16 / R0)));
        v[sl] = packw(wq, xv[sl], u0 ? self_pair : other);
      }
    }
    fft_reg_v<NC, C, NT, true, 2, 0, true>(v, ex, PS, tw2, store);
  } else {
    auto load = [&](int c, int k) -> float2 {
      const int f = 4 * g + c / RB;
      if (f >= nf) return make_float2(0.f, 0.f);
      const float2* row = spec + f * fstride + (r0 + c % RB) * NC;
      return pack(k, row[k], (k == 0) ? make_float2(0.f, 0.f) : row[NC - k]);
    };
    fft_reg<NC, C, NT, true, true, 0, true>(ex, PS, tw2, load, store);
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < NC * RB; idx += blockDim.x) {
    const int r = idx / NC, j = idx % NC;
    const float2* src = res + j * PS + r;
    const float2 z0 = src[0], z1 = src[RB], z2 = src[2 * RB], z3 = src[3 * RB];
    const long long at = (static_cast<long long>(g) * N * N + r0 + r) * N + 2 * j;
    if constexpr (BF16) {  // four bins of a point as bfloat16 (8 bytes), rounded to nearest even
      uint4 v;
      v.x = bf16x2(z0.x, z1.x);
      v.y = bf16x2(z2.x, z3.x);
      v.z = bf16x2(z0.y, z1.y);
      v.w = bf16x2(z2.y, z3.y);
      *reinterpret_cast<uint4*>(reinterpret_cast<uint2*>(out) + at) = v;
    } else {
      float4* o = out + at;
      o[0] = make_float4(z0.x, z1.x, z2.x, z3.x);
      o[1] = make_float4(z0.y, z1.y, z2.y, z3.y);
    }
  }
}

// z-pass of the field reconstruction with the multipole window fused in.
// grid (nc/T, n/2 + 1): CTA (x-tile, iy) transforms the rows iy and n - iy together (one row for
// iy = 0; the y-Nyquist row iy = n/2 is zero).  The two rows share |n|^2 at every (x, z), so
// one gather of the window table serves both.  For its own stage-0 points each thread keeps
// delta_hat * R_lm(n-hat) of both rows (with the real sign of i^l) and the window-table row of
// |n|^2 in shared memory.  Bins are taken four at a time: one float4 gather of the window
// table [n2][nbp] per point gives the values of four fields, and the gather of the next four is
// issued before the current four are transformed, so its latency hides behind them.  Field f
// (bin b0 + f) is delta_hat * R * J_f(|n|^2) (* i for odd l); its z-transformed tile goes to
// out + f * fstride.
template <int N, int T>
struct AlmZ {
  static constexpr int NT = RegThreads<N, T, 512>::NT;
  static constexpr int PPT = N * T / NT;
  static constexpr int PADR = 2;  // exchange padding, 2 elements per 2 points (conflict-free for T = 8)
  static constexpr int MINB = NT >= 512 ? 1 : 512 / NT;  // at least 16 warps per SM
  static constexpr size_t smem() {
    return (StageTw<N>::SIZE + 2 * static_cast<size_t>(PPT) * NT + static_cast<size_t>(N) * T + N) *
               sizeof(float2) +
           static_cast<size_t>(PPT) * NT * sizeof(int);
  }
};

template <int N, int T>
__global__ void __launch_bounds__(AlmZ<N, T>::NT, AlmZ<N, T>::MINB)
    k_alm_z(const float2* __restrict__ dhat, float2* __restrict__ out, long long fstride, int nf,
            const float4* __restrict__ jt4, int nbp4, int l, int m, const float2* __restrict__ twg,
            const float* __restrict__ phi) {
  constexpr int NC = N / 2;
  constexpr int NT = AlmZ<N, T>::NT;
  constexpr int PPT = AlmZ<N, T>::PPT;
  constexpr int PADR = AlmZ<N, T>::PADR;
  extern __shared__ float2 sm[];
  float2* tw = sm;                      // per-stage twiddles
  float2* pd = tw + StageTw<N>::SIZE;   // [2][PPT][NT] delta_hat * angular factor of the two rows
  float2* ex = pd + 2 * PPT * NT;       // [N][T] exchange (+ padding)
  int* pn = reinterpret_cast<int*>(ex + N * T + N);  // [PPT][NT] window-table rows
  const int x0 = blockIdx.x * T;
  const int iy = blockIdx.y;
  const int iy2 = (N - iy) & (N - 1);        // the mirror row (iy itself for iy = 0)
  const int nrow = (iy == 0) ? 1 : 2;
  // offsets within one field (n^3 / 2 < 2^31)
  const int colbase[2] = {iy * NC + x0, iy2 * NC + x0};
  constexpr int zstride = N * NC;
  if (iy == N / 2) {  // y-Nyquist row: the window is zero
    for (int f = 0; f < nf; ++f)
      for (int idx = threadIdx.x; idx < N * T; idx += blockDim.x) {
        const int z = idx / T, c = idx % T;
        out[f * fstride + colbase[0] + z * zstride + c] = make_float2(0.f, 0.f);
      }
    return;
  }
  stage_tw_fill<N>(tw, twg, 1);
  const float sgn = ((l & 3) < 2) ? 1.f : -1.f;  // real part of i^l (or of i^{l-1} for odd l)
  const int ny = signed_freq(iy, N);
  float4 jn[PPT];
#pragma unroll
  for (int s = 0; s < PPT; ++s) {
    int c, z;
    reg_slot<N, T, NT, false>(s, c, z);
    const int nz = signed_freq(z, N), nx = x0 + c;
    const bool nyq = (z == N / 2);
    const int row = nyq ? 0 : (nx * nx + ny * ny + nz * nz) * nbp4;
    pn[s * NT + threadIdx.x] = row;
    const float pxz = __ldg(phi + nx) * __ldg(phi + z);
    const float a = nyq ? 0.f
                        : sgn * ylm_dev(l, m, static_cast<float>(nx), static_cast<float>(ny), static_cast<float>(nz)) *
                              (pxz * __ldg(phi + iy));
    pd[s * NT + threadIdx.x] = cscale(dhat[colbase[0] + z * zstride + c], a);
    if (nrow == 2) {
      const float a2 = nyq ? 0.f
                           : sgn *
                                 ylm_dev(l, m, static_cast<float>(nx), static_cast<float>(-ny), static_cast<float>(nz)) *
                                 (pxz * __ldg(phi + iy2));
      pd[(PPT + s) * NT + threadIdx.x] = cscale(dhat[colbase[1] + z * zstride + c], a2);
    }
    jn[s] = __ldg(jt4 + row);
  }
  __syncthreads();
  for (int g = 0; 4 * g < nf; ++g) {
    float4 jv[PPT];
#pragma unroll
    for (int s = 0; s < PPT; ++s) jv[s] = jn[s];
    if (4 * (g + 1) < nf) {
#pragma unroll
      for (int s = 0; s < PPT; ++s) jn[s] = __ldg(jt4 + pn[s * NT + threadIdx.x] + g + 1);
    }
    const int nj = (nf - 4 * g) < 4 ? (nf - 4 * g) : 4;
    for (int j = 0; j < nj; ++j) {
      const int f = 4 * g + j;
      for (int r = 0; r < nrow; ++r) {
        float2 v[PPT];
#pragma unroll
        for (int s = 0; s < PPT; ++s) {
          const float jj = j == 0 ? jv[s].x : j == 1 ? jv[s].y : j == 2 ? jv[s].z : jv[s].w;
          v[s] = cscale(pd[(r * PPT + s) * NT + threadIdx.x], jj);
          if (l & 1) v[s] = mul_i(v[s]);
        }
        float2* of = out + f * fstride + colbase[r];
        auto store = [&](int c, int z, float2 val) { of[z * zstride + c] = val; };
        fft_reg_v<N, T, NT, true, false, PADR>(v, ex, T, tw, store);
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// Adjoint (transpose) passes of the field reconstruction, for gradients.
//
// x-pass R2C of four bin-interleaved real fields (one group [z][y][x][4]) into four plain
// half spectra without the x-Nyquist column: the half-length complex transform of
// z[j] = (x[2j], x[2j+1]) followed by X[k] = E[k] + W_N^k O[k].  grid (n*n/RB, ngroups).
template <int N, int RB>
__global__ void __launch_bounds__(RegThreads<N / 2, 4 * RB, 256>::NT)
    k_r2c_x4(const float4* __restrict__ in, int nf, float2* __restrict__ spec, long long fstride,
             const float2* __restrict__ twg) {
  constexpr int NC = N / 2, C = 4 * RB, PS = C + 1;
  constexpr int NT = RegThreads<NC, C, 256>::NT;
  extern __shared__ float2 sm[];
  float2* tw = sm;                       // W_N^e, e < N
  float2* tw2 = sm + N;                  // per-stage twiddles of the length-NC transform
  float2* ex = tw2 + StageTw<NC>::SIZE;  // [NC][PS] exchange, then the outputs
  float2* res = ex;
  const int g = blockIdx.y;
  const long long r0 = static_cast<long long>(blockIdx.x) * RB;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = twg[i];
  stage_tw_fill<NC>(tw2, twg, 2);
  __syncthreads();
  auto load = [&](int c, int k) -> float2 {
    const int j = c / RB, r = c % RB;
    const float4* row = in + (static_cast<long long>(g) * N * N + r0 + r) * N;
    const float4 a = row[2 * k], b = row[2 * k + 1];
    const float* fa = reinterpret_cast<const float*>(&a);
    const float* fb = reinterpret_cast<const float*>(&b);
    return make_float2(fa[j], fb[j]);
  };
  auto store = [&](int c, int k, float2 v) { res[k * PS + c] = v; };
  fft_reg<NC, C, NT, false, true, 0, true>(ex, PS, tw2, load, store);
  __syncthreads();
  for (int idx = threadIdx.x; idx < NC * C; idx += blockDim.x) {
    const int c = idx / NC, k = idx % NC;
    const int f = 4 * g + c / RB;
    if (f >= nf) continue;
    const float2 zk = res[k * PS + c];
    const float2 zm = cconj(res[((NC - k) & (NC - 1)) * PS + c]);
    const float2 e = cscale(cadd(zk, zm), 0.5f);
    const float2 dd = csub(zk, zm);
    const float2 od = make_float2(0.5f * dd.y, -0.5f * dd.x);
    spec[f * fstride + (r0 + c % RB) * NC + k] = cadd(e, cmul(tw[k], od));
  }
}

// Adjoint z-pass: forward z-transform of nf x,y-transformed spectra and the transposed window,
// gk += sum_f (-1)^l K_lm,f(n) spec_f(n) with K = i^l R_lm J_f (|n|^2) as in the forward pass.
// grid (nc/T, n).
template <int N, int T>
__global__ void __launch_bounds__(RegThreads<N, T, 512>::NT)
    k_adj_z(const float2* __restrict__ spec, long long fstride, int nf, const float4* __restrict__ jt4, int nbp4,
            int l, int m, float2* __restrict__ gk, const float2* __restrict__ twg, const float* __restrict__ phi) {
  constexpr int NC = N / 2;
  constexpr int NT = RegThreads<N, T, 512>::NT;
  extern __shared__ float2 sm[];
  float2* tw = sm;                      // per-stage twiddles
  float2* ex = tw + StageTw<N>::SIZE;   // [N][T] (+ N padding)
  float2* acc = ex + N * T + N;         // [N][T] sum over fields
  float* ang = reinterpret_cast<float*>(acc + N * T);  // [N][T]
  int* n2 = reinterpret_cast<int*>(ang + N * T);        // [N][T]
  const int x0 = blockIdx.x * T;
  const int iy = blockIdx.y;
  if (iy == N / 2) return;  // the window vanishes on the y-Nyquist plane
  const long long colbase = static_cast<long long>(iy) * NC + x0;
  const long long zstride = static_cast<long long>(N) * NC;
  stage_tw_fill<N>(tw, twg, 1);
  // (-1)^l i^l = (-i)^l = sgn * (-i)^(l mod 2): sgn = +1 for l mod 4 in {0, 1}, -1 otherwise
  const float sgn = ((l & 3) < 2) ? 1.f : -1.f;
  const int ny = signed_freq(iy, N);
  for (int idx = threadIdx.x; idx < N * T; idx += blockDim.x) {
    const int z = idx / T, c = idx % T;
    const int nz = signed_freq(z, N), nx = x0 + c;
    const bool nyq = (z == N / 2);
    n2[idx] = nyq ? 0 : nx * nx + ny * ny + nz * nz;
    ang[idx] = nyq ? 0.f
                   : sgn * ylm_dev(l, m, static_cast<float>(nx), static_cast<float>(ny), static_cast<float>(nz)) *
                         (__ldg(phi + nx) * __ldg(phi + iy) * __ldg(phi + z));
    acc[idx] = make_float2(0.f, 0.f);
  }
  __syncthreads();
  const float* jt = reinterpret_cast<const float*>(jt4);
  for (int f = 0; f < nf; ++f) {
    const float2* sf = spec + f * fstride;
    auto load = [&](int c, int z) { return sf[colbase + z * zstride + c]; };
    auto store = [&](int c, int z, float2 v) {
      const int idx = z * T + c;
      const float a = ang[idx] * __ldg(jt + static_cast<long long>(n2[idx]) * 4 * nbp4 + f);
      acc[idx] = cadd(acc[idx], cscale(v, a));
    };
    fft_reg<N, T, NT, false, false, 2>(ex, T, tw, load, store);
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < N * T; idx += blockDim.x) {
    const int z = idx / T, c = idx % T;
    float2 v = acc[idx];
    if (l & 1) v = make_float2(v.y, -v.x);  // times -i
    float2* o = gk + colbase + z * zstride + c;
    *o = cadd(*o, v);
  }
}

// ---------------------------------------------------------------------------------------
namespace {

constexpr int kTz = 8;   // columns per z-pass (window) tile
constexpr int kTy = 16;  // columns per plain pencil tile
constexpr int kRB = 8;   // rows per x-pass tile
constexpr int kRB4 = 4;  // rows per four-field x-pass tile

template <typename K>
int set_smem(K kernel, size_t bytes) {
  return ensure_smem(reinterpret_cast<const void*>(kernel), bytes);
}

inline int check_launch() { return cudaGetLastError() == cudaSuccess ? ZETA_OK : ZETA_ECUDA; }

// dynamic shared memory of the pencil pass (twiddles + [N][T] exchange)
template <int N, int T>
constexpr size_t axis_smem() {
  return (StageTw<N>::SIZE + static_cast<size_t>(N) * T) * sizeof(float2);
}
// four-field x-pass: W_N, half-length twiddles, [N/2][4 RB + 1] exchange
template <int N, int RB>
constexpr size_t x4_smem() {
  return (N + StageTw<N / 2>::SIZE + static_cast<size_t>(N / 2) * (4 * RB + 1)) * sizeof(float2);
}

template <int N>
int r2c_impl(const zeta_ctx* c, const float* delta, float2* dhat, cudaStream_t s) {
  constexpr int NC = N / 2;
  constexpr int T = kTy < NC ? kTy : NC;
  StageScope prof(c, ST_R2C, 3, s);
  size_t smx = (N + NC + NC * (kRB + 1)) * sizeof(float2);
  if (set_smem(k_r2c_x<N, kRB>, smx)) return ZETA_ECUDA;
  k_r2c_x<N, kRB><<<N * N / kRB, 256, smx, s>>>(delta, dhat, c->d_tw);
  size_t sma = axis_smem<N, T>();
  if (set_smem(k_fft_axis<N, T, false, 1>, sma) || set_smem(k_fft_axis<N, T, false, 2>, sma)) return ZETA_ECUDA;
  k_fft_axis<N, T, false, 1><<<dim3(NC / T, N, 1), RegThreads<N, T, 512>::NT, sma, s>>>(dhat, 0, c->d_tw);
  k_fft_axis<N, T, false, 2><<<dim3(NC / T, N, 1), RegThreads<N, T, 512>::NT, sma, s>>>(dhat, 0, c->d_tw);
  return check_launch();
}

template <int N>
int c2r_impl(const zeta_ctx* c, float2* data, int nf, cudaStream_t s, bool do_y) {
  constexpr int NC = N / 2;
  constexpr int T = kTy < NC ? kTy : NC;
  const long long fstride = static_cast<long long>(N) * N * NC;
  if (do_y) {
    StageScope prof(c, ST_ALM_Y, 1, s);
    size_t sma = axis_smem<N, T>();
    if (set_smem(k_fft_axis<N, T, true, 1>, sma)) return ZETA_ECUDA;
    k_fft_axis<N, T, true, 1><<<dim3(NC / T, N, nf), RegThreads<N, T, 512>::NT, sma, s>>>(data, fstride, c->d_tw);
  }
  StageScope prof(c, ST_ALM_X, 1, s);
  size_t smx = (N + NC + NC * (kRB + 1)) * sizeof(float2);
  if (set_smem(k_c2r_x<N, kRB>, smx)) return ZETA_ECUDA;
  k_c2r_x<N, kRB><<<dim3(N * N / kRB, nf), 256, smx, s>>>(data, fstride, c->d_tw);
  return check_launch();
}

// The three passes of the field reconstruction, each on one of two tile shapes (the context's
// alm_shape, chosen by zeta_autotune; 0 is the default): z-pass columns T (8 or 4), y-pass
// columns TY (16 or 8), x-pass rows RB (4 or 2).
template <int N, int T>
int alm_z_pass(const zeta_ctx* c, const float2* dhat, int l, int b0, int m, int nf, float2* spec, cudaStream_t s) {
  constexpr int NC = N / 2;
  const long long fstride = static_cast<long long>(N) * N * NC;
  StageScope prof(c, ST_ALM_Z, 1, s);
  const size_t smz = AlmZ<N, T>::smem();
  if (set_smem(k_alm_z<N, T>, smz)) return ZETA_ECUDA;
  const int nbp4 = (c->p.nbins + 3) / 4;
  const float4* jt4 = reinterpret_cast<const float4*>(c->d_jtab) + static_cast<long long>(l) * c->nn2 * nbp4 + b0 / 4;
  k_alm_z<N, T><<<dim3(NC / T, N / 2 + 1), AlmZ<N, T>::NT, smz, s>>>(dhat, spec, fstride, nf, jt4, nbp4, l, m,
                                                                      c->d_tw, c->d_phi);
  return check_launch();
}

template <int N, int TY>
int alm_y_pass(const zeta_ctx* c, int nf, float2* spec, cudaStream_t s) {
  constexpr int NC = N / 2;
  const long long fstride = static_cast<long long>(N) * N * NC;
  StageScope prof(c, ST_ALM_Y, 1, s);
  const size_t sma = axis_smem<N, TY>();
  if (set_smem(k_fft_axis<N, TY, true, 1>, sma)) return ZETA_ECUDA;
  k_fft_axis<N, TY, true, 1><<<dim3(NC / TY, N, nf), RegThreads<N, TY, 512>::NT, sma, s>>>(spec, fstride, c->d_tw);
  return check_launch();
}

template <int N, int RB>
int alm_x_pass(const zeta_ctx* c, int nf, const float2* spec, float* out, cudaStream_t s, bool bf16) {
  constexpr int NC = N / 2;
  const long long fstride = static_cast<long long>(N) * N * NC;
  StageScope prof(c, ST_ALM_X, 1, s);
  const size_t smx = x4_smem<N, RB>();
  const int ng4 = (nf + 3) / 4;
  if (bf16) {
    if (set_smem(k_c2r_x4<N, RB, true>, smx)) return ZETA_ECUDA;
    k_c2r_x4<N, RB, true><<<dim3(N * N / RB, ng4), RegThreads<N / 2, 4 * RB, 256>::NT, smx, s>>>(
        spec, fstride, nf, reinterpret_cast<float4*>(out), c->d_tw);
  } else {
    if (set_smem(k_c2r_x4<N, RB>, smx)) return ZETA_ECUDA;
    k_c2r_x4<N, RB><<<dim3(N * N / RB, ng4), RegThreads<N / 2, 4 * RB, 256>::NT, smx, s>>>(
        spec, fstride, nf, reinterpret_cast<float4*>(out), c->d_tw);
  }
  return check_launch();
}

template <int N>
int alm_impl(const zeta_ctx* c, const float2* dhat, int l, int m, int b0, int nf, float2* spec, float* out,
             cudaStream_t s, bool bf16) {
  constexpr int NC = N / 2;
  constexpr int T0 = kTz < NC ? kTz : NC, T1 = 4 < NC ? 4 : NC;
  constexpr int Y0 = kTy < NC ? kTy : NC, Y1 = 8 < NC ? 8 : NC;
  int rc = c->alm_shape[0] ? alm_z_pass<N, T1>(c, dhat, l, b0, m, nf, spec, s)
                           : alm_z_pass<N, T0>(c, dhat, l, b0, m, nf, spec, s);
  if (rc != ZETA_OK) return rc;
  rc = c->alm_shape[1] ? alm_y_pass<N, Y1>(c, nf, spec, s) : alm_y_pass<N, Y0>(c, nf, spec, s);
  if (rc != ZETA_OK) return rc;
  return c->alm_shape[2] ? alm_x_pass<N, 2>(c, nf, spec, out, s, bf16) : alm_x_pass<N, kRB4>(c, nf, spec, out, s, bf16);
}

// Full inverse of nf half spectra in place: z-, y- and x-passes.
template <int N>
int c2r_full(const zeta_ctx* c, float2* data, int nf, cudaStream_t s) {
  constexpr int NC = N / 2;
  constexpr int T = kTy < NC ? kTy : NC;
  const long long fstride = static_cast<long long>(N) * N * NC;
  size_t sma = axis_smem<N, T>();
  if (set_smem(k_fft_axis<N, T, true, 2>, sma)) return ZETA_ECUDA;
  StageScope prof(c, ST_ALM_Z, 1, s);
  k_fft_axis<N, T, true, 2><<<dim3(NC / T, N, nf), RegThreads<N, T, 512>::NT, sma, s>>>(data, fstride, c->d_tw);
  if (check_launch()) return ZETA_ECUDA;
  return c2r_impl<N>(c, data, nf, s, true);
}

}  // namespace

#define ZK_DISPATCH_N(n, CALL) \
  switch (n) {                 \
    case 16: return CALL(16);  \
    case 32: return CALL(32);  \
    case 64: return CALL(64);  \
    case 128: return CALL(128); \
    case 256: return CALL(256); \
    case 512: return CALL(512); \
    default: return ZETA_ENOTSUP; \
  }

int launch_r2c(const zeta_ctx* c, const float* delta, float2* dhat, cudaStream_t s) {
#define ZK_CALL(NN) r2c_impl<NN>(c, delta, dhat, s)
  ZK_DISPATCH_N(c->n, ZK_CALL)
#undef ZK_CALL
}

int launch_alm(const zeta_ctx* c, const float2* dhat, int l, int m, int b0, int nf, float2* spec, float* out,
               cudaStream_t s, bool bf16) {
#define ZK_CALL(NN) alm_impl<NN>(c, dhat, l, m, b0, nf, spec, out, s, bf16)
  ZK_DISPATCH_N(c->n, ZK_CALL)
#undef ZK_CALL
}

template <int N>
int adj_impl(const zeta_ctx* c, const float* fields, int nf, float2* spec, int l, int m, float2* gk, cudaStream_t s) {
  constexpr int NC = N / 2;
  constexpr int TY = kTy < NC ? kTy : NC;
  constexpr int TZ = kTz < NC ? kTz : NC;
  constexpr int RB = kRB4;
  const long long fstride = static_cast<long long>(N) * N * NC;
  StageScope prof(c, ST_ADJ_FFT, 3, s);
  const size_t smx = x4_smem<N, RB>();
  if (set_smem(k_r2c_x4<N, RB>, smx)) return ZETA_ECUDA;
  k_r2c_x4<N, RB><<<dim3(N * N / RB, (nf + 3) / 4), RegThreads<N / 2, 4 * RB, 256>::NT, smx, s>>>(
      reinterpret_cast<const float4*>(fields), nf, spec, fstride, c->d_tw);
  const size_t sma = axis_smem<N, TY>();
  if (set_smem(k_fft_axis<N, TY, false, 1>, sma)) return ZETA_ECUDA;
  k_fft_axis<N, TY, false, 1><<<dim3(NC / TY, N, nf), RegThreads<N, TY, 512>::NT, sma, s>>>(spec, fstride, c->d_tw);
  const size_t smz = (StageTw<N>::SIZE + 2 * static_cast<size_t>(N) * TZ + N) * sizeof(float2) +
                     2 * static_cast<size_t>(N) * TZ * 4;
  if (set_smem(k_adj_z<N, TZ>, smz)) return ZETA_ECUDA;
  const int nbp4 = (c->p.nbins + 3) / 4;
  const float4* jt4 = reinterpret_cast<const float4*>(c->d_jtab) + static_cast<long long>(l) * c->nn2 * nbp4;
  k_adj_z<N, TZ><<<dim3(NC / TZ, N), RegThreads<N, TZ, 512>::NT, smz, s>>>(spec, fstride, nf, jt4, nbp4, l, m, gk,
                                                                          c->d_tw, c->d_phi);
  return check_launch();
}

int launch_adj_spectral(const zeta_ctx* c, const float* fields, int nf, float2* spec, int l, int m, float2* gk,
                        cudaStream_t s) {
#define ZK_CALL(NN) adj_impl<NN>(c, fields, nf, spec, l, m, gk, s)
  ZK_DISPATCH_N(c->n, ZK_CALL)
#undef ZK_CALL
}

int launch_c2r_inplace(const zeta_ctx* c, float2* data, int nf, cudaStream_t s) {
#define ZK_CALL(NN) c2r_full<NN>(c, data, nf, s)
  ZK_DISPATCH_N(c->n, ZK_CALL)
#undef ZK_CALL
}

// out = dhat * W(|n|^2) on the stored half spectrum, zero on the Nyquist planes (the table holds
// the primary-vertex tophat with the 1/N_g of the inverse transform)
__global__ void k_primary_mul(const float2* __restrict__ dhat, const float* __restrict__ w, int n,
                              float2* __restrict__ out) {
  const int nc = n / 2;
  const long long total = static_cast<long long>(n) * n * nc;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long long>(blockDim.x) * gridDim.x) {
    const int ix = static_cast<int>(i % nc), iy = static_cast<int>((i / nc) % n),
              iz = static_cast<int>(i / (static_cast<long long>(nc) * n));
    float2 v = make_float2(0.f, 0.f);
    if (iy != n / 2 && iz != n / 2) {
      const int fy = signed_freq(iy, n), fz = signed_freq(iz, n);
      v = cscale(dhat[i], __ldg(w + (ix * ix + fy * fy + fz * fz)));
    }
    out[i] = v;
  }
}

int launch_primary(const zeta_ctx* c, const float2* dhat, float* out, cudaStream_t s) {
  if (!c->d_wprim) return ZETA_EINVAL;
  {
    StageScope prof(c, ST_R2C, 1, s);
    k_primary_mul<<<c->num_sms * 8, 256, 0, s>>>(dhat, c->d_wprim, c->n, reinterpret_cast<float2*>(out));
    if (check_launch()) return ZETA_ECUDA;
  }
  return launch_c2r_inplace(c, reinterpret_cast<float2*>(out), 1, s);
}

}  // namespace zk
