// Shared-memory FFT building blocks for sm_103a.
//
// A CTA transforms T independent sequences ("columns") of length L = 2^p that sit in
// shared memory point-major: element (point k, column c) lives at buf[k * PS + c].
// The transform is an in-place decimation-in-frequency Cooley-Tukey with radix-8
// butterflies in registers (one radix-2 or radix-4 stage absorbs log2(L) mod 3), so a
// 512-point transform is three passes over shared memory.  After the last stage the
// spectrum sits in mixed-radix digit-reversed order; `fft_pos_of` gives the position of
// each natural index and readers gather through it, which keeps every global write
// coalesced.  Twiddles W_L^e = exp(-2 pi i e / L) come from a host-built float64 table
// rounded to float32; the inverse transform conjugates them.  Unnormalised both ways.
#pragma once
#include <cuda_runtime.h>

namespace zk {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 z) {
  return INV ? make_float2(-z.y, z.x) : make_float2(z.y, -z.x);
}
__device__ __forceinline__ float2 mul_i(float2 z) { return make_float2(-z.y, z.x); }

template <int R, bool INV>
__device__ __forceinline__ void dft_small(float2* x);

template <>
__device__ __forceinline__ void dft_small<2, false>(float2* x) {
  float2 a = x[0], b = x[1];
  x[0] = cadd(a, b);
  x[1] = csub(a, b);
}
template <>
__device__ __forceinline__ void dft_small<2, true>(float2* x) {
  dft_small<2, false>(x);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3) {
  float2 s02 = cadd(x0, x2), d02 = csub(x0, x2);
  float2 s13 = cadd(x1, x3), d13 = mul_mi<INV>(csub(x1, x3));
  x0 = cadd(s02, s13);
  x2 = csub(s02, s13);
  x1 = cadd(d02, d13);
  x3 = csub(d02, d13);
}

template <>
__device__ __forceinline__ void dft_small<4, false>(float2* x) { dft4<false>(x[0], x[1], x[2], x[3]); }
template <>
__device__ __forceinline__ void dft_small<4, true>(float2* x) { dft4<true>(x[0], x[1], x[2], x[3]); }

template <bool INV>
__device__ __forceinline__ void dft8(float2* x) {
  // even/odd split: E = DFT4(x0,x2,x4,x6), O = DFT4(x1,x3,x5,x7); y_p = E_p + W8^p O_p
  float2 e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
  float2 o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  const float r = 0.70710678118654752f;
  // W8^1 = (1 -/+ i)/sqrt2, W8^2 = -/+ i, W8^3 = (-1 -/+ i)/sqrt2   (forward/inverse)
  float2 t1 = INV ? make_float2(r * (o1.x - o1.y), r * (o1.x + o1.y))
                  : make_float2(r * (o1.x + o1.y), r * (o1.y - o1.x));
  float2 t2 = mul_mi<INV>(o2);
  float2 t3 = INV ? make_float2(-r * (o3.x + o3.y), r * (o3.x - o3.y))
                  : make_float2(r * (o3.y - o3.x), -r * (o3.x + o3.y));
  x[0] = cadd(e0, o0);
  x[4] = csub(e0, o0);
  x[1] = cadd(e1, t1);
  x[5] = csub(e1, t1);
  x[2] = cadd(e2, t2);
  x[6] = csub(e2, t2);
  x[3] = cadd(e3, t3);
  x[7] = csub(e3, t3);
}
template <>
__device__ __forceinline__ void dft_small<8, false>(float2* x) { dft8<false>(x); }
template <>
__device__ __forceinline__ void dft_small<8, true>(float2* x) { dft8<true>(x); }

// Radix of stage s for a length-L transform: the first stage takes log2(L) mod 3 (if any),
// all others are radix 8.
template <int L>
struct FftPlan {
  static constexpr int LOG = (L <= 1) ? 0 : 1 + FftPlan<L / 2>::LOG;
  static constexpr int REM = LOG % 3;
  static constexpr int NST = LOG / 3 + (REM ? 1 : 0);
  static __host__ __device__ constexpr int radix(int s) { return (s == 0 && REM) ? (1 << REM) : 8; }
};
template <>
struct FftPlan<1> {
  static constexpr int LOG = 0;
  static constexpr int REM = 0;
  static constexpr int NST = 0;
  static __host__ __device__ constexpr int radix(int) { return 1; }
};

// Position (after all DIF stages) that holds natural index k.
template <int L>
__device__ __forceinline__ int fft_pos_of(int k) {
  int pos = 0, m = L;
#pragma unroll
  for (int s = 0; s < FftPlan<L>::NST; ++s) {
    const int R = FftPlan<L>::radix(s);
    m /= R;
    pos += (k % R) * m;
    k /= R;
  }
  return pos;
}
// Natural index held at position pos.
template <int L>
__device__ __forceinline__ int fft_index_at(int pos) {
  int k = 0, m = L, w = 1;
#pragma unroll
  for (int s = 0; s < FftPlan<L>::NST; ++s) {
    const int R = FftPlan<L>::radix(s);
    m /= R;
    k += ((pos / m) % R) * w;
    w *= R;
  }
  return k;
}

// One DIF stage of radix R on a span Ls (sub-transform length), all T columns.
template <int L, int R, bool INV>
__device__ __forceinline__ void dif_stage(float2* buf, int PS, int T, int Ls, const float2* tw) {
  const int m = Ls / R;
  const int ntask = (L / R) * T;
  const int tstride = L / Ls;  // W_Ls^e = W_L^{e * L / Ls}
  for (int task = threadIdx.x; task < ntask; task += blockDim.x) {
    const int col = task % T;
    const int k = task / T;
    const int j = k % m;
    const int base = (k / m) * Ls + j;
    float2 x[R];
#pragma unroll
    for (int q = 0; q < R; ++q) x[q] = buf[(base + q * m) * PS + col];
    dft_small<R, INV>(x);
    if (m > 1) {
#pragma unroll
      for (int p = 1; p < R; ++p) {
        float2 w = tw[(p * j * tstride) & (L - 1)];
        if (INV) w.y = -w.y;
        x[p] = cmul(x[p], w);
      }
    }
#pragma unroll
    for (int p = 0; p < R; ++p) buf[(base + p * m) * PS + col] = x[p];
  }
}

// Full transform of T columns of length L in shared memory.  tw: W_L^e for e < L (forward
// sign), in shared memory.  Starts and ends with __syncthreads().
template <int L, bool INV>
__device__ __forceinline__ void fft_smem(float2* buf, int PS, int T, const float2* tw) {
  __syncthreads();
  int Ls = L;
#pragma unroll
  for (int s = 0; s < FftPlan<L>::NST; ++s) {
    const int R = FftPlan<L>::radix(s);
    if (R == 8) dif_stage<L, 8, INV>(buf, PS, T, Ls, tw);
    else if (R == 4) dif_stage<L, 4, INV>(buf, PS, T, Ls, tw);
    else dif_stage<L, 2, INV>(buf, PS, T, Ls, tw);
    Ls /= R;
    __syncthreads();
  }
}

}  // namespace zk
