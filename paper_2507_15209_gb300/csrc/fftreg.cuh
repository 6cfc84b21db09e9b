// Register-staged FFT for sm_103a: the butterflies of every stage run in registers and
// shared memory is touched only to exchange data between stages.
//
// A CTA of NT threads transforms T independent sequences ("columns") of length L = 2^p.
// Stage s (radix R_s, span LS_s, M_s = LS_s / R_s) has (L / R_s) * T butterfly tasks; a task
// (col, k) reads points base + q*M_s (base = (k / M_s) * LS_s + k % M_s) and writes them back in
// place, decimation-in-frequency order.  Every thread owns L*T/NT points in every stage:
//   * stage 0 takes its inputs straight from a caller functor load(col, point) (global
//     memory, with any pre-multiplication fused in);
//   * between stages the outputs go to shared memory [point][PS] and the next stage's inputs
//     are read back (one exchange = one write + one read per point);
//   * the last stage hands each output to store(col, natural_index, value).
// So a 512-point transform costs two exchanges instead of a shared-memory pass per stage.
// Tasks are assigned column-fastest (pencils: columns contiguous in global memory), except
// that in ROWS mode stage 0 assigns them point-fastest so that rows load coalesced.
// Twiddles come from a per-stage table in shared memory, [stage][j][3] = W_LS^j, W_LS^2j,
// W_LS^4j (the odd powers formed by at most two multiplications), so that the lanes of a warp,
// which hold consecutive j, read consecutive entries instead of strided ones.
// The exchange buffer may be padded by PADR elements every PADR points (PADR = 0: none),
// which keeps the last stage of narrow (T = 8) pencils free of bank conflicts.
#pragma once
#include "fft.cuh"

namespace zk {

template <int L>
__host__ __device__ constexpr int plan_radix(int s) {
  return FftPlan<L>::radix(s);
}
template <int L>
__host__ __device__ constexpr int plan_span(int S) {
  int ls = L;
  for (int s = 0; s < S; ++s) ls /= plan_radix<L>(s);
  return ls;
}

// Stage-0 task mappings (MAP, later stages always column-fastest, which keeps every
// shared-memory exchange free of bank conflicts):
//   0  column-fastest (pencils: columns contiguous in global memory);
//   1  rows: point-fastest, so that rows load coalesced;
//   2  mirror-paired rows: thread u of a column takes tasks k = u and k = KC - u (u = 0: k = 0 and
//      k = KC/2), KC = L / R, with its tasks alternating between the two; then the points
//      p and L - p of a half-length real-to-complex packing sit in the same thread (task pairs
//      (2j, 2j + 1), point q against R - 1 - q).  Needs an even number of tasks per thread.
template <int L, int T, int NT, int MAP, int R>
__device__ __forceinline__ void reg_task(int i, int& col, int& k) {
  const int t = threadIdx.x + i * NT;
  if constexpr (MAP == 2) {
    constexpr int KC = L / R, H = KC / 2;
    const int u = threadIdx.x % H, cidx = threadIdx.x / H;
    col = cidx + (i >> 1) * (NT / H);
    k = (i & 1) == 0 ? u : (u == 0 ? H : KC - u);
  } else if constexpr (MAP == 1) {
    k = t % (L / R);
    col = t / (L / R);
  } else {
    col = t % T;
    k = t / T;
  }
}

// Layout of the per-stage twiddle table: stage S starts at off(S) and holds 3 entries per
// butterfly offset j < M_S.
template <int L>
struct StageTw {
  static __host__ __device__ constexpr int off(int S) {
    int o = 0;
    for (int s = 0; s < S; ++s) o += 3 * (plan_span<L>(s) / plan_radix<L>(s));
    return o;
  }
  static constexpr int SIZE = off(FftPlan<L>::NST);
};

// Fill the table (all threads of the CTA; a barrier must follow).  twg holds W_G^e, e < G,
// for a length G = L * gstep, so W_L^e = twg[e * gstep].
template <int L>
__device__ __forceinline__ void stage_tw_fill(float2* dst, const float2* __restrict__ twg, int gstep) {
  constexpr int NST = FftPlan<L>::NST;
  for (int i = threadIdx.x; i < StageTw<L>::SIZE; i += blockDim.x) {
    int S = 0;
    while (S + 1 < NST && i >= StageTw<L>::off(S + 1)) ++S;
    const int r = i - StageTw<L>::off(S);
    const int j = r / 3, p = r % 3;
    const int TS = L / plan_span<L>(S);
    const int e = ((1 << p) * j * TS) & (L - 1);
    dst[i] = twg[e * gstep];
  }
}

// Twiddle multiply of the R outputs of butterfly j of span LS: y_p *= W_LS^{p j}; t is the
// stage's part of the table.
template <int R, int LS, bool INV>
__device__ __forceinline__ void twiddle(float2* y, int j, const float2* t) {
  if (LS == R) return;  // M == 1: all twiddles are 1
  const float2* e = t + 3 * j;
  float2 w1 = e[0];
  if (INV) w1.y = -w1.y;
  y[1] = cmul(y[1], w1);
  if (R >= 4) {
    float2 w2 = e[1];
    if (INV) w2.y = -w2.y;
    y[2] = cmul(y[2], w2);
    y[3] = cmul(y[3], cmul(w2, w1));
    if (R == 8) {
      float2 w4 = e[2];
      if (INV) w4.y = -w4.y;
      const float2 w3 = cmul(w2, w1);
      y[4] = cmul(y[4], w4);
      y[5] = cmul(y[5], cmul(w4, w1));
      y[6] = cmul(y[6], cmul(w4, w2));
      y[7] = cmul(y[7], cmul(w4, w3));
    }
  }
}

// Exchange-buffer index of point pt of column col: PADR elements of padding after every
// PADR points (PADR = 0: none).  For 8-byte elements the two half-warps are served
// separately; with T = 8 columns the padded pitch puts the two points that a half-warp reads
// in the last stage 16 banks apart.
template <int PADR>
__device__ __forceinline__ int ex_index(int pt, int col, int PS) {
  return pt * PS + col + (PADR ? (pt / PADR) * PADR : 0);
}

template <int L, int T, int NT, bool INV, int ROWS, int PADR, int S>
struct RegStage {
  static constexpr int R = plan_radix<L>(S);
  static constexpr int LS = plan_span<L>(S);
  static constexpr int M = LS / R;
  static constexpr int PPT = L * T / NT;
  static constexpr int NTASK = PPT / R;

  __device__ __forceinline__ static int base_of(int k) { return (k / M) * LS + (k % M); }

  static constexpr int RM = S == 0 ? ROWS : 0;  // task mapping of this stage
  // butterflies + twiddles of this stage on v (inputs in task order)
  __device__ __forceinline__ static void compute(float2* v, const float2* tw) {
#pragma unroll
    for (int i = 0; i < NTASK; ++i) {
      int col, k;
      reg_task<L, T, NT, RM, R>(i, col, k);
      dft_small<R, INV>(v + i * R);
      twiddle<R, LS, INV>(v + i * R, k % M, tw + StageTw<L>::off(S));
    }
  }
  // write this stage's outputs to shared memory
  __device__ __forceinline__ static void put(const float2* v, float2* sm, int PS) {
#pragma unroll
    for (int i = 0; i < NTASK; ++i) {
      int col, k;
      reg_task<L, T, NT, RM, R>(i, col, k);
      const int b = base_of(k);
#pragma unroll
      for (int p = 0; p < R; ++p) sm[ex_index<PADR>(b + p * M, col, PS)] = v[i * R + p];
    }
  }
  // read this stage's inputs from shared memory
  __device__ __forceinline__ static void get(float2* v, const float2* sm, int PS) {
#pragma unroll
    for (int i = 0; i < NTASK; ++i) {
      int col, k;
      reg_task<L, T, NT, RM, R>(i, col, k);
      const int b = base_of(k);
#pragma unroll
      for (int q = 0; q < R; ++q) v[i * R + q] = sm[ex_index<PADR>(b + q * M, col, PS)];
    }
  }
};

// SYNC_OUT: barrier before the last stage hands out its outputs (lets the caller's store
// reuse the exchange buffer).
template <int L, int T, int NT, bool INV, int ROWS, int PADR, bool SYNC_OUT, int S>
struct RegRun {
  template <class Store>
  __device__ __forceinline__ static void run(float2* v, float2* sm, int PS, const float2* tw, Store& store) {
    using St = RegStage<L, T, NT, INV, ROWS, PADR, S>;
    constexpr int NST = FftPlan<L>::NST;
    St::compute(v, tw);
    if constexpr (S + 1 < NST) {
      using Nx = RegStage<L, T, NT, INV, ROWS, PADR, S + 1>;
      __syncthreads();  // previous readers of sm are done
      St::put(v, sm, PS);
      __syncthreads();
      Nx::get(v, sm, PS);
      RegRun<L, T, NT, INV, ROWS, PADR, SYNC_OUT, S + 1>::run(v, sm, PS, tw, store);
    } else {
      if constexpr (SYNC_OUT) __syncthreads();
#pragma unroll
      for (int i = 0; i < St::NTASK; ++i) {
        int col, k;
        reg_task<L, T, NT, St::RM, St::R>(i, col, k);
        const int b = St::base_of(k);
#pragma unroll
        for (int p = 0; p < St::R; ++p) store(col, fft_index_at<L>(b + p * St::M), v[i * St::R + p]);
      }
    }
  }
};

// Stage-0 input slot of a thread: slot i*R0 + q holds point k + q*M0 of column col, where
// (col, k) is the thread's task i.  Callers that precompute per-point data use this order.
template <int L, int T, int NT, int ROWS>
__device__ __forceinline__ void reg_slot(int slot, int& col, int& point) {
  using S0 = RegStage<L, T, NT, false, ROWS, 0, 0>;
  int k;
  reg_task<L, T, NT, ROWS, S0::R>(slot / S0::R, col, k);
  point = k + (slot % S0::R) * S0::M;
}

// Full transform of inputs already in registers (slot order of reg_slot).
template <int L, int T, int NT, bool INV, int ROWS, int PADR = 0, bool SYNC_OUT = false, class Store>
__device__ __forceinline__ void fft_reg_v(float2* v, float2* sm, int PS, const float2* tw, Store& store) {
  RegRun<L, T, NT, INV, ROWS, PADR, SYNC_OUT, 0>::run(v, sm, PS, tw, store);
}

// Full transform.  load(col, point) -> float2 gives the input; store(col, index, value)
// receives each output at its natural index.  sm: [L][PS] float2 exchange buffer (PS >= T,
// plus L elements of padding when PADR > 0; odd PS in ROWS mode keeps the exchange conflict-free);
// tw: the per-stage table of StageTw<L> (forward sign) in shared memory.  No barrier after
// the stores.
template <int L, int T, int NT, bool INV, int ROWS, int PADR = 0, bool SYNC_OUT = false, class Load, class Store>
__device__ __forceinline__ void fft_reg(float2* sm, int PS, const float2* tw, Load& load, Store& store) {
  constexpr int PPT = L * T / NT;
  float2 v[PPT];
#pragma unroll
  for (int s = 0; s < PPT; ++s) {
    int col, point;
    reg_slot<L, T, NT, ROWS>(s, col, point);
    v[s] = load(col, point);
  }
  RegRun<L, T, NT, INV, ROWS, PADR, SYNC_OUT, 0>::run(v, sm, PS, tw, store);
}

}  // namespace zk
