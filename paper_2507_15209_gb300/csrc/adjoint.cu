// Adjoint (reverse-mode) kernels for gradients of a scalar loss L = sum_l sum_ij W_l[i,j]
// zeta_l[i,j] (field-level inference).  With S_l = (W_l + W_l^T)/2 and the reconstruction
// a_b = A_b delta, A_b = IDFT diag(K_b) DFT, the transpose is A_b^T = (-1)^l IDFT diag(K_b) DFT,
// so every (l, m) adds (-1)^l sum_b K_b DFT(h_b) to one k-space accumulator that is transformed
// back once at the end (fft.cu: launch_adj_spectral, launch_c2r_inplace).
//   node form:      q += sum S a a,  h_b = 2 delta (S a)_b          dL/d delta = (q + IDFT)/N_g
//   particle form:  per particle c_b = (2 w_p / W)(S f)_b; the direct term sum_b c_b grad f_b;
//                   h_b = assignment of c_b;  the mass term's share -2 Mhat delta_hat c_l(k) in
//                   k-space; dL/dx_p = direct + (N_g w_p / W) grad(interpolated dL/d delta).
// The particle scatter uses float atomics, so those gradients are reproducible only to float32
// rounding; everything else is order-fixed.
#include "zeta_internal.h"

namespace zk {
namespace {

constexpr int kAT = 256;

template <int D>
__device__ __forceinline__ void bs_w(float t, float* w, float* dw) {
  if (D == 2) {
    w[0] = 1.f - t;
    w[1] = t;
    dw[0] = -1.f;
    dw[1] = 1.f;
  } else {
    const float t2 = t * t, t3 = t2 * t, s = 1.f - t;
    w[0] = s * s * s * (1.f / 6.f);
    w[1] = (3.f * t3 - 6.f * t2 + 4.f) * (1.f / 6.f);
    w[2] = (-3.f * t3 + 3.f * t2 + 3.f * t + 1.f) * (1.f / 6.f);
    w[3] = t3 * (1.f / 6.f);
    dw[0] = -0.5f * s * s;
    dw[1] = 1.5f * t2 - 2.f * t;
    dw[2] = -1.5f * t2 + t + 0.5f;
    dw[3] = 0.5f * t2;
  }
}

__device__ __forceinline__ int cell_t(float x, double inv_h, int n, float& t) {
  const double u = static_cast<double>(x) * inv_h;
  const double v = u - floor(u / n) * n;
  int c = static_cast<int>(floor(v));
  const double fr = v - c;
  if (c >= n) c -= n;
  t = static_cast<float>(fr);
  if (t >= 1.f) t = 0.99999994f;
  return c;
}

template <int NBP>
__global__ void __launch_bounds__(kAT) k_adj_node(const float* __restrict__ delta, float4* __restrict__ f4, long long ng,
                                                  int nb, const float* __restrict__ S, float* __restrict__ q) {
  constexpr int G = NBP / 4;
  __shared__ float s_s[NBP * NBP];
  for (int i = threadIdx.x; i < NBP * NBP; i += blockDim.x) {
    const int r = i / NBP, c = i % NBP;
    s_s[i] = (r < nb && c < nb) ? S[r * nb + c] : 0.f;
  }
  __syncthreads();
  const int ngrp = (nb + 3) / 4;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < ng;
       i += static_cast<long long>(blockDim.x) * gridDim.x) {
    float a[NBP];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const float4 v = (g < ngrp) ? f4[g * ng + i] : make_float4(0.f, 0.f, 0.f, 0.f);
      a[4 * g] = v.x;
      a[4 * g + 1] = v.y;
      a[4 * g + 2] = v.z;
      a[4 * g + 3] = v.w;
    }
    const float d = delta[i];
    float qs = 0.f;
    float h[NBP];
#pragma unroll
    for (int b = 0; b < NBP; ++b) {
      float t = 0.f;
#pragma unroll
      for (int b2 = 0; b2 < NBP; ++b2) t = fmaf(s_s[b * NBP + b2], a[b2], t);
      qs = fmaf(a[b], t, qs);
      h[b] = 2.f * d * t;
    }
    q[i] += qs;
#pragma unroll
    for (int g = 0; g < G; ++g)
      if (g < ngrp) f4[g * ng + i] = make_float4(h[4 * g], h[4 * g + 1], h[4 * g + 2], h[4 * g + 3]);
  }
}

// gk(n) -= 2 Mhat(n) delta_hat(n) (2l+1)/(4 pi) sum_bb' S[b,b'] T_b(n) T_b'(n), non-Nyquist modes
__global__ void __launch_bounds__(kAT) k_adj_mass(const float2* __restrict__ dhat, const float* __restrict__ jt, int nbp,
                                                  const float* __restrict__ mhat, int n, int nb, const float* __restrict__ S,
                                                  float coef, float2* __restrict__ gk) {
  __shared__ float s_s[kMaxBins * kMaxBins];
  for (int i = threadIdx.x; i < nb * nb; i += blockDim.x) s_s[i] = S[i];
  __syncthreads();
  const int nc = n / 2;
  const long long total = static_cast<long long>(n) * n * nc;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long long>(blockDim.x) * gridDim.x) {
    const int ix = static_cast<int>(i % nc), iy = static_cast<int>((i / nc) % n),
              iz = static_cast<int>(i / (static_cast<long long>(nc) * n));
    if (iy == n / 2 || iz == n / 2) continue;
    const int fy = iy < n / 2 ? iy : iy - n, fz = iz < n / 2 ? iz : iz - n;
    const long long n2 = static_cast<long long>(ix) * ix + fy * fy + fz * fz;
    const float* tb = jt + n2 * nbp;
    float c = 0.f;
    for (int b = 0; b < nb; ++b) {
      float t = 0.f;
      for (int b2 = 0; b2 < nb; ++b2) t = fmaf(s_s[b * nb + b2], __ldg(tb + b2), t);
      c = fmaf(__ldg(tb + b), t, c);
    }
    const float f = 2.f * coef * c * mhat[ix] * mhat[iy] * mhat[iz];
    const float2 d = dhat[i];
    gk[i] = make_float2(gk[i].x - f * d.x, gk[i].y - f * d.y);
  }
}

// Particle adjoint: persistent CTAs over tiles, batches of kAPB particles.
// particles per batch: keeps the static shared memory of a CTA under 48 KB
template <int NBP>
struct AdjBatch {
  static constexpr int APB = NBP >= 24 ? 64 : 128;
};

template <int NBP, int D>
__global__ void __launch_bounds__(kAT)
    k_adj_points(const float4* __restrict__ sorted, const long long* __restrict__ tile_start,
                 const int* __restrict__ sidx, const float4* __restrict__ f4, long long ng, int n, int nb, double inv_h,
                 const float* __restrict__ S, const double* __restrict__ wsum, float4* __restrict__ h4,
                 float* __restrict__ direct) {
  constexpr int OFF = D / 2 - 1;
  constexpr int kAPB = AdjBatch<NBP>::APB;
  __shared__ float s_s[NBP * NBP];
  __shared__ int4 org[kAPB];
  __shared__ float bw[kAPB][6 * D];    // wx, wy, wz, dwx, dwy, dwz (derivatives already / H)
  __shared__ float fv[kAPB][NBP];      // f_b, then c_b
  __shared__ float gv[kAPB][NBP][3];   // grad f_b
  __shared__ float pw[kAPB];
  for (int i = threadIdx.x; i < NBP * NBP; i += blockDim.x) {
    const int r = i / NBP, c = i % NBP;
    s_s[i] = (r < nb && c < nb) ? S[r * nb + c] : 0.f;
  }
  const float wscale = static_cast<float>(2.0 / wsum[0]);
  const float hinv = static_cast<float>(inv_h);
  const int ngrp = (nb + 3) / 4;
  const int nt = n / kTile;
  const long long ntiles = static_cast<long long>(nt) * nt * nt;
  const int mask = n - 1;
  // full batches of kAPB consecutive particles of the tile-sorted catalogue (a tile holds few
  // particles at galaxy-catalogue densities; consecutive tiles keep the batch's stencils close together)
  const long long ptot = tile_start[ntiles];
  {
    for (long long bs = static_cast<long long>(blockIdx.x) * kAPB; bs < ptot;
         bs += static_cast<long long>(gridDim.x) * kAPB) {
      const int cnt = static_cast<int>((ptot - bs) < kAPB ? (ptot - bs) : kAPB);
      __syncthreads();
      if (threadIdx.x < cnt) {
        const int me = threadIdx.x;
        const float4 pp = sorted[bs + me];
        float tx, ty, tz;
        const int cx = cell_t(pp.x, inv_h, n, tx), cy = cell_t(pp.y, inv_h, n, ty), cz = cell_t(pp.z, inv_h, n, tz);
        float w[D], dw[D];
        bs_w<D>(tx, w, dw);
        for (int o = 0; o < D; ++o) {
          bw[me][o] = w[o];
          bw[me][3 * D + o] = dw[o] * hinv;
        }
        bs_w<D>(ty, w, dw);
        for (int o = 0; o < D; ++o) {
          bw[me][D + o] = w[o];
          bw[me][4 * D + o] = dw[o] * hinv;
        }
        bs_w<D>(tz, w, dw);
        for (int o = 0; o < D; ++o) {
          bw[me][2 * D + o] = w[o];
          bw[me][5 * D + o] = dw[o] * hinv;
        }
        org[me] = make_int4(cx - OFF, cy - OFF, cz - OFF, 0);
        pw[me] = (isfinite(pp.w) && isfinite(pp.x) && isfinite(pp.y) && isfinite(pp.z)) ? pp.w : 0.f;
      }
      __syncthreads();
      // values and gradients of every field group at every particle of the batch
      for (int task = threadIdx.x; task < cnt * ngrp; task += blockDim.x) {
        const int p = task % cnt, g = task / cnt;
        const int4 o = org[p];
        const float* w = bw[p];
        const float4* base = f4 + g * ng;
        float4 v0 = make_float4(0.f, 0.f, 0.f, 0.f), gx = v0, gy = v0, gz = v0;
        for (int oz = 0; oz < D; ++oz) {
          const long long zrow = static_cast<long long>((o.z + oz) & mask) * n;
          for (int oy = 0; oy < D; ++oy) {
            const float4* row = base + (zrow + ((o.y + oy) & mask)) * n;
            const float wyz = w[2 * D + oz] * w[D + oy];
            const float dy = w[2 * D + oz] * w[4 * D + oy];
            const float dz = w[5 * D + oz] * w[D + oy];
            for (int ox = 0; ox < D; ++ox) {
              const float4 v = __ldg(row + ((o.x + ox) & mask));
              const float a = wyz * w[ox], ax = wyz * w[3 * D + ox], ay = dy * w[ox], az = dz * w[ox];
              v0.x = fmaf(a, v.x, v0.x); v0.y = fmaf(a, v.y, v0.y); v0.z = fmaf(a, v.z, v0.z); v0.w = fmaf(a, v.w, v0.w);
              gx.x = fmaf(ax, v.x, gx.x); gx.y = fmaf(ax, v.y, gx.y); gx.z = fmaf(ax, v.z, gx.z); gx.w = fmaf(ax, v.w, gx.w);
              gy.x = fmaf(ay, v.x, gy.x); gy.y = fmaf(ay, v.y, gy.y); gy.z = fmaf(ay, v.z, gy.z); gy.w = fmaf(ay, v.w, gy.w);
              gz.x = fmaf(az, v.x, gz.x); gz.y = fmaf(az, v.y, gz.y); gz.z = fmaf(az, v.z, gz.z); gz.w = fmaf(az, v.w, gz.w);
            }
          }
        }
        const float vv[4] = {v0.x, v0.y, v0.z, v0.w};
        const float xx[4] = {gx.x, gx.y, gx.z, gx.w};
        const float yy[4] = {gy.x, gy.y, gy.z, gy.w};
        const float zz[4] = {gz.x, gz.y, gz.z, gz.w};
        for (int j = 0; j < 4; ++j) {
          fv[p][4 * g + j] = vv[j];
          gv[p][4 * g + j][0] = xx[j];
          gv[p][4 * g + j][1] = yy[j];
          gv[p][4 * g + j][2] = zz[j];
        }
      }
      __syncthreads();
      // per particle: c = (2 w / W) S f, the direct term, then c replaces f
      if (threadIdx.x < cnt) {
        const int p = threadIdx.x;
        float c[NBP];
        for (int b = 0; b < NBP; ++b) {
          float t = 0.f;
          for (int b2 = 0; b2 < NBP; ++b2) t = fmaf(s_s[b * NBP + b2], (b2 < 4 * ngrp) ? fv[p][b2] : 0.f, t);
          c[b] = wscale * pw[p] * t;
        }
        float dx = 0.f, dy = 0.f, dz = 0.f;
        for (int b = 0; b < 4 * ngrp && b < NBP; ++b) {
          dx = fmaf(c[b], gv[p][b][0], dx);
          dy = fmaf(c[b], gv[p][b][1], dy);
          dz = fmaf(c[b], gv[p][b][2], dz);
        }
        const long long oi = sidx[bs + p];
        direct[3 * oi] += dx;
        direct[3 * oi + 1] += dy;
        direct[3 * oi + 2] += dz;
        for (int b = 0; b < NBP; ++b) fv[p][b] = c[b];
      }
      __syncthreads();
      // scatter c_b with the assignment stencil
      for (int task = threadIdx.x; task < cnt * ngrp; task += blockDim.x) {
        const int p = task % cnt, g = task / cnt;
        const int4 o = org[p];
        const float* w = bw[p];
        const float4 cv = make_float4(fv[p][4 * g], fv[p][4 * g + 1], fv[p][4 * g + 2], fv[p][4 * g + 3]);
        float4* base = h4 + g * ng;
        for (int oz = 0; oz < D; ++oz) {
          const long long zrow = static_cast<long long>((o.z + oz) & mask) * n;
          for (int oy = 0; oy < D; ++oy) {
            float4* row = base + (zrow + ((o.y + oy) & mask)) * n;
            const float wyz = w[2 * D + oz] * w[D + oy];
            for (int ox = 0; ox < D; ++ox) {
              const float a = wyz * w[ox];
              atomicAdd(row + ((o.x + ox) & mask), make_float4(a * cv.x, a * cv.y, a * cv.z, a * cv.w));
            }
          }
        }
      }
    }
  }
}

__global__ void k_adj_finish_node(const float* __restrict__ q, const float* __restrict__ g, long long ng, float inv_ng,
                                  float* __restrict__ grad) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < ng;
       i += static_cast<long long>(blockDim.x) * gridDim.x)
    grad[i] = (q[i] + g[i]) * inv_ng;
}

template <int D>
__global__ void k_adj_finish_particles(const float4* __restrict__ parts, long long np, const float* __restrict__ gd, int n,
                                       double inv_h, const double* __restrict__ wsum, const float* __restrict__ direct,
                                       float* __restrict__ grad) {
  constexpr int OFF = D / 2 - 1;
  const int mask = n - 1;
  const float scale = static_cast<float>(static_cast<double>(n) * n * n / wsum[0]);
  const float hinv = static_cast<float>(inv_h);
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < np;
       i += static_cast<long long>(blockDim.x) * gridDim.x) {
    const float4 pp = parts[i];
    float tx, ty, tz;
    const int cx = cell_t(pp.x, inv_h, n, tx), cy = cell_t(pp.y, inv_h, n, ty), cz = cell_t(pp.z, inv_h, n, tz);
    float wx[D], wy[D], wz[D], dx[D], dy[D], dz[D];
    bs_w<D>(tx, wx, dx);
    bs_w<D>(ty, wy, dy);
    bs_w<D>(tz, wz, dz);
    float g0 = 0.f, g1 = 0.f, g2 = 0.f;
    for (int oz = 0; oz < D; ++oz)
      for (int oy = 0; oy < D; ++oy) {
        const long long row = (static_cast<long long>((cz - OFF + oz) & mask) * n + ((cy - OFF + oy) & mask)) * n;
        for (int ox = 0; ox < D; ++ox) {
          const float v = __ldg(gd + row + ((cx - OFF + ox) & mask));
          g0 = fmaf(dx[ox] * wy[oy] * wz[oz], v, g0);
          g1 = fmaf(wx[ox] * dy[oy] * wz[oz], v, g1);
          g2 = fmaf(wx[ox] * wy[oy] * dz[oz], v, g2);
        }
      }
    const float f = (isfinite(pp.w) ? pp.w : 0.f) * scale * hinv;
    grad[3 * i] = direct[3 * i] + f * g0;
    grad[3 * i + 1] = direct[3 * i + 1] + f * g1;
    grad[3 * i + 2] = direct[3 * i + 2] + f * g2;
  }
}

inline int grid1(long long work, int sms) {
  long long g = (work + kAT - 1) / kAT;
  const long long cap = static_cast<long long>(sms) * 16;
  return static_cast<int>(g < 1 ? 1 : (g > cap ? cap : g));
}
inline int nbp_of(int nb) { return nb <= 8 ? 8 : nb <= 16 ? 16 : nb <= 24 ? 24 : 32; }

}  // namespace

int launch_adj_node_point(const zeta_ctx* c, const float* delta, float* fields, const float* S, float* q,
                          cudaStream_t s) {
  StageScope prof(c, ST_ADJ_POINT, 1, s);
  float4* f4 = reinterpret_cast<float4*>(fields);
  const int g = grid1(c->ng, c->num_sms);
  switch (nbp_of(c->p.nbins)) {
    case 8: k_adj_node<8><<<g, kAT, 0, s>>>(delta, f4, c->ng, c->p.nbins, S, q); break;
    case 16: k_adj_node<16><<<g, kAT, 0, s>>>(delta, f4, c->ng, c->p.nbins, S, q); break;
    case 24: k_adj_node<24><<<g, kAT, 0, s>>>(delta, f4, c->ng, c->p.nbins, S, q); break;
    default: k_adj_node<32><<<g, kAT, 0, s>>>(delta, f4, c->ng, c->p.nbins, S, q); break;
  }
  return cudaGetLastError() == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
}

int launch_adj_mass(const zeta_ctx* c, const float2* dhat, int l, const float* S, float2* gk, cudaStream_t s) {
  StageScope prof(c, ST_ADJ_OTHER, 1, s);
  const int nbp = 4 * ((c->p.nbins + 3) / 4);
  const float* jt = c->d_jtab + static_cast<long long>(l) * c->nn2 * nbp;
  const float coef = static_cast<float>((2.0 * l + 1.0) / (4.0 * 3.14159265358979323846));
  k_adj_mass<<<grid1(c->ng / 2, c->num_sms), kAT, 0, s>>>(dhat, jt, nbp, c->d_mhat, c->n, c->p.nbins, S, coef, gk);
  return cudaGetLastError() == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
}

int launch_adj_points(const zeta_ctx* c, const float4* sorted, const int64_t* tile_start, const int* sorted_idx,
                      const float* fields, const float* S, const double* wsum, float* hfield, float* direct,
                      cudaStream_t s) {
  StageScope prof(c, ST_ADJ_POINT, 1, s);
  const auto* ts = reinterpret_cast<const long long*>(tile_start);
  const auto* f4 = reinterpret_cast<const float4*>(fields);
  auto* h4 = reinterpret_cast<float4*>(hfield);
  const double inv_h = c->n / c->p.box;
  const int g = c->num_sms * 4;
  const int nb = c->p.nbins;
#define ZK_ADJ(P, DD) \
  k_adj_points<P, DD><<<g, kAT, 0, s>>>(sorted, ts, sorted_idx, f4, c->ng, c->n, nb, inv_h, S, wsum, h4, direct)
  const int nbp = nbp_of(nb);
  if (c->p.dsup == 2) {
    if (nbp == 8) ZK_ADJ(8, 2); else if (nbp == 16) ZK_ADJ(16, 2); else if (nbp == 24) ZK_ADJ(24, 2); else ZK_ADJ(32, 2);
  } else {
    if (nbp == 8) ZK_ADJ(8, 4); else if (nbp == 16) ZK_ADJ(16, 4); else if (nbp == 24) ZK_ADJ(24, 4); else ZK_ADJ(32, 4);
  }
#undef ZK_ADJ
  return cudaGetLastError() == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
}

int launch_adj_finish_node(const zeta_ctx* c, const float* q, const float* g, float* grad, cudaStream_t s) {
  StageScope prof(c, ST_ADJ_OTHER, 1, s);
  k_adj_finish_node<<<grid1(c->ng, c->num_sms), kAT, 0, s>>>(q, g, c->ng, static_cast<float>(1.0 / c->ng), grad);
  return cudaGetLastError() == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
}

int launch_adj_finish_particles(const zeta_ctx* c, const float4* parts, int64_t np, const float* gdelta,
                                const double* wsum, const float* direct, float* grad, cudaStream_t s) {
  StageScope prof(c, ST_ADJ_OTHER, 1, s);
  const double inv_h = c->n / c->p.box;
  if (c->p.dsup == 2)
    k_adj_finish_particles<2><<<grid1(np, c->num_sms), kAT, 0, s>>>(parts, np, gdelta, c->n, inv_h, wsum, direct, grad);
  else
    k_adj_finish_particles<4><<<grid1(np, c->num_sms), kAT, 0, s>>>(parts, np, gdelta, c->n, inv_h, wsum, direct, grad);
  return cudaGetLastError() == cudaSuccess ? ZETA_OK : ZETA_ECUDA;
}

}  // namespace zk
