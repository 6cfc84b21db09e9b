// Host float64 tables of the method (Fig. 1 step (3): tabulating the k-space windows).
//
//  * jbar_l(k; b): the radial window of bin b, the r^2-weighted shell average of the
//    spherical Bessel function j_l(k r) (the vertex window of Eq. 3PCF-multipole-window
//    averaged over a radial bin).  Integrated by Gauss-Legendre on sub-intervals no longer
//    than 3 radians of k r; j_0..j_L come from the three-term recurrence, upward when x > L
//    and Miller's downward recurrence (normalised to sin x / x) otherwise, with the power
//    series for x < 1.  Indexed by the integer |n|^2, so each lattice wavevector reads the
//    exact value of its own |k|.
//  * Real spherical harmonics: constants of the fully normalised associated-Legendre
//    recurrence.
//  * B-spline mass (Gram) values M(a) = beta_{2D}(a) and the per-cell Gauss-Legendre
//    quadrature used by the connection-coefficient sum (Eq. con-coeff), from the explicit
//    truncated-power form of the centred cardinal B-spline.
//  * The vertex windows of Sec. 3: the spherical tophat W_TH(kR) = 3 (sin x - x cos x) / x^3
//    that may multiply every secondary vertex (and smooth the primary one), the point-radius
//    shell j_l(k r) of Eq. 3PCF-multipole-window, and the basis power spectrum Phi-hat (Fig. 1
//    step (3)) as a per-axis factor sinc^{2D}(pi n_d / n).
//  * DFT twiddles.
#include <cmath>
#include <cstdlib>
#include <thread>
#include <utility>
#include <vector>

#include "zeta_internal.h"

namespace zk {
namespace {

constexpr double kPi = 3.14159265358979323846;

void gauss_legendre(int q, std::vector<double>& x, std::vector<double>& w) {
  x.assign(q, 0.0);
  w.assign(q, 0.0);
  for (int i = 0; i < q; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (q + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= q; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      // p1 = P_q(z), p0 = P_{q-1}(z)
      double dp = q * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) {
        p0 = 1.0;
        p1 = z;
        for (int k = 2; k <= q; ++k) {
          double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        dp = q * (z * p1 - p0) / (z * z - 1.0);
        break;
      }
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= q; ++k) {
      double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    const double dp = q * (z * p1 - p0) / (z * z - 1.0);
    x[i] = -z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// j_0 .. j_L at x >= 0 into j[0..L] (j must hold max(L, 1) + 1 values).
void sph_bessel_all(int L, double x, double* j) {
  if (x == 0.0) {
    j[0] = 1.0;
    for (int l = 1; l <= L; ++l) j[l] = 0.0;
    return;
  }
  if (x < 1.0) {
    // j_l(x) = x^l / (2l+1)!! * sum_k (-x^2/2)^k / (k! (2l+3)(2l+5)...(2l+2k+1))
    double lead = 1.0;  // x^l / (2l+1)!!
    for (int l = 0; l <= L; ++l) {
      if (l > 0) lead *= x / (2.0 * l + 1.0);
      double term = 1.0, sum = 1.0;
      for (int k = 1; k < 30; ++k) {
        term *= -0.5 * x * x / (k * (2.0 * l + 2.0 * k + 1.0));
        sum += term;
        if (std::fabs(term) < 1e-18 * std::fabs(sum)) break;
      }
      j[l] = lead * sum;
    }
    return;
  }
  const double s = std::sin(x), c = std::cos(x);
  const double j0 = s / x;
  const double j1 = s / (x * x) - c / x;
  if (x > L) {
    j[0] = j0;
    if (L >= 1) j[1] = j1;
    for (int l = 1; l < L; ++l) j[l + 1] = (2.0 * l + 1.0) / x * j[l] - j[l - 1];
    return;
  }
  const int lstart = L + 30 + static_cast<int>(x);
  std::vector<double> f(lstart + 2, 0.0);
  f[lstart] = 1e-300;
  for (int l = lstart; l >= 1; --l) {
    f[l - 1] = (2.0 * l + 1.0) / x * f[l] - f[l + 1];
    if (std::fabs(f[l - 1]) > 1e250) {  // rescale to stay finite
      for (int q = l - 1; q <= lstart; ++q) f[q] *= 1e-250;
    }
  }
  // f is proportional to the minimal solution j_l; normalise on the larger of j_0, j_1
  const double scale = (std::fabs(j0) >= std::fabs(j1)) ? j0 / f[0] : j1 / f[1];
  for (int l = 0; l <= L; ++l) j[l] = f[l] * scale;
}

double cardinal_bspline(int order, double x) {
  // centred cardinal B-spline of the given order (degree order-1, support [-order/2, order/2])
  double sum = 0.0, binom = 1.0, fact = 1.0;
  for (int k = 1; k < order; ++k) fact *= k;
  for (int jj = 0; jj <= order; ++jj) {
    const double t = x + 0.5 * order - jj;
    if (t > 0.0) sum += ((jj & 1) ? -binom : binom) * std::pow(t, order - 1);
    binom = binom * (order - jj) / (jj + 1.0);
  }
  return sum / fact;
}

// Accumulate sum_q w_q r_q^2 j_l(k r_q) over [r_lo, r_hi) for l <= L into num[0..L].
void shell_moments(int L, double k, double r_lo, double r_hi, const std::vector<double>& gx,
                   const std::vector<double>& gw, double* num) {
  const int nsub = std::max(1, static_cast<int>(std::ceil(k * (r_hi - r_lo) / 3.0)));
  const double h = (r_hi - r_lo) / nsub;
  double jl[kMaxL + 2];
  for (int l = 0; l <= L; ++l) num[l] = 0.0;
  for (int s = 0; s < nsub; ++s) {
    const double a = r_lo + s * h;
    for (size_t q = 0; q < gx.size(); ++q) {
      const double r = a + 0.5 * h * (gx[q] + 1.0);
      sph_bessel_all(L, k * r, jl);
      const double wr = 0.5 * h * gw[q] * r * r;
      for (int l = 0; l <= L; ++l) num[l] += wr * jl[l];
    }
  }
}

}  // namespace

void host_jbar_values(int l, double box, double r_lo, double r_hi, const int64_t* n2, int64_t count,
                      double* out) {
  std::vector<double> gx, gw;
  gauss_legendre(12, gx, gw);
  const double den = (r_hi * r_hi * r_hi - r_lo * r_lo * r_lo) / 3.0;
  double num[kMaxL + 2];
  for (int64_t i = 0; i < count; ++i) {
    const double k = 2.0 * kPi / box * std::sqrt(static_cast<double>(n2[i]));
    shell_moments(l, k, r_lo, r_hi, gx, gw, num);
    out[i] = num[l] / den;
  }
}

double tophat_window(double x) {
  if (std::fabs(x) < 1e-2) {
    const double x2 = x * x;
    return 1.0 - x2 / 10.0 + x2 * x2 / 280.0;
  }
  return 3.0 * (std::sin(x) - x * std::cos(x)) / (x * x * x);
}

void host_jbar_table(int n, double box, int lmax, int nbins, const double* edges, std::vector<float>& out) {
  VertexSpec v;
  v.edges = edges;
  host_window_table(n, box, lmax, nbins, v, out);
}

void host_window_table(int n, double box, int lmax, int nbins, const VertexSpec& v, std::vector<float>& out) {
  const int64_t nn2 = table_n2_count(n);
  const double ng = static_cast<double>(n) * n * n;
  const double pref = std::sqrt(4.0 * kPi) / ng;
  const int nbp = 4 * ((nbins + 3) / 4);
  out.assign(static_cast<size_t>(lmax + 1) * nn2 * nbp, 0.0f);
  std::vector<double> gx, gw;
  gauss_legendre(12, gx, gw);
  unsigned nth = std::thread::hardware_concurrency();
  if (nth == 0) nth = 1;
  if (nth > 64) nth = 64;
  auto work = [&](unsigned t) {
    double num[kMaxL + 2];
    for (int64_t i = t; i < nn2; i += nth) {
      const double k = 2.0 * kPi / box * std::sqrt(static_cast<double>(i));
      const double wth = v.tophat > 0.0 ? tophat_window(k * v.tophat) : 1.0;
      for (int b = 0; b < nbins; ++b) {
        double den = 1.0;
        if (v.radial == ZETA_RADIAL_POINT) {
          sph_bessel_all(lmax, k * v.radii[b], num);
        } else {
          const double r_lo = v.edges[b], r_hi = v.edges[b + 1];
          den = (r_hi * r_hi * r_hi - r_lo * r_lo * r_lo) / 3.0;
          shell_moments(lmax, k, r_lo, r_hi, gx, gw, num);
        }
        for (int l = 0; l <= lmax; ++l)
          out[(static_cast<size_t>(l) * nn2 + i) * nbp + b] = static_cast<float>(pref * wth * num[l] / den);
      }
    }
  };
  std::vector<std::thread> pool;
  for (unsigned t = 1; t < nth; ++t) pool.emplace_back(work, t);
  work(0);
  for (auto& th : pool) th.join();
}

void host_twiddles(int n, std::vector<float2>& out) {
  out.resize(n);
  for (int e = 0; e < n; ++e) {
    const double ang = 2.0 * kPi * e / n;
    out[e] = make_float2(static_cast<float>(std::cos(ang)), static_cast<float>(-std::sin(ang)));
  }
}

void host_ylm_constants(double* mm, double* a, double* b) {
  for (int m = 0; m <= kMaxL; ++m) {
    double prod = 1.0;
    for (int k = 1; k <= m; ++k) prod *= (2.0 * k - 1.0) / (2.0 * k);
    mm[m] = std::sqrt((2.0 * m + 1.0) / (4.0 * kPi) * prod);
  }
  for (int l = 0; l <= kMaxL; ++l) {
    for (int m = 0; m <= kMaxL; ++m) {
      double av = 0.0, bv = 0.0;
      if (l >= m + 1) {
        const double l2 = static_cast<double>(l) * l, m2 = static_cast<double>(m) * m;
        av = std::sqrt((4.0 * l2 - 1.0) / (l2 - m2));
        if (l >= m + 2) bv = std::sqrt((2.0 * l + 1.0) * ((l - 1.0) * (l - 1.0) - m2) / ((2.0 * l - 3.0) * (l2 - m2)));
      }
      a[l * (kMaxL + 1) + m] = av;
      b[l * (kMaxL + 1) + m] = bv;
    }
  }
}

// ---- the genus-4 Daubechies scaling function (dsup = 3; Sec. 2.2, D_sup = 3) ----
// Low-pass taps h_k = (1 + s, 3 + s, 3 - s, 1 - s) / (4 sqrt2), s = sqrt3, and the two-scale
// relation phi(x) = sqrt2 sum_k h_k phi(2x - k), support [0, 3].
static void daub4_taps(double* h) {
  const double s = std::sqrt(3.0), d = 4.0 * std::sqrt(2.0);
  h[0] = (1.0 + s) / d;
  h[1] = (3.0 + s) / d;
  h[2] = (3.0 - s) / d;
  h[3] = (1.0 - s) / d;
}

void host_daub4_dyadic(int level, std::vector<double>& out) {
  double h[4];
  daub4_taps(h);
  const double r2 = std::sqrt(2.0);
  // the integers: phi(1) = sqrt2 (h1 phi(1) + h0 phi(2)) with phi(1) + phi(2) = 1
  const double ratio = r2 * h[0] / (1.0 - r2 * h[1]);  // phi(1) / phi(2)
  const double p2 = 1.0 / (1.0 + ratio);
  std::vector<double> cur = {0.0, ratio * p2, p2, 0.0};
  for (int j = 0; j < level; ++j) {
    const int64_t unit = int64_t(1) << j;  // points per unit at level j
    const int64_t m = 6 * unit;            // last index at level j + 1
    std::vector<double> nxt(static_cast<size_t>(m + 1), 0.0);
    for (int64_t k = 0; k <= m; ++k) {
      if ((k & 1) == 0) {
        nxt[k] = cur[k / 2];
        continue;
      }
      double v = 0.0;  // phi(k / 2^(j+1)) = sqrt2 sum_i h_i phi(k / 2^j - i)
      for (int i = 0; i < 4; ++i) {
        const int64_t src = k - i * unit;
        if (src >= 0 && src <= 3 * unit) v += h[i] * cur[src];
      }
      nxt[k] = r2 * v;
    }
    cur.swap(nxt);
  }
  out.swap(cur);
}

double host_daub4_power(double omega) {
  // |phi-hat|^2 = prod_{j>=1} |m0(omega / 2^j)|^2 with |m0(w)|^2 = cos^4(w/2) (1 + 2 sin^2(w/2)) and
  // prod_{j>=1} cos(omega / 2^(j+1)) = sin(omega/2) / (omega/2)
  const double x = 0.5 * omega;
  const double sinc = x == 0.0 ? 1.0 : std::sin(x) / x;
  double p = sinc * sinc * sinc * sinc;
  double w = 0.25 * omega;
  for (int j = 0; j < 64 && w != 0.0; ++j, w *= 0.5) {
    const double sw = std::sin(w);
    p *= 1.0 + 2.0 * sw * sw;
  }
  return p;
}

// Solves the square system a x = b (size m, row-major a) by Gaussian elimination with partial
// pivoting; a and b are overwritten.
static void solve_dense(int m, std::vector<double>& a, std::vector<double>& b, std::vector<double>& x) {
  for (int c = 0; c < m; ++c) {
    int piv = c;
    for (int r = c + 1; r < m; ++r)
      if (std::fabs(a[r * m + c]) > std::fabs(a[piv * m + c])) piv = r;
    if (piv != c) {
      for (int k = 0; k < m; ++k) std::swap(a[c * m + k], a[piv * m + k]);
      std::swap(b[c], b[piv]);
    }
    for (int r = c + 1; r < m; ++r) {
      const double f = a[r * m + c] / a[c * m + c];
      if (f == 0.0) continue;
      for (int k = c; k < m; ++k) a[r * m + k] -= f * a[c * m + k];
      b[r] -= f * b[c];
    }
  }
  x.assign(m, 0.0);
  for (int r = m - 1; r >= 0; --r) {
    double v = b[r];
    for (int k = r + 1; k < m; ++k) v -= a[r * m + k] * x[k];
    x[r] = v / a[r * m + r];
  }
}

void host_daub4_gamma(double* g) {
  // Gamma(a, b) = int phi(x) phi(x-a) phi(x-b) dx, |a|, |b| <= 2, index (a+2) * 5 + (b+2):
  // the two-scale relation gives Gamma(a, b) = sqrt2 sum_{i,j,k} h_i h_j h_k Gamma(2a+j-i, 2b+k-i)
  // (zero where the supports do not overlap, |a - b| >= 3), and the partition of unity with the
  // orthonormality of phi gives sum_b Gamma(a, b) = [a == 0].  The stacked (25 + 5) x 25 system
  // is solved through its normal equations.
  double h[4];
  daub4_taps(h);
  const double r2 = std::sqrt(2.0);
  const int m = 25, rows = 30;
  std::vector<double> a(static_cast<size_t>(rows) * m, 0.0), rhs(rows, 0.0);
  for (int ia = -2; ia <= 2; ++ia)
    for (int ib = -2; ib <= 2; ++ib) {
      const int r = (ia + 2) * 5 + (ib + 2);
      a[r * m + r] -= 1.0;
      if (std::abs(ia - ib) >= 3) continue;  // the equation reads Gamma = 0 there
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j)
          for (int k = 0; k < 4; ++k) {
            const int p = 2 * ia + j - i, q = 2 * ib + k - i;
            if (p < -2 || p > 2 || q < -2 || q > 2 || std::abs(p - q) >= 3) continue;
            a[r * m + (p + 2) * 5 + (q + 2)] += r2 * h[i] * h[j] * h[k];
          }
    }
  for (int ia = -2; ia <= 2; ++ia) {
    const int r = 25 + ia + 2;
    for (int ib = -2; ib <= 2; ++ib) a[r * m + (ia + 2) * 5 + (ib + 2)] = 1.0;
    rhs[r] = ia == 0 ? 1.0 : 0.0;
  }
  std::vector<double> ata(static_cast<size_t>(m) * m, 0.0), atb(m, 0.0), x;
  for (int i = 0; i < m; ++i) {
    for (int j = 0; j < m; ++j) {
      double v = 0.0;
      for (int r = 0; r < rows; ++r) v += a[r * m + i] * a[r * m + j];
      ata[i * m + j] = v;
    }
    double v = 0.0;
    for (int r = 0; r < rows; ++r) v += a[r * m + i] * rhs[r];
    atb[i] = v;
  }
  solve_dense(m, ata, atb, x);
  for (int i = 0; i < m; ++i) g[i] = x[i];
}

void host_daub4_gamma_split(std::vector<double>& lam, std::vector<double>& u) {
  // gamma = U diag(lam) U^T by cyclic Jacobi rotations (gamma is symmetric 5 x 5)
  double g[25];
  host_daub4_gamma(g);
  double a[5][5], v[5][5];
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) {
      a[i][j] = 0.5 * (g[i * 5 + j] + g[j * 5 + i]);
      v[i][j] = i == j ? 1.0 : 0.0;
    }
  for (int sweep = 0; sweep < 64; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < 5; ++i)
      for (int j = i + 1; j < 5; ++j) off += a[i][j] * a[i][j];
    if (off < 1e-34) break;
    for (int p = 0; p < 5; ++p)
      for (int q = p + 1; q < 5; ++q) {
        if (a[p][q] == 0.0) continue;
        const double th = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
        const double t = (th >= 0.0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < 5; ++k) {  // columns p, q
          const double akp = a[k][p], akq = a[k][q];
          a[k][p] = c * akp - s * akq;
          a[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < 5; ++k) {  // rows p, q
          const double apk = a[p][k], aqk = a[q][k];
          a[p][k] = c * apk - s * aqk;
          a[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < 5; ++k) {
          const double vkp = v[k][p], vkq = v[k][q];
          v[k][p] = c * vkp - s * vkq;
          v[k][q] = s * vkp + c * vkq;
        }
      }
  }
  lam.assign(5, 0.0);
  u.assign(25, 0.0);
  for (int k = 0; k < 5; ++k) {
    lam[k] = a[k][k];
    for (int o = 0; o < 5; ++o) u[o * 5 + k] = v[o][k];  // u[o][k]: offset o - 2, eigenvector k
  }
}

void host_mass_1d(int dsup, double* out) {
  if (dsup == 3) {  // orthonormal basis: M(a) = [a == 0]
    for (int a = -2; a <= 2; ++a) out[a + 2] = a == 0 ? 1.0 : 0.0;
    return;
  }
  for (int a = -(dsup - 1); a <= dsup - 1; ++a) out[a + dsup - 1] = cardinal_bspline(2 * dsup, a);
}

static void mass_hat_f64(int n, int dsup, double* out) {
  double m[16];
  host_mass_1d(dsup, m);
  for (int k = 0; k < n; ++k) {
    double v = m[dsup - 1];
    for (int a = 1; a < dsup; ++a) v += 2.0 * m[dsup - 1 + a] * std::cos(2.0 * kPi * k * a / n);
    out[k] = v;
  }
}

void host_mass_hat(int n, int dsup, std::vector<float>& out, bool with_phi) {
  std::vector<double> v(n), ph;
  mass_hat_f64(n, dsup, v.data());
  if (with_phi) host_phi_hat_1d(n, dsup, ph);
  out.resize(n);
  for (int k = 0; k < n; ++k) out[k] = static_cast<float>(with_phi ? v[k] * ph[k] * ph[k] : v[k]);
}

void host_phi_hat_1d(int n, int dsup, std::vector<double>& out) {
  out.resize(n);
  for (int i = 0; i < n; ++i) {
    const int f = i < n / 2 ? i : i - n;
    if (dsup == 3) {
      out[i] = host_daub4_power(2.0 * kPi * f / n);
      continue;
    }
    const double x = kPi * f / n;
    const double sinc = f == 0 ? 1.0 : std::sin(x) / x;
    out[i] = std::pow(sinc, 2 * dsup);
  }
}

void host_tophat_table(int n, double box, double radius, std::vector<float>& out) {
  const int64_t nn2 = table_n2_count(n);
  out.resize(nn2);
  const double ng = static_cast<double>(n) * n * n;
  for (int64_t i = 0; i < nn2; ++i)
    out[i] = static_cast<float>(tophat_window(2.0 * kPi / box * std::sqrt(static_cast<double>(i)) * radius) / ng);
}

void host_cell_quadrature(int q, int dsup, std::vector<double>& t, std::vector<double>& wq,
                          std::vector<double>& beta) {
  std::vector<double> gx, gw;
  gauss_legendre(q, gx, gw);
  t.resize(q);
  wq.resize(q);
  beta.resize(static_cast<size_t>(q) * dsup);
  for (int i = 0; i < q; ++i) {
    t[i] = 0.5 * (gx[i] + 1.0);
    wq[i] = 0.5 * gw[i];
    for (int o = 0; o < dsup; ++o) beta[i * dsup + o] = cardinal_bspline(dsup, t[i] + dsup / 2 - 1 - o);
  }
}

}  // namespace zk

extern "C" int zeta_host_jbar(int l, double box, double r_lo, double r_hi, const int64_t* n2, int64_t count,
                              double* out) {
  if (l < 0 || l > zk::kMaxL || !(box > 0) || !(r_lo > 0) || !(r_hi > r_lo) || count < 0 || (count && (!n2 || !out)))
    return ZETA_EINVAL;
  for (int64_t i = 0; i < count; ++i)
    if (n2[i] < 0) return ZETA_EINVAL;
  zk::host_jbar_values(l, box, r_lo, r_hi, n2, count, out);
  return ZETA_OK;
}

extern "C" int zeta_host_jbar_table(int n, double box, int lmax, int nbins, const double* edges, float* out) {
  if (n < 4 || n > 512 || (n & (n - 1)) || !(box > 0) || lmax < 0 || lmax > zk::kMaxL || nbins < 1 ||
      nbins > zk::kMaxBins || !edges || !out)
    return ZETA_EINVAL;
  if (!(edges[0] > 0)) return ZETA_EINVAL;
  for (int b = 0; b < nbins; ++b)
    if (!(edges[b + 1] > edges[b])) return ZETA_EINVAL;
  std::vector<float> t;
  zk::host_jbar_table(n, box, lmax, nbins, edges, t);
  for (size_t i = 0; i < t.size(); ++i) out[i] = t[i];
  return ZETA_OK;
}

extern "C" int zeta_host_window_table(const zeta_params* p, float* out) {
  if (!p || !out || p->n < 4 || p->n > 512 || (p->n & (p->n - 1)) || !(p->box > 0) || p->lmax < 0 ||
      p->lmax > zk::kMaxL || p->nbins < 1 || p->nbins > zk::kMaxBins || p->tophat < 0 || !std::isfinite(p->tophat))
    return ZETA_EINVAL;
  zk::VertexSpec v;
  v.radial = p->radial;
  v.edges = p->edges;
  v.radii = p->radii;
  v.tophat = p->tophat;
  if (p->radial == ZETA_RADIAL_POINT) {
    if (!p->radii) return ZETA_EINVAL;
    for (int b = 0; b < p->nbins; ++b)
      if (!(p->radii[b] > 0) || !std::isfinite(p->radii[b])) return ZETA_EINVAL;
  } else if (p->radial == ZETA_RADIAL_SHELL) {
    if (!p->edges || !(p->edges[0] > 0)) return ZETA_EINVAL;
    for (int b = 0; b < p->nbins; ++b)
      if (!(p->edges[b + 1] > p->edges[b])) return ZETA_EINVAL;
  } else {
    return ZETA_EINVAL;
  }
  std::vector<float> t;
  zk::host_window_table(p->n, p->box, p->lmax, p->nbins, v, t);
  for (size_t i = 0; i < t.size(); ++i) out[i] = t[i];
  return ZETA_OK;
}

extern "C" int zeta_host_phi_hat(int n, int dsup, double* out) {
  if (n < 2 || n > (1 << 20) || dsup < 2 || dsup > 4 || !out) return ZETA_EINVAL;
  std::vector<double> v;
  zk::host_phi_hat_1d(n, dsup, v);
  for (int i = 0; i < n; ++i) out[i] = v[i];
  return ZETA_OK;
}

extern "C" int zeta_host_mass_hat(int n, int dsup, double* out) {
  if (n < 2 || n > (1 << 20) || dsup < 2 || dsup > 4 || !out) return ZETA_EINVAL;
  zk::mass_hat_f64(n, dsup, out);
  return ZETA_OK;
}

extern "C" int zeta_host_cell_quadrature(int q, int dsup, double* t, double* wq, double* beta) {
  if (q < 1 || q > 32 || (dsup != 2 && dsup != 4) || !t || !wq || !beta) return ZETA_EINVAL;
  std::vector<double> tv, wv, bv;
  zk::host_cell_quadrature(q, dsup, tv, wv, bv);
  for (int i = 0; i < q; ++i) {
    t[i] = tv[i];
    wq[i] = wv[i];
  }
  for (size_t i = 0; i < bv.size(); ++i) beta[i] = bv[i];
  return ZETA_OK;
}

extern "C" int zeta_host_daub4_dyadic(int level, double* out) {
  if (level < 0 || level > 20 || !out) return ZETA_EINVAL;
  std::vector<double> v;
  zk::host_daub4_dyadic(level, v);
  for (size_t i = 0; i < v.size(); ++i) out[i] = v[i];
  return ZETA_OK;
}

extern "C" int zeta_host_daub4_gamma(double* gamma, double* lam, double* u) {
  if (!gamma) return ZETA_EINVAL;
  zk::host_daub4_gamma(gamma);
  if (lam && u) {
    std::vector<double> l, uv;
    zk::host_daub4_gamma_split(l, uv);
    for (int k = 0; k < 5; ++k) lam[k] = l[k];
    for (int k = 0; k < 25; ++k) u[k] = uv[k];
  }
  return ZETA_OK;
}

extern "C" double zeta_host_ylm(int l, int m, double vx, double vy, double vz) {
  if (l < 0 || l > zk::kMaxL || m < -l || m > l) return 0.0;
  // constants built once; a function-local static is initialised thread-safely (C++11)
  struct Consts {
    double mm[zk::kMaxL + 1], a[(zk::kMaxL + 1) * (zk::kMaxL + 1)], b[(zk::kMaxL + 1) * (zk::kMaxL + 1)];
    Consts() { zk::host_ylm_constants(mm, a, b); }
  };
  static const Consts k;
  const double* mm = k.mm;
  const double* a = k.a;
  const double* b = k.b;
  const double r2 = vx * vx + vy * vy + vz * vz;
  if (r2 == 0.0) return l == 0 ? 1.0 / std::sqrt(4.0 * 3.14159265358979323846) : 0.0;
  const double rinv = 1.0 / std::sqrt(r2);
  const double ct = vz * rinv, sx = vx * rinv, sy = vy * rinv;
  const int am = m < 0 ? -m : m;
  double cr = 1.0, ci = 0.0;
  for (int k = 0; k < am; ++k) {
    const double t = cr * sx - ci * sy;
    ci = cr * sy + ci * sx;
    cr = t;
  }
  double qm1 = 0.0, qc = mm[am];
  for (int ll = am + 1; ll <= l; ++ll) {
    const double qn = a[ll * (zk::kMaxL + 1) + am] * ct * qc - b[ll * (zk::kMaxL + 1) + am] * qm1;
    qm1 = qc;
    qc = qn;
  }
  const double ang = (m == 0) ? 1.0 : std::sqrt(2.0) * (m > 0 ? cr : ci);
  return qc * ang;
}

extern "C" int zeta_host_legendre_sum(int lmax, int nb, const double* zeta_l, int nmu, const double* mu, double* out) {
  if (lmax < 0 || nb < 1 || nmu < 1 || !zeta_l || !mu || !out) return ZETA_EINVAL;
  const size_t nb2 = static_cast<size_t>(nb) * nb;
  for (int i = 0; i < nmu; ++i) {
    if (!(mu[i] >= -1.0 && mu[i] <= 1.0)) return ZETA_EINVAL;
    double* o = out + i * nb2;
    for (size_t e = 0; e < nb2; ++e) o[e] = 0.0;
    double p0 = 1.0, p1 = mu[i];
    for (int l = 0; l <= lmax; ++l) {
      const double pl = l == 0 ? p0 : p1;
      for (size_t e = 0; e < nb2; ++e) o[e] += pl * zeta_l[l * nb2 + e];
      if (l >= 1) {
        const double p2 = ((2.0 * l + 1.0) * mu[i] * p1 - l * p0) / (l + 1.0);
        p0 = p1;
        p1 = p2;
      }
    }
  }
  return ZETA_OK;
}

extern "C" int zeta_host_reduced_q(int count, const double* zeta, const double* xi1, const double* xi2,
                                   const double* xi3, double* q) {
  if (count < 0 || (count && (!zeta || !xi1 || !xi2 || !xi3 || !q))) return ZETA_EINVAL;
  for (int i = 0; i < count; ++i)
    q[i] = zeta[i] / (xi1[i] * xi2[i] + xi2[i] * xi3[i] + xi3[i] * xi1[i]);
  return ZETA_OK;
}
