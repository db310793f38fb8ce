// Host-side builders: Fourier continuation tables (Sec. 4), FFT plans,
// twiddle and chirp tables.  Everything here runs once per context.
//
// Quad precision: the FC(Gram) trigonometric least squares is ill-conditioned
// (condition number ~1e16), so it is solved with Householder QR in IEEE
// binary128 (x86-64: __float128/libquadmath; aarch64: long double), and the
// twiddles/chirps are evaluated there too, then rounded once to FP64.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "fcsph_internal.h"

#if defined(__x86_64__)
#include <quadmath.h>
typedef __float128 qreal;
static inline qreal qcos(qreal x) { return cosq(x); }
static inline qreal qsin(qreal x) { return sinq(x); }
static inline qreal qsqrt(qreal x) { return sqrtq(x); }
static inline qreal qabs(qreal x) { return fabsq(x); }
static const qreal QPI = M_PIq;
#elif defined(__aarch64__)
typedef long double qreal;  // IEEE binary128 on aarch64 Linux
static inline qreal qcos(qreal x) { return cosl(x); }
static inline qreal qsin(qreal x) { return sinl(x); }
static inline qreal qsqrt(qreal x) { return sqrtl(x); }
static inline qreal qabs(qreal x) { return fabsl(x); }
static const qreal QPI = 3.141592653589793238462643383279502884L;
#else
#error "fcsph needs a binary128 type (x86-64 or aarch64)"
#endif

namespace fcsph {

// ---------------------------------------------------------------------------
// Dense least squares min ||A X - B|| by Householder QR (A: m x n, m >= n,
// full column rank; B: m x k).  Row-major storage.  Returns X (n x k).
static std::vector<qreal> lsq_qr(std::vector<qreal> A, int m, int n, std::vector<qreal> B, int k) {
  for (int c = 0; c < n; ++c) {
    qreal norm = 0;
    for (int r = c; r < m; ++r) norm += A[r * n + c] * A[r * n + c];
    norm = qsqrt(norm);
    qreal alpha = A[c * n + c] > 0 ? -norm : norm;
    std::vector<qreal> v(m - c);
    for (int r = c; r < m; ++r) v[r - c] = A[r * n + c];
    v[0] -= alpha;
    qreal vv = 0;
    for (qreal x : v) vv += x * x;
    if (vv == 0) continue;
    for (int j = c; j < n; ++j) {
      qreal s = 0;
      for (int r = c; r < m; ++r) s += v[r - c] * A[r * n + j];
      s = 2 * s / vv;
      for (int r = c; r < m; ++r) A[r * n + j] -= s * v[r - c];
    }
    for (int j = 0; j < k; ++j) {
      qreal s = 0;
      for (int r = c; r < m; ++r) s += v[r - c] * B[r * k + j];
      s = 2 * s / vv;
      for (int r = c; r < m; ++r) B[r * k + j] -= s * v[r - c];
    }
  }
  std::vector<qreal> X(n * k);
  for (int j = 0; j < k; ++j) {
    for (int r = n - 1; r >= 0; --r) {
      qreal s = B[r * k + j];
      for (int c = r + 1; c < n; ++c) s -= A[r * n + c] * X[c * k + j];
      X[r * k + j] = s / A[r * n + r];
    }
  }
  return X;
}

// FC(Gram), Sec. 4.5: the right-wall data (matching nodes u = 0..d-1, wall at
// u = d-1, unit = dy) are represented by their degree-(d-1) polynomial and
// continued by a trigonometric polynomial of period T = 2(2d + C - 2) with
// K = floor(T/4) modes, fitted in the least-squares sense to that polynomial
// on [0, d-1] and to zero on [d+C, 2d+C-1] (20 points per unit interval on
// both).  Evaluated at the C continuation nodes u = d..d+C-1; the left wall
// is the mirror image.  E = [E_r | E_l], E_l[c][a] = E_r[C-1-c][d-1-a].
static void gram_table(int d, int C, std::vector<double>* E) {
  const int T = 2 * (2 * d + C - 2);
  const int K = T / 4;
  const int ovs = 20;
  const int npi = (d - 1) * ovs + 1;  // fit points per interval
  const int m = 2 * npi, n = 2 * K + 1;
  std::vector<qreal> A(m * n), B(m * d, 0);
  const int per = ovs * T;  // angles are 2 pi * (k * U mod per) / per, U = ovs * u
  for (int r = 0; r < m; ++r) {
    const int U = r < npi ? r : ovs * (d + C) + (r - npi);
    A[r * n + 0] = 1;
    for (int kk = 1; kk <= K; ++kk) {
      const qreal ang = 2 * QPI * (qreal)((long long)kk * U % per) / (qreal)per;
      A[r * n + 2 * kk - 1] = qcos(ang);
      A[r * n + 2 * kk] = qsin(ang);
    }
    if (r < npi) {  // Lagrange basis of the matching nodes at u = U / ovs
      const qreal u = (qreal)U / ovs;
      for (int a = 0; a < d; ++a) {
        qreal v = 1;
        for (int b = 0; b < d; ++b)
          if (b != a) v *= (u - b) / (qreal)(a - b);
        B[r * d + a] = v;
      }
    }
  }
  std::vector<qreal> X = lsq_qr(A, m, n, B, d);
  std::vector<double> Er(C * d);
  for (int c = 0; c < C; ++c) {
    const int U = ovs * (d + c);
    std::vector<qreal> row(n);
    row[0] = 1;
    for (int kk = 1; kk <= K; ++kk) {
      const qreal ang = 2 * QPI * (qreal)((long long)kk * U % per) / (qreal)per;
      row[2 * kk - 1] = qcos(ang);
      row[2 * kk] = qsin(ang);
    }
    for (int a = 0; a < d; ++a) {
      qreal s = 0;
      for (int j = 0; j < n; ++j) s += row[j] * X[j * d + a];
      Er[c * d + a] = (double)s;
    }
  }
  E->assign(C * 2 * d, 0.0);
  for (int c = 0; c < C; ++c)
    for (int a = 0; a < d; ++a) {
      (*E)[c * 2 * d + a] = Er[c * d + a];
      (*E)[c * 2 * d + d + a] = Er[(C - 1 - c) * d + (d - 1 - a)];
    }
}

// The paper's FC, Sec. 4.1-4.4 (Eqs. 14-29), coordinates in units of dy:
// least-squares fit of degree p to n_match wall values (QR, Eq. 20), with the
// Neumann row [0 .. 0 1 0 | 0] appended for bc = NEUMANN (Eq. 28);
// continuation node j = 1..C: right fit at xi = j, left fit at
// xi = -(C + 1 - j), quintic blend with t = (j-1)/(C-1) (Eqs. 24-25).
static void paper_table(int nm, int C, int p, int bc, std::vector<double>* E) {
  E->assign(C * 2 * nm, 0.0);
  for (int side = 0; side < 2; ++side) {  // 0: right wall block, 1: left
    const int rows = nm + (bc == FCSPH_NEUMANN ? 1 : 0);
    std::vector<qreal> V(rows * (p + 1), 0), I(rows * nm, 0);
    for (int i = 0; i < nm; ++i) {
      const qreal xi = side == 0 ? (qreal)(i - (nm - 1)) : (qreal)i;
      for (int c = 0; c <= p; ++c) {
        qreal v = 1;
        for (int e = 0; e < p - c; ++e) v *= xi;
        V[i * (p + 1) + c] = v;  // [xi^p ... xi 1]
      }
      I[i * nm + i] = 1;
    }
    if (bc == FCSPH_NEUMANN) V[nm * (p + 1) + (p - 1)] = 1;
    std::vector<qreal> Cop = lsq_qr(V, rows, p + 1, I, nm);  // (p+1) x nm
    for (int j = 1; j <= C; ++j) {
      const qreal t = (qreal)(j - 1) / (qreal)(C - 1);
      const qreal sg = 10 * t * t * t - 15 * t * t * t * t + 6 * t * t * t * t * t;
      const qreal w = side == 0 ? 1 - sg : sg;
      const qreal xi = side == 0 ? (qreal)j : -(qreal)(C + 1 - j);
      for (int a = 0; a < nm; ++a) {
        qreal s = 0;
        for (int c = 0; c <= p; ++c) {
          qreal v = 1;
          for (int e = 0; e < p - c; ++e) v *= xi;
          s += v * Cop[c * nm + a];
        }
        (*E)[(j - 1) * 2 * nm + side * nm + a] = (double)(w * s);
      }
    }
  }
}

int fc_table_build(const fcsph_fc* fc, int bc, std::vector<double>* E, std::string* err) {
  if (!fc || fc->n_match < 2 || fc->n_cont < 2 || fc->n_match > 16 || fc->n_cont > 128) {
    if (err) *err = "fc: need 2 <= n_match <= 16 and 2 <= n_cont <= 128";
    return FCSPH_EINVAL;
  }
  if (fc->variant == FCSPH_FC_GRAM) {
    gram_table(fc->n_match, fc->n_cont, E);
    return FCSPH_OK;
  }
  if (fc->variant == FCSPH_FC_PAPER) {
    if (fc->poly_deg < 1 || fc->poly_deg >= fc->n_match) {
      if (err) *err = "fc: paper variant needs 1 <= poly_deg < n_match";
      return FCSPH_EINVAL;
    }
    paper_table(fc->n_match, fc->n_cont, fc->poly_deg, bc, E);
    return FCSPH_OK;
  }
  if (err) *err = "fc: unknown variant";
  return FCSPH_EINVAL;
}

// ---------------------------------------------------------------------------
// FFT plans.

static void roots(int n, std::vector<double>* re, std::vector<double>* im) {
  re->resize(n);
  im->resize(n);
  for (int e = 0; e < n; ++e) {
    const qreal ang = -2 * QPI * (qreal)e / (qreal)n;
    (*re)[e] = (double)qcos(ang);
    (*im)[e] = (double)qsin(ang);
  }
}

bool factor_direct(int n, Plan1* p) {
  // radix order: larger primes, 7s, 5s, a 3 then 9s, a 4 or 2 then 8s.  The
  // first Stockham stages store at a stride of their radix; odd radices
  // first keep those stores free of shared-memory bank conflicts, and the
  // radix-8 stages come last, when consecutive threads store consecutive
  // elements.
  int cnt[32] = {0};
  std::vector<int> big;
  int r = n;
  for (int q : {2, 3, 5, 7}) {
    while (r % q == 0) {
      ++cnt[q];
      r /= q;
    }
  }
  for (int q = 11; q * q <= r; q += 2)
    while (r % q == 0) {
      big.push_back(q);
      r /= q;
    }
  if (r > 1) big.push_back(r);
  for (int q : big)
    if (q > kMaxDirectPrime) return false;
  std::vector<int> rad;
  while (cnt[2] >= 3) {
    rad.push_back(8);
    cnt[2] -= 3;
  }
  if (cnt[2] == 2) rad.push_back(4);
  if (cnt[2] == 1) rad.push_back(2);
  while (cnt[3] >= 2) {
    rad.push_back(9);
    cnt[3] -= 2;
  }
  if (cnt[3] == 1) rad.push_back(3);
  for (int i = 0; i < cnt[5]; ++i) rad.push_back(5);
  for (int i = 0; i < cnt[7]; ++i) rad.push_back(7);
  for (int q : big) rad.push_back(q);
  if ((int)rad.size() > kMaxStages) return false;
  std::reverse(rad.begin(), rad.end());
  plan_set_radices(p, n, rad.data(), (int)rad.size());
  return true;
}

// exp(-k^2 h^2 / 4) for the m angular wavenumbers 2 pi kappa / (m d) of an
// m-point periodic axis (kappa signed, Nyquist positive), first `count` entries.
std::vector<double> gauss_axis(int m, double d, double h, int count) {
  std::vector<double> out(count);
  for (int a = 0; a < count; ++a) {
    const int kappa = (2 * a <= m) ? a : a - m;
    const qreal k = 2 * QPI * (qreal)kappa / ((qreal)m * (qreal)d);
    const qreal e = k * k * (qreal)h * (qreal)h / 4;
#if defined(__x86_64__)
    out[a] = (double)expq(-e);
#else
    out[a] = (double)expl(-e);
#endif
  }
  return out;
}

// Eq. 16 closed form on the extended grid: W_hat = e^{-s} sum_{m<family}
// s^m / m!, s = |k|^2 h^2 / 4, for every row q = ky nz + kq (ky < hy, the y
// half-spectrum; kq < nz) and kx index < mx; kx and kz signed (Nyquist
// positive), ky >= 0.  e^{-s} is the product of the per-axis factors ex, ey,
// ez (gauss_axis, quad precision, rounded once each); s and the series are
// evaluated in FP64, so the table is within a few FP64 ulps and identical on
// every host.  Entry q mx + kx.
std::vector<double> what_table(const std::vector<double>& ex, const std::vector<double>& ey,
                               const std::vector<double>& ez, int mx, int my, int nz, int hy, double dx, double dy,
                               double dz, double h, int family) {
  std::vector<double> out((size_t)hy * nz * mx);
  const double pi = 3.14159265358979323846;
  const double ckx = 2.0 * pi / (mx * dx), cky = 2.0 * pi / (my * dy), ckz = nz > 1 ? 2.0 * pi / (nz * dz) : 0.0;
  const double hh = h * h * 0.25;
  for (int ky = 0; ky < hy; ++ky)
    for (int kq = 0; kq < nz; ++kq) {
      const int kz = (2 * kq <= nz) ? kq : kq - nz;
      const double kyw = cky * ky, kzw = ckz * kz;
      const double kyz2 = kyw * kyw + kzw * kzw;
      const double eyz = ey[ky] * ez[kq];
      for (int a = 0; a < mx; ++a) {
        const int kx = (2 * a <= mx) ? a : a - mx;
        const double kxw = ckx * kx;
        const double s = (kxw * kxw + kyz2) * hh;
        double term = 1.0, sum = 1.0;
        for (int m = 1; m < family; ++m) {
          term = term * s / m;
          sum += term;
        }
        out[((size_t)ky * nz + kq) * mx + a] = ex[a] * eyz * sum;
      }
    }
  return out;
}

int smooth_at_least(int n) {
  for (int m = n;; ++m) {
    int r = m;
    for (int q : {2, 3, 5, 7})
      while (r % q == 0) r /= q;
    if (r == 1) return m;
  }
}

static bool is_prime(int n) {
  if (n < 2) return false;
  for (int q = 2; q * q <= n; ++q)
    if (n % q == 0) return false;
  return true;
}

static long long powmod(long long b, long long e, long long m) {
  long long r = 1;
  b %= m;
  while (e > 0) {
    if (e & 1) r = r * b % m;
    b = b * b % m;
    e >>= 1;
  }
  return r;
}

// Smallest primitive root of the prime p.
static int primitive_root(int p) {
  std::vector<int> qs;
  int r = p - 1;
  for (int q = 2; q * q <= r; ++q)
    if (r % q == 0) {
      qs.push_back(q);
      while (r % q == 0) r /= q;
    }
  if (r > 1) qs.push_back(r);
  for (int g = 2; g < p; ++g) {
    bool ok = true;
    for (int q : qs)
      if (powmod(g, (p - 1) / q, p) == 1) {
        ok = false;
        break;
      }
    if (ok) return g;
  }
  return 1;
}

FftPlan make_plan(int n, Pool* pool, std::vector<double>* bre, std::vector<double>* bim) {
  FftPlan P;
  std::vector<double> r, i;
  if (factor_direct(n, &P.base)) {
    roots(n, &r, &i);
    P.base.tw = pool->add(r, i);
    P.bs = 0;
    return P;
  }
  if (is_prime(n) && factor_direct(n - 1, &P.sub)) {
    // Rader: X_{g^-m} = x_0 + (a * b)_m, a_q = x_{g^q}, b_s = w^{g^-s}, cyclic of length n - 1
    P.rd = 1;
    plan_set_radices(&P.base, n, nullptr, 0);
    const int m = n - 1;
    roots(m, &r, &i);
    P.sub.tw = pool->add(r, i);
    const long long g = primitive_root(n);
    const long long ginv = powmod(g, n - 2, n);
    std::vector<double> gi(m), si(m), z(m, 0.0);
    bre->assign(m, 0.0);
    bim->assign(m, 0.0);
    for (int q = 0; q < m; ++q) {
      gi[q] = (double)powmod(g, q, n);
      si[q] = (double)powmod(ginv, q, n);
      const qreal ang = -2 * QPI * (qreal)((long long)si[q]) / (qreal)n;
      (*bre)[q] = (double)qcos(ang);
      (*bim)[q] = (double)qsin(ang);
    }
    P.gidx = pool->add(gi, z);
    P.sidx = pool->add(si, z);
    P.bhat = pool->add(std::vector<double>(m, 0.0), std::vector<double>(m, 0.0));
    return P;
  }
  P.bs = 1;
  plan_set_radices(&P.base, n, nullptr, 0);
  const int m = smooth_at_least(2 * n - 1);
  factor_direct(m, &P.sub);
  roots(m, &r, &i);
  P.sub.tw = pool->add(r, i);
  std::vector<double> cr(n), ci(n);
  for (int j = 0; j < n; ++j) {  // chirp exp(i pi j^2 / n), exponent reduced mod 2n
    const long long e = ((long long)j * j) % (2LL * n);
    const qreal ang = QPI * (qreal)e / (qreal)n;
    cr[j] = (double)qcos(ang);
    ci[j] = (double)qsin(ang);
  }
  P.chirp = pool->add(cr, ci);
  bre->assign(m, 0.0);
  bim->assign(m, 0.0);
  for (int j = 0; j < n; ++j) {
    (*bre)[j] = cr[j];
    (*bim)[j] = ci[j];
    if (j > 0) {
      (*bre)[m - j] = cr[j];
      (*bim)[m - j] = ci[j];
    }
  }
  P.bhat = pool->add(std::vector<double>(m, 0.0), std::vector<double>(m, 0.0));
  return P;
}

}  // namespace fcsph
