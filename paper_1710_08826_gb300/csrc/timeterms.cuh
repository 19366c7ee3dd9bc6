// timeterms.cuh -- decay-time machinery shared by the time-dependent amplitude models
// (td4.cu: four-body; dalitz.cu: three-body): the Faddeeva function w(z) (Weideman's
// rational approximation, J. A. C. Weideman, SIAM J. Numer. Anal. 31 (1994) 1497; host and
// device), the convolution E(g; t, s) of e^{-g t'} (t' >= 0) with a Gaussian resolution for
// real and complex g, and the mixing terms with their derivatives.  The formulas are stated
// at the top of td4.cu.
//
// The rate needs the four terms only through
//   R = |A|^2 P + |B|^2 Q + Re(A B*) T_sh + Im(A B*) T_s,
//   P = (T_ch + T_c)/2,  Q = (T_ch - T_c)/2,
// i.e. the convolutions of e^{-G t'} [cosh(y G t') +- cos(x G t')]/2, e^{-G t'} sinh(y G t')
// and e^{-G t'} sin(x G t').  For small mixing Q, T_sh and T_s are tiny differences of nearly
// equal convolved exponentials (Q = O(x^2 + y^2), T_sh = O(y)): formed as such differences in
// FP32 they keep only a few significant digits, and so do their derivatives.  Where
// z = max(|x|, |y|) G (max(t, 0) + 6 s) is small they are therefore summed as power series in
// the moments of the resolution-convolved exponential,
//   M_n(t) = int_0^inf t'^n e^{-G t'} N(t - t'; 0, s) dt',
//   u_n = G^n M_n / n!,
//   P = sum_m a_m u_2m,  Q = sum_m b_m u_2m,  T_sh = sum_m y^(2m+1) u_(2m+1),
//   T_s = sum_m (-1)^m x^(2m+1) u_(2m+1),
//   a_m, b_m = (y^2m +- (-1)^m x^2m) / 2,
// from the Taylor series of cosh and cos, with every term of one sign for t > G s^2.  The
// moments follow from M_0 = E(G) (one erfcx) by the recurrence obtained by integrating
// t' N(t - t') by parts,
//   M_1 = (t - G s^2) M_0 + s^2 N(t),  M_(n+1) = (t - G s^2) M_n + n s^2 M_(n-1),
// i.e. u_(n+1) = (G (t - G s^2) u_n + G^2 s^2 u_(n-1)) / (n + 1).  Derivatives:
//   G d u_n / d G = n u_n - (n + 1) u_(n+1)        (d M_n / d G = -M_(n+1)),
//   d u_n / d s = s d^2 u_n / d t^2                 (heat equation of the Gaussian)
//              = s [G^2 (u_n - 2 u_(n-1) + u_(n-2)) + c_n],
//   c_0 = N'(t) - G N(t), c_1 = G N(t), c_n = 0 for n >= 2 (from d M_n / d t = n M_(n-1)
//   - G M_n + [n = 0] N(t)).  Elsewhere (large mixing) the terms come from the Faddeeva path,
// where the differences are not small.
#pragma once

#include <cmath>
#include <vector>

#include "common.cuh"

namespace goo {

constexpr int kWMax = 40;
constexpr int kWN32 = 24, kWN64 = 40;

// ---------------------------------------------------------------------------------------
// Faddeeva function (Weideman); host and device, any floating type
// ---------------------------------------------------------------------------------------
template <typename T>
__host__ __device__ inline void faddeeva(T zr, T zi, const T* a, int N, T L, T& wr, T& wi) {
  // D = L - i z = (L + zi) - i zr;  1/D = conj(D)/|D|^2
  const T dr = L + zi, di = -zr;
  const T inv = T(1) / (dr * dr + di * di);
  const T ir = dr * inv, ii = -di * inv;
  // Z = (L + i z)/D = ((L - zi) + i zr)/D
  const T nr = L - zi, ni = zr;
  const T Zr = nr * ir - ni * ii, Zi = nr * ii + ni * ir;
  T pr = a[N - 1], pi = T(0);
  for (int j = N - 2; j >= 0; --j) {
    const T tr = pr * Zr - pi * Zi + a[j];
    pi = pr * Zi + pi * Zr;
    pr = tr;
  }
  // w = (1/D) (2 p / D + 1/sqrt(pi))
  const T qr = T(2) * (pr * ir - pi * ii) + T(0.56418958354775628695), qi = T(2) * (pr * ii + pi * ir);
  wr = ir * qr - ii * qi;
  wi = ir * qi + ii * qr;
}

static void weideman_coeffs(int N, double* a, double* L) {
  const int M = 2 * N, M2 = 2 * M;
  const double Lv = std::sqrt(N / std::sqrt(2.0));
  std::vector<double> f(M2, 0.0);
  for (int k = -M + 1; k <= M - 1; ++k) {
    const double th = k * M_PI / M, t = Lv * std::tan(th / 2.0);
    f[k + M] = std::exp(-t * t) * (Lv * Lv + t * t);
  }
  std::vector<double> g(M2);
  for (int j = 0; j < M2; ++j) g[j] = f[(j + M) % M2];  // the half-length rotation
  for (int m = 1; m <= N; ++m) {
    double re = 0.0;
    for (int j = 0; j < M2; ++j) re += g[j] * std::cos(2.0 * M_PI * (double)j * m / M2);
    a[m - 1] = re / M2;
  }
  *L = Lv;
}

struct WeidemanTables {
  double a32[kWMax], a64[kWMax];
  double L32, L64;
  WeidemanTables() {
    weideman_coeffs(kWN32, a32, &L32);
    weideman_coeffs(kWN64, a64, &L64);
  }
};

static const WeidemanTables& weideman() {
  static const WeidemanTables t;
  return t;
}

// ---------------------------------------------------------------------------------------
// decay-time terms
// ---------------------------------------------------------------------------------------
template <typename T>
struct TimeTerms {
  T P, Q, Tsh, Ts;
  T d[4][4];  // d[param][term], param = x, y, tau, sigma_t; term = P, Q, sh, s
};

// Orders of the moment series: u_0 .. u_(2K+2) (the G-derivative of u_(2K+1) needs
// u_(2K+2)), and the largest z = max(|x|,|y|) G (max(t,0) + 6 s) at which the truncated
// series is used.  FP32: K = 4, z <= 0.5 (first omitted term of Q below 1e-8 of Q);
// FP64: K = 6, z <= 0.35 (below 1e-16 of Q).
template <typename T>
struct SeriesOrder {
  static constexpr int K = sizeof(T) == 4 ? 4 : 6;
  static constexpr double zmax = sizeof(T) == 4 ? 0.5 : 0.35;
};

// Per-theta constants of the decay-time terms in the path's precision: the series
// coefficients and their derivatives, prepared on the host in FP64 from the rounded x, y.
template <typename T>
struct TimeCoef {
  static constexpr int K = SeriesOrder<T>::K;
  T G, x, y, s;
  T zs;                        // max(|x|, |y|) G
  T a[K + 1], b[K + 1];        // P, Q coefficients of u_2m (a_0 = 1, b_0 = 0)
  T ysh[K + 1], xs[K + 1];     // T_sh, T_s coefficients of u_(2m+1)
  T dax[K + 1], day[K + 1];    // d a_m / dx (= -d b_m / dx), d a_m / dy (= d b_m / dy)
  T dshy[K + 1], dsx[K + 1];   // d ysh_m / dy, d xs_m / dx
  // the order in use, K - 1 or K, and the largest z at which it meets the truncation
  // criterion: K - 1 when that covers every event the dataset's time range admits
  int ku;
  T zmax_ku;
  T is2, is2h;  // 1 / s^2 and 1 / (2 s^2), so that no event divides by them
};

#ifndef __CUDACC_RTC__
// t_hi: the upper limit of the observed time (events above it take the Faddeeva path where
// the order in use does not cover them, so it decides the speed, not the result).
template <typename T>
inline void fill_time_coef(TimeCoef<T>& c, double x64, double y64, double tau, double s64,
                           double t_hi = HUGE_VAL) {
  constexpr int K = TimeCoef<T>::K;
  c.G = (T)(1.0 / tau);
  c.x = (T)x64;
  c.y = (T)y64;
  c.s = (T)s64;
  const double x = (double)c.x, y = (double)c.y, G = (double)c.G;
  c.zs = (T)(std::fmax(std::fabs(x), std::fabs(y)) * G);
  c.is2 = (T)(1.0 / ((double)c.s * (double)c.s));
  c.is2h = (T)(0.5 / ((double)c.s * (double)c.s));
  for (int m = 0; m <= K; ++m) {
    const double sg = (m & 1) ? -1.0 : 1.0;
    const double y2m = std::pow(y, 2 * m), x2m = std::pow(x, 2 * m);
    c.a[m] = (T)(0.5 * (y2m + sg * x2m));
    c.b[m] = (T)(0.5 * (y2m - sg * x2m));
    c.day[m] = (T)(m > 0 ? m * std::pow(y, 2 * m - 1) : 0.0);
    c.dax[m] = (T)(m > 0 ? sg * m * std::pow(x, 2 * m - 1) : 0.0);
    c.ysh[m] = (T)(y2m * y);
    c.xs[m] = (T)(sg * x2m * x);
    c.dshy[m] = (T)((2 * m + 1) * y2m);
    c.dsx[m] = (T)(sg * (2 * m + 1) * x2m);
  }
  c.b[0] = (T)0;
  // the first omitted term against the leading one is about z^(2k) 2 / (2k + 2)! at order k;
  // order K - 1 meets the bound that order K meets at SeriesOrder<T>::zmax up to zk1
  auto ratio = [](double z, int k) { return std::pow(z, 2.0 * k) * 2.0 / std::tgamma(2.0 * k + 3.0); };
  const double eps = ratio(SeriesOrder<T>::zmax, K);
  const double zk1 = std::pow(eps * std::tgamma(2.0 * (K - 1) + 3.0) / 2.0, 1.0 / (2.0 * (K - 1)));
  const double zdata = (double)c.zs * (std::fmax(t_hi, 0.0) + 6.0 * (double)c.s);
  c.ku = zdata < zk1 ? K - 1 : K;
  c.zmax_ku = (T)(zdata < zk1 ? zk1 : SeriesOrder<T>::zmax);
}
#endif

template <typename T>
__device__ __forceinline__ T td_erfcx(T u) {
  if constexpr (sizeof(T) == 4) return erfcxf(u);
  else return erfcx(u);
}

template <typename T>
__device__ __forceinline__ T td_exp(T v) {
  if constexpr (sizeof(T) == 4) return expf(v);
  else return exp(v);
}

// E(g) for real g, with dE/dg and dE/ds (gauss = exp(-t^2/2s^2), k = 1/(sqrt(2 pi)))
template <typename T>
__device__ __forceinline__ void conv_real(T g, T t, T s, T gauss, T& E, T& dEg, T& dEs) {
  const T u = (g * s * s - t) * (T(0.70710678118654752440) / s);
  if (u >= T(0)) {
    E = T(0.5) * gauss * td_erfcx<T>(u);
  } else {
    E = td_exp<T>(T(0.5) * g * g * s * s - g * t) - T(0.5) * gauss * td_erfcx<T>(-u);
  }
  const T k = T(0.39894228040143267794);
  dEg = (g * s * s - t) * E - s * k * gauss;
  dEs = g * g * s * E - (g * s * s + t) / (s * s) * k * gauss;
}

// E(g) for complex g = (gr, gi), with dE/dg and dE/ds
template <typename T>
__device__ __forceinline__ void conv_complex(T gr, T gi, T t, T s, T gauss, const T* wa, int wN, T wL, T& Er, T& Ei,
                                             T& dgr, T& dgi, T& dsr, T& dsi) {
  const T c = T(0.70710678118654752440) / s;
  const T ur = (gr * s * s - t) * c, ui = gi * s * s * c;
  T wr, wi;
  if (ur >= T(0)) {
    faddeeva<T>(-ui, ur, wa, wN, wL, wr, wi);  // w(i u)
    Er = T(0.5) * gauss * wr;
    Ei = T(0.5) * gauss * wi;
  } else {
    faddeeva<T>(ui, -ur, wa, wN, wL, wr, wi);  // w(-i u)
    const T er = T(0.5) * (gr * gr - gi * gi) * s * s - gr * t, ei = gr * gi * s * s - gi * t;
    const T mag = td_exp<T>(er);
    T sn, cs;
    if constexpr (sizeof(T) == 4) sincosf(ei, &sn, &cs);
    else sincos(ei, &sn, &cs);
    Er = mag * cs - T(0.5) * gauss * wr;
    Ei = mag * sn - T(0.5) * gauss * wi;
  }
  const T k = T(0.39894228040143267794);
  // dE/dg = (g s^2 - t) E - s k gauss
  const T ar = gr * s * s - t, ai = gi * s * s;
  dgr = ar * Er - ai * Ei - s * k * gauss;
  dgi = ar * Ei + ai * Er;
  // dE/ds = g^2 s E - (g s^2 + t)/s^2 k gauss
  const T g2r = (gr * gr - gi * gi) * s, g2i = T(2) * gr * gi * s;
  dsr = g2r * Er - g2i * Ei - (gr * s * s + t) / (s * s) * k * gauss;
  dsi = g2r * Ei + g2i * Er - gi * k * gauss;
}

// The decay-time terms at the observed time t from the convolved exponentials (Faddeeva
// path, any mixing) and their derivatives with respect to (x, y, tau, sigma_t), for
// Gamma = G, mixing (x, y), resolution s; gauss = exp(-t^2 / 2 s^2).
template <typename T>
__device__ __forceinline__ void time_terms_direct(T G, T x, T y, T s, const T* wa, int wN, T wL, T t, T gauss,
                                                  TimeTerms<T>& R) {
  const T gp = G * (T(1) - y), gm = G * (T(1) + y);
  T Ep, dEgp, dEsp, Em, dEgm, dEsm;
  conv_real<T>(gp, t, s, gauss, Ep, dEgp, dEsp);
  conv_real<T>(gm, t, s, gauss, Em, dEgm, dEsm);
  T Ecr, Eci, dgr, dgi, dsr, dsi;
  conv_complex<T>(G, -G * x, t, s, gauss, wa, wN, wL, Ecr, Eci, dgr, dgi, dsr, dsi);
  const T Tch = T(0.5) * (Ep + Em);
  R.P = T(0.5) * (Tch + Ecr);
  R.Q = T(0.5) * (Tch - Ecr);
  R.Tsh = T(0.5) * (Ep - Em);
  R.Ts = Eci;
  // per parameter the derivatives of (T_ch, T_c) map to P, Q as the terms do
  T dch[4], dc[4];
  // x: dgc/dx = -i G  ->  (-iG)(dgr + i dgi) = G dgi - i G dgr
  dch[0] = T(0);
  dc[0] = G * dgi;
  R.d[0][2] = T(0);
  R.d[0][3] = -G * dgr;
  // y: dg+/dy = -G, dg-/dy = +G
  dch[1] = T(0.5) * G * (dEgm - dEgp);
  dc[1] = T(0);
  R.d[1][2] = -T(0.5) * G * (dEgp + dEgm);
  R.d[1][3] = T(0);
  // tau: dg/dtau = -g G
  dch[2] = -T(0.5) * G * (dEgp * gp + dEgm * gm);
  dc[2] = -G * (dgr * G - dgi * (-G * x));  // Re((dgr + i dgi)(-gc G)), gc = (G, -G x)
  R.d[2][2] = -T(0.5) * G * (dEgp * gp - dEgm * gm);
  R.d[2][3] = -G * (dgr * (-G * x) + dgi * G);
  // sigma_t
  dch[3] = T(0.5) * (dEsp + dEsm);
  dc[3] = dsr;
  R.d[3][2] = T(0.5) * (dEsp - dEsm);
  R.d[3][3] = dsi;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    R.d[j][0] = T(0.5) * (dch[j] + dc[j]);
    R.d[j][1] = T(0.5) * (dch[j] - dc[j]);
  }
}

// The decay-time terms by the moment series of order KU (small mixing; see the top of this
// file).
template <typename T, int KU>
__device__ __forceinline__ void time_terms_series(const TimeCoef<T>& c, T t, T gauss, TimeTerms<T>& R) {
  constexpr int K = KU;
  constexpr int NU = 2 * K + 3;
  const T G = c.G, s = c.s;
  const T s2 = s * s;
  T E0, dEg_unused, dEs_unused;
  conv_real<T>(G, t, s, gauss, E0, dEg_unused, dEs_unused);
  const T phi = T(0.39894228040143267794) / s * gauss;  // N(t; 0, s)
  const T v = t - G * s2;
  const T Gv = G * v, G2s2 = G * G * s2;
  T u[NU];
  u[0] = E0;
  u[1] = G * (v * E0 + s2 * phi);
#pragma unroll
  for (int n = 1; n < NU - 1; ++n) u[n + 1] = (Gv * u[n] + G2s2 * u[n - 1]) * T(1.0 / (n + 1));
  // d u_n / d s (heat equation) and G d u_n / d G
  const T G2 = G * G;
  auto su = [&](int n) -> T {
    const T um1 = n >= 1 ? u[n - 1] : T(0), um2 = n >= 2 ? u[n - 2] : T(0);
    const T cn = n == 0 ? (-t * c.is2 - G) * phi : (n == 1 ? G * phi : T(0));
    return s * (G2 * ((u[n] - um1) - (um1 - um2)) + cn);
  };
  auto gu = [&](int n) -> T { return T(n) * u[n] - T(n + 1) * u[n + 1]; };
  T P = u[0], Q = T(0), Tsh = T(0), Ts = T(0);
  T Px = T(0), Py = T(0), PG = gu(0), Ps = su(0), QG = T(0), Qs = T(0);
  T Shy = T(0), ShG = T(0), Shs = T(0), Sx = T(0), SG = T(0), Ss = T(0);
#pragma unroll
  for (int m = 1; m <= K; ++m) {
    const T ue = u[2 * m];
    P += c.a[m] * ue;
    Q += c.b[m] * ue;
    Px += c.dax[m] * ue;
    Py += c.day[m] * ue;
    const T ge = gu(2 * m), se = su(2 * m);
    PG += c.a[m] * ge;
    QG += c.b[m] * ge;
    Ps += c.a[m] * se;
    Qs += c.b[m] * se;
  }
#pragma unroll
  for (int m = 0; m <= K; ++m) {
    const T uo = u[2 * m + 1];
    Tsh += c.ysh[m] * uo;
    Ts += c.xs[m] * uo;
    Shy += c.dshy[m] * uo;
    Sx += c.dsx[m] * uo;
    const T go = gu(2 * m + 1), so = su(2 * m + 1);
    ShG += c.ysh[m] * go;
    SG += c.xs[m] * go;
    Shs += c.ysh[m] * so;
    Ss += c.xs[m] * so;
  }
  R.P = P;
  R.Q = Q;
  R.Tsh = Tsh;
  R.Ts = Ts;
  // x: P and Q move oppositely; T_sh does not depend on x, T_s not on y
  R.d[0][0] = Px;
  R.d[0][1] = -Px;
  R.d[0][2] = T(0);
  R.d[0][3] = Sx;
  R.d[1][0] = Py;
  R.d[1][1] = Py;
  R.d[1][2] = Shy;
  R.d[1][3] = T(0);
  // tau: d / d tau = -G (G d / d G)
  R.d[2][0] = -G * PG;
  R.d[2][1] = -G * QG;
  R.d[2][2] = -G * ShG;
  R.d[2][3] = -G * SG;
  R.d[3][0] = Ps;
  R.d[3][1] = Qs;
  R.d[3][2] = Shs;
  R.d[3][3] = Ss;
}

// The decay-time terms at the observed time t and their derivatives: the moment series of the
// order in use where z = max(|x|, |y|) G (max(t, 0) + 6 s) is below its limit (c.zmax_ku),
// else the Faddeeva path.
template <typename T>
__device__ __forceinline__ void time_terms_g(const TimeCoef<T>& c, const T* wa, int wN, T wL, T t, TimeTerms<T>& R) {
  const T gauss = td_exp<T>(-t * t * c.is2h);
  const T z = c.zs * ((t > T(0) ? t : T(0)) + T(6) * c.s);
  if (z < c.zmax_ku) {
    // the same order for every event of a launch (a uniform branch)
    if (c.ku == TimeCoef<T>::K) time_terms_series<T, TimeCoef<T>::K>(c, t, gauss, R);
    else time_terms_series<T, TimeCoef<T>::K - 1>(c, t, gauss, R);
  } else {
    time_terms_direct<T>(c.G, c.x, c.y, c.s, wa, wN, wL, t, gauss, R);
  }
}


}  // namespace goo
