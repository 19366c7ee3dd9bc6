// timeterms.cuh -- decay-time machinery shared by the time-dependent amplitude models
// (td4.cu: four-body; dalitz.cu: three-body): the Faddeeva function w(z) (Weideman's
// rational approximation, J. A. C. Weideman, SIAM J. Numer. Anal. 31 (1994) 1497; host and
// device), the convolution E(g; t, s) of e^{-g t'} (t' >= 0) with a Gaussian resolution for
// real and complex g, and the four mixing terms T_ch, T_sh, T_c, T_s with their derivatives.
// The formulas are stated at the top of td4.cu.
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
  T Tch, Tsh, Tc, Ts;
  T d[4][4];  // d[param][term], param = x, y, tau, sigma_t; term = ch, sh, c, s
};

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

// The four decay-time terms at the observed time t and their derivatives with respect to
// (x, y, tau, sigma_t), for Gamma = G, mixing (x, y), resolution s.
template <typename T>
__device__ __forceinline__ void time_terms_g(T G, T x, T y, T s, const T* wa, int wN, T wL, T t, TimeTerms<T>& R) {
  const T gauss = td_exp<T>(-t * t / (T(2) * s * s));
  const T gp = G * (T(1) - y), gm = G * (T(1) + y);
  T Ep, dEgp, dEsp, Em, dEgm, dEsm;
  conv_real<T>(gp, t, s, gauss, Ep, dEgp, dEsp);
  conv_real<T>(gm, t, s, gauss, Em, dEgm, dEsm);
  T Ecr, Eci, dgr, dgi, dsr, dsi;
  conv_complex<T>(G, -G * x, t, s, gauss, wa, wN, wL, Ecr, Eci, dgr, dgi, dsr, dsi);
  R.Tch = T(0.5) * (Ep + Em);
  R.Tsh = T(0.5) * (Ep - Em);
  R.Tc = Ecr;
  R.Ts = Eci;
  // x: dgc/dx = -i G  ->  (-iG)(dgr + i dgi) = G dgi - i G dgr
  R.d[0][0] = T(0);
  R.d[0][1] = T(0);
  R.d[0][2] = G * dgi;
  R.d[0][3] = -G * dgr;
  // y: dg+/dy = -G, dg-/dy = +G
  R.d[1][0] = T(0.5) * G * (dEgm - dEgp);
  R.d[1][1] = -T(0.5) * G * (dEgp + dEgm);
  R.d[1][2] = T(0);
  R.d[1][3] = T(0);
  // tau: dg/dtau = -g G
  R.d[2][0] = -T(0.5) * G * (dEgp * gp + dEgm * gm);
  R.d[2][1] = -T(0.5) * G * (dEgp * gp - dEgm * gm);
  R.d[2][2] = -G * (dgr * G - dgi * (-G * x));  // Re((dgr + i dgi)(-gc G)), gc = (G, -G x)
  R.d[2][3] = -G * (dgr * (-G * x) + dgi * G);
  // sigma_t
  R.d[3][0] = T(0.5) * (dEsp + dEsm);
  R.d[3][1] = T(0.5) * (dEsp - dEsm);
  R.d[3][2] = dsr;
  R.d[3][3] = dsi;
}


}  // namespace goo
