// td4.cu -- the time-dependent four-body amplitude model: amplitude cache, MC Gram matrix,
// and the NLL + adjoint gradient with mixing and a Gaussian decay-time resolution.
//
// Paper: a time-dependent amplitude analysis of four-body decays for a mixing measurement
// is among GooFit's amplitude PDFs (Sec. 5); phase-space MC samples give the normalisation
// (Sec. 5); partial results are cached in structure-of-arrays form (Sec. 4).  The paper
// prints no formulas; the model (fixed by the oracle) is:
//   observables m12, m34, c12 = cos th12, c34 = cos th34, phi, t;
//   a_k = F(m12) F(m34) W_k(c12, c34, phi),  F = BW(m^2) (q/q0)^L B_L(r q)/B_L(r q0),
//   BW(s) = 1/(m0^2 - s - i m0 G(m)),  G(m) = G0 (q/q0)^(2L+1) (m0/m) (B_L(rq)/B_L(rq0))^2;
//   A = sum_k c_k a_k (free), B = sum_k b_k a_k (fixed);
//   R = (|A|^2+|B|^2)/2 T_ch + (|A|^2-|B|^2)/2 T_c + Re(AB*) T_sh + Im(AB*) T_s,
//   T_ch, T_sh = (E(G(1-y)) +- E(G(1+y)))/2,  T_c + i T_s = E(G(1 - i x)),  G = 1/tau,
//   E(g; t, s) = e^{-g t'} (t' >= 0) convolved with N(0, s):
//     Re u >= 0:  E = 1/2 exp(-t^2/2s^2) w(i u),  u = (g s^2 - t)/(s sqrt 2)
//     Re u <  0:  E = exp(g^2 s^2/2 - g t) - 1/2 exp(-t^2/2s^2) w(-i u);
//   N = <|A|^2+|B|^2>/2 I_ch + <|A|^2-|B|^2>/2 I_c + Re<AB*> I_sh + Im<AB*> I_s over the MC
//   (Gram matrix <a_k a_l*>), I_ch = tau/(1-y^2), I_sh = y tau/(1-y^2), I_c = tau/(1+x^2),
//   I_s = x tau/(1+x^2);  NLL = -sum log R + n log N.
// The Faddeeva function w(z), Im z >= 0, is Weideman's rational approximation (J. A. C.
// Weideman, SIAM J. Numer. Anal. 31 (1994) 1497):
//   w(z) = 2 p(Z)/(L - iz)^2 + (1/sqrt pi)/(L - iz),  Z = (L + iz)/(L - iz),  L = sqrt(N/sqrt 2),
// p a polynomial of degree N-1 whose coefficients come from a discrete Fourier transform of
// exp(-t^2)(L^2 + t^2) at t = L tan(theta/2) (computed here on the host in FP64); N = 24 in
// the FP32 path and 40 in the FP64 path.  The real-argument terms use erfcx.
//
// Gradient lanes per event: log R; Re, Im of a_k V / R with
// V = (T_ch + T_c) A* + (T_sh - i T_s) B* (dR/dRe c_k = Re(a_k V), dR/dIm c_k = -Im(a_k V));
// and dR/d(x, y, tau, sigma_t) / R.  The last block forms the NLL and its gradient in FP64.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "dalitz.cuh"
#include "model.cuh"
#include "timeterms.cuh"

namespace goo {

constexpr int kTdMaxAmp = 16;

struct Td4Amp {
  int ang, L1, L2, pad;
  double m0a, g0a, q0a, b0a;  // resonance in the 12 pair: m0, width, q(m0), B_L(r q(m0))
  double m0b, g0b, q0b, b0b;  // resonance in the 34 pair
};

struct Td4Dev {
  int K, pad;
  double m1, m2, m3, m4, r;
  Td4Amp amp[kTdMaxAmp];
};

template <typename T>
struct Td4Args {
  T cr[kTdMaxAmp], ci[kTdMaxAmp], br[kTdMaxAmp], bi[kTdMaxAmp];
  T G, x, y, s;  // 1/tau, mixing, resolution in the path's precision
  TimeCoef<T> tc;  // the same with the moment-series coefficients (timeterms.cuh)
  T wa[kWMax];   // Weideman coefficients (constant term first)
  T wL;
  int wN, K, n_params, planes;
  int par_re[kTdMaxAmp], par_im[kTdMaxAmp], par_t[4];
  int64_t n_total;  // events of the dataset (cache plane length)
  // the normalisation at theta, formed on the host in FP64 from the cached Gram matrix
  // (td4_norm_terms): N, log N, (dN / d Re c_k) / N, (dN / d Im c_k) / N and (dN / dx) / N,
  // (dN / dy) / N, (tau dN / d tau) / N
  double nrm_N, nrm_logN, nrm_ur[kTdMaxAmp], nrm_ui[kTdMaxAmp], nrm_dt[3];
};


// ---------------------------------------------------------------------------------------
// amplitude cache
// ---------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T td_barrier(int L, T z) {
  if (L == 0) return T(1);
  if (L == 1) return sqrt(T(1) / (T(1) + z));
  return sqrt(T(9) / (T(9) + T(3) * z + z * z));
}

template <typename T>
__device__ __forceinline__ void td_lineshape(T m, T m0, T g0, T q0, T b0, int L, T ma, T mb, T r, T& fr, T& fi) {
  const T m2 = m * m;
  const T lam = (m2 - (ma + mb) * (ma + mb)) * (m2 - (ma - mb) * (ma - mb));
  const T q = sqrt(lam > T(0) ? lam : T(0)) / (T(2) * m);
  const T ratio = td_barrier<T>(L, (r * q) * (r * q)) / b0;
  const T qq = q / q0;
  T qL = T(1);
  for (int l = 0; l < L; ++l) qL *= qq;
  const T width = g0 * qL * qL * qq * (m0 / m) * ratio * ratio;
  const T dr = m0 * m0 - m2, di = m0 * width;  // BW = 1/(dr - i di) = (dr + i di)/|.|^2
  const T inv = T(1) / (dr * dr + di * di);
  const T scale = qL * ratio * inv;
  fr = dr * scale;
  fi = di * scale;
}

template <typename T>
__device__ __forceinline__ void td_angular(int ang, T c12, T c34, T phi, T& wr, T& wi) {
  const T s12 = sqrt(fmax(T(1) - c12 * c12, T(0))), s34 = sqrt(fmax(T(1) - c34 * c34, T(0)));
  const T p2 = T(0.5) * (T(3) * c12 * c12 - T(1));
  wi = T(0);
  switch (ang) {
    case GOO_ANG_SS: wr = T(1); break;
    case GOO_ANG_VS0: wr = c12; break;
    case GOO_ANG_SV0: wr = c34; break;
    case GOO_ANG_VV0: wr = c12 * c34; break;
    case GOO_ANG_VVPAR: wr = s12 * s34 * cos(phi); break;
    case GOO_ANG_VVPERP: wr = T(0); wi = s12 * s34 * sin(phi); break;
    case GOO_ANG_TS0: wr = p2; break;
    default: wr = p2 * c34; break;  // GOO_ANG_TV0
  }
}

template <typename T>
struct Td4Cols {
  const T* c[5];  // m12, m34, c12, c34, phi
};

// Cache layout as for the three-body model: FP32 ceil(K/2) planes of float4 (re_k, im_k,
// re_k+1, im_k+1), FP64 K planes of double2; plane p of an n-event dataset at p * n.
template <typename T>
__global__ void td4_cache_kernel(const Td4Dev* __restrict__ tdp, Td4Cols<T> cols, int64_t n, void* cache_v) {
  __shared__ Td4Dev td;
  for (int i = threadIdx.x; i < (int)(sizeof(Td4Dev) / 4); i += blockDim.x) ((int*)&td)[i] = ((const int*)tdp)[i];
  __syncthreads();
  const int K = td.K;
  const T r = (T)td.r;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const T m12 = cols.c[0][i], m34 = cols.c[1][i], c12 = cols.c[2][i], c34 = cols.c[3][i], phi = cols.c[4][i];
    for (int k = 0; k < K; ++k) {
      const Td4Amp& A = td.amp[k];
      T f1r, f1i, f2r, f2i, wr, wi;
      td_lineshape<T>(m12, (T)A.m0a, (T)A.g0a, (T)A.q0a, (T)A.b0a, A.L1, (T)td.m1, (T)td.m2, r, f1r, f1i);
      td_lineshape<T>(m34, (T)A.m0b, (T)A.g0b, (T)A.q0b, (T)A.b0b, A.L2, (T)td.m3, (T)td.m4, r, f2r, f2i);
      td_angular<T>(A.ang, c12, c34, phi, wr, wi);
      const T fr = f1r * f2r - f1i * f2i, fi = f1r * f2i + f1i * f2r;
      const T ar = fr * wr - fi * wi, ai = fr * wi + fi * wr;
      if constexpr (sizeof(T) == 4) {
        float* plane = (float*)((float4*)cache_v + (int64_t)(k / 2) * n + i);
        plane[2 * (k & 1)] = ar;
        plane[2 * (k & 1) + 1] = ai;
      } else {
        ((double2*)cache_v)[(int64_t)k * n + i] = make_double2(ar, ai);
      }
    }
    if constexpr (sizeof(T) == 4) {
      if (K & 1) {  // zero the unused half of the last plane
        float* plane = (float*)((float4*)cache_v + (int64_t)(K / 2) * n + i);
        plane[2] = plane[3] = 0.f;
      }
    }
  }
}

template <typename T>
__device__ __forceinline__ void time_terms(const Td4Args<T>& a, T t, TimeTerms<T>& R) {
  time_terms_g<T>(a.tc, a.wa, a.wN, a.wL, t, R);
}

// ---------------------------------------------------------------------------------------
// NLL kernels
// ---------------------------------------------------------------------------------------
template <int KB, bool GRAD>
struct TdLanes {
  static constexpr int NS = GRAD ? 1 + 2 * KB + 4 : 1;
};

template <typename T, int KB>
struct TdAcc {
  Kahan lf32;
  double lf64 = 0.0;
  T lre[KB], lim[KB], lt[4];
  unsigned bad = 0;
};

// One event from its amplitudes (ar, ai) and observed time t.
template <typename T, int KB, bool GRAD>
__device__ __forceinline__ void td4_event(const Td4Args<T>& a, const T (&ar)[KB], const T (&ai)[KB], T t,
                                          TdAcc<T, KB>& acc) {
  T Ar = T(0), Ai = T(0), Br = T(0), Bi = T(0);
#pragma unroll
  for (int k = 0; k < KB; ++k) {
    Ar += a.cr[k] * ar[k] - a.ci[k] * ai[k];
    Ai += a.cr[k] * ai[k] + a.ci[k] * ar[k];
    Br += a.br[k] * ar[k] - a.bi[k] * ai[k];
    Bi += a.br[k] * ai[k] + a.bi[k] * ar[k];
  }
  TimeTerms<T> tt;
  time_terms<T>(a, t, tt);
  const T AA = Ar * Ar + Ai * Ai, BB = Br * Br + Bi * Bi;
  const T ABr = Ar * Br + Ai * Bi, ABi = Ai * Br - Ar * Bi;  // A conj(B)
  // R = |A|^2 P + |B|^2 Q + Re(A B*) T_sh + Im(A B*) T_s with P, Q = (T_ch +- T_c)/2
  const T R = AA * tt.P + BB * tt.Q + ABr * tt.Tsh + ABi * tt.Ts;
  if (!(R > T(0))) {
    acc.bad++;
    return;
  }
  if constexpr (sizeof(T) == 4) acc.lf32.add(logf(R));
  else acc.lf64 += log(R);
  if constexpr (GRAD) {
    const T invR = T(1) / R;
    // V / R, V = (T_ch + T_c) A* + (T_sh - i T_s) B* = 2 P A* + (T_sh - i T_s) B*
    const T c1 = T(2) * tt.P * invR, sh = tt.Tsh * invR, ss = tt.Ts * invR;
    const T Vr = c1 * Ar + sh * Br - ss * Bi;
    const T Vi = -c1 * Ai - sh * Bi - ss * Br;
#pragma unroll
    for (int k = 0; k < KB; ++k) {
      acc.lre[k] += ar[k] * Vr - ai[k] * Vi;     // Re(a_k V) / R
      acc.lim[k] += -(ar[k] * Vi + ai[k] * Vr);  // -Im(a_k V) / R
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
      acc.lt[j] += (AA * tt.d[j][0] + BB * tt.d[j][1] + ABr * tt.d[j][2] + ABi * tt.d[j][3]) * invR;
  }
}

// The FP32 form of td4_event in the staged kernel.  The amplitudes come as (re, im) pairs
// straight from the float4 planes, and A = sum c_k a_k is formed from two packed sums,
// (sum cr_k re_k, sum cr_k im_k) and (sum ci_k re_k, sum ci_k im_k), B likewise: four packed
// FMAs per amplitude instead of eight scalar ones.  log2 R is accumulated (td4_finish scales
// the FP32 sum by ln 2 once per thread) and 1/R is the hardware reciprocal.
template <int KB, bool GRAD>
__device__ __forceinline__ void td4_event_f32(const Td4Args<float>& a, const float2 (&am)[KB], float t,
                                              TdAcc<float, KB>& acc) {
  using namespace pk;
  float2 P1 = splat(0.f), P2 = splat(0.f), Q1 = splat(0.f), Q2 = splat(0.f);
#pragma unroll
  for (int k = 0; k < KB; ++k) {
    P1 = fma(splat(a.cr[k]), am[k], P1);
    P2 = fma(splat(a.ci[k]), am[k], P2);
    Q1 = fma(splat(a.br[k]), am[k], Q1);
    Q2 = fma(splat(a.bi[k]), am[k], Q2);
  }
  const float Ar = P1.x - P2.y, Ai = P1.y + P2.x, Br = Q1.x - Q2.y, Bi = Q1.y + Q2.x;
  TimeTerms<float> tt;
  time_terms<float>(a, t, tt);
  const float AA = Ar * Ar + Ai * Ai, BB = Br * Br + Bi * Bi;
  const float ABr = Ar * Br + Ai * Bi, ABi = Ai * Br - Ar * Bi;  // A conj(B)
  const float R = AA * tt.P + BB * tt.Q + ABr * tt.Tsh + ABi * tt.Ts;
  if (!(R > 0.f)) {
    acc.bad++;
    return;
  }
  acc.lf32.add(lg2(R));
  if constexpr (GRAD) {
    const float invR = rcp(R);
    const float c1 = 2.f * tt.P * invR, sh = tt.Tsh * invR, ss = tt.Ts * invR;
    const float Vr = c1 * Ar + sh * Br - ss * Bi;
    const float Vi = -c1 * Ai - sh * Bi - ss * Br;
#pragma unroll
    for (int k = 0; k < KB; ++k) {
      acc.lre[k] += am[k].x * Vr - am[k].y * Vi;     // Re(a_k V) / R
      acc.lim[k] += -(am[k].x * Vi + am[k].y * Vr);  // -Im(a_k V) / R
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
      acc.lt[j] += (AA * tt.d[j][0] + BB * tt.d[j][1] + ABr * tt.d[j][2] + ABi * tt.d[j][3]) * invR;
  }
}

// Block and last-block reductions, then the FP64 combination with the normalisation terms the
// host formed from the Gram matrix (they depend on theta and the MC sample only, not on the
// events: an O(K^2) quadratic form, whose FP64 latency chain had been the last block's tail).
template <typename T, int KB, bool GRAD>
__device__ __forceinline__ void td4_finish(const Td4Args<T>& a, TdAcc<T, KB>& acc, int64_t begin, int64_t end,
                                           float2* partials, unsigned* counters, double* result, int out_mode,
                                           ddf* s_red, unsigned* s_bad) {
  constexpr int NS = TdLanes<KB, GRAD>::NS;
  ddf v[NS];
  // the FP32 kernel sums log2 R (td4_event_f32)
  v[0] = (sizeof(T) == 4) ? dd_mul(acc.lf32.value(), ddf{kLn2Hi, kLn2Lo}) : dd_from_double(acc.lf64);
  if constexpr (GRAD) {
#pragma unroll
    for (int k = 0; k < KB; ++k) {
      v[1 + 2 * k] = (sizeof(T) == 4) ? ddf{(float)acc.lre[k], 0.f} : dd_from_double((double)acc.lre[k]);
      v[2 + 2 * k] = (sizeof(T) == 4) ? ddf{(float)acc.lim[k], 0.f} : dd_from_double((double)acc.lim[k]);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
      v[1 + 2 * KB + j] = (sizeof(T) == 4) ? ddf{(float)acc.lt[j], 0.f} : dd_from_double((double)acc.lt[j]);
  }
  unsigned bad = acc.bad;
  for (int m = 16; m > 0; m >>= 1) bad += __shfl_xor_sync(0xffffffffu, bad, m);
  if ((threadIdx.x & 31) == 0) s_bad[threadIdx.x >> 5] = bad;
  block_reduce_to_partials<NS>(v, NS, partials, s_red);
  if (threadIdx.x == 0) {
    unsigned b = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += s_bad[w];
    if (b) atomicAdd(counters + 1, b);
  }
  __shared__ double s_out[NS];
  if (!last_block_ticket(counters, gridDim.x)) return;
  // every other block added to these words before its ticket (and a fence): plain L2 reads,
  // issued before the reduction so that their latency overlaps it
  unsigned nbad = 0u, status = 0u;
  if (threadIdx.x == 0) {
    nbad = __ldcg(counters + 1);
    status = __ldcg(counters + kStatusWord);
  }
  reduce_partials(partials, NS, gridDim.x, s_out, s_red, blockDim.x);
  const double nev = (double)(end - begin);
  const int K = a.K;
  const int P = a.n_params;
  const int off = out_mode == 0 ? 2 : 3;
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    double g = 0.0;
    if (GRAD) {
      for (int k = 0; k < K; ++k) {
        if (a.par_re[k] == p) g += -s_out[1 + 2 * k] + nev * a.nrm_ur[k];
        if (a.par_im[k] == p) g += -s_out[2 + 2 * k] - nev * a.nrm_ui[k];
      }
      const int o = 1 + 2 * KB;
      for (int j = 0; j < 4; ++j)
        if (a.par_t[j] == p) g += -s_out[o + j] + (j < 3 ? nev * a.nrm_dt[j] : 0.0);
    }
    result[off + p] = g;
  }
  if (threadIdx.x == 0) {
    counters[1] = 0u;
    counters[kStatusWord] = 0u;
    *counters = 0u;  // the ticket
    const double nb = status ? -1.0 : (double)nbad;  // a wait that gave up: negative count
    result[0] = -s_out[0] + nev * a.nrm_logN;
    if (out_mode == 0) {
      result[1] = nb;
      result[2 + P] = a.nrm_N;
    } else {
      result[1] = 0.0;
      result[2] = nb;
    }
  }
  result_complete(result, P > 1 ? P : 1);
}

// FP64: direct loads, one event per thread per grid-stride step.
template <int KB, bool GRAD>
__global__ void __launch_bounds__(kBlock, 2) td4_nll_f64_kernel(const __grid_constant__ Td4Args<double> a,
                                                                const double2* __restrict__ cache,
                                                                const double* __restrict__ tcol, int64_t begin,
                                                                int64_t end, float2* partials, unsigned* counters,
                                                                double* result, int out_mode) {
  constexpr int NS = TdLanes<KB, GRAD>::NS;
  __shared__ ddf s_red[(kBlock / 32) * NS > kBlock ? (kBlock / 32) * NS : kBlock];
  __shared__ unsigned s_bad[kBlock / 32];
  TdAcc<double, KB> acc;
#pragma unroll
  for (int k = 0; k < KB; ++k) acc.lre[k] = acc.lim[k] = 0.0;
#pragma unroll
  for (int j = 0; j < 4; ++j) acc.lt[j] = 0.0;
  const int K = a.K;
  const int64_t n = a.n_total;
  for (int64_t i = begin + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < end;
       i += (int64_t)gridDim.x * blockDim.x) {
    double ar[KB], ai[KB];
#pragma unroll
    for (int k = 0; k < KB; ++k) {
      double2 v = make_double2(0.0, 0.0);
      if (k < K) v = cache[(int64_t)k * n + i];
      ar[k] = v.x;
      ai[k] = v.y;
    }
    td4_event<double, KB, GRAD>(a, ar, ai, tcol[i], acc);
  }
  td4_finish<double, KB, GRAD>(a, acc, begin, end, partials, counters, result, out_mode, s_red, s_bad);
}

// FP32: tiles of kTdTile events (aligned to multiples of kTdTile) of every amplitude plane
// and of the time column staged in shared memory by bulk copies, kTdStages tiles ahead;
// block b takes tiles tb0 + b, + gridDim.x, ...; ragged first / last tiles read global
// memory.  Dynamic shared memory: kTdStages * (planes * kTdTile float4 + kTdTile float).
constexpr int kTdTile = kBlock;  // one event per thread per tile
constexpr int kTdStages = 4;

template <int KB, bool GRAD>
__global__ void __launch_bounds__(kBlock, 2) td4_nll_f32_kernel(const __grid_constant__ Td4Args<float> a,
                                                                const float4* __restrict__ cache,
                                                                const float* __restrict__ tcol, int64_t begin,
                                                                int64_t end, float2* partials, unsigned* counters,
                                                                double* result, int out_mode) {
  constexpr int NS = TdLanes<KB, GRAD>::NS;
  constexpr int TE = kTdTile, NST = kTdStages;
  __shared__ ddf s_red[(kBlock / 32) * NS > kBlock ? (kBlock / 32) * NS : kBlock];
  __shared__ unsigned s_bad[kBlock / 32];
  __shared__ __align__(8) uint64_t s_bar[NST];
  extern __shared__ __align__(128) float4 s_tile[];  // per stage: planes x TE float4, then TE float
  const int planes = a.planes;
  const int64_t n = a.n_total;
  const size_t stage_f4 = (size_t)planes * TE + TE / 4;
  const int64_t tb0 = begin / TE, tb1 = (end + TE - 1) / TE;
  auto tile_of = [&](int j) { return tb0 + blockIdx.x + (int64_t)j * gridDim.x; };
  auto full = [&](int64_t t) { return t * TE >= begin && (t + 1) * TE <= end; };
  auto issue = [&](int j) {
    const int64_t t = tile_of(j);
    if (t >= tb1) return;
    uint64_t* bar = &s_bar[j % NST];
    float4* base = s_tile + (size_t)(j % NST) * stage_f4;
    if (full(t)) {
      mbar_arrive_expect_tx(bar, (unsigned)(planes * TE * sizeof(float4) + TE * sizeof(float)));
      for (int p = 0; p < planes; ++p) bulk_load(base + (size_t)p * TE, cache + (int64_t)p * n + t * TE, TE * sizeof(float4), bar);
      bulk_load(base + (size_t)planes * TE, tcol + t * TE, TE * sizeof(float), bar);
    } else {
      mbar_arrive(bar);
    }
  };
  if (threadIdx.x == 0) {
    for (int st = 0; st < NST; ++st) mbar_init(&s_bar[st], 1);
    mbar_init_fence();
    for (int j = 0; j < NST; ++j) issue(j);
  }
  TdAcc<float, KB> acc;
#pragma unroll
  for (int k = 0; k < KB; ++k) acc.lre[k] = acc.lim[k] = 0.f;
#pragma unroll
  for (int j = 0; j < 4; ++j) acc.lt[j] = 0.f;
  __syncthreads();  // barriers initialised before any thread waits on them
  const long long wlim = tile_wait_limit(counters);
  int j = 0;
  bool failed = false;
  for (; tile_of(j) < tb1; ++j) {
    const int64_t t = tile_of(j);
    const int st = j % NST;
    const bool ok_wait = mbar_wait(&s_bar[st], (unsigned)(j / NST) & 1u, wlim);
    if (ok_wait) {
      const float4* sb = s_tile + (size_t)st * stage_f4;
      const float* stt = (const float*)(sb + (size_t)planes * TE);
      const bool staged = full(t);
      for (int e = threadIdx.x; e < TE; e += blockDim.x) {
        const int64_t i = t * TE + e;
        if (!staged && (i < begin || i >= end)) continue;
        float2 am[KB];
#pragma unroll
        for (int p = 0; p < KB / 2; ++p) {
          float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
          if (p < planes) v = staged ? sb[(size_t)p * TE + e] : __ldg(cache + (int64_t)p * n + i);
          am[2 * p] = make_float2(v.x, v.y);
          am[2 * p + 1] = make_float2(v.z, v.w);
        }
        const float tv = staged ? stt[e] : __ldg(tcol + i);
        td4_event_f32<KB, GRAD>(a, am, tv, acc);
      }
    }
    if (__syncthreads_or(!ok_wait)) {
      failed = true;
      break;
    }
    if (threadIdx.x == 0) {
      fence_proxy_async();
      issue(j + NST);
    }
  }
  if (failed) {
    // a copy did not arrive in time: record it, then wait (again bounded) for this block's
    // copies still in flight before the block's shared memory is released
    if (threadIdx.x == 0) {
      atomicOr(counters + kStatusWord, 1u);
      for (int jj = j; jj < j + NST && tile_of(jj) < tb1; ++jj) mbar_wait(&s_bar[jj % NST], (unsigned)(jj / NST) & 1u);
    }
    __syncthreads();
  }
  td4_finish<float, KB, GRAD>(a, acc, begin, end, partials, counters, result, out_mode, s_red, s_bad);
}

// per-event log f = log R - log N (goo_eval_logf)
template <typename T, int KB>
__global__ void td4_logf_kernel(const __grid_constant__ Td4Args<T> a, const void* cache_v, const T* __restrict__ tcol,
                                double logN, double* __restrict__ out) {
  const int K = a.K;
  const int64_t n = a.n_total;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    T ar[KB], ai[KB];
#pragma unroll
    for (int k = 0; k < KB; ++k) {
      ar[k] = ai[k] = T(0);
      if (k < K) {
        if constexpr (sizeof(T) == 4) {
          const float4 v = ((const float4*)cache_v)[(int64_t)(k / 2) * n + i];
          ar[k] = (k & 1) ? v.z : v.x;
          ai[k] = (k & 1) ? v.w : v.y;
        } else {
          const double2 v = ((const double2*)cache_v)[(int64_t)k * n + i];
          ar[k] = v.x;
          ai[k] = v.y;
        }
      }
    }
    TdAcc<T, KB> acc;
    td4_event<T, KB, false>(a, ar, ai, tcol[i], acc);
    const double lr = (sizeof(T) == 4) ? dd_to_double(acc.lf32.value()) : acc.lf64;
    out[i] = acc.bad ? -HUGE_VAL : lr - logN;
  }
}

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------
struct Td4Model {
  int K = 0;
  int par_re[kTdMaxAmp], par_im[kTdMaxAmp], par_t[4];
  double br[kTdMaxAmp], bi[kTdMaxAmp];
  Td4Dev host{};
  Td4Dev* dev = nullptr;
  double* gram_dev[2] = {nullptr, nullptr};
  double gram_host[2][kTdMaxAmp * kTdMaxAmp * 2];
  uint64_t gram_key[2] = {0, 0};
  const goo_dataset* mc = nullptr;
  uint64_t key = 0;
};

static double two_body_q(double m, double ma, double mb) {
  const double lam = (m * m - (ma + mb) * (ma + mb)) * (m * m - (ma - mb) * (ma - mb));
  return std::sqrt(lam > 0 ? lam : 0.0) / (2.0 * m);
}

static double barrier_host(int L, double z) {
  if (L == 0) return 1.0;
  if (L == 1) return std::sqrt(1.0 / (1.0 + z));
  return std::sqrt(9.0 / (9.0 + 3.0 * z + z * z));
}

static void spins_of(int ang, int& L1, int& L2) {
  static const int s1[8] = {0, 1, 0, 1, 1, 1, 2, 2}, s2[8] = {0, 0, 1, 1, 1, 1, 0, 1};
  L1 = s1[ang];
  L2 = s2[ang];
}

int build_td4_model(goo_ctx* ctx, const goo_node* nodes, int n_nodes, int n_params, int n_obs, goo_model* m) {
  const goo_node& root = nodes[n_nodes - 1];
  if (n_obs != 6) return set_error(GOO_ERR_ARG, "GOO_OP_TD4 needs the 6 observables m12, m34, c12, c34, phi, t");
  if (root.n_child < 1 || root.n_child > kTdMaxAmp)
    return set_error(GOO_ERR_UNSUPPORTED, "GOO_OP_TD4 with %d amplitudes (1..%d)", root.n_child, kTdMaxAmp);
  Td4Model* d = new Td4Model();
  m->td4 = d;
  m->kind = 2;
  Td4Dev& h = d->host;
  h.K = d->K = root.n_child;
  h.m1 = root.dval[1];
  h.m2 = root.dval[2];
  h.m3 = root.dval[3];
  h.m4 = root.dval[4];
  h.r = root.dval[5];
  const double M = root.dval[0];
  if (!(M > h.m1 + h.m2 + h.m3 + h.m4) || h.r < 0)
    return set_error(GOO_ERR_ARG, "GOO_OP_TD4: parent mass below threshold or negative barrier radius");
  for (int j = 0; j < 4; ++j) {
    if (root.par[j] < 0 || root.par[j] >= n_params)
      return set_error(GOO_ERR_ARG, "GOO_OP_TD4: time parameter %d has index %d", j, root.par[j]);
    d->par_t[j] = root.par[j];
  }
  for (int k = 0; k < d->K; ++k) {
    const goo_node& a = nodes[root.child[k]];
    if (a.op != GOO_OP_AMP4) return set_error(GOO_ERR_ARG, "GOO_OP_TD4 child %d is not GOO_OP_AMP4", k);
    if (a.ival[0] < GOO_ANG_SS || a.ival[0] > GOO_ANG_TV0) return set_error(GOO_ERR_ARG, "angular type %d", a.ival[0]);
    for (int j = 0; j < 2; ++j)
      if (a.par[j] < 0 || a.par[j] >= n_params) return set_error(GOO_ERR_ARG, "amplitude %d coefficient index", k);
    d->par_re[k] = a.par[0];
    d->par_im[k] = a.par[1];
    d->br[k] = a.dval[4];
    d->bi[k] = a.dval[5];
    Td4Amp& A = h.amp[k];
    A.ang = a.ival[0];
    spins_of(A.ang, A.L1, A.L2);
    A.m0a = a.dval[0];
    A.g0a = a.dval[1];
    A.m0b = a.dval[2];
    A.g0b = a.dval[3];
    if (!(A.m0a > h.m1 + h.m2) || !(A.m0b > h.m3 + h.m4) || !(A.g0a > 0) || !(A.g0b > 0))
      return set_error(GOO_ERR_ARG, "amplitude %d: resonance below its pair threshold or width <= 0", k);
    A.q0a = two_body_q(A.m0a, h.m1, h.m2);
    A.q0b = two_body_q(A.m0b, h.m3, h.m4);
    A.b0a = barrier_host(A.L1, (h.r * A.q0a) * (h.r * A.q0a));
    A.b0b = barrier_host(A.L2, (h.r * A.q0b) * (h.r * A.q0b));
  }
  uint64_t key = 1469598103934665603ull;  // FNV-1a over the lineshape constants
  const unsigned char* bytes = (const unsigned char*)&h;
  for (size_t i = 0; i < sizeof(Td4Dev); ++i) key = (key ^ bytes[i]) * 1099511628211ull;
  d->key = key;
  if (cudaMalloc(&d->dev, sizeof(Td4Dev)) != cudaSuccess || cudaMalloc(&d->gram_dev[0], sizeof(double) * 2 * kTdMaxAmp * kTdMaxAmp) != cudaSuccess ||
      cudaMalloc(&d->gram_dev[1], sizeof(double) * 2 * kTdMaxAmp * kTdMaxAmp) != cudaSuccess) {
    cudaGetLastError();
    return set_error(GOO_ERR_OOM, "goo_model_build: four-body model tables");
  }
  GOO_CUDA_TRY(cudaMemcpyAsync(d->dev, &h, sizeof(Td4Dev), cudaMemcpyHostToDevice, ctx->stream));
  GOO_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  (void)weideman();
  return GOO_OK;
}

void td4_free(goo_model* m) {
  Td4Model* d = m->td4;
  if (!d) return;
  if (d->dev) cudaFree(d->dev);
  for (auto& g : d->gram_dev)
    if (g) cudaFree(g);
  delete d;
  m->td4 = nullptr;
}

int td4_set_norm(goo_model* m, const goo_norm_spec* spec) {
  if (spec->kind != GOO_NORM_MC || !spec->mc)
    return set_error(GOO_ERR_UNSUPPORTED, "the four-body model is normalised with GOO_NORM_MC and a phase-space sample");
  if (spec->mc->ncols < 5) return set_error(GOO_ERR_ARG, "the MC sample needs the five phase-space columns");
  m->td4->mc = spec->mc;
  m->td4->gram_key[0] = m->td4->gram_key[1] = 0;
  m->norm = *spec;
  return GOO_OK;
}

static int td4_cache(goo_model* m, const goo_dataset* ds_c, int precision, const void** out) {
  goo_dataset* ds = const_cast<goo_dataset*>(ds_c);
  Td4Model& d = *m->td4;
  goo_ctx* ctx = m->ctx;
  const int pi = precision == GOO_F32 ? 0 : 1;
  const uint64_t key = d.key ^ (uint64_t)(uintptr_t)m ^ (uint64_t)(pi + 3) * 0x9e3779b97f4a7c15ull ^
                       ds->epoch * 0xd6e8feb86659fd93ull;
  CacheSlot& slot = ds->cache[pi];
  const int64_t n = ds->n;
  const size_t bytes = pi == 0 ? (size_t)((d.K + 1) / 2) * (size_t)n * sizeof(float4) : (size_t)d.K * (size_t)n * sizeof(double2);
  if (slot.ptr && slot.key == key && slot.bytes >= bytes) {
    *out = slot.ptr;
    return GOO_OK;
  }
  if (!slot.ptr || slot.bytes < bytes) {
    if (slot.ptr) cudaFree(slot.ptr);
    slot.ptr = nullptr;
    slot.bytes = 0;
    if (cudaMalloc(&slot.ptr, bytes > 0 ? bytes : 16) != cudaSuccess) {
      cudaGetLastError();
      return set_error(GOO_ERR_OOM, "amplitude cache of %zu bytes does not fit", bytes);
    }
    slot.bytes = bytes;
  }
  if (n > 0) {
    const int nb = grid_blocks(ctx, n, 4);
    if (pi == 0) {
      Td4Cols<float> c{};
      for (int j = 0; j < 5; ++j) c.c[j] = ds->d32[j];
      LaunchScope ls(ctx, "td4_cache_f32");
      td4_cache_kernel<float><<<nb, kBlock, 0, ctx->stream>>>(d.dev, c, n, slot.ptr);
    } else {
      Td4Cols<double> c{};
      for (int j = 0; j < 5; ++j) c.c[j] = ds->d64[j];
      LaunchScope ls(ctx, "td4_cache_f64");
      td4_cache_kernel<double><<<nb, kBlock, 0, ctx->stream>>>(d.dev, c, n, slot.ptr);
    }
    GOO_CUDA_TRY(cudaGetLastError());
  }
  slot.key = key;
  *out = slot.ptr;
  return GOO_OK;
}

template <typename T>
static int td4_gram_launch(goo_model* m, const void* cache, int64_t n, int pi) {
  Td4Model& d = *m->td4;
  goo_ctx* ctx = m->ctx;
  constexpr int KB = 15;
  constexpr int NS = 2 * (KB + 1);
  int bps = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, gram_kernel<T, KB>, kBlock, 0) != cudaSuccess || bps < 1) {
    cudaGetLastError();
    bps = 1;
  }
  int64_t nbx = (n + kBlock - 1) / kBlock;
  const int64_t cap = ((int64_t)ctx->num_sms * bps + d.K - 1) / d.K;
  if (nbx > cap) nbx = cap;
  if (nbx < 1) nbx = 1;
  GOO_TRY(ensure_partials(ctx, (size_t)nbx * d.K * NS));
  {
    LaunchScope ls(ctx, sizeof(T) == 4 ? "td4_gram_f32" : "td4_gram_f64");
    gram_kernel<T, KB><<<dim3((unsigned)nbx, d.K), kBlock, 0, ctx->stream>>>(cache, n, d.K, 0, ctx->scratch.partials,
                                                                            ctx->scratch.counters, d.gram_dev[pi]);
  }
  GOO_CUDA_TRY(cudaGetLastError());
  return GOO_OK;
}

static int td4_ensure_gram(goo_model* m, int precision) {
  Td4Model& d = *m->td4;
  const int pi = precision == GOO_F32 ? 0 : 1;
  if (!d.mc) return set_error(GOO_ERR_STATE, "the four-body model has no MC normalisation sample (goo_model_set_norm)");
  if (d.K > 15) return set_error(GOO_ERR_UNSUPPORTED, "the Gram matrix supports at most 15 amplitudes");
  const uint64_t key = d.key ^ (uint64_t)(uintptr_t)d.mc ^ (uint64_t)(pi + 11) ^ d.mc->epoch * 0xd6e8feb86659fd93ull;
  if (d.gram_key[pi] == key) return GOO_OK;
  if (d.mc->n < 1) return set_error(GOO_ERR_ARG, "the MC normalisation sample is empty");
  const void* cache = nullptr;
  GOO_TRY(td4_cache(m, d.mc, precision, &cache));
  if (pi == 0) GOO_TRY(td4_gram_launch<float>(m, cache, d.mc->n, pi));
  else GOO_TRY(td4_gram_launch<double>(m, cache, d.mc->n, pi));
  GOO_CUDA_TRY(cudaMemcpyAsync(d.gram_host[pi], d.gram_dev[pi], sizeof(double) * 2 * d.K * d.K, cudaMemcpyDeviceToHost,
                               m->ctx->stream));
  GOO_CUDA_TRY(cudaStreamSynchronize(m->ctx->stream));
  d.gram_key[pi] = key;
  return GOO_OK;
}

template <typename T>
static void td4_args(const goo_model* m, const double* theta, int64_t n_total, Td4Args<T>& a) {
  const Td4Model& d = *m->td4;
  std::memset(&a, 0, sizeof a);
  a.K = d.K;
  a.planes = (d.K + 1) / 2;
  a.n_params = m->n_params;
  a.n_total = n_total;
  for (int k = 0; k < d.K; ++k) {
    a.cr[k] = (T)theta[d.par_re[k]];
    a.ci[k] = (T)theta[d.par_im[k]];
    a.br[k] = (T)d.br[k];
    a.bi[k] = (T)d.bi[k];
    a.par_re[k] = d.par_re[k];
    a.par_im[k] = d.par_im[k];
  }
  for (int j = 0; j < 4; ++j) a.par_t[j] = d.par_t[j];
  fill_time_coef<T>(a.tc, theta[d.par_t[0]], theta[d.par_t[1]], theta[d.par_t[2]], theta[d.par_t[3]], m->hi[5]);
  a.x = a.tc.x;
  a.y = a.tc.y;
  a.G = a.tc.G;
  a.s = a.tc.s;
  const WeidemanTables& w = weideman();
  a.wN = sizeof(T) == 4 ? kWN32 : kWN64;
  for (int j = 0; j < a.wN; ++j) a.wa[j] = (T)(sizeof(T) == 4 ? w.a32[j] : w.a64[j]);
  a.wL = (T)(sizeof(T) == 4 ? w.L32 : w.L64);
}

// The normalisation at theta from the host copy of the Gram matrix (td4_ensure_gram keeps it
// current), in FP64 and at the precision-rounded parameters the kernel uses:
//   v_c = G conj(c), v_b = G conj(b),  <|A|^2> = Re c.v_c, <|B|^2> = Re b.v_b, <A B*> = c.v_b,
//   N = <|A|^2+|B|^2>/2 I_ch + <|A|^2-|B|^2>/2 I_c + Re<AB*> I_sh + Im<AB*> I_s,
//   dN / d Re c_k = Re((I_ch + I_c) v_c,k + (I_sh - i I_s) v_b,k), dN / d Im c_k = -Im(same),
// with the time integrals' derivatives for x, y and tau.
template <typename T>
static void td4_norm_terms(const goo_model* m, int precision, Td4Args<T>& a) {
  const Td4Model& d = *m->td4;
  const int pi = precision == GOO_F32 ? 0 : 1;
  const int K = d.K;
  const double x = (double)a.x, y = (double)a.y, tau = 1.0 / (double)a.G;
  const double iy = 1.0 / (1 - y * y), ix = 1.0 / (1 + x * x);
  const double Ich = tau * iy, Ish = y * tau * iy, Ic = tau * ix, Is = x * tau * ix;
  double vcr[kTdMaxAmp], vci[kTdMaxAmp], vbr[kTdMaxAmp], vbi[kTdMaxAmp];
  double aa = 0, bb = 0, abr = 0, abi = 0;
  for (int k = 0; k < K; ++k) {
    vcr[k] = vci[k] = vbr[k] = vbi[k] = 0.0;
    for (int l = 0; l < K; ++l) {
      const double gr = d.gram_host[pi][2 * (k * K + l)], gi = d.gram_host[pi][2 * (k * K + l) + 1];
      const double clr = (double)a.cr[l], cli = (double)a.ci[l], blr = (double)a.br[l], bli = (double)a.bi[l];
      vcr[k] += gr * clr + gi * cli;  // G_kl conj(c_l)
      vci[k] += gi * clr - gr * cli;
      vbr[k] += gr * blr + gi * bli;
      vbi[k] += gi * blr - gr * bli;
    }
    const double ckr = (double)a.cr[k], cki = (double)a.ci[k], bkr = (double)a.br[k], bki = (double)a.bi[k];
    aa += ckr * vcr[k] - cki * vci[k];  // Re(c_k v_c,k)
    bb += bkr * vbr[k] - bki * vbi[k];
    abr += ckr * vbr[k] - cki * vbi[k];  // c_k v_b,k (summed: <A B*>)
    abi += ckr * vbi[k] + cki * vbr[k];
  }
  const double N = 0.5 * (aa + bb) * Ich + 0.5 * (aa - bb) * Ic + abr * Ish + abi * Is;
  const double invN = 1.0 / N;
  for (int k = 0; k < K; ++k) {
    a.nrm_ur[k] = ((Ich + Ic) * vcr[k] + Ish * vbr[k] + Is * vbi[k]) * invN;
    a.nrm_ui[k] = ((Ich + Ic) * vci[k] + Ish * vbi[k] - Is * vbr[k]) * invN;
  }
  a.nrm_N = N;
  a.nrm_logN = std::log(N);
  const double ix2 = ix * ix, iy2 = iy * iy;
  const double dxc = -2 * x * tau * ix2, dxs = tau * (1 - x * x) * ix2;
  const double dych = 2 * y * tau * iy2, dysh = tau * (1 + y * y) * iy2;
  a.nrm_dt[0] = (0.5 * (aa - bb) * dxc + abi * dxs) * invN;  // (dN/dx) / N
  a.nrm_dt[1] = (0.5 * (aa + bb) * dych + abr * dysh) * invN;
  a.nrm_dt[2] = (0.5 * (aa + bb) * iy + 0.5 * (aa - bb) * ix + abr * y * iy + abi * x * ix) * invN;  // tau dN/dtau / N
}

static int td4_check_theta(const goo_model* m, const double* theta) {
  const Td4Model& d = *m->td4;
  const double x = theta[d.par_t[0]], y = theta[d.par_t[1]], tau = theta[d.par_t[2]], s = theta[d.par_t[3]];
  if (!(tau > 0) || !(s > 0) || !(std::fabs(y) < 1) || !std::isfinite(x))
    return set_error(GOO_ERR_ARG, "four-body model: needs tau > 0, sigma_t > 0, |y| < 1 (tau=%g sigma=%g y=%g)", tau, s, y);
  return GOO_OK;
}

constexpr int kMaxDevicesTd = 64;

template <int KB, bool GRAD>
static int launch_td4_f32(goo_model* m, const void* cache, const goo_dataset* ds, int64_t begin, int64_t end,
                          const double* theta, int out_mode) {
  goo_ctx* ctx = m->ctx;
  Td4Args<float> a;
  td4_args<float>(m, theta, ds->n, a);
  td4_norm_terms<float>(m, GOO_F32, a);
  const size_t smem = (size_t)kTdStages * ((size_t)a.planes * kTdTile * sizeof(float4) + kTdTile * sizeof(float));
  static bool configured[kMaxDevicesTd] = {};
  if (ctx->device < 0 || ctx->device >= kMaxDevicesTd) return set_error(GOO_ERR_ARG, "device %d", ctx->device);
  if (!configured[ctx->device]) {
    GOO_CUDA_TRY(cudaFuncSetAttribute(td4_nll_f32_kernel<KB, GRAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)((size_t)kTdStages * ((KB / 2) * kTdTile * sizeof(float4) + kTdTile * sizeof(float)))));
    configured[ctx->device] = true;
  }
  const int occ = cached_occupancy((const void*)td4_nll_f32_kernel<KB, GRAD>, ctx->device, kBlock, smem);
  const int64_t tiles = (end + kTdTile - 1) / kTdTile - begin / kTdTile;
  const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)ctx->num_sms * occ));
  GOO_TRY(ensure_partials(ctx, (size_t)nb * TdLanes<KB, GRAD>::NS));
  {
    LaunchScope ls(ctx, GRAD ? "td4_nll_grad_f32" : "td4_nll_f32");
    td4_nll_f32_kernel<KB, GRAD><<<nb, kBlock, smem, ctx->stream>>>(a, (const float4*)cache, ds->d32[5], begin, end,
                                                                   ctx->scratch.partials, ctx->scratch.counters,
                                                                   ctx->scratch.result_out, out_mode);
  }
  GOO_CUDA_TRY(cudaGetLastError());
  return GOO_OK;
}

template <int KB, bool GRAD>
static int launch_td4_f64(goo_model* m, const void* cache, const goo_dataset* ds, int64_t begin, int64_t end,
                          const double* theta, int out_mode) {
  goo_ctx* ctx = m->ctx;
  Td4Args<double> a;
  td4_args<double>(m, theta, ds->n, a);
  td4_norm_terms<double>(m, GOO_F64, a);
  static int occ = 0;
  if (occ == 0 && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, td4_nll_f64_kernel<KB, GRAD>, kBlock, 0) != cudaSuccess ||
                   occ < 1)) {
    cudaGetLastError();
    occ = 1;
  }
  const int nb = grid_blocks(ctx, end - begin, occ);
  GOO_TRY(ensure_partials(ctx, (size_t)nb * TdLanes<KB, GRAD>::NS));
  {
    LaunchScope ls(ctx, GRAD ? "td4_nll_grad_f64" : "td4_nll_f64");
    td4_nll_f64_kernel<KB, GRAD><<<nb, kBlock, 0, ctx->stream>>>(a, (const double2*)cache, ds->d64[5], begin, end,
                                                                ctx->scratch.partials, ctx->scratch.counters,
                                                                ctx->scratch.result_out, out_mode);
  }
  GOO_CUDA_TRY(cudaGetLastError());
  return GOO_OK;
}

template <bool GRAD>
static int td4_launch(goo_model* m, const void* cache, const goo_dataset* ds, int64_t begin, int64_t end,
                      const double* theta, int precision, int out_mode) {
  const bool small = m->td4->K <= 10;
  if (precision == GOO_F32)
    return small ? launch_td4_f32<10, GRAD>(m, cache, ds, begin, end, theta, out_mode)
                 : launch_td4_f32<16, GRAD>(m, cache, ds, begin, end, theta, out_mode);
  return small ? launch_td4_f64<10, GRAD>(m, cache, ds, begin, end, theta, out_mode)
               : launch_td4_f64<16, GRAD>(m, cache, ds, begin, end, theta, out_mode);
}

int td4_nll(goo_model* m, const goo_dataset* ds, int64_t begin, int64_t end, const double* theta, int precision,
            bool grad, double* out, int out_mode) {
  goo_ctx* ctx = m->ctx;
  // the record goes to the mapped host copy; the host polls its fields
  MappedResult mapped(ctx);
  const int P = m->n_params;
  if (ds->ncols < 6) return set_error(GOO_ERR_ARG, "the four-body model needs 6 dataset columns");
  GOO_TRY(td4_check_theta(m, theta));
  GOO_TRY(td4_ensure_gram(m, precision));
  const int nout = (out_mode == 0 ? 2 : 3) + P;
  if (end <= begin) {
    for (int i = 0; i < nout; ++i) out[i] = 0.0;
    return GOO_OK;
  }
  const void* cache = nullptr;
  GOO_TRY(td4_cache(m, ds, precision, &cache));
  GOO_TRY((grad ? td4_launch<true>(m, cache, ds, begin, end, theta, precision, out_mode)
                : td4_launch<false>(m, cache, ds, begin, end, theta, precision, out_mode)));
  return read_result_mapped(ctx, nout, out);
}

// N at theta from the host copy of the Gram matrix (the same formula as the kernels' last block)
static double td4_norm_host(const goo_model* m, const double* theta, int precision) {
  const Td4Model& d = *m->td4;
  const int pi = precision == GOO_F32 ? 0 : 1;
  const bool f32 = precision == GOO_F32;
  auto rnd = [&](double v) { return f32 ? (double)(float)v : v; };
  double aa = 0, bb = 0, abr = 0, abi = 0;
  const int K = d.K;
  for (int k = 0; k < K; ++k) {
    const double ckr = rnd(theta[d.par_re[k]]), cki = rnd(theta[d.par_im[k]]), bkr = rnd(d.br[k]), bki = rnd(d.bi[k]);
    double vcr = 0, vci = 0, vbr = 0, vbi = 0;
    for (int l = 0; l < K; ++l) {
      const double gr = d.gram_host[pi][2 * (k * K + l)], gi = d.gram_host[pi][2 * (k * K + l) + 1];
      const double clr = rnd(theta[d.par_re[l]]), cli = rnd(theta[d.par_im[l]]), blr = rnd(d.br[l]), bli = rnd(d.bi[l]);
      vcr += gr * clr + gi * cli;
      vci += gi * clr - gr * cli;
      vbr += gr * blr + gi * bli;
      vbi += gi * blr - gr * bli;
    }
    aa += ckr * vcr - cki * vci;
    bb += bkr * vbr - bki * vbi;
    abr += ckr * vbr - cki * vbi;
    abi += ckr * vbi + cki * vbr;
  }
  const double x = rnd(theta[d.par_t[0]]), y = rnd(theta[d.par_t[1]]);
  const double tau = 1.0 / rnd(1.0 / theta[d.par_t[2]]);
  return 0.5 * (aa + bb) * tau / (1 - y * y) + 0.5 * (aa - bb) * tau / (1 + x * x) + abr * y * tau / (1 - y * y) +
         abi * x * tau / (1 + x * x);
}

int td4_normalise(goo_model* m, const double* theta, int precision, double* norm_out) {
  GOO_TRY(td4_check_theta(m, theta));
  GOO_TRY(td4_ensure_gram(m, precision));
  *norm_out = td4_norm_host(m, theta, precision);
  return GOO_OK;
}

int td4_eval_logf(goo_model* m, const goo_dataset* ds, const double* theta, int precision, double* logf_dev) {
  goo_ctx* ctx = m->ctx;
  if (ds->ncols < 6) return set_error(GOO_ERR_ARG, "the four-body model needs 6 dataset columns");
  GOO_TRY(td4_check_theta(m, theta));
  GOO_TRY(td4_ensure_gram(m, precision));
  if (ds->n == 0) return GOO_OK;
  const double logN = std::log(td4_norm_host(m, theta, precision));
  const void* cache = nullptr;
  GOO_TRY(td4_cache(m, ds, precision, &cache));
  const int nb = grid_blocks(ctx, ds->n, 4);
  LaunchScope ls(ctx, "td4_logf");
  const bool small = m->td4->K <= 10;
  if (precision == GOO_F32) {
    Td4Args<float> a;
    td4_args<float>(m, theta, ds->n, a);
    if (small) td4_logf_kernel<float, 10><<<nb, kBlock, 0, ctx->stream>>>(a, cache, ds->d32[5], logN, logf_dev);
    else td4_logf_kernel<float, 16><<<nb, kBlock, 0, ctx->stream>>>(a, cache, ds->d32[5], logN, logf_dev);
  } else {
    Td4Args<double> a;
    td4_args<double>(m, theta, ds->n, a);
    if (small) td4_logf_kernel<double, 10><<<nb, kBlock, 0, ctx->stream>>>(a, cache, ds->d64[5], logN, logf_dev);
    else td4_logf_kernel<double, 16><<<nb, kBlock, 0, ctx->stream>>>(a, cache, ds->d64[5], logN, logf_dev);
  }
  GOO_CUDA_TRY(cudaGetLastError());
  return GOO_OK;
}

int td4_gram(goo_model* m, int precision, double* out, int* K_out) {
  GOO_TRY(td4_ensure_gram(m, precision));
  const int pi = precision == GOO_F32 ? 0 : 1;
  std::memcpy(out, m->td4->gram_host[pi], sizeof(double) * 2 * m->td4->K * m->td4->K);
  *K_out = m->td4->K;
  return GOO_OK;
}

int td4_amplitudes(goo_model* m, const goo_dataset* ds, int precision, const void** cache, int* n_amp) {
  if (ds->ncols < 5) return set_error(GOO_ERR_ARG, "the four-body model needs the five phase-space columns");
  GOO_TRY(td4_cache(m, ds, precision, cache));
  GOO_CUDA_TRY(cudaStreamSynchronize(m->ctx->stream));
  *n_amp = m->td4->K;
  return GOO_OK;
}

}  // namespace goo

// Host evaluation of the library's Faddeeva approximation (the same code the kernels run),
// exposed so that it can be checked against an independent implementation on the CPU.
extern "C" int goo_faddeeva(double re, double im, int precision, double* out) {
  using namespace goo;
  if (!out) return set_error(GOO_ERR_ARG, "goo_faddeeva: NULL output");
  if (!(im >= 0.0)) return set_error(GOO_ERR_ARG, "goo_faddeeva: Im z must be >= 0");
  const WeidemanTables& w = weideman();
  if (precision == GOO_F32) {
    float a[kWMax];
    for (int j = 0; j < kWN32; ++j) a[j] = (float)w.a32[j];
    float wr, wi;
    faddeeva<float>((float)re, (float)im, a, kWN32, (float)w.L32, wr, wi);
    out[0] = wr;
    out[1] = wi;
  } else if (precision == GOO_F64) {
    double wr, wi;
    faddeeva<double>(re, im, w.a64, kWN64, w.L64, wr, wi);
    out[0] = wr;
    out[1] = wi;
  } else {
    return set_error(GOO_ERR_ARG, "goo_faddeeva: precision=%d", precision);
  }
  return GOO_OK;
}
