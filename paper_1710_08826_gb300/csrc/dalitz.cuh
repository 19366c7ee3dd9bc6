// dalitz.cuh -- device code shared by the amplitude-model kernels (dalitz.cu) and the
// toy-MC server (serve.cu): lineshape constants, the Breit-Wigner amplitude of one
// resonance, and the loads of the cached amplitudes of one event.  The formulas are stated
// at the top of dalitz.cu.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace goo {

constexpr int kMaxAmp = 16;

template <typename T>
struct BwConstT {
  int spin, pair;  // pair 0: (12)+3, 1: (13)+2, 2: (23)+1
  T m0sq, m0w;     // m0^2, m0 * Gamma0
  T inv_q0sq;      // 1 / q0^2
  T r2, rp2;       // resonance and parent barrier radii squared
  T thrP, thrM;    // (mA + mB)^2, (mA - mB)^2
  T pthrP, pthrM;  // (M + mC)^2, (M - mC)^2
  T zconst;        // (mA^2 - mB^2)(M^2 - mC^2)
  T inv4M2;        // 1 / (4 M^2)
  T Fz0;           // 1 + z0 (L=1) or 9 + 3 z0 + z0^2 (L=2)
  T m0;            // m0
};
using BwConst = BwConstT<double>;

struct DalitzDev {
  int nbw;              // number of Breit-Wigner amplitudes (cached)
  double sumsq;         // M^2 + m1^2 + m2^2 + m3^2  (s23 = sumsq - s12 - s13)
  BwConstT<double> bw[kMaxAmp];
  BwConstT<float> bwf[kMaxAmp];  // the same constants rounded to float (FP32 path)
};

template <typename T>
__device__ __forceinline__ const BwConstT<T>& bw_of(const DalitzDev& d, int k);
template <>
__device__ __forceinline__ const BwConstT<double>& bw_of<double>(const DalitzDev& d, int k) { return d.bw[k]; }
template <>
__device__ __forceinline__ const BwConstT<float>& bw_of<float>(const DalitzDev& d, int k) { return d.bwf[k]; }

// ---------------------------------------------------------------------------------------
// amplitude of one Breit-Wigner resonance at (s12, s13, s23), in precision T
// ---------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void bw_amp(const BwConstT<T>& b, T s12, T s13, T s23, T& re, T& im) {
  const int L = b.spin;
  T s, sac, sbc;
  if (b.pair == 0) {
    s = s12;
    sac = s13;
    sbc = s23;
  } else if (b.pair == 1) {
    s = s13;
    sac = s12;
    sbc = s23;
  } else {
    s = s23;
    sac = s12;
    sbc = s13;
  }
  const T lam1 = (s - T(b.thrP)) * (s - T(b.thrM));
  T q2 = lam1 / (T(4) * s);
  q2 = q2 > T(0) ? q2 : T(0);
  const T z = T(b.r2) * q2;
  const T t = q2 * T(b.inv_q0sq);
  const T st = sqrt(t);
  T ratio2, pw;
  if (L == 0) {
    ratio2 = T(1);
    pw = st;
  } else if (L == 1) {
    ratio2 = T(b.Fz0) / (T(1) + z);
    pw = t * st;
  } else {
    ratio2 = T(b.Fz0) / (T(9) + T(3) * z + z * z);
    pw = t * t * st;
  }
  const T rs = T(1) / sqrt(s);
  const T m0 = b.m0;
  const T di = T(b.m0w) * pw * m0 * rs * ratio2;  // m0 Gamma(s)
  const T dr = T(b.m0sq) - s;
  const T inv = T(1) / (dr * dr + di * di);
  const T lam2 = (s - T(b.pthrP)) * (s - T(b.pthrM));
  T zp = T(b.rp2) * lam2 * T(b.inv4M2);
  zp = zp > T(0) ? zp : T(0);
  T parent, spinf;
  if (L == 0) {
    parent = T(1);
    spinf = T(1);
  } else if (L == 1) {
    parent = T(1) / sqrt(T(1) + zp);
    spinf = sac - sbc - T(b.zconst) / s;
  } else {
    parent = T(3) / sqrt(T(9) + T(3) * zp + zp * zp);
    const T z1 = sac - sbc - T(b.zconst) / s;
    spinf = z1 * z1 - lam1 * lam2 / (T(3) * s * s);
  }
  const T scale = sqrt(ratio2) * parent * spinf * inv;
  re = dr * scale;
  im = di * scale;
}

// Loads the nbw cached amplitudes of event i (compile-time bound KB, runtime nbw).
template <int KB>
__device__ __forceinline__ void load_amps(const float4* __restrict__ cache, int64_t n, int64_t i, int nbw,
                                          float (&ar)[KB + 1], float (&ai)[KB + 1]) {
#pragma unroll
  for (int p = 0; p < (KB + 1) / 2; ++p) {
    if (2 * p < nbw) {
      const float4 v = __ldg(cache + (int64_t)p * n + i);
      ar[2 * p] = v.x;
      ai[2 * p] = v.y;
      if (2 * p + 1 < KB) {
        ar[2 * p + 1] = v.z;
        ai[2 * p + 1] = v.w;
      }
    } else {
      ar[2 * p] = ai[2 * p] = 0.f;
      if (2 * p + 1 < KB) ar[2 * p + 1] = ai[2 * p + 1] = 0.f;
    }
  }
}

template <int KB>
__device__ __forceinline__ void load_amps(const double2* __restrict__ cache, int64_t n, int64_t i, int nbw,
                                          double (&ar)[KB + 1], double (&ai)[KB + 1]) {
#pragma unroll
  for (int k = 0; k < KB; ++k) {
    if (k < nbw) {
      const double2 v = cache[(int64_t)k * n + i];
      ar[k] = v.x;
      ai[k] = v.y;
    } else {
      ar[k] = ai[k] = 0.0;
    }
  }
}

// One event of a coherent sum in packed FP32 form.  With a_k = (Re A_k, Im A_k) held as a
// register pair and cre_k = (Re c_k, Re c_k), cim_k = (Im c_k, Im c_k):
//   P = sum_k Re c_k a_k,  Q = sum_k Im c_k a_k,  S = (P.x - Q.y) + i (P.y + Q.x),
// and the gradient lanes A_k conj(S) / |S|^2 = (t_r + i t_i) A_k are accumulated as
//   G1_k += t_r a_k,  G2_k += t_i a_k   (Re = G1.x - G2.y, Im = G1.y + G2.x at the end),
// so each amplitude costs two packed fma for S and two for the gradient.
template <int KA, bool GRAD>
__device__ __forceinline__ void coh_event_pk(const float2 (&cre)[KA], const float2 (&cim)[KA], const float2 (&a)[KA],
                                             Kahan& lf, float2 (&G1)[KA], float2 (&G2)[KA], unsigned& bad) {
  float2 P = pk::mul(cre[0], a[0]), Q = pk::mul(cim[0], a[0]);
#pragma unroll
  for (int k = 1; k < KA; ++k) {
    P = pk::fma(cre[k], a[k], P);
    Q = pk::fma(cim[k], a[k], Q);
  }
  const float sr = P.x - Q.y, si = P.y + Q.x;
  const float s2 = fmaf(sr, sr, si * si);
  if (s2 > 0.f) {
    lf.add(pk::kLn2 * pk::lg2(s2));
    if constexpr (GRAD) {
      const float inv = pk::rcp(s2);
      const float2 tr = pk::splat(sr * inv), ti = pk::splat(-si * inv);  // conj(S) / |S|^2
#pragma unroll
      for (int k = 0; k < KA; ++k) {
        G1[k] = pk::fma(tr, a[k], G1[k]);
        G2[k] = pk::fma(ti, a[k], G2[k]);
      }
    }
  } else {
    bad++;
  }
}

// ---------------------------------------------------------------------------------------
template <typename T, int KB>
__global__ void __launch_bounds__(kBlock, 2) gram_kernel(const void* cache_v, int64_t n, int nbw, int has_nr,
                                                         float2* partials, unsigned* counters, double* gram_out) {
  constexpr int KA = KB + 1;
  constexpr int NS = 2 * KA;
  __shared__ ddf s_red[(kBlock / 32) * NS > kBlock ? (kBlock / 32) * NS : kBlock];
  using Vec = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  const Vec* cache = (const Vec*)cache_v;
  const int k = blockIdx.y;  // row, in slot numbering (BW slots, NR = KB)
  const int krow = k < nbw ? k : KB;
  Kahan kr[KA], ki[KA];
  double dr[KA], di[KA];
#pragma unroll
  for (int l = 0; l < KA; ++l) dr[l] = di[l] = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    T ar[KA], ai[KA];
    load_amps<KB>(cache, n, i, nbw, ar, ai);
    ar[KB] = has_nr ? T(1) : T(0);
    ai[KB] = T(0);
    T xr = T(0), xi = T(0);
#pragma unroll
    for (int l = 0; l < KA; ++l)
      if (l == krow) {
        xr = ar[l];
        xi = ai[l];
      }
#pragma unroll
    for (int l = 0; l < KA; ++l) {
      // A_k conj(A_l)
      const T pr = xr * ar[l] + xi * ai[l];
      const T pi = xi * ar[l] - xr * ai[l];
      if constexpr (sizeof(T) == 4) {
        kr[l].add(pr);
        ki[l].add(pi);
      } else {
        dr[l] += pr;
        di[l] += pi;
      }
    }
  }
  ddf v[NS];
#pragma unroll
  for (int l = 0; l < KA; ++l) {
    v[2 * l] = (sizeof(T) == 4) ? kr[l].value() : dd_from_double(dr[l]);
    v[2 * l + 1] = (sizeof(T) == 4) ? ki[l].value() : dd_from_double(di[l]);
  }
  const int nbx = gridDim.x;
  {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      ddf w = dd_warp_sum(v[s]);
      if (lane == 0) s_red[warp * NS + s] = w;
    }
    __syncthreads();
    if (threadIdx.x < NS) {
      ddf acc = s_red[threadIdx.x];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) acc = dd_add(acc, s_red[w * NS + threadIdx.x]);
      partials[((size_t)k * nbx + blockIdx.x) * NS + threadIdx.x] = make_float2(acc.hi, acc.lo);
    }
  }
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = atomicAdd(counters, 1u) == (unsigned)(nbx * gridDim.y - 1);
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  // G in model order: BW amplitudes 0..nbw-1, then NR at index nbw
  const int K = nbw + (has_nr ? 1 : 0);
  for (int lane_id = threadIdx.x; lane_id < (int)gridDim.y * NS; lane_id += blockDim.x) {
    const int kk = lane_id / NS, s = lane_id % NS;
    const int l = s / 2;
    ddf acc = {0.f, 0.f};
    for (int b = 0; b < nbx; ++b) {
      const float2 p = __ldcg(partials + ((size_t)kk * nbx + b) * NS + s);
      acc = dd_add(acc, {p.x, p.y});
    }
    const int krow_model = kk;                              // rows were launched in model order
    const int lcol_model = l < nbw ? l : (l == KB ? nbw : -1);
    // upper triangle from row k, mirrored with conjugation: G is Hermitian by construction
    if (lcol_model >= krow_model && lcol_model < K && krow_model < K) {
      double v = dd_to_double(acc) / (double)n;
      if ((s & 1) && lcol_model == krow_model) v = 0.0;
      gram_out[2 * (krow_model * K + lcol_model) + (s & 1)] = v;
      gram_out[2 * (lcol_model * K + krow_model) + (s & 1)] = (s & 1) ? -v : v;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) *counters = 0u;
}

// The same amplitude with the parts of its denominator D = (m0^2 - s) - i m0 Gamma(s):
// dr = m0^2 - s, di = m0 Gamma(s), inv = 1 / |D|^2, so that 1 / D = (dr + i di) inv.  The
// floating-lineshape kernels form d log A / d m0 and d log A / d Gamma0 from them.
template <typename T>
__device__ __forceinline__ void bw_amp_parts(const BwConstT<T>& b, T s12, T s13, T s23, T& re, T& im, T& dr,
                                             T& di, T& inv) {
  const int L = b.spin;
  T s, sac, sbc;
  if (b.pair == 0) {
    s = s12;
    sac = s13;
    sbc = s23;
  } else if (b.pair == 1) {
    s = s13;
    sac = s12;
    sbc = s23;
  } else {
    s = s23;
    sac = s12;
    sbc = s13;
  }
  const T lam1 = (s - T(b.thrP)) * (s - T(b.thrM));
  T q2 = lam1 / (T(4) * s);
  q2 = q2 > T(0) ? q2 : T(0);
  const T z = T(b.r2) * q2;
  const T t = q2 * T(b.inv_q0sq);
  const T st = sqrt(t);
  T ratio2, pw;
  if (L == 0) {
    ratio2 = T(1);
    pw = st;
  } else if (L == 1) {
    ratio2 = T(b.Fz0) / (T(1) + z);
    pw = t * st;
  } else {
    ratio2 = T(b.Fz0) / (T(9) + T(3) * z + z * z);
    pw = t * t * st;
  }
  const T rs = T(1) / sqrt(s);
  di = T(b.m0w) * pw * T(b.m0) * rs * ratio2;
  dr = T(b.m0sq) - s;
  inv = T(1) / (dr * dr + di * di);
  const T lam2 = (s - T(b.pthrP)) * (s - T(b.pthrM));
  T zp = T(b.rp2) * lam2 * T(b.inv4M2);
  zp = zp > T(0) ? zp : T(0);
  T parent, spinf;
  if (L == 0) {
    parent = T(1);
    spinf = T(1);
  } else if (L == 1) {
    parent = T(1) / sqrt(T(1) + zp);
    spinf = sac - sbc - T(b.zconst) / s;
  } else {
    parent = T(3) / sqrt(T(9) + T(3) * zp + zp * zp);
    const T z1 = sac - sbc - T(b.zconst) / s;
    spinf = z1 * z1 - lam1 * lam2 / (T(3) * s * s);
  }
  const T scale = sqrt(ratio2) * parent * spinf * inv;
  re = dr * scale;
  im = di * scale;
}

}  // namespace goo
