// dalitz.cu -- three-body amplitude (Dalitz-plot) models: amplitude cache, MC Gram matrix
// and the coherent-sum NLL with its adjoint gradient.
//
// Paper: GooFit carries dedicated amplitude PDFs for three-body decays (Sec. 1), whose
// components are complex amplitudes with the density given by the squared magnitude of
// their sum (Sec. 1, footnote); PDFs cache partial results in structure-of-arrays form
// and recompute them only when their parameters change (Sec. 4); MC phase-space samples
// provide the normalisation integral (Sec. 5).
//
// Model (isobar convention; the paper prints no formulas):
//   S(x) = sum_k c_k A_k(x),  f = |S|^2 / N,  N = c^H G c,  G_kl = mean over the MC sample
//   of A_k conj(A_l);  NLL = -sum_i log |S_i|^2 + n log N.
//   A_R(s12, s13) = BW(s_AB) * B_L(r q)/B_L(r q0) * B_L(r_par p*) * Z_L for resonance R in
//   pair (A, B) with bachelor C, where
//     q^2  = lambda(s, mA^2, mB^2) / (4 s),   p*^2 = lambda(M^2, s, mC^2) / (4 M^2),
//     B_0 = 1, B_1(z) = sqrt(1/(1+z)), B_2(z) = sqrt(9/(9+3z+z^2)),   z = r^2 q^2,
//     Gamma(s) = G0 (q/q0)^(2L+1) (m0/sqrt s) (B_L(z)/B_L(z0))^2,
//     BW(s) = 1 / (m0^2 - s - i m0 Gamma(s)),
//     Z_0 = 1,  Z_1 = s_AC - s_BC - (mA^2 - mB^2)(M^2 - mC^2)/s,
//     Z_2 = Z_1^2 - lambda(s, mA^2, mB^2) lambda(M^2, s, mC^2) / (3 s^2)
//   (Z_1 = -4 q k cos(theta) and Z_2 = 16 q^2 k^2 (cos^2 - 1/3) in the resonance frame).
//   lambda(s, a^2, b^2) is evaluated in its factorised form (s-(a+b)^2)(s-(a-b)^2).
//
// Gradient: d|S|^2/d Re c_k = 2 Re(A_k conj S), d|S|^2/d Im c_k = -2 Im(A_k conj S), and
// for the normalisation dN/d Re c_k = 2 Re(v_k), dN/d Im c_k = -2 Im(v_k), v = G conj(c).
// The event kernel accumulates sum_i A_k conj(S_i) / |S_i|^2 (2K lanes) and sum log|S|^2.
//
// FP32 path: amplitudes and S in FP32, Kahan per thread, double-float across threads; the
// final FP64 combination takes c at the FP32-rounded values the kernel used, so the NLL is
// the exact likelihood at those coefficients.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "dalitz.cuh"
#include "timeterms.cuh"
#include "model.cuh"

namespace goo {

struct DalitzModel {
  int K = 0;                       // amplitudes, BWs first then the NR (if any)
  int nbw = 0;
  bool has_nr = false;
  int par_re[kMaxAmp], par_im[kMaxAmp];
  int par_m0[kMaxAmp], par_w[kMaxAmp];
  int spin[kMaxAmp], pair[kMaxAmp];
  int col12 = 0, col13 = 1;
  double M = 0, m1 = 0, m2 = 0, m3 = 0, r_res = 0, r_par = 0;
  DalitzDev host{};
  DalitzDev* dev = nullptr;
  uint64_t ls_key = 0;             // lineshape version of `host`/`dev`
  // Gram matrices (K x K complex, row-major, FP64) per precision, with their keys
  double* gram_dev[2] = {nullptr, nullptr};
  double gram_host[2][kMaxAmp * kMaxAmp * 2];
  uint64_t gram_key[2] = {0, 0};
  const goo_dataset* mc = nullptr;
  bool floating = false;           // GOO_LINESHAPE_FLOATING: no cache, lineshape gradients
  double* ls_mc = nullptr;         // MC-pass lane sums of the floating-lineshape path (device)
  bool polar = false;              // GOO_COEF_POLAR: the coefficient parameters are (r, phi)
  // time-dependent three-body model (GOO_OP_TD3)
  bool td = false;
  int col_t = 2;
  int par_t[4] = {-1, -1, -1, -1};  // x, y, tau, sigma_t
  double* gram3_dev[2] = {nullptr, nullptr};  // per precision: G_aa, G_bb, G_ab (K x K complex each)
  double gram3_host[2][3 * kMaxAmp * kMaxAmp * 2];
  uint64_t gram3_key[2] = {0, 0};
};

// Cache layout.  FP32: ceil(nbw/2) planes of float4 (re_k, im_k, re_k+1, im_k+1) per event;
// FP64: nbw planes of double2 (re, im) per event.  Plane p of an n-event dataset starts at
// element p * n.
__global__ void amp_cache_f32_kernel(const DalitzDev* __restrict__ dd, const float* __restrict__ s12c,
                                     const float* __restrict__ s13c, int64_t n, float4* __restrict__ cache) {
  __shared__ DalitzDev s_dd;
  for (int i = threadIdx.x; i < (int)(sizeof(DalitzDev) / 4); i += blockDim.x)
    ((int*)&s_dd)[i] = ((const int*)dd)[i];
  __syncthreads();
  const int nbw = s_dd.nbw;
  const int planes = (nbw + 1) / 2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float a = s12c[i], b = s13c[i];
    const float c = (float)(s_dd.sumsq - (double)a - (double)b);
    for (int p = 0; p < planes; ++p) {
      float r0, i0, r1 = 0.f, i1 = 0.f;
      bw_amp<float>(s_dd.bwf[2 * p], a, b, c, r0, i0);
      if (2 * p + 1 < nbw) bw_amp<float>(s_dd.bwf[2 * p + 1], a, b, c, r1, i1);
      cache[(int64_t)p * n + i] = make_float4(r0, i0, r1, i1);
    }
  }
}

__global__ void amp_cache_f64_kernel(const DalitzDev* __restrict__ dd, const double* __restrict__ s12c,
                                     const double* __restrict__ s13c, int64_t n, double2* __restrict__ cache) {
  __shared__ DalitzDev s_dd;
  for (int i = threadIdx.x; i < (int)(sizeof(DalitzDev) / 4); i += blockDim.x)
    ((int*)&s_dd)[i] = ((const int*)dd)[i];
  __syncthreads();
  const int nbw = s_dd.nbw;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double a = s12c[i], b = s13c[i];
    const double c = s_dd.sumsq - a - b;
    for (int k = 0; k < nbw; ++k) {
      double re, im;
      bw_amp<double>(s_dd.bw[k], a, b, c, re, im);
      cache[(int64_t)k * n + i] = make_double2(re, im);
    }
  }
}

// ---------------------------------------------------------------------------------------
// coherent NLL (+ gradient lanes) over events [begin, end) of one dataset
// ---------------------------------------------------------------------------------------
template <typename T>
struct CohArgs {
  T cr[kMaxAmp], ci[kMaxAmp];  // coefficients (BWs first, then NR)
  int nbw, K, has_nr;
  int par_re[kMaxAmp], par_im[kMaxAmp];
  int n_params;
  int64_t n_total;             // events of the dataset (cache plane length)
  int polar;                   // the coefficient parameters are (r, phi): c = r e^{i phi}
  double jc[kMaxAmp], js[kMaxAmp], jr[kMaxAmp];  // cos phi, sin phi, r per amplitude (polar)
  // the normalisation at theta, formed on the host in FP64 from the cached Gram matrix
  // (coh_norm_terms): N, log N and 2 v_k / N with v_k = sum_l G_kl conj(c_l)
  double nrm_N, nrm_logN, nrm_vr[kMaxAmp], nrm_vi[kMaxAmp];
};

// A gradient over (Re c, Im c) of amplitude k mapped to its parameters (FP64): unchanged, or
// for polar coefficients d/dr = cos(phi) d/dRe + sin(phi) d/dIm and
// d/dphi = r (-sin(phi) d/dRe + cos(phi) d/dIm).
__device__ __forceinline__ void coef_chain(int polar, double c, double s, double r, double& gre, double& gim) {
  if (!polar) return;
  const double u = c * gre + s * gim, v = r * (c * gim - s * gre);
  gre = u;
  gim = v;
}

template <typename T, int KB, bool GRAD>
struct CohLanes {
  static constexpr int NS = GRAD ? 1 + 2 * (KB + 1) : 1;
};

// Per-thread accumulators of the coherent kernels.
template <typename T, int KB>
struct CohAcc {
  Kahan lf32;
  double lf64 = 0.0;
  T gre[KB + 1], gim[KB + 1];
  unsigned bad = 0;
};

// One event: S = sum_k c_k A_k, log |S|^2 and the lanes Re / Im of A_k conj(S) / |S|^2.
template <typename T, int KB, bool GRAD>
__device__ __forceinline__ void coh_event(const T (&cr)[KB + 1], const T (&ci)[KB + 1], const T (&ar)[KB + 1],
                                          const T (&ai)[KB + 1], CohAcc<T, KB>& acc) {
  constexpr int KA = KB + 1;
  T sr = T(0), si = T(0);
#pragma unroll
  for (int k = 0; k < KA; ++k) {
    sr += cr[k] * ar[k] - ci[k] * ai[k];
    si += cr[k] * ai[k] + ci[k] * ar[k];
  }
  const T s2 = sr * sr + si * si;
  if (s2 > T(0)) {
    if constexpr (sizeof(T) == 4) {
      acc.lf32.add(__logf(s2));
    } else {
      acc.lf64 += log(s2);
    }
    if constexpr (GRAD) {
      const T inv = T(1) / s2;
      const T tr = sr * inv, ti = -si * inv;  // conj(S) / |S|^2
#pragma unroll
      for (int k = 0; k < KA; ++k) {
        acc.gre[k] += ar[k] * tr - ai[k] * ti;
        acc.gim[k] += ar[k] * ti + ai[k] * tr;
      }
    }
  } else {
    acc.bad++;
  }
}

// Block and last-block reductions of the lanes, then the FP64 combination with the
// normalisation terms the host formed from the Gram matrix at the coefficients the kernel used
// (they depend on theta and the MC sample only: an O(K^2) quadratic form that would otherwise
// be an FP64 latency chain on the last block).
template <typename T, int KB, bool GRAD>
__device__ __forceinline__ void coh_finish(const CohArgs<T>& a, CohAcc<T, KB>& acc, int64_t begin, int64_t end,
                                           float2* partials, unsigned* counters, double* result, int out_mode,
                                           ddf* s_red, unsigned* s_bad) {
  constexpr int NS = CohLanes<T, KB, GRAD>::NS;
  constexpr int KA = KB + 1;
  ddf v[NS];
  v[0] = (sizeof(T) == 4) ? acc.lf32.value() : dd_from_double(acc.lf64);
  if constexpr (GRAD) {
#pragma unroll
    for (int k = 0; k < KA; ++k) {
      v[1 + 2 * k] = (sizeof(T) == 4) ? ddf{(float)acc.gre[k], 0.f} : dd_from_double((double)acc.gre[k]);
      v[2 + 2 * k] = (sizeof(T) == 4) ? ddf{(float)acc.gim[k], 0.f} : dd_from_double((double)acc.gim[k]);
    }
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
  // thread p gathers the gradient of parameter p (parameters may be shared) in a fixed order
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    double g = 0.0;
    if (GRAD)
      for (int k = 0; k < K; ++k) {
        const int slot = (k < a.nbw) ? k : KB;  // NR lives in the last slot
        double gre = -2.0 * s_out[1 + 2 * slot] + nev * a.nrm_vr[k];
        double gim = 2.0 * s_out[2 + 2 * slot] - nev * a.nrm_vi[k];
        coef_chain(a.polar, a.jc[k], a.js[k], a.jr[k], gre, gim);
        if (a.par_re[k] == p) g += gre;
        if (a.par_im[k] == p) g += gim;
      }
    result[off + p] = g;
  }
  if (threadIdx.x == 0) {
    counters[1] = 0u;
    counters[kStatusWord] = 0u;
    *counters = 0u;  // the ticket
    const double nll = -s_out[0] + nev * a.nrm_logN;
    // a device wait that gave up is reported as a negative event count
    const double nb = status ? -1.0 : (double)nbad;
    result[0] = nll;
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

template <typename T, int KB>
__device__ __forceinline__ void coh_coeffs(const CohArgs<T>& a, T (&cr)[KB + 1], T (&ci)[KB + 1]) {
  const int nbw = a.nbw;
#pragma unroll
  for (int k = 0; k < KB; ++k) {
    cr[k] = k < nbw ? a.cr[k] : T(0);
    ci[k] = k < nbw ? a.ci[k] : T(0);
  }
  cr[KB] = a.has_nr ? a.cr[nbw] : T(0);
  ci[KB] = a.has_nr ? a.ci[nbw] : T(0);
}

// Direct form (one event per thread per grid-stride step); the FP64 path uses it.
template <typename T, int KB, bool GRAD>
__global__ void __launch_bounds__(kBlock, 2) coh_nll_kernel(const __grid_constant__ CohArgs<T> a, const void* cache_v,
                                                            int64_t begin, int64_t end, float2* partials,
                                                            unsigned* counters, double* result, int out_mode) {
  constexpr int NS = CohLanes<T, KB, GRAD>::NS;
  constexpr int KA = KB + 1;  // BW slots + NR slot
  __shared__ ddf s_red[(kBlock / 32) * NS > kBlock ? (kBlock / 32) * NS : kBlock];
  __shared__ unsigned s_bad[kBlock / 32];
  using Vec = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  const Vec* cache = (const Vec*)cache_v;
  const int nbw = a.nbw;
  T cr[KA], ci[KA];
  coh_coeffs<T, KB>(a, cr, ci);
  CohAcc<T, KB> acc;
#pragma unroll
  for (int k = 0; k < KA; ++k) acc.gre[k] = acc.gim[k] = T(0);
  const int64_t n = a.n_total;
  for (int64_t i = begin + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < end;
       i += (int64_t)gridDim.x * blockDim.x) {
    T ar[KA], ai[KA];
    load_amps<KB>(cache, n, i, nbw, ar, ai);
    ar[KB] = T(1);
    ai[KB] = T(0);
    coh_event<T, KB, GRAD>(cr, ci, ar, ai, acc);
  }
  coh_finish<T, KB, GRAD>(a, acc, begin, end, partials, counters, result, out_mode, s_red, s_bad);
}

// FP32 form with the amplitude-cache tiles staged in shared memory.  A tile holds
// kCohTile events of every float4 plane (aligned to multiples of kCohTile); one thread
// issues a bulk copy per plane kCohStages tiles ahead, and block b takes tiles
// tb0 + b, tb0 + b + gridDim.x, ...  Ragged first / last tiles are read from global memory.
// Dynamic shared memory: kCohStages * n_planes * kCohTile float4.
constexpr int kCohTile = kStagedBlock;  // one event per thread per tile
constexpr int kCohStages = 3;

template <int KB, bool GRAD>
__global__ void __launch_bounds__(kStagedBlock, 1) coh_nll_staged_kernel(const __grid_constant__ CohArgs<float> a,
                                                                   const float4* __restrict__ cache, int64_t begin,
                                                                   int64_t end, float2* partials, unsigned* counters,
                                                                   double* result, int out_mode) {
  constexpr int NS = CohLanes<float, KB, GRAD>::NS;
  constexpr int KA = KB + 1;
  constexpr int TE = kCohTile;
  constexpr int NST = kCohStages;
  __shared__ ddf s_red[(kStagedBlock / 32) * NS > kStagedBlock ? (kStagedBlock / 32) * NS : kStagedBlock];
  __shared__ unsigned s_bad[kStagedBlock / 32];
  __shared__ __align__(8) uint64_t s_bar[NST];
  extern __shared__ __align__(128) float4 s_amp[];  // [NST][planes][TE]
  const int nbw = a.nbw;
  const int planes = (nbw + 1) / 2;
  const int64_t n = a.n_total;
  const int64_t tb0 = begin / TE, tb1 = (end + TE - 1) / TE;
  auto tile_of = [&](int j) { return tb0 + blockIdx.x + (int64_t)j * gridDim.x; };
  auto full = [&](int64_t t) { return t * TE >= begin && (t + 1) * TE <= end; };
  auto buf = [&](int st, int p) { return s_amp + ((size_t)st * planes + p) * TE; };
  const unsigned withhold = withheld_tile(counters);  // the failure-detection test hook
  auto issue = [&](int j) {
    const int64_t t = tile_of(j);
    if (t >= tb1 || (withhold && j == (int)withhold - 1)) return;
    uint64_t* bar = &s_bar[j % NST];
    if (full(t)) {
      mbar_arrive_expect_tx(bar, (unsigned)(planes * TE * sizeof(float4)));
      for (int p = 0; p < planes; ++p) bulk_load(buf(j % NST, p), cache + (int64_t)p * n + t * TE, TE * sizeof(float4), bar);
    } else {
      mbar_arrive(bar);
    }
  };
  if (threadIdx.x == 0) {
    for (int st = 0; st < NST; ++st) mbar_init(&s_bar[st], 1);
    mbar_init_fence();
    for (int j = 0; j < NST; ++j) issue(j);
  }
  float2 cre[KA], cim[KA];
  {
    float cr[KA], ci[KA];
    coh_coeffs<float, KB>(a, cr, ci);
#pragma unroll
    for (int k = 0; k < KA; ++k) {
      cre[k] = pk::splat(cr[k]);
      cim[k] = pk::splat(ci[k]);
    }
  }
  Kahan lf;
  float2 G1[KA], G2[KA];
#pragma unroll
  for (int k = 0; k < KA; ++k) G1[k] = G2[k] = pk::splat(0.f);
  unsigned bad = 0;
  __syncthreads();  // barriers initialised before any thread waits on them
  const long long wlim = tile_wait_limit(counters);
  int j = 0;
  bool failed = false;
  for (; tile_of(j) < tb1; ++j) {
    const int64_t t = tile_of(j);
    const int st = j % NST;
    const bool ok_wait = mbar_wait(&s_bar[st], (unsigned)(j / NST) & 1u, wlim);
    if (ok_wait) {
      const float4* sb = buf(st, 0);  // plane p of the tile at sb + p * TE
      const bool staged = full(t);
#pragma unroll 1
      for (int e = threadIdx.x; e < TE; e += blockDim.x) {
        const int64_t i = t * TE + e;
        if (!staged && (i < begin || i >= end)) continue;
        float2 amp[KA];
#pragma unroll
        for (int p = 0; p < (KB + 1) / 2; ++p) {
          float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
          if (p < planes) v = staged ? sb[p * TE + e] : __ldg(cache + (int64_t)p * n + i);
          amp[2 * p] = make_float2(v.x, v.y);
          if (2 * p + 1 < KB) amp[2 * p + 1] = make_float2(v.z, v.w);
        }
        amp[KB] = make_float2(1.f, 0.f);
        coh_event_pk<KA, GRAD>(cre, cim, amp, lf, G1, G2, bad);
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
      for (int jj = j; jj < j + NST && tile_of(jj) < tb1; ++jj)
        if (!(withhold && jj == (int)withhold - 1)) mbar_wait(&s_bar[jj % NST], (unsigned)(jj / NST) & 1u);
    }
    __syncthreads();
  }
  CohAcc<float, KB> acc;
  acc.lf32 = lf;
  acc.bad = bad;
#pragma unroll
  for (int k = 0; k < KA; ++k) {
    acc.gre[k] = G1[k].x - G2[k].y;
    acc.gim[k] = G1[k].y + G2[k].x;
  }
  coh_finish<float, KB, GRAD>(a, acc, begin, end, partials, counters, result, out_mode, s_red, s_bad);
}

// per-event log f = log|S|^2 - log N
template <typename T, int KB>
__global__ void coh_logf_kernel(const __grid_constant__ CohArgs<T> a, const void* cache_v, double logN,
                                double* __restrict__ out) {
  constexpr int KA = KB + 1;
  using Vec = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  const Vec* cache = (const Vec*)cache_v;
  const int nbw = a.nbw;
  const int64_t n = a.n_total;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    T ar[KA], ai[KA];
    load_amps<KB>(cache, n, i, nbw, ar, ai);
    ar[KB] = T(1);
    ai[KB] = T(0);
    T sr = T(0), si = T(0);
#pragma unroll
    for (int k = 0; k < KA; ++k) {
      const T c_r = k < nbw ? a.cr[k] : (k == KB && a.has_nr ? a.cr[nbw] : T(0));
      const T c_i = k < nbw ? a.ci[k] : (k == KB && a.has_nr ? a.ci[nbw] : T(0));
      sr += c_r * ar[k] - c_i * ai[k];
      si += c_r * ai[k] + c_i * ar[k];
    }
    const T s2 = sr * sr + si * si;
    out[i] = s2 > T(0) ? log((double)s2) - logN : -HUGE_VAL;
  }
}

// ---------------------------------------------------------------------------------------
// Gram matrix over an MC cache: block (x, k) accumulates row k, G_kl for all l, over its
// share of the MC events.  Lanes: 2 per l (re, im).  K <= kMaxAmp incl. the NR amplitude.
// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------
static double kallen(double a, double b, double c) { return a * a + b * b + c * c - 2 * a * b - 2 * a * c - 2 * b * c; }

static void pair_masses(const DalitzModel& d, int pair, double& mA, double& mB, double& mC) {
  if (pair == 0) {
    mA = d.m1;
    mB = d.m2;
    mC = d.m3;
  } else if (pair == 1) {
    mA = d.m1;
    mB = d.m3;
    mC = d.m2;
  } else {
    mA = d.m2;
    mB = d.m3;
    mC = d.m1;
  }
}

// Coefficient k of the amplitude sum from its two parameters: (Re, Im), or (r, phi) with
// GOO_COEF_POLAR.
static void coef(const DalitzModel& d, const double* theta, int k, double& re, double& im) {
  const double u = theta[d.par_re[k]], v = theta[d.par_im[k]];
  if (d.polar) {
    re = u * std::cos(v);
    im = u * std::sin(v);
  } else {
    re = u;
    im = v;
  }
}

// The polar Jacobian entries (cos phi, sin phi, r) of every amplitude into kernel arguments.
template <typename A>
static void fill_jacobian(const DalitzModel& d, const double* theta, A& a) {
  a.polar = d.polar ? 1 : 0;
  for (int k = 0; k < d.K; ++k) {
    a.jc[k] = d.polar ? std::cos(theta[d.par_im[k]]) : 1.0;
    a.js[k] = d.polar ? std::sin(theta[d.par_im[k]]) : 0.0;
    a.jr[k] = d.polar ? theta[d.par_re[k]] : 1.0;
  }
}

static uint64_t lineshape_key(const DalitzModel& d, const double* theta) {
  uint64_t h = 1469598103934665603ull;
  for (int k = 0; k < d.nbw; ++k) {
    double v[2] = {theta[d.par_m0[k]], theta[d.par_w[k]]};
    const unsigned char* p = (const unsigned char*)v;
    for (size_t j = 0; j < sizeof v; ++j) h = (h ^ p[j]) * 1099511628211ull;
  }
  return h ? h : 1;
}

// Lineshape constants for the current theta (FP64, once per lineshape version).
// ---------------------------------------------------------------------------------------
// floating lineshapes (masses and widths free; paper Sec. 4: the cache is then invalid at
// every step).  No amplitude cache: each evaluation runs a pass over the MC sample and one
// over the events, and both evaluate every Breit-Wigner amplitude from (s12, s13) with the
// parts of its denominator D = m0^2 - s - i m0 Gamma(s), which give
//   d log A / d m0     = rho - (2 m0 - i kappa m0 Gamma(s)) / D,
//   d log A / d Gamma0 = i m0 Gamma(s) / (Gamma0 D),
// where rho = d log(B_L(z) / B_L(z0)) / d m0 (through q0) and kappa = d log(m0 Gamma(s)) /
// d m0 = 2 / m0 - (2L + 1) d log q0 / d m0 + 2 rho are constants of the resonance (the
// spin and parent-barrier factors do not depend on m0 or Gamma0).  Lanes: 0 = sum log |S|^2
// (events) or sum |S|^2 (MC); then per amplitude slot Re / Im of A_k conj(S) w; then per
// resonance Re(c_k A_k conj(S) w d log A_k / d m0) and the same for Gamma0, with w = 1 / |S|^2
// for events and 1 for MC points.  The event pass's last block combines both passes:
//   NLL = -sum log |S|^2 + n log(sum_MC |S|^2 / n_MC),
//   d NLL / d p = -sum_events (d |S|^2 / d p) / |S|^2 + n (sum_MC d |S|^2 / d p) / sum_MC |S|^2.
// ---------------------------------------------------------------------------------------
template <typename T>
struct LsConst {
  T cr[kMaxAmp], ci[kMaxAmp];          // coefficients by slot: resonances, then the NR in slot KB
  T rho[kMaxAmp], kappa[kMaxAmp], two_m0[kMaxAmp], inv_g0[kMaxAmp];
  int par_m0[kMaxAmp], par_w[kMaxAmp];
};

template <int KB, bool GRAD>
struct LsLanes {
  static constexpr int NS = GRAD ? 1 + 2 * (KB + 1) + 2 * KB : 1;
};

// Dynamic shared memory of a floating-lineshape block: per thread, the five parts (re, im,
// dr, di, inv) of each resonance's amplitude and the NS - 1 gradient lanes, as columns of
// kBlock values (thread t at offset t: conflict-free), with the gradient only.
template <typename T, int KB, bool GRAD>
constexpr size_t ls_smem() {
  return GRAD ? (size_t)(5 * KB + LsLanes<KB, GRAD>::NS - 1) * kBlock * sizeof(T) : 0;
}

// The resonances are visited in a run-time loop (not unrolled) whose state lives in those
// shared-memory columns, so that the kernel needs few registers.
template <typename T, int KB, bool GRAD, bool MC>
__global__ void __launch_bounds__(kBlock)
    coh_ls_kernel(const __grid_constant__ CohArgs<T> a, const __grid_constant__ LsConst<T> c,
                  const DalitzDev* __restrict__ ddp, const T* __restrict__ c12, const T* __restrict__ c13,
                  int64_t begin, int64_t end, const double* __restrict__ mc_sums, double n_mc, float2* partials,
                  unsigned* counters, double* out, int out_mode) {
  constexpr int KA = KB + 1;
  constexpr int NS = LsLanes<KB, GRAD>::NS;
  __shared__ DalitzDev s_dd;
  __shared__ ddf s_red[(kBlock / 32) * NS > kBlock ? (kBlock / 32) * NS : kBlock];
  __shared__ unsigned s_bad[kBlock / 32];
  __shared__ double s_out[NS];
  extern __shared__ __align__(16) unsigned char s_dyn[];
  T* s_a = reinterpret_cast<T*>(s_dyn);  // [5][KB][kBlock]
  T* s_l = s_a + 5 * KB * kBlock;        // [NS - 1][kBlock]
  const int t = threadIdx.x;
  for (int i = t; i < (int)(sizeof(DalitzDev) / 4); i += blockDim.x) ((int*)&s_dd)[i] = ((const int*)ddp)[i];
  if constexpr (GRAD)
    for (int j = 0; j < NS - 1; ++j) s_l[j * kBlock + t] = T(0);
  __syncthreads();
  const int nbw = s_dd.nbw;
  const T cnr = c.cr[KB], cni = c.ci[KB];
  Kahan lf32;
  double lf64 = 0.0;
  unsigned bad = 0;
  for (int64_t i = begin + blockIdx.x * (int64_t)blockDim.x + t; i < end; i += (int64_t)gridDim.x * blockDim.x) {
    const T x12 = c12[i], x13 = c13[i];
    T x23;
    if constexpr (sizeof(T) == 4) x23 = (float)(s_dd.sumsq - (double)x12 - (double)x13);
    else x23 = s_dd.sumsq - x12 - x13;
    T sr = cnr, si = cni;  // the non-resonant amplitude is 1
#pragma unroll 1
    for (int k = 0; k < nbw; ++k) {
      T ar, ai, dr, di, iv;
      bw_amp_parts<T>(bw_of<T>(s_dd, k), x12, x13, x23, ar, ai, dr, di, iv);
      sr += c.cr[k] * ar - c.ci[k] * ai;
      si += c.cr[k] * ai + c.ci[k] * ar;
      if constexpr (GRAD) {
        T* col = s_a + k * kBlock + t;
        col[0] = ar;
        col[KB * kBlock] = ai;
        col[2 * KB * kBlock] = dr;
        col[3 * KB * kBlock] = di;
        col[4 * KB * kBlock] = iv;
      }
    }
    const T s2 = sr * sr + si * si;
    if (!MC && !(s2 > T(0))) {
      ++bad;
      continue;
    }
    if constexpr (sizeof(T) == 4) lf32.add(MC ? s2 : __logf(s2));
    else lf64 += MC ? s2 : log(s2);
    if constexpr (GRAD) {
      const T w = MC ? T(1) : T(1) / s2;
      const T tr = sr * w, ti = -si * w;  // conj(S) w
      s_l[(2 * KB) * kBlock + t] += tr;   // the non-resonant slot: A = 1
      s_l[(2 * KB + 1) * kBlock + t] += ti;
#pragma unroll 1
      for (int k = 0; k < nbw; ++k) {
        const T* col = s_a + k * kBlock + t;
        const T ar = col[0], ai = col[KB * kBlock], dr = col[2 * KB * kBlock], di = col[3 * KB * kBlock],
                iv = col[4 * KB * kBlock];
        const T ur = ar * tr - ai * ti, ui = ar * ti + ai * tr;                      // A_k conj(S) w
        const T vr = c.cr[k] * ur - c.ci[k] * ui, vi = c.cr[k] * ui + c.ci[k] * ur;  // c_k A_k conj(S) w
        const T e2 = di * iv;
        const T lmr = c.rho[k] - (c.two_m0[k] * dr + c.kappa[k] * di * di) * iv;
        const T lmi = -(c.two_m0[k] - c.kappa[k] * dr) * e2;
        const T lgr = -di * e2 * c.inv_g0[k], lgi = dr * e2 * c.inv_g0[k];
        T* lane = s_l + 2 * k * kBlock + t;
        lane[0] += ur;
        lane[kBlock] += ui;
        lane[2 * KA * kBlock] += vr * lmr - vi * lmi;
        lane[(2 * KA + 1) * kBlock] += vr * lgr - vi * lgi;
      }
    }
  }
  ddf v[NS];
  v[0] = (sizeof(T) == 4) ? lf32.value() : dd_from_double(lf64);
  if constexpr (GRAD) {
#pragma unroll
    for (int j = 0; j < NS - 1; ++j) {
      const T x = s_l[j * kBlock + t];
      v[1 + j] = (sizeof(T) == 4) ? ddf{(float)x, 0.f} : dd_from_double((double)x);
    }
  }
  for (int m = 16; m > 0; m >>= 1) bad += __shfl_xor_sync(0xffffffffu, bad, m);
  if ((threadIdx.x & 31) == 0) s_bad[threadIdx.x >> 5] = bad;
  block_reduce_to_partials<NS>(v, NS, partials, s_red);
  if (threadIdx.x == 0) {
    unsigned b = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += s_bad[w];
    if (b) atomicAdd(counters + 1, b);
  }
  if (!last_block_ticket(counters, gridDim.x)) return;
  reduce_partials(partials, NS, gridDim.x, s_out, s_red, blockDim.x);
  if constexpr (MC) {
    // the MC pass ends with its lane sums (read by the event pass that follows it)
    for (int t = threadIdx.x; t < NS; t += blockDim.x) out[t] = s_out[t];
    if (threadIdx.x == 0) *counters = 0u;  // the ticket
    return;
  }
  const double nev = (double)(end - begin);
  const double Smc = mc_sums[0];
  const int P = a.n_params;
  const int off = out_mode == 0 ? 2 : 3;
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    double g = 0.0;
    if (GRAD) {
      for (int kk = 0; kk < a.K; ++kk) {
        const int sl = kk < a.nbw ? kk : KB;  // the NR lives in the last slot
        double gre = -2.0 * s_out[1 + 2 * sl] + 2.0 * nev * mc_sums[1 + 2 * sl] / Smc;
        double gim = 2.0 * s_out[2 + 2 * sl] - 2.0 * nev * mc_sums[2 + 2 * sl] / Smc;
        coef_chain(a.polar, a.jc[kk], a.js[kk], a.jr[kk], gre, gim);
        if (a.par_re[kk] == p) g += gre;
        if (a.par_im[kk] == p) g += gim;
      }
      for (int k = 0; k < a.nbw; ++k) {
        const int o = 1 + 2 * KA + 2 * k;
        if (c.par_m0[k] == p) g += -2.0 * s_out[o] + 2.0 * nev * mc_sums[o] / Smc;
        if (c.par_w[k] == p) g += -2.0 * s_out[o + 1] + 2.0 * nev * mc_sums[o + 1] / Smc;
      }
    }
    out[off + p] = g;
  }
  if (threadIdx.x == 0) {
    // every other block added to these words before its ticket (and a fence): plain L2 reads
    const unsigned nbad = __ldcg(counters + 1);
    const unsigned status = __ldcg(counters + kStatusWord);
    counters[1] = 0u;
    counters[kStatusWord] = 0u;
    *counters = 0u;  // the ticket
    const double N = Smc / n_mc;
    const double nb = status ? -1.0 : (double)nbad;  // a device wait that gave up: negative count
    out[0] = -s_out[0] + nev * log(N);
    if (out_mode == 0) {
      out[1] = nb;
      out[2 + P] = N;
    } else {
      out[1] = 0.0;
      out[2] = nb;
    }
  }
  result_complete(out);
}

// ---------------------------------------------------------------------------------------
// time-dependent three-body model (GOO_OP_TD3; paper Sec. 5, Table 2).  The anti-particle's
// amplitudes are the same lineshapes at the exchanged point, abar_k(s12, s13) =
// a_k(s13, s12) (a second cache built from the exchanged columns); A = sum c_k a_k,
// B = sum c_k abar_k with the same coefficients.  Per event the four decay-time terms of the
// four-body model (timeterms.cuh) give
//   R = (|A|^2+|B|^2)/2 T_ch + (|A|^2-|B|^2)/2 T_c + Re(AB*) T_sh + Im(AB*) T_s,
// and the gradient lanes Re / -Im of (a_k V_A + abar_k V_B) / R with
//   V_A = (T_ch + T_c) A* + (T_sh - i T_s) B*,  V_B = (T_ch - T_c) B* + (T_sh + i T_s) A*,
// plus d R / d(x, y, tau, sigma_t) / R.  N comes from three MC Gram matrices,
//   <|A|^2> = c^T G_aa c*, <|B|^2> = c^T G_bb c*, <AB*> = c^T G_ab c*,
// and the closed-form time integrals.
// ---------------------------------------------------------------------------------------

// G_kl = mean over the events of X_k conj(Y_l) (k, l < K; the amplitude nbw is the constant
// NR amplitude 1 when present), one block per (k, l), FP64 sums in a fixed order.
template <typename T>
__global__ void __launch_bounds__(kBlock) gram_cross_kernel(const void* xv, const void* yv, int64_t n, int nbw, int K,
                                                            double* out) {
  const int k = blockIdx.x / K, l = blockIdx.x % K;
  auto amp = [&](const void* c, int j, int64_t i, double& re, double& im) {
    if (j >= nbw) {
      re = 1.0;
      im = 0.0;
    } else if constexpr (sizeof(T) == 4) {
      const float4 v = ((const float4*)c)[(int64_t)(j / 2) * n + i];
      re = (double)((j & 1) ? v.z : v.x);
      im = (double)((j & 1) ? v.w : v.y);
    } else {
      const double2 v = ((const double2*)c)[(int64_t)j * n + i];
      re = v.x;
      im = v.y;
    }
  };
  double sr = 0.0, si = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    double xr, xi, yr, yi;
    amp(xv, k, i, xr, xi);
    amp(yv, l, i, yr, yi);
    sr += xr * yr + xi * yi;  // X conj(Y)
    si += xi * yr - xr * yi;
  }
  __shared__ double s_r[kBlock / 32], s_i[kBlock / 32];
  for (int m = 16; m > 0; m >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, m);
    si += __shfl_xor_sync(0xffffffffu, si, m);
  }
  if ((threadIdx.x & 31) == 0) {
    s_r[threadIdx.x >> 5] = sr;
    s_i[threadIdx.x >> 5] = si;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0.0, ti = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      tr += s_r[w];
      ti += s_i[w];
    }
    out[2 * (k * K + l)] = tr / (double)n;
    out[2 * (k * K + l) + 1] = ti / (double)n;
  }
}

constexpr int kTd3KB = 15;  // resonance slots of the time-dependent three-body kernels (NR in slot 15)

template <typename T>
struct Td3Args {
  T cr[kTd3KB + 1], ci[kTd3KB + 1];  // coefficients by slot: resonances, then the NR in slot kTd3KB
  T G, x, y, s;                      // 1/tau, mixing, resolution in the path's precision
  TimeCoef<T> tc;                    // the same with the moment-series coefficients
  T wa[kWMax];                       // Weideman coefficients
  T wL;
  int wN, nbw, K, n_params;
  int par_re[kMaxAmp], par_im[kMaxAmp], par_t[4];  // parameter of each amplitude (tree order)
  int64_t n_total;                   // events of the dataset (cache plane length)
  int polar;                         // the coefficient parameters are (r, phi)
  double jc[kMaxAmp], js[kMaxAmp], jr[kMaxAmp];  // cos phi, sin phi, r per amplitude (polar)
  // the normalisation at theta, formed on the host in FP64 from the cached Gram matrices
  // (td3_norm_terms): N, log N, (dN / d Re c_k) / N, (dN / d Im c_k) / N (tree order) and
  // (dN / dx) / N, (dN / dy) / N, (tau dN / d tau) / N
  double nrm_N, nrm_logN, nrm_re[kMaxAmp], nrm_im[kMaxAmp], nrm_dt[3];
};

template <bool GRAD>
struct Td3Lanes {
  static constexpr int NS = GRAD ? 1 + 2 * (kTd3KB + 1) + 4 : 1;
};

template <typename T, bool GRAD>
__global__ void __launch_bounds__(kBlock, 2)
    td3_nll_kernel(const __grid_constant__ Td3Args<T> a, const void* __restrict__ cache_a,
                   const void* __restrict__ cache_b, const T* __restrict__ tcol, int64_t begin, int64_t end,
                   float2* partials, unsigned* counters, double* out, int out_mode) {
  constexpr int KB = kTd3KB, KA = KB + 1;
  constexpr int NS = Td3Lanes<GRAD>::NS;
  __shared__ ddf s_red[(kBlock / 32) * NS > kBlock ? (kBlock / 32) * NS : kBlock];
  __shared__ unsigned s_bad[kBlock / 32];
  __shared__ double s_out[NS];
  const int64_t n = a.n_total;
  const int nbw = a.nbw;
  // the amplitude pair of slot k (< nbw) at event i: a_k and abar_k
  auto load = [&](int k, int64_t i, T& ar, T& ai, T& br, T& bi) {
    if constexpr (sizeof(T) == 4) {
      const float4 va = __ldg((const float4*)cache_a + (int64_t)(k / 2) * n + i);
      const float4 vb = __ldg((const float4*)cache_b + (int64_t)(k / 2) * n + i);
      ar = (k & 1) ? va.z : va.x;
      ai = (k & 1) ? va.w : va.y;
      br = (k & 1) ? vb.z : vb.x;
      bi = (k & 1) ? vb.w : vb.y;
    } else {
      const double2 va = __ldg((const double2*)cache_a + (int64_t)k * n + i);
      const double2 vb = __ldg((const double2*)cache_b + (int64_t)k * n + i);
      ar = va.x;
      ai = va.y;
      br = vb.x;
      bi = vb.y;
    }
  };
  // FP32: all amplitude planes of the event are requested before any is used (loads
  // predicated on the plane count rather than a loop exit, so none waits on the arithmetic of
  // the one before), and kept for the gradient lanes
  constexpr int NP = sizeof(T) == 4 ? (KB + 1) / 2 : 1;
  float4 pa[NP], pb[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) pa[q] = pb[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  auto get = [&](int k, int64_t i, T& ar, T& ai, T& br, T& bi) {
    if constexpr (sizeof(T) == 4) {
      const float4 va = pa[k / 2], vb = pb[k / 2];
      ar = (k & 1) ? va.z : va.x;
      ai = (k & 1) ? va.w : va.y;
      br = (k & 1) ? vb.z : vb.x;
      bi = (k & 1) ? vb.w : vb.y;
    } else {
      load(k, i, ar, ai, br, bi);
    }
  };
  Kahan lf32;
  double lf64 = 0.0;
  T lre[KA], lim[KA], lt[4];
#pragma unroll
  for (int k = 0; k < KA; ++k) lre[k] = lim[k] = T(0);
#pragma unroll
  for (int j = 0; j < 4; ++j) lt[j] = T(0);
  unsigned bad = 0;
  for (int64_t i = begin + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < end;
       i += (int64_t)gridDim.x * blockDim.x) {
    const T t = tcol[i];
    if constexpr (sizeof(T) == 4) {
#pragma unroll
      for (int q = 0; q < NP; ++q)
        if (2 * q < nbw) {
          pa[q] = __ldg((const float4*)cache_a + (int64_t)q * n + i);
          pb[q] = __ldg((const float4*)cache_b + (int64_t)q * n + i);
        }
    }
    T Ar = a.cr[KB], Ai = a.ci[KB], Br = a.cr[KB], Bi = a.ci[KB];  // the NR amplitude is 1 for both
    if constexpr (sizeof(T) == 4) {
      // FP32: the sums as packed (re, im) FMAs on the planes' halves, (sum cr_k a_k) and
      // (sum ci_k a_k) per cache, combined once: four packed FMAs per amplitude, not eight
      using namespace pk;
      float2 P1 = make_float2(Ar, Ai), P2 = splat(0.f), Q1 = make_float2(Br, Bi), Q2 = splat(0.f);
#pragma unroll
      for (int k = 0; k < KB; ++k) {
        if (k >= nbw) break;
        const float4 va = pa[k / 2], vb = pb[k / 2];
        const float2 ak = (k & 1) ? make_float2(va.z, va.w) : make_float2(va.x, va.y);
        const float2 bk = (k & 1) ? make_float2(vb.z, vb.w) : make_float2(vb.x, vb.y);
        P1 = fma(splat(a.cr[k]), ak, P1);
        P2 = fma(splat(a.ci[k]), ak, P2);
        Q1 = fma(splat(a.cr[k]), bk, Q1);
        Q2 = fma(splat(a.ci[k]), bk, Q2);
      }
      Ar = P1.x - P2.y;
      Ai = P1.y + P2.x;
      Br = Q1.x - Q2.y;
      Bi = Q1.y + Q2.x;
    } else {
#pragma unroll
      for (int k = 0; k < KB; ++k) {
        if (k >= nbw) break;
        T ar, ai, br, bi;
        get(k, i, ar, ai, br, bi);
        Ar += a.cr[k] * ar - a.ci[k] * ai;
        Ai += a.cr[k] * ai + a.ci[k] * ar;
        Br += a.cr[k] * br - a.ci[k] * bi;
        Bi += a.cr[k] * bi + a.ci[k] * br;
      }
    }
    TimeTerms<T> tt;
    time_terms_g<T>(a.tc, a.wa, a.wN, a.wL, t, tt);
    const T AA = Ar * Ar + Ai * Ai, BB = Br * Br + Bi * Bi;
    const T ABr = Ar * Br + Ai * Bi, ABi = Ai * Br - Ar * Bi;  // A conj(B)
    // R = |A|^2 P + |B|^2 Q + Re(A B*) T_sh + Im(A B*) T_s with P, Q = (T_ch +- T_c)/2
    const T R = AA * tt.P + BB * tt.Q + ABr * tt.Tsh + ABi * tt.Ts;
    if (!(R > T(0))) {
      ++bad;
      continue;
    }
    if constexpr (sizeof(T) == 4) lf32.add(pk::lg2(R));  // log2 R, scaled by ln 2 at the end
    else lf64 += log(R);
    if constexpr (GRAD) {
      T invR;
      if constexpr (sizeof(T) == 4) invR = pk::rcp(R);
      else invR = T(1) / R;
      const T cp = T(2) * tt.P * invR, cm = T(2) * tt.Q * invR, sh = tt.Tsh * invR, ss = tt.Ts * invR;
      // V_A / R = cp A* + (sh - i ss) B*,  V_B / R = cm B* + (sh + i ss) A*
      const T VAr = cp * Ar + sh * Br - ss * Bi, VAi = -cp * Ai - sh * Bi - ss * Br;
      const T VBr = cm * Br + sh * Ar + ss * Ai, VBi = -cm * Bi - sh * Ai + ss * Ar;
#pragma unroll
      for (int k = 0; k < KB; ++k) {
        if (k >= nbw) break;
        T ar, ai, br, bi;
        get(k, i, ar, ai, br, bi);
        const T qr = ar * VAr - ai * VAi + br * VBr - bi * VBi;  // Re(a V_A + abar V_B) / R
        const T qi = ar * VAi + ai * VAr + br * VBi + bi * VBr;
        lre[k] += qr;
        lim[k] -= qi;
      }
      lre[KB] += VAr + VBr;  // the NR slot (a = abar = 1)
      lim[KB] -= VAi + VBi;
#pragma unroll
      for (int j = 0; j < 4; ++j)
        lt[j] += (AA * tt.d[j][0] + BB * tt.d[j][1] + ABr * tt.d[j][2] + ABi * tt.d[j][3]) * invR;
    }
  }
  ddf v[NS];
  v[0] = (sizeof(T) == 4) ? dd_mul(lf32.value(), ddf{kLn2Hi, kLn2Lo}) : dd_from_double(lf64);
  if constexpr (GRAD) {
#pragma unroll
    for (int k = 0; k < KA; ++k) {
      v[1 + 2 * k] = (sizeof(T) == 4) ? ddf{(float)lre[k], 0.f} : dd_from_double((double)lre[k]);
      v[2 + 2 * k] = (sizeof(T) == 4) ? ddf{(float)lim[k], 0.f} : dd_from_double((double)lim[k]);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
      v[1 + 2 * KA + j] = (sizeof(T) == 4) ? ddf{(float)lt[j], 0.f} : dd_from_double((double)lt[j]);
  }
  for (int m = 16; m > 0; m >>= 1) bad += __shfl_xor_sync(0xffffffffu, bad, m);
  if ((threadIdx.x & 31) == 0) s_bad[threadIdx.x >> 5] = bad;
  block_reduce_to_partials<NS>(v, NS, partials, s_red);
  if (threadIdx.x == 0) {
    unsigned b = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += s_bad[w];
    if (b) atomicAdd(counters + 1, b);
  }
  if (!last_block_ticket(counters, gridDim.x)) return;
  // The last block reduces the lanes and combines them with the normalisation terms the host
  // formed from the three Gram matrices (they depend on theta and the MC sample only).
  // Every other block added to the counter words before its ticket (and a fence): plain L2
  // reads, issued before the reduction so that their latency overlaps it.
  unsigned nbad = 0u, status = 0u;
  if (threadIdx.x == 0) {
    nbad = __ldcg(counters + 1);
    status = __ldcg(counters + kStatusWord);
  }
  reduce_partials(partials, NS, gridDim.x, s_out, s_red, blockDim.x);
  const int K = a.K;
  const double nev = (double)(end - begin);
  const int P = a.n_params;
  const int off = out_mode == 0 ? 2 : 3;
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    double g = 0.0;
    if (GRAD) {
      for (int kk = 0; kk < K; ++kk) {
        const int sl = kk < nbw ? kk : KB;
        double gre = -s_out[1 + 2 * sl] + nev * a.nrm_re[kk], gim = -s_out[2 + 2 * sl] + nev * a.nrm_im[kk];
        coef_chain(a.polar, a.jc[kk], a.js[kk], a.jr[kk], gre, gim);
        if (a.par_re[kk] == p) g += gre;
        if (a.par_im[kk] == p) g += gim;
      }
      const int o = 1 + 2 * KA;
      for (int j = 0; j < 4; ++j)
        if (a.par_t[j] == p) g += -s_out[o + j] + (j < 3 ? nev * a.nrm_dt[j] : 0.0);
    }
    out[off + p] = g;
  }
  if (threadIdx.x == 0) {
    counters[1] = 0u;
    counters[kStatusWord] = 0u;
    *counters = 0u;  // the ticket
    const double nb = status ? -1.0 : (double)nbad;  // a device wait that gave up: negative count
    out[0] = -s_out[0] + nev * a.nrm_logN;
    if (out_mode == 0) {
      out[1] = nb;
      out[2 + P] = a.nrm_N;
    } else {
      out[1] = 0.0;
      out[2] = nb;
    }
  }
  result_complete(out, P > 1 ? P : 1);
}

static int dalitz_constants(goo_model* m, const double* theta) {
  DalitzModel& d = *m->dalitz;
  const uint64_t key = lineshape_key(d, theta);
  if (key == d.ls_key) return GOO_OK;
  DalitzDev& h = d.host;
  h.nbw = d.nbw;
  const double M = d.M;
  h.sumsq = M * M + d.m1 * d.m1 + d.m2 * d.m2 + d.m3 * d.m3;
  for (int k = 0; k < d.nbw; ++k) {
    BwConst& b = h.bw[k];
    const int L = d.spin[k];
    double mA, mB, mC;
    pair_masses(d, d.pair[k], mA, mB, mC);
    const double m0 = theta[d.par_m0[k]], g0 = theta[d.par_w[k]];
    if (!(m0 > mA + mB) || !(g0 > 0))
      return set_error(GOO_ERR_ARG, "amplitude %d: mass %g must exceed its threshold %g and width %g be > 0", k, m0,
                       mA + mB, g0);
    b.spin = L;
    b.pair = d.pair[k];
    b.m0sq = m0 * m0;
    b.m0w = m0 * g0;
    const double q0sq = kallen(m0 * m0, mA * mA, mB * mB) / (4 * m0 * m0);
    b.inv_q0sq = 1.0 / q0sq;
    b.r2 = d.r_res * d.r_res;
    b.rp2 = d.r_par * d.r_par;
    b.thrP = (mA + mB) * (mA + mB);
    b.thrM = (mA - mB) * (mA - mB);
    b.pthrP = (M + mC) * (M + mC);
    b.pthrM = (M - mC) * (M - mC);
    b.zconst = (mA * mA - mB * mB) * (M * M - mC * mC);
    b.inv4M2 = 1.0 / (4 * M * M);
    const double z0 = b.r2 * q0sq;
    b.Fz0 = (L == 1) ? 1.0 + z0 : (L == 2 ? 9.0 + 3.0 * z0 + z0 * z0 : 1.0);
    b.m0 = m0;
    BwConstT<float>& f = h.bwf[k];
    f.spin = b.spin;
    f.pair = b.pair;
    f.m0sq = (float)b.m0sq;
    f.m0w = (float)b.m0w;
    f.inv_q0sq = (float)b.inv_q0sq;
    f.r2 = (float)b.r2;
    f.rp2 = (float)b.rp2;
    f.thrP = (float)b.thrP;
    f.thrM = (float)b.thrM;
    f.pthrP = (float)b.pthrP;
    f.pthrM = (float)b.pthrM;
    f.zconst = (float)b.zconst;
    f.inv4M2 = (float)b.inv4M2;
    f.Fz0 = (float)b.Fz0;
    f.m0 = (float)b.m0;
  }
  goo_ctx* ctx = m->ctx;
  GOO_CUDA_TRY(cudaMemcpyAsync(d.dev, &h, sizeof(DalitzDev), cudaMemcpyHostToDevice, ctx->stream));
  GOO_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  d.ls_key = key;
  d.gram_key[0] = d.gram_key[1] = 0;
  d.gram3_key[0] = d.gram3_key[1] = 0;
  return GOO_OK;
}

// Builds (if stale) the amplitude cache of `ds` in `precision`; returns its device pointer.
// With `exchanged`, the amplitudes at the exchanged Dalitz point (s13, s12): the anti-particle
// amplitudes of the time-dependent three-body model.
static int ensure_cache(goo_model* m, const goo_dataset* ds_c, int precision, const void** out,
                        bool exchanged = false) {
  goo_dataset* ds = const_cast<goo_dataset*>(ds_c);
  DalitzModel& d = *m->dalitz;
  goo_ctx* ctx = m->ctx;
  const int pi = precision == GOO_F32 ? 0 : 1;
  const uint64_t key = d.ls_key ^ (uint64_t)(uintptr_t)m ^ (uint64_t)(pi + 1 + (exchanged ? 4 : 0)) * 0x9e3779b97f4a7c15ull ^
                       ds->epoch * 0xd6e8feb86659fd93ull;
  CacheSlot& slot = ds->cache[pi + (exchanged ? 2 : 0)];
  const int ca = exchanged ? d.col13 : d.col12, cb = exchanged ? d.col12 : d.col13;
  const int64_t n = ds->n;
  const size_t bytes = pi == 0 ? (size_t)((d.nbw + 1) / 2) * (size_t)n * sizeof(float4)
                               : (size_t)d.nbw * (size_t)n * sizeof(double2);
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
  if (n > 0 && d.nbw > 0) {
    const int nb = grid_blocks(ctx, n, 4);
    if (pi == 0) {
      LaunchScope ls(ctx, "amp_cache_f32");
      amp_cache_f32_kernel<<<nb, kBlock, 0, ctx->stream>>>(d.dev, ds->d32[ca], ds->d32[cb], n, (float4*)slot.ptr);
    } else {
      LaunchScope ls(ctx, "amp_cache_f64");
      amp_cache_f64_kernel<<<nb, kBlock, 0, ctx->stream>>>(d.dev, ds->d64[ca], ds->d64[cb], n, (double2*)slot.ptr);
    }
    GOO_CUDA_TRY(cudaGetLastError());
  }
  slot.key = key;
  *out = slot.ptr;
  return GOO_OK;
}

template <typename T, int KB>
static int launch_gram(goo_model* m, const void* cache, int64_t n, int pi) {
  DalitzModel& d = *m->dalitz;
  goo_ctx* ctx = m->ctx;
  constexpr int NS = 2 * (KB + 1);
  int bps = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, gram_kernel<T, KB>, kBlock, 0) != cudaSuccess || bps < 1) {
    cudaGetLastError();
    bps = 1;
  }
  const int K = d.K;
  int64_t nbx = (n + kBlock - 1) / kBlock;
  const int64_t cap = ((int64_t)ctx->num_sms * bps + K - 1) / K;
  if (nbx > cap) nbx = cap;
  if (nbx < 1) nbx = 1;
  GOO_TRY(ensure_partials(ctx, (size_t)nbx * K * NS));
  {
    LaunchScope ls(ctx, sizeof(T) == 4 ? "gram_f32" : "gram_f64");
    gram_kernel<T, KB><<<dim3((unsigned)nbx, K), kBlock, 0, ctx->stream>>>(
        cache, n, d.nbw, d.has_nr ? 1 : 0, ctx->scratch.partials, ctx->scratch.counters, d.gram_dev[pi]);
  }
  GOO_CUDA_TRY(cudaGetLastError());
  return GOO_OK;
}

static int ensure_gram(goo_model* m, int precision) {
  DalitzModel& d = *m->dalitz;
  const int pi = precision == GOO_F32 ? 0 : 1;
  if (!d.mc) return set_error(GOO_ERR_STATE, "amplitude model has no MC normalisation sample (goo_model_set_norm)");
  const uint64_t key = d.ls_key ^ (uint64_t)(uintptr_t)d.mc ^ (uint64_t)(pi + 7) ^ d.mc->epoch * 0xd6e8feb86659fd93ull;
  if (d.gram_key[pi] == key) return GOO_OK;
  const void* cache = nullptr;
  GOO_TRY(ensure_cache(m, d.mc, precision, &cache));
  if (d.mc->n < 1) return set_error(GOO_ERR_ARG, "the MC normalisation sample is empty");
  if (pi == 0) {
    GOO_TRY((d.nbw <= 8 ? launch_gram<float, 8>(m, cache, d.mc->n, pi) : launch_gram<float, 15>(m, cache, d.mc->n, pi)));
  } else {
    GOO_TRY((d.nbw <= 8 ? launch_gram<double, 8>(m, cache, d.mc->n, pi) : launch_gram<double, 15>(m, cache, d.mc->n, pi)));
  }
  GOO_CUDA_TRY(cudaMemcpyAsync(d.gram_host[pi], d.gram_dev[pi], sizeof(double) * 2 * d.K * d.K, cudaMemcpyDeviceToHost,
                               m->ctx->stream));
  GOO_CUDA_TRY(cudaStreamSynchronize(m->ctx->stream));
  d.gram_key[pi] = key;
  return GOO_OK;
}

template <typename T>
static void fill_args(const DalitzModel& d, const double* theta, int n_params, int64_t n_total, CohArgs<T>& a) {
  std::memset(&a, 0, sizeof a);
  a.nbw = d.nbw;
  a.K = d.K;
  a.has_nr = d.has_nr ? 1 : 0;
  a.n_params = n_params;
  a.n_total = n_total;
  for (int k = 0; k < d.K; ++k) {
    double re, im;
    coef(d, theta, k, re, im);
    a.cr[k] = (T)re;
    a.ci[k] = (T)im;
    a.par_re[k] = d.par_re[k];
    a.par_im[k] = d.par_im[k];
  }
  fill_jacobian(d, theta, a);
}

// The normalisation at theta from the host copy of the Gram matrix (ensure_gram keeps it
// current), in FP64 at the precision-rounded coefficients the kernel uses:
//   v_k = sum_l G_kl conj(c_l),  N = sum_k Re(c_k v_k),  dN / d Re c_k = 2 Re v_k,
//   dN / d Im c_k = -2 Im v_k.
template <typename T>
static void coh_norm_terms(const DalitzModel& d, const double* G, CohArgs<T>& a) {
  const int K = d.K;
  double vr[kMaxAmp], vi[kMaxAmp], N = 0.0;
  for (int k = 0; k < K; ++k) {
    vr[k] = vi[k] = 0.0;
    for (int l = 0; l < K; ++l) {
      const double gr = G[2 * (k * K + l)], gi = G[2 * (k * K + l) + 1];
      const double clr = (double)a.cr[l], cli = (double)a.ci[l];
      vr[k] += gr * clr + gi * cli;
      vi[k] += gi * clr - gr * cli;
    }
    N += (double)a.cr[k] * vr[k] - (double)a.ci[k] * vi[k];
  }
  const double invN = 1.0 / N;
  for (int k = 0; k < K; ++k) {
    a.nrm_vr[k] = 2.0 * vr[k] * invN;
    a.nrm_vi[k] = 2.0 * vi[k] * invN;
  }
  a.nrm_N = N;
  a.nrm_logN = std::log(N);
}

constexpr int kMaxDevicesCoh = 64;

template <int KB, bool GRAD>
static int launch_coh_staged(goo_model* m, const void* cache, const goo_dataset* ds, int64_t begin, int64_t end,
                             const double* theta, int out_mode, int pi) {
  DalitzModel& d = *m->dalitz;
  goo_ctx* ctx = m->ctx;
  const int planes = (d.nbw + 1) / 2;
  const size_t smem = (size_t)kCohStages * planes * kCohTile * sizeof(float4);
  static bool configured[kMaxDevicesCoh] = {};
  if (ctx->device < 0 || ctx->device >= kMaxDevicesCoh) return set_error(GOO_ERR_ARG, "device %d", ctx->device);
  if (!configured[ctx->device]) {
    GOO_CUDA_TRY(cudaFuncSetAttribute(coh_nll_staged_kernel<KB, GRAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)((size_t)kCohStages * ((KB + 1) / 2) * kCohTile * sizeof(float4))));
    configured[ctx->device] = true;
  }
  const int occ = cached_occupancy((const void*)coh_nll_staged_kernel<KB, GRAD>, ctx->device, kStagedBlock, smem);
  const int64_t tiles = (end + kCohTile - 1) / kCohTile - begin / kCohTile;
  const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)ctx->num_sms * occ));
  constexpr int NS = CohLanes<float, KB, GRAD>::NS;
  GOO_TRY(ensure_partials(ctx, (size_t)nb * NS));
  CohArgs<float> a;
  fill_args<float>(d, theta, m->n_params, ds->n, a);
  coh_norm_terms<float>(d, d.gram_host[pi], a);
  {
    LaunchScope ls(ctx, GRAD ? "coh_nll_grad_f32" : "coh_nll_f32");
    coh_nll_staged_kernel<KB, GRAD><<<nb, kStagedBlock, smem, ctx->stream>>>(a, (const float4*)cache, begin, end,
                                                                       ctx->scratch.partials, ctx->scratch.counters,
                                                                       ctx->scratch.result_out, out_mode);
  }
  GOO_CUDA_TRY(cudaGetLastError());
  return GOO_OK;
}

template <typename T, int KB, bool GRAD>
static int launch_coh(goo_model* m, const void* cache, const goo_dataset* ds, int64_t begin, int64_t end,
                      const double* theta, int out_mode, int pi) {
  if constexpr (sizeof(T) == 4) return launch_coh_staged<KB, GRAD>(m, cache, ds, begin, end, theta, out_mode, pi);
  DalitzModel& d = *m->dalitz;
  goo_ctx* ctx = m->ctx;
  static int occ = 0;
  if (occ == 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, coh_nll_kernel<T, KB, GRAD>, kBlock, 0) != cudaSuccess ||
        occ < 1) {
      cudaGetLastError();
      occ = 1;
    }
  }
  const int nb = grid_blocks(ctx, end - begin, occ);
  constexpr int NS = CohLanes<T, KB, GRAD>::NS;
  GOO_TRY(ensure_partials(ctx, (size_t)nb * NS));
  CohArgs<T> a;
  fill_args<T>(d, theta, m->n_params, ds->n, a);
  coh_norm_terms<T>(d, d.gram_host[pi], a);
  {
    LaunchScope ls(ctx, sizeof(T) == 4 ? (GRAD ? "coh_nll_grad_f32" : "coh_nll_f32")
                                       : (GRAD ? "coh_nll_grad_f64" : "coh_nll_f64"));
    coh_nll_kernel<T, KB, GRAD><<<nb, kBlock, 0, ctx->stream>>>(a, cache, begin, end, ctx->scratch.partials,
                                                                ctx->scratch.counters, ctx->scratch.result_out,
                                                                out_mode);
  }
  GOO_CUDA_TRY(cudaGetLastError());
  return GOO_OK;
}

template <typename T, bool GRAD>
static int launch_coh_sel(goo_model* m, const void* cache, const goo_dataset* ds, int64_t begin, int64_t end,
                          const double* theta, int out_mode, int pi) {
  if (m->dalitz->nbw <= 8) return launch_coh<T, 8, GRAD>(m, cache, ds, begin, end, theta, out_mode, pi);
  return launch_coh<T, 15, GRAD>(m, cache, ds, begin, end, theta, out_mode, pi);
}

// Constants of the floating-lineshape kernels at theta (FP64 on the host, rounded to T):
// the coefficients by slot and, per resonance (mass m0, width Gamma0, spin L, daughters A, B),
//   d(q0^2) / d m0 = (m0^4 - (mA + mB)^2 (mA - mB)^2) / (2 m0^3),
//   rho   = F'(z0) / (2 F(z0)) r^2 d(q0^2) / d m0   (F(z) = 1 + z for L = 1, 9 + 3z + z^2 for
//           L = 2: the squared barrier ratio is F(z0) / F(z); rho = 0 for L = 0),
//   kappa = 2 / m0 - (2L + 1) d(q0^2) / d m0 / (2 q0^2) + 2 rho.
template <typename T>
static void fill_ls(const DalitzModel& d, const double* theta, LsConst<T>& c) {
  std::memset(&c, 0, sizeof c);
  for (int k = 0; k < d.nbw; ++k) {
    double re, im;
    coef(d, theta, k, re, im);
    c.cr[k] = (T)re;
    c.ci[k] = (T)im;
    c.par_m0[k] = d.par_m0[k];
    c.par_w[k] = d.par_w[k];
    double mA, mB, mC;
    pair_masses(d, d.pair[k], mA, mB, mC);
    const int L = d.spin[k];
    const double m0 = theta[d.par_m0[k]], g0 = theta[d.par_w[k]];
    const double u = m0 * m0, thrP = (mA + mB) * (mA + mB), thrM = (mA - mB) * (mA - mB);
    const double q0sq = kallen(u, mA * mA, mB * mB) / (4 * u);
    const double dq0sq = (u * u - thrP * thrM) / (2 * m0 * m0 * m0);
    const double r2 = d.r_res * d.r_res, z0 = r2 * q0sq;
    double rho = 0.0;
    if (L == 1) rho = 0.5 / (1.0 + z0) * r2 * dq0sq;
    if (L == 2) rho = 0.5 * (3.0 + 2.0 * z0) / (9.0 + 3.0 * z0 + z0 * z0) * r2 * dq0sq;
    const double kappa = 2.0 / m0 - (2 * L + 1) * dq0sq / (2.0 * q0sq) + 2.0 * rho;
    c.rho[k] = (T)rho;
    c.kappa[k] = (T)kappa;
    c.two_m0[k] = (T)(2.0 * m0);
    c.inv_g0[k] = (T)(1.0 / g0);
  }
  for (int k = d.nbw; k < kMaxAmp; ++k) c.par_m0[k] = c.par_w[k] = -1;
}

template <typename T, int KB, bool GRAD, bool MC>
static int launch_ls(goo_model* m, const goo_dataset* ds, int64_t begin, int64_t end, const double* theta,
                     double* out, int out_mode) {
  DalitzModel& d = *m->dalitz;
  goo_ctx* ctx = m->ctx;
  constexpr size_t smem = ls_smem<T, KB, GRAD>();
  static int occ[2] = {0, 0};
  int& o = occ[MC ? 1 : 0];
  if (o == 0) {
    if (smem > 48 * 1024)
      GOO_CUDA_TRY(cudaFuncSetAttribute(coh_ls_kernel<T, KB, GRAD, MC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, coh_ls_kernel<T, KB, GRAD, MC>, kBlock, smem) != cudaSuccess ||
        o < 1) {
      cudaGetLastError();
      o = 1;
    }
  }
  const int nb = grid_blocks(ctx, end - begin, o);
  constexpr int NS = LsLanes<KB, GRAD>::NS;
  GOO_TRY(ensure_partials(ctx, (size_t)nb * NS));
  CohArgs<T> a;
  fill_args<T>(d, theta, m->n_params, ds->n, a);
  LsConst<T> c;
  fill_ls<T>(d, theta, c);
  if (d.has_nr) {
    double re, im;
    coef(d, theta, d.nbw, re, im);
    c.cr[KB] = (T)re;
    c.ci[KB] = (T)im;
  }
  const T* c12 = sizeof(T) == 4 ? (const T*)ds->d32[d.col12] : (const T*)ds->d64[d.col12];
  const T* c13 = sizeof(T) == 4 ? (const T*)ds->d32[d.col13] : (const T*)ds->d64[d.col13];
  {
    LaunchScope ls(ctx, MC ? (sizeof(T) == 4 ? "coh_ls_mc_f32" : "coh_ls_mc_f64")
                           : (sizeof(T) == 4 ? (GRAD ? "coh_ls_grad_f32" : "coh_ls_f32")
                                             : (GRAD ? "coh_ls_grad_f64" : "coh_ls_f64")));
    coh_ls_kernel<T, KB, GRAD, MC><<<nb, kBlock, smem, ctx->stream>>>(
        a, c, d.dev, c12, c13, begin, end, d.ls_mc, (double)(d.mc ? d.mc->n : 0), ctx->scratch.partials,
        ctx->scratch.counters, out, out_mode);
  }
  GOO_CUDA_TRY(cudaGetLastError());
  return GOO_OK;
}

// The floating-lineshape evaluation: the MC pass, then the event pass over [begin, end).
template <typename T, bool GRAD>
static int launch_ls_pair(goo_model* m, const goo_dataset* ds, int64_t begin, int64_t end, const double* theta,
                          int out_mode) {
  DalitzModel& d = *m->dalitz;
  if (d.nbw <= 8) {
    GOO_TRY((launch_ls<T, 8, GRAD, true>(m, d.mc, 0, d.mc->n, theta, d.ls_mc, 0)));
    return launch_ls<T, 8, GRAD, false>(m, ds, begin, end, theta, m->ctx->scratch.result_out, out_mode);
  }
  GOO_TRY((launch_ls<T, 15, GRAD, true>(m, d.mc, 0, d.mc->n, theta, d.ls_mc, 0)));
  return launch_ls<T, 15, GRAD, false>(m, ds, begin, end, theta, m->ctx->scratch.result_out, out_mode);
}

// The three MC Gram matrices of the time-dependent three-body model (G_aa, G_bb, G_ab) in
// `precision`, rebuilt when the lineshapes or the MC sample change; a host copy for
// goo_normalise.
static int ensure_td_grams(goo_model* m, int precision) {
  DalitzModel& d = *m->dalitz;
  goo_ctx* ctx = m->ctx;
  const int pi = precision == GOO_F32 ? 0 : 1;
  if (!d.mc) return set_error(GOO_ERR_STATE, "amplitude model has no MC normalisation sample (goo_model_set_norm)");
  if (d.mc->n < 1) return set_error(GOO_ERR_ARG, "the MC normalisation sample is empty");
  const uint64_t key = d.ls_key ^ (uint64_t)(uintptr_t)d.mc ^ (uint64_t)(pi + 11) ^ d.mc->epoch * 0xd6e8feb86659fd93ull;
  if (d.gram3_key[pi] == key) return GOO_OK;
  const void *ca = nullptr, *cb = nullptr;
  GOO_TRY(ensure_cache(m, d.mc, precision, &ca));
  GOO_TRY(ensure_cache(m, d.mc, precision, &cb, true));
  const int K = d.K;
  double* g = d.gram3_dev[pi];
  const void* pairs[3][2] = {{ca, ca}, {cb, cb}, {ca, cb}};
  for (int q = 0; q < 3; ++q) {
    LaunchScope ls(ctx, pi == 0 ? "td3_gram_f32" : "td3_gram_f64");
    if (pi == 0)
      gram_cross_kernel<float><<<K * K, kBlock, 0, ctx->stream>>>(pairs[q][0], pairs[q][1], d.mc->n, d.nbw, K,
                                                                 g + (size_t)q * 2 * K * K);
    else
      gram_cross_kernel<double><<<K * K, kBlock, 0, ctx->stream>>>(pairs[q][0], pairs[q][1], d.mc->n, d.nbw, K,
                                                                  g + (size_t)q * 2 * K * K);
  }
  GOO_CUDA_TRY(cudaGetLastError());
  GOO_CUDA_TRY(cudaMemcpyAsync(d.gram3_host[pi], g, sizeof(double) * 3 * 2 * K * K, cudaMemcpyDeviceToHost,
                               ctx->stream));
  GOO_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  d.gram3_key[pi] = key;
  return GOO_OK;
}

template <typename T>
static void fill_td3(const DalitzModel& d, const double* theta, int n_params, int64_t n_total, Td3Args<T>& a,
                     double t_hi) {
  std::memset(&a, 0, sizeof a);
  for (int k = 0; k < d.K; ++k) {
    const int sl = k < d.nbw ? k : kTd3KB;
    double re, im;
    coef(d, theta, k, re, im);
    a.cr[sl] = (T)re;
    a.ci[sl] = (T)im;
    a.par_re[k] = d.par_re[k];
    a.par_im[k] = d.par_im[k];
  }
  fill_time_coef<T>(a.tc, theta[d.par_t[0]], theta[d.par_t[1]], theta[d.par_t[2]], theta[d.par_t[3]], t_hi);
  a.x = a.tc.x;
  a.y = a.tc.y;
  a.G = a.tc.G;
  a.s = a.tc.s;
  for (int j = 0; j < 4; ++j) a.par_t[j] = d.par_t[j];
  const WeidemanTables& w = weideman();
  a.wN = sizeof(T) == 4 ? kWN32 : kWN64;
  for (int j = 0; j < a.wN; ++j) a.wa[j] = (T)(sizeof(T) == 4 ? w.a32[j] : w.a64[j]);
  a.wL = (T)(sizeof(T) == 4 ? w.L32 : w.L64);
  a.nbw = d.nbw;
  a.K = d.K;
  a.n_params = n_params;
  a.n_total = n_total;
  fill_jacobian(d, theta, a);
}

// The normalisation at theta from the host copies of the three Gram matrices G_aa, G_bb, G_ab
// (ensure_td_grams keeps them current), in FP64 at the precision-rounded parameters the kernel
// uses.  With v_a = G_aa conj(c), v_b = G_bb conj(c), u = G_ab conj(c), w = c^T G_ab:
//   <|A|^2> = Re c.v_a, <|B|^2> = Re c.v_b, <A B*> = c.u,
//   N = (<|A|^2> + <|B|^2>)/2 I_ch + (<|A|^2> - <|B|^2>)/2 I_c + Re<AB*> I_sh + Im<AB*> I_s,
//   d<|A|^2> / d Re c_k = 2 Re v_a,k, / d Im c_k = -2 Im v_a,k;
//   d<AB*> / d Re c_k = u_k + w_k, / d Im c_k = i (u_k - w_k);
// and the time integrals' derivatives for x, y and tau.
template <typename T>
static void td3_norm_terms(const DalitzModel& d, const double* G, Td3Args<T>& a) {
  const int K = d.K;
  const double* Gaa = G;
  const double* Gbb = G + 2 * K * K;
  const double* Gab = G + 4 * K * K;
  auto cf = [&](int j, double& r, double& im) {
    const int sl = j < d.nbw ? j : kTd3KB;
    r = (double)a.cr[sl];
    im = (double)a.ci[sl];
  };
  const double x = (double)a.x, y = (double)a.y, tau = 1.0 / (double)a.G;
  const double iy = 1.0 / (1 - y * y), ix = 1.0 / (1 + x * x);
  const double Ich = tau * iy, Ish = y * tau * iy, Ic = tau * ix, Is = x * tau * ix;
  double var[kMaxAmp], vai[kMaxAmp], vbr[kMaxAmp], vbi[kMaxAmp], ur[kMaxAmp], ui[kMaxAmp], wr[kMaxAmp], wi[kMaxAmp];
  double PA = 0, PB = 0, Xr = 0, Xi = 0;
  for (int k = 0; k < K; ++k) {
    var[k] = vai[k] = vbr[k] = vbi[k] = ur[k] = ui[k] = wr[k] = wi[k] = 0.0;
    for (int l = 0; l < K; ++l) {
      double clr, cli;
      cf(l, clr, cli);
      const double ar_ = Gaa[2 * (k * K + l)], ai_ = Gaa[2 * (k * K + l) + 1];
      const double br_ = Gbb[2 * (k * K + l)], bi_ = Gbb[2 * (k * K + l) + 1];
      const double xr_ = Gab[2 * (k * K + l)], xi_ = Gab[2 * (k * K + l) + 1];
      const double yr_ = Gab[2 * (l * K + k)], yi_ = Gab[2 * (l * K + k) + 1];
      var[k] += ar_ * clr + ai_ * cli;  // G_aa[k][l] conj(c_l)
      vai[k] += ai_ * clr - ar_ * cli;
      vbr[k] += br_ * clr + bi_ * cli;
      vbi[k] += bi_ * clr - br_ * cli;
      ur[k] += xr_ * clr + xi_ * cli;  // G_ab[k][l] conj(c_l)
      ui[k] += xi_ * clr - xr_ * cli;
      wr[k] += clr * yr_ - cli * yi_;  // c_l G_ab[l][k]
      wi[k] += clr * yi_ + cli * yr_;
    }
    double ckr, cki;
    cf(k, ckr, cki);
    PA += ckr * var[k] - cki * vai[k];  // Re(c_k v_a,k)
    PB += ckr * vbr[k] - cki * vbi[k];
    Xr += ckr * ur[k] - cki * ui[k];  // c_k u_k (summed: <A B*>)
    Xi += ckr * ui[k] + cki * ur[k];
  }
  const double N = 0.5 * (PA + PB) * Ich + 0.5 * (PA - PB) * Ic + Xr * Ish + Xi * Is;
  const double invN = 1.0 / N;
  for (int k = 0; k < K; ++k) {
    const double dre = 0.5 * (2 * var[k] + 2 * vbr[k]) * Ich + 0.5 * (2 * var[k] - 2 * vbr[k]) * Ic +
                       (ur[k] + wr[k]) * Ish + (ui[k] + wi[k]) * Is;
    const double dim = 0.5 * (-2 * vai[k] - 2 * vbi[k]) * Ich + 0.5 * (-2 * vai[k] + 2 * vbi[k]) * Ic -
                       (ui[k] - wi[k]) * Ish + (ur[k] - wr[k]) * Is;
    a.nrm_re[k] = dre * invN;
    a.nrm_im[k] = dim * invN;
  }
  a.nrm_N = N;
  a.nrm_logN = std::log(N);
  const double ix2 = ix * ix, iy2 = iy * iy;
  const double dxc = -2 * x * tau * ix2, dxs = tau * (1 - x * x) * ix2;
  const double dych = 2 * y * tau * iy2, dysh = tau * (1 + y * y) * iy2;
  a.nrm_dt[0] = (0.5 * (PA - PB) * dxc + Xi * dxs) * invN;
  a.nrm_dt[1] = (0.5 * (PA + PB) * dych + Xr * dysh) * invN;
  a.nrm_dt[2] = (0.5 * (PA + PB) * iy + 0.5 * (PA - PB) * ix + Xr * y * iy + Xi * x * ix) * invN;
}

template <typename T, bool GRAD>
static int launch_td3(goo_model* m, const goo_dataset* ds, int64_t begin, int64_t end, const double* theta,
                      const void* ca, const void* cb, int out_mode) {
  DalitzModel& d = *m->dalitz;
  goo_ctx* ctx = m->ctx;
  const int pi = sizeof(T) == 4 ? 0 : 1;
  static int occ[2] = {0, 0};
  int& o = occ[pi];
  if (o == 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, td3_nll_kernel<T, GRAD>, kBlock, 0) != cudaSuccess || o < 1) {
      cudaGetLastError();
      o = 1;
    }
  }
  const int nb = grid_blocks(ctx, end - begin, o);
  constexpr int NS = Td3Lanes<GRAD>::NS;
  GOO_TRY(ensure_partials(ctx, (size_t)nb * NS));
  Td3Args<T> a;
  fill_td3<T>(d, theta, m->n_params, ds->n, a, m->hi[d.col_t]);
  td3_norm_terms<T>(d, d.gram3_host[pi], a);
  const T* tcol = sizeof(T) == 4 ? (const T*)ds->d32[d.col_t] : (const T*)ds->d64[d.col_t];
  {
    LaunchScope ls(ctx, sizeof(T) == 4 ? (GRAD ? "td3_nll_grad_f32" : "td3_nll_f32")
                                       : (GRAD ? "td3_nll_grad_f64" : "td3_nll_f64"));
    td3_nll_kernel<T, GRAD><<<nb, kBlock, 0, ctx->stream>>>(a, ca, cb, tcol, begin, end, ctx->scratch.partials,
                                                            ctx->scratch.counters, ctx->scratch.result_out,
                                                            out_mode);
  }
  GOO_CUDA_TRY(cudaGetLastError());
  return GOO_OK;
}

// N of the time-dependent three-body model at theta from the host copy of the Gram matrices.
static double td3_norm_host(const DalitzModel& d, const double* G, const double* theta, bool f32) {
  const int K = d.K;
  auto cf = [&](int k, double& r, double& i) {
    coef(d, theta, k, r, i);
    if (f32) {
      r = (double)(float)r;
      i = (double)(float)i;
    }
  };
  double PA = 0, PB = 0, Xr = 0, Xi = 0;
  for (int k = 0; k < K; ++k)
    for (int l = 0; l < K; ++l) {
      double ckr, cki, clr, cli;
      cf(k, ckr, cki);
      cf(l, clr, cli);
      const double pr = ckr * clr + cki * cli, pim = cki * clr - ckr * cli;  // c_k conj(c_l)
      const double* Gs[3] = {G, G + 2 * K * K, G + 4 * K * K};
      const double gr[3] = {Gs[0][2 * (k * K + l)], Gs[1][2 * (k * K + l)], Gs[2][2 * (k * K + l)]};
      const double gi[3] = {Gs[0][2 * (k * K + l) + 1], Gs[1][2 * (k * K + l) + 1], Gs[2][2 * (k * K + l) + 1]};
      PA += pr * gr[0] - pim * gi[0];
      PB += pr * gr[1] - pim * gi[1];
      Xr += pr * gr[2] - pim * gi[2];
      Xi += pr * gi[2] + pim * gr[2];
    }
  double x = theta[d.par_t[0]], y = theta[d.par_t[1]], tau = theta[d.par_t[2]];
  if (f32) {
    x = (double)(float)x;
    y = (double)(float)y;
    tau = 1.0 / (double)(float)(1.0 / tau);
  }
  const double Ich = tau / (1 - y * y), Ish = y * tau / (1 - y * y), Ic = tau / (1 + x * x), Is = x * tau / (1 + x * x);
  return 0.5 * (PA + PB) * Ich + 0.5 * (PA - PB) * Ic + Xr * Ish + Xi * Is;
}

int build_dalitz_model(goo_ctx* ctx, const goo_node* nodes, int n_nodes, int n_params, int n_obs, const double* lo,
                       const double* hi, goo_model* m) {
  const goo_node& root = nodes[n_nodes - 1];
  if (root.n_child < 1 || root.n_child > kMaxAmp)
    return set_error(GOO_ERR_UNSUPPORTED, "coherent sum of %d amplitudes (1..%d)", root.n_child, kMaxAmp);
  if (n_obs < 2 || root.obs[0] < 0 || root.obs[1] < 0 || root.obs[0] >= n_obs || root.obs[1] >= n_obs)
    return set_error(GOO_ERR_ARG, "coherent node needs observables s12 and s13");
  DalitzModel* d = new DalitzModel();
  m->dalitz = d;
  m->kind = 1;
  d->col12 = root.obs[0];
  d->col13 = root.obs[1];
  if (root.op == GOO_OP_TD3) {
    d->td = true;
    d->col_t = root.ival[0];
    if (n_obs < 3 || d->col_t < 0 || d->col_t >= n_obs || d->col_t == d->col12 || d->col_t == d->col13)
      return set_error(GOO_ERR_ARG, "GOO_OP_TD3 needs a decay-time observable (ival[0]) besides s12 and s13");
    for (int j = 0; j < 4; ++j) {
      if (root.par[j] < 0 || root.par[j] >= n_params)
        return set_error(GOO_ERR_ARG, "GOO_OP_TD3: time parameter %d has index %d", j, root.par[j]);
      d->par_t[j] = root.par[j];
    }
  }
  d->M = root.dval[0];
  d->m1 = root.dval[1];
  d->m2 = root.dval[2];
  d->m3 = root.dval[3];
  d->r_res = root.dval[4];
  d->r_par = root.dval[5];
  if (!(d->M > d->m1 + d->m2 + d->m3) || d->m1 < 0 || d->m2 < 0 || d->m3 < 0)
    return set_error(GOO_ERR_ARG, "parent mass %g below the sum of the daughter masses", d->M);
  auto check_par = [&](int p) { return p >= 0 && p < n_params; };
  // BWs first (in tree order), then the NR amplitude
  for (int pass = 0; pass < 2; ++pass) {
    for (int c = 0; c < root.n_child; ++c) {
      const goo_node& a = nodes[root.child[c]];
      if (a.op != GOO_OP_BW && a.op != GOO_OP_NR)
        return set_error(GOO_ERR_ARG, "coherent child %d has op %d (BW or NR expected)", c, a.op);
      if ((pass == 0) != (a.op == GOO_OP_BW)) continue;
      const int k = d->K++;
      if (!check_par(a.par[2]) || !check_par(a.par[3]))
        return set_error(GOO_ERR_ARG, "amplitude %d has no coefficient parameters", c);
      d->par_re[k] = a.par[2];
      d->par_im[k] = a.par[3];
      if (a.op == GOO_OP_BW) {
        if (!check_par(a.par[0]) || !check_par(a.par[1]))
          return set_error(GOO_ERR_ARG, "BW amplitude %d has no mass/width parameters", c);
        if (a.ival[0] < 0 || a.ival[0] > 2) return set_error(GOO_ERR_UNSUPPORTED, "BW spin %d (0..2)", a.ival[0]);
        if (a.ival[1] < 0 || a.ival[1] > 2) return set_error(GOO_ERR_ARG, "BW pair %d (0..2)", a.ival[1]);
        d->par_m0[k] = a.par[0];
        d->par_w[k] = a.par[1];
        d->spin[k] = a.ival[0];
        d->pair[k] = a.ival[1];
        d->nbw++;
      } else {
        if (d->has_nr) return set_error(GOO_ERR_UNSUPPORTED, "at most one non-resonant amplitude");
        d->has_nr = true;
      }
    }
  }
  if (d->nbw > 15) return set_error(GOO_ERR_UNSUPPORTED, "at most 15 resonances");
  if (d->td && std::fabs(d->m2 - d->m3) > 1e-12 * d->M)
    return set_error(GOO_ERR_ARG, "GOO_OP_TD3: the CP-conjugate particles 2 and 3 need equal masses (%g, %g)", d->m2,
                     d->m3);
  if (d->td) {
    for (int i = 0; i < 2; ++i)
      if (cudaMalloc(&d->gram3_dev[i], sizeof(double) * 3 * 2 * kMaxAmp * kMaxAmp) != cudaSuccess) {
        cudaGetLastError();
        return set_error(GOO_ERR_OOM, "cannot allocate the amplitude model");
      }
  }
  (void)lo;
  (void)hi;
  if (cudaMalloc(&d->dev, sizeof(DalitzDev)) != cudaSuccess ||
      cudaMalloc(&d->gram_dev[0], sizeof(double) * 2 * kMaxAmp * kMaxAmp) != cudaSuccess ||
      cudaMalloc(&d->gram_dev[1], sizeof(double) * 2 * kMaxAmp * kMaxAmp) != cudaSuccess) {
    cudaGetLastError();
    return set_error(GOO_ERR_OOM, "cannot allocate the amplitude model");
  }
  m->norm.kind = GOO_NORM_MC;
  (void)ctx;
  return GOO_OK;
}

int dalitz_set_norm(goo_model* m, const goo_norm_spec* spec) {
  if (spec->kind != GOO_NORM_MC || !spec->mc)
    return set_error(GOO_ERR_UNSUPPORTED, "amplitude models are normalised with an MC sample (GOO_NORM_MC)");
  const goo_dataset* mc = spec->mc;
  DalitzModel& d = *m->dalitz;
  if (mc->ctx != m->ctx) return set_error(GOO_ERR_ARG, "MC sample belongs to another context");
  if (mc->ncols <= d.col12 || mc->ncols <= d.col13) return set_error(GOO_ERR_ARG, "MC sample lacks s12/s13 columns");
  d.mc = mc;
  d.gram_key[0] = d.gram_key[1] = 0;
  d.gram3_key[0] = d.gram3_key[1] = 0;
  m->norm = *spec;
  return GOO_OK;
}

void dalitz_free(goo_model* m) {
  DalitzModel* d = m->dalitz;
  if (!d) return;
  if (d->dev) cudaFree(d->dev);
  for (int i = 0; i < 2; ++i)
    if (d->gram_dev[i]) cudaFree(d->gram_dev[i]);
  if (d->ls_mc) cudaFree(d->ls_mc);
  for (int i = 0; i < 2; ++i)
    if (d->gram3_dev[i]) cudaFree(d->gram3_dev[i]);
  delete d;
  m->dalitz = nullptr;
}

static double quad_form(const DalitzModel& d, const double* G, const double* theta, bool f32) {
  double N = 0.0;
  for (int k = 0; k < d.K; ++k)
    for (int l = 0; l < d.K; ++l) {
      double ckr, cki, clr, cli;
      coef(d, theta, k, ckr, cki);
      coef(d, theta, l, clr, cli);
      if (f32) {
        ckr = (double)(float)ckr;
        cki = (double)(float)cki;
        clr = (double)(float)clr;
        cli = (double)(float)cli;
      }
      const double gr = G[2 * (k * d.K + l)], gi = G[2 * (k * d.K + l) + 1];
      // Re(c_k conj(c_l) G_kl)
      const double pr = ckr * clr + cki * cli, pim = cki * clr - ckr * cli;
      N += pr * gr - pim * gi;
    }
  return N;
}

int dalitz_normalise(goo_model* m, const double* theta, int precision, double* norm_out) {
  GOO_TRY(dalitz_constants(m, theta));
  if (m->dalitz->td) {
    GOO_TRY(ensure_td_grams(m, precision));
    norm_out[0] = td3_norm_host(*m->dalitz, m->dalitz->gram3_host[precision == GOO_F32 ? 0 : 1], theta,
                                precision == GOO_F32);
    return GOO_OK;
  }
  GOO_TRY(ensure_gram(m, precision));
  const int pi = precision == GOO_F32 ? 0 : 1;
  norm_out[0] = quad_form(*m->dalitz, m->dalitz->gram_host[pi], theta, precision == GOO_F32);
  return GOO_OK;
}

int dalitz_nll(goo_model* m, const goo_dataset* ds, int64_t begin, int64_t end, const double* theta, int precision,
               bool grad, double* out, int out_mode) {
  DalitzModel& d = *m->dalitz;
  goo_ctx* ctx = m->ctx;
  // the record goes to the mapped host copy; the host polls its fields
  MappedResult mapped(ctx);
  const int P = m->n_params;
  if (ds->ncols <= d.col12 || ds->ncols <= d.col13) return set_error(GOO_ERR_ARG, "dataset lacks s12/s13 columns");
  GOO_TRY(dalitz_constants(m, theta));
  const int nout = (out_mode == 0 ? 2 : 3) + P;
  if (d.td) {
    // time-dependent three-body model: amplitude caches at the event and the exchanged point
    if (ds->ncols <= d.col_t) return set_error(GOO_ERR_ARG, "dataset lacks the decay-time column");
    GOO_TRY(ensure_td_grams(m, precision));
    if (end <= begin) {
      for (int i = 0; i < nout; ++i) out[i] = 0.0;
      return GOO_OK;
    }
    const void *ca = nullptr, *cb = nullptr;
    GOO_TRY(ensure_cache(m, ds, precision, &ca));
    GOO_TRY(ensure_cache(m, ds, precision, &cb, true));
    if (precision == GOO_F32) {
      GOO_TRY((grad ? launch_td3<float, true>(m, ds, begin, end, theta, ca, cb, out_mode)
                    : launch_td3<float, false>(m, ds, begin, end, theta, ca, cb, out_mode)));
    } else {
      GOO_TRY((grad ? launch_td3<double, true>(m, ds, begin, end, theta, ca, cb, out_mode)
                    : launch_td3<double, false>(m, ds, begin, end, theta, ca, cb, out_mode)));
    }
  } else if (d.floating) {
    // no cache and no Gram matrix: an MC pass and an event pass, lineshape gradients included
    if (!d.mc) return set_error(GOO_ERR_STATE, "amplitude model has no MC normalisation sample (goo_model_set_norm)");
    if (d.mc->n < 1) return set_error(GOO_ERR_ARG, "the MC normalisation sample is empty");
    if (end <= begin) {
      for (int i = 0; i < nout; ++i) out[i] = 0.0;
      return GOO_OK;
    }
    if (!d.ls_mc && cudaMalloc(&d.ls_mc, 64 * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      d.ls_mc = nullptr;
      return set_error(GOO_ERR_OOM, "floating-lineshape work space");
    }
    if (precision == GOO_F32) {
      GOO_TRY((grad ? launch_ls_pair<float, true>(m, ds, begin, end, theta, out_mode)
                    : launch_ls_pair<float, false>(m, ds, begin, end, theta, out_mode)));
    } else {
      GOO_TRY((grad ? launch_ls_pair<double, true>(m, ds, begin, end, theta, out_mode)
                    : launch_ls_pair<double, false>(m, ds, begin, end, theta, out_mode)));
    }
  } else {
  GOO_TRY(ensure_gram(m, precision));
  const int pi = precision == GOO_F32 ? 0 : 1;
  if (end <= begin) {
    for (int i = 0; i < nout; ++i) out[i] = 0.0;
    return GOO_OK;
  }
  const void* cache = nullptr;
  GOO_TRY(ensure_cache(m, ds, precision, &cache));
  if (precision == GOO_F32) {
    GOO_TRY((grad ? launch_coh_sel<float, true>(m, cache, ds, begin, end, theta, out_mode, pi)
                  : launch_coh_sel<float, false>(m, cache, ds, begin, end, theta, out_mode, pi)));
  } else {
    GOO_TRY((grad ? launch_coh_sel<double, true>(m, cache, ds, begin, end, theta, out_mode, pi)
                  : launch_coh_sel<double, false>(m, cache, ds, begin, end, theta, out_mode, pi)));
  }
  }
  return read_result_mapped(ctx, nout, out);
}

int dalitz_eval_logf(goo_model* m, const goo_dataset* ds, const double* theta, int precision, double* logf_dev) {
  DalitzModel& d = *m->dalitz;
  goo_ctx* ctx = m->ctx;
  if (d.td) return set_error(GOO_ERR_UNSUPPORTED, "goo_eval_logf of the time-dependent three-body model");
  if (ds->ncols <= d.col12 || ds->ncols <= d.col13) return set_error(GOO_ERR_ARG, "dataset lacks s12/s13 columns");
  GOO_TRY(dalitz_constants(m, theta));
  GOO_TRY(ensure_gram(m, precision));
  if (ds->n == 0) return GOO_OK;
  const int pi = precision == GOO_F32 ? 0 : 1;
  const double logN = std::log(quad_form(d, d.gram_host[pi], theta, precision == GOO_F32));
  const void* cache = nullptr;
  GOO_TRY(ensure_cache(m, ds, precision, &cache));
  const int nb = grid_blocks(ctx, ds->n, 4);
  LaunchScope ls(ctx, "coh_logf");
  if (precision == GOO_F32) {
    CohArgs<float> a;
    fill_args<float>(d, theta, m->n_params, ds->n, a);
    if (d.nbw <= 8) coh_logf_kernel<float, 8><<<nb, kBlock, 0, ctx->stream>>>(a, cache, logN, logf_dev);
    else coh_logf_kernel<float, 15><<<nb, kBlock, 0, ctx->stream>>>(a, cache, logN, logf_dev);
  } else {
    CohArgs<double> a;
    fill_args<double>(d, theta, m->n_params, ds->n, a);
    if (d.nbw <= 8) coh_logf_kernel<double, 8><<<nb, kBlock, 0, ctx->stream>>>(a, cache, logN, logf_dev);
    else coh_logf_kernel<double, 15><<<nb, kBlock, 0, ctx->stream>>>(a, cache, logN, logf_dev);
  }
  GOO_CUDA_TRY(cudaGetLastError());
  return GOO_OK;
}

// Host copies of the Gram matrix (K x K complex, model amplitude order: resonances in tree
// order, then the non-resonant amplitude) and of the per-event amplitude cache (test access).
int dalitz_gram(goo_model* m, const double* theta, int precision, double* out, int* K_out) {
  if (m->dalitz->td) return set_error(GOO_ERR_UNSUPPORTED, "goo_gram: the time-dependent three-body model has three");
  GOO_TRY(dalitz_constants(m, theta));
  GOO_TRY(ensure_gram(m, precision));
  const int pi = precision == GOO_F32 ? 0 : 1;
  const int K = m->dalitz->K;
  std::memcpy(out, m->dalitz->gram_host[pi], sizeof(double) * 2 * K * K);
  *K_out = K;
  return GOO_OK;
}

int dalitz_amplitudes(goo_model* m, const goo_dataset* ds, const double* theta, int precision, const void** cache,
                      int* nbw) {
  GOO_TRY(dalitz_constants(m, theta));
  GOO_TRY(ensure_cache(m, ds, precision, cache));
  *nbw = m->dalitz->nbw;
  GOO_CUDA_TRY(cudaStreamSynchronize(m->ctx->stream));
  return GOO_OK;
}

int dalitz_server_info(goo_model* m, const double* theta, AmpModelInfo* info) {
  if (m->kind != 1) return set_error(GOO_ERR_STATE, "toy server needs an amplitude model");
  if (m->dalitz->td) return set_error(GOO_ERR_UNSUPPORTED, "toy server of the time-dependent three-body model");
  if (m->dalitz->polar) return set_error(GOO_ERR_UNSUPPORTED, "toy server with polar coefficients");
  GOO_TRY(dalitz_constants(m, theta));
  GOO_TRY(ensure_gram(m, GOO_F32));
  const DalitzModel& d = *m->dalitz;
  info->dalitz_dev = d.dev;
  info->gram_dev = d.gram_dev[0];
  info->K = d.K;
  info->nbw = d.nbw;
  info->has_nr = d.has_nr ? 1 : 0;
  for (int k = 0; k < d.K; ++k) {
    info->par_re[k] = d.par_re[k];
    info->par_im[k] = d.par_im[k];
  }
  info->M = d.M;
  info->m1 = d.m1;
  info->m2 = d.m2;
  info->m3 = d.m3;
  info->lo12 = (d.m1 + d.m2) * (d.m1 + d.m2);
  info->hi12 = (d.M - d.m3) * (d.M - d.m3);
  info->lo13 = (d.m1 + d.m3) * (d.m1 + d.m3);
  info->hi13 = (d.M - d.m2) * (d.M - d.m2);
  return GOO_OK;
}

}  // namespace goo

namespace goo {
int dalitz_set_lineshapes(goo_model* m, int mode) {
  if (mode != GOO_LINESHAPE_CACHED && mode != GOO_LINESHAPE_FLOATING)
    return set_error(GOO_ERR_ARG, "goo_model_set_lineshapes: mode %d", mode);
  if (m->dalitz->td && mode == GOO_LINESHAPE_FLOATING)
    return set_error(GOO_ERR_UNSUPPORTED, "floating lineshapes of the time-dependent three-body model");
  m->dalitz->floating = mode == GOO_LINESHAPE_FLOATING;
  return GOO_OK;
}

bool dalitz_lineshape_param(const goo_model* m, int p) {
  const DalitzModel& d = *m->dalitz;
  for (int k = 0; k < d.nbw; ++k)
    if (d.par_m0[k] == p || d.par_w[k] == p) return true;
  return false;
}

bool dalitz_floating(const goo_model* m) { return m->dalitz->floating; }

int dalitz_set_coefficients(goo_model* m, int form) {
  if (form != GOO_COEF_CARTESIAN && form != GOO_COEF_POLAR)
    return set_error(GOO_ERR_ARG, "goo_model_set_coefficients: form %d", form);
  m->dalitz->polar = form == GOO_COEF_POLAR;
  return GOO_OK;
}
bool dalitz_time_dependent(const goo_model* m) { return m->dalitz->td; }
}  // namespace goo
