// tree.cu -- sum/product PDF models: flattening, parameter preparation, grid
// normalisation and the fused per-event NLL (+ adjoint gradient) kernel.
//
// Paper: PDFs are composed from basic PDFs by combination PDFs (Fig. 1; Sec. 1) and the
// time of a fit goes into evaluating the function at every point of the dataset (Sec. 1).
//
// Model semantics (the paper prints no formulas; RooFit conventions, Sec. 1):
//   leaf shapes       GAUSS exp(-(x-mu)^2/2s^2), EXPO exp(l x), POLY2 1+a1 x+a2 x^2,
//                     ARGUS m u^p exp(c u) with u = 1 - m^2/m0^2 (0 for u <= 0)
//   PROD              product of its children (disjoint observables)
//   ADD               sum_k w_k child_k / norm(child_k), w_k = frac_k, last = 1 - sum(frac)
// The host flattens any such tree into a sum of products
//   f(x) = sum_k w_k U_k(x) / N_k,   U_k = product of the leaves of product k,
// where w_k is a product of ADD fractions (or one minus their sum) and N_k is the integral
// of U_k: the product of the leaves' closed forms (ANALYTIC) or the midpoint sum over a
// grid of product k's observables (GRID).  This equals the recursive definition whenever
// PROD children act on disjoint observables.
//
// Per event every value is carried as r * exp(a) (a "log-domain" pair) so that tiny
// densities (far Gaussian tails, exponentials) never underflow:
//   U_k = r_k exp(a_k),  log f = M + log S,  M = max_k (a_k - log N_k),
//   S = sum_k w_k r_k exp(a_k - log N_k - M).
// Adjoint gradient: with c_k = r_k exp(a_k - log N_k - M) / S (so the share of product k in
// f is w_k c_k), the per-event derivative is
//   d log f / d theta = sum_k [ w_k c_k d log U_k/d theta + c_k d w_k/d theta
//                              - w_k c_k d log N_k/d theta ],
// so the kernel only accumulates C_k = sum_i c_k and A_{k,l,j} = sum_i c_k d log U_leaf/d theta_j
// per leaf parameter; the last block maps these lanes to d NLL / d theta in FP64.
//
// FP32 path precision: offsets of an observable (mu, m0), the weights w_k and the offsets
// -log N_k are passed as float hi + lo pairs, so that FP32 rounding of a constant does not
// bias the fit; per-event rounding is random and averages out.  Closed-form norms in the
// FP32 path are taken at the FP32-rounded parameters the kernel actually uses, so the NLL is
// the exact likelihood of those parameters.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "model.cuh"
#include "jit.cuh"
#include "sop_kernels.cuh"

namespace goo {

// =======================================================================================
// parameter preparation (a1): per-theta derived constants, computed on the host in FP64
// and uploaded with theta in one copy (O(number of leaves) work)
// =======================================================================================
static double gauss_log_norm(double lo, double hi, double mu, double sig, double* dmu, double* dsig) {
  // N = sig sqrt(pi/2) [erf(b) - erf(a)], a = (lo-mu)/(sqrt2 sig), b = (hi-mu)/(sqrt2 sig)
  const double r2 = 1.4142135623730951, c = 1.2533141373155003;  // sqrt(2), sqrt(pi/2)
  double a = (lo - mu) / (r2 * sig), b = (hi - mu) / (r2 * sig);
  double diff;
  if (a > 0.0) diff = erfc(a) - erfc(b);
  else if (b < 0.0) diff = erfc(-b) - erfc(-a);
  else diff = erf(b) - erf(a);
  double N = sig * c * diff;
  double ga = exp(-a * a), gb = exp(-b * b);
  // dN/dmu = g(lo) - g(hi);  dN/dsig = (N - [(x-mu) g(x)]_lo^hi) / sig
  *dmu = (ga - gb) / N;
  *dsig = (N - ((hi - mu) * gb - (lo - mu) * ga)) / (sig * N);
  return log(N);
}

static double expo_log_norm(double lo, double hi, double lam, double* dlam) {
  const double d = hi - lo;
  if (fabs(lam * d) < 1e-5) {
    // N = d (1 + lam (lo+hi)/2 + ...),  d log N / d lam = mean of x + lam d^2/12 + ...
    *dlam = 0.5 * (lo + hi) + lam * d * d / 12.0;
    return log(d) + lam * 0.5 * (lo + hi) + lam * lam * d * d / 24.0;
  }
  double logN;
  if (lam < 0.0) logN = lam * lo + log(expm1(lam * d) / lam);
  else logN = lam * hi + log(-expm1(-lam * d) / lam);
  // d log N / d lam = (hi e^{lam hi} - lo e^{lam lo}) / (e^{lam hi} - e^{lam lo}) - 1/lam
  const double mean = (lam < 0.0) ? (hi * exp(lam * d) - lo) / (exp(lam * d) - 1.0)
                                  : (hi - lo * exp(-lam * d)) / (1.0 - exp(-lam * d));
  *dlam = mean - 1.0 / lam;
  return logN;
}

static double poly2_log_norm(double lo, double hi, double a1, double a2, double* da1, double* da2) {
  double i1 = 0.5 * (hi * hi - lo * lo), i2 = (hi * hi * hi - lo * lo * lo) / 3.0;
  double N = (hi - lo) + a1 * i1 + a2 * i2;
  *da1 = i1 / N;
  *da2 = i2 / N;
  return log(N);
}

// Upper bound of the leaf's log-domain exponent a over [lo, hi] (grid reference scale).
static double leaf_max_exponent(int op, double lo, double hi, const double* d) {
  if (op == GOO_OP_GAUSS) {
    double mu = d[0], is = d[1];
    double x = mu < lo ? lo : (mu > hi ? hi : mu);
    double z = (x - mu) * is;
    return -0.5 * z * z;
  }
  if (op == GOO_OP_EXPO) return fmax(d[0] * lo, d[0] * hi);
  if (op == GOO_OP_ARGUS) {
    double m0 = d[0], c = d[2], p = d[3];
    double umax = 1.0 - lo * lo / (m0 * m0);
    if (umax <= 0.0) return 0.0;
    double u = (c < 0.0) ? fmin(-p / c, umax) : umax;
    if (u <= 0.0) u = umax;
    return p * log(u) + c * u;
  }
  return 0.0;
}

// Fills the per-theta fields of a model block whose static fields (opcodes, columns,
// parameter indices, products, ADD tables, grid geometry) are already set: per-leaf FP32 and
// FP64 constants, per-product weights w_k and dw/dtheta, the grid reference exponents, and
// for analytic normalisation log N_k with d log N_k / d theta.  In the FP32 path the closed
// forms are taken at the FP32-rounded parameters the kernels use.
void host_prep(ModelDev& h, const double* theta, int precision) {
  const bool analytic = h.norm_kind == GOO_NORM_ANALYTIC;
  const bool f32 = precision == GOO_F32;
  double logN_leaf[kMaxComp * kMaxLeaf] = {0};
  double dlog_leaf[kMaxComp * kMaxLeaf][3] = {{0}};
  double amax_leaf[kMaxComp * kMaxLeaf] = {0};
  for (int k = 0; k < h.nK; ++k) {
    for (int l = 0; l < h.comp[k].n_leaf; ++l) {
      const int t = k * kMaxLeaf + l;
      LeafDev& L = h.leaf[t];
      const double lo = h.lo[L.col], hi = h.hi[L.col];
      const double p0 = L.par[0] >= 0 ? theta[L.par[0]] : 0.0;
      const double p1 = L.par[1] >= 0 ? theta[L.par[1]] : 0.0;
      const double p2 = L.par[2] >= 0 ? theta[L.par[2]] : 0.0;
      for (int i = 0; i < 6; ++i) {
        L.d[i] = 0.0;
        L.f[i] = 0.f;
      }
      double g0 = 0.0, g1 = 0.0;
      switch (L.op) {
        case GOO_OP_GAUSS: {
          L.d[0] = p0;
          L.d[1] = 1.0 / p1;
          const float hi32 = (float)p0;
          L.f[0] = hi32;
          L.f[1] = (float)(p0 - (double)hi32);
          L.f[2] = (float)(1.0 / p1);
          if (analytic) {
            const double mu = f32 ? (double)L.f[0] + (double)L.f[1] : p0;
            const double sg = f32 ? 1.0 / (double)L.f[2] : p1;
            logN_leaf[t] = gauss_log_norm(lo, hi, mu, sg, &g0, &g1);
          } else {
            amax_leaf[t] = leaf_max_exponent(L.op, lo, hi, L.d);
          }
          break;
        }
        case GOO_OP_EXPO:
          L.d[0] = p0;
          L.f[0] = (float)p0;
          if (analytic) logN_leaf[t] = expo_log_norm(lo, hi, f32 ? (double)L.f[0] : p0, &g0);
          else amax_leaf[t] = leaf_max_exponent(L.op, lo, hi, L.d);
          break;
        case GOO_OP_POLY2:
          L.d[0] = p0;
          L.d[1] = p1;
          L.f[0] = (float)p0;
          L.f[1] = (float)p1;
          if (analytic)
            logN_leaf[t] = poly2_log_norm(lo, hi, f32 ? (double)L.f[0] : p0, f32 ? (double)L.f[1] : p1, &g0, &g1);
          break;
        case GOO_OP_ARGUS: {
          L.d[0] = p0;
          L.d[1] = 1.0 / (p0 * p0);
          L.d[2] = p1;
          L.d[3] = p2;
          L.d[4] = 2.0 / p0;
          const float hi32 = (float)p0;
          L.f[0] = hi32;
          L.f[1] = (float)(p0 - (double)hi32);
          L.f[2] = (float)(1.0 / (p0 * p0));
          L.f[3] = (float)p1;
          L.f[4] = (float)p2;
          L.f[5] = (float)(2.0 / p0);
          if (!analytic) amax_leaf[t] = leaf_max_exponent(L.op, lo, hi, L.d);
          break;
        }
        default:
          break;
      }
      dlog_leaf[t][0] = g0;
      dlog_leaf[t][1] = g1;
      L.a_ref = amax_leaf[t];
      L.a_ref_hi = (float)amax_leaf[t];
      L.a_ref_lo = (float)(amax_leaf[t] - (double)L.a_ref_hi);
    }
  }
  for (int k = 0; k < kMaxComp; ++k)
    for (int p = 0; p < kMaxParams; ++p) {
      h.dw[k][p] = 0.0;
      if (analytic) h.dlogN[k][p] = 0.0;
    }
  for (int k = 0; k < h.nK; ++k) {
    CompDev& C = h.comp[k];
    double fac[8];
    double w = 1.0;
    for (int f = 0; f < C.n_fac; ++f) {
      const AddDev& A = h.add[C.fac_add[f]];
      double v;
      if (C.fac_pos[f] < A.n_child - 1) {
        v = theta[A.frac[C.fac_pos[f]]];
      } else {
        v = 1.0;
        for (int j = 0; j < A.n_child - 1; ++j) v -= theta[A.frac[j]];
      }
      fac[f] = v;
      w *= v;
    }
    // dw/dtheta: product rule over the ADD factors
    for (int f = 0; f < C.n_fac; ++f) {
      const AddDev& A = h.add[C.fac_add[f]];
      double rest = 1.0;
      for (int g = 0; g < C.n_fac; ++g)
        if (g != f) rest *= fac[g];
      if (C.fac_pos[f] < A.n_child - 1) {
        h.dw[k][A.frac[C.fac_pos[f]]] += rest;
      } else {
        for (int j = 0; j < A.n_child - 1; ++j) h.dw[k][A.frac[j]] -= rest;
      }
    }
    C.w = w;
    C.w_hi = (float)w;
    C.w_lo = (float)(w - (double)C.w_hi);
    double amax = 0.0;
    for (int l = 0; l < C.n_leaf; ++l) amax += amax_leaf[k * kMaxLeaf + l];
    C.a_ref = amax;
    C.a_ref_hi = (float)amax;
    C.a_ref_lo = (float)(amax - (double)C.a_ref_hi);
    if (analytic) {
      double logN = 0.0;
      for (int l = 0; l < C.n_leaf; ++l) {
        const int li = k * kMaxLeaf + l;
        logN += logN_leaf[li];
        const LeafDev& L = h.leaf[li];
        for (int j = 0; j < 3; ++j)
          if (L.par[j] >= 0) h.dlogN[k][L.par[j]] += dlog_leaf[li][j];
      }
      C.log_norm = logN;
      C.off_hi = (float)(-logN);
      C.off_lo = (float)(-logN - (double)C.off_hi);
    }
  }
}

// =======================================================================================
// grid normalisation: per product k, midpoint sum of U_k over the grid of its observables
// and of U_k * d log(leaf)/d par.  Work unit: a segment of kSeg points along the last grid
// dimension; leaves on the other observables are evaluated once per segment (they are
// constant along it).  The last dimension's coordinates are computed once per block into
// shared memory (double-float in the FP32 path).  Lanes per product: 0 = sum U exp(-a_ref),
// 1 + l*3 + j = sum U d_lj.
// =======================================================================================
constexpr int kSeg = 16;
constexpr int kGridCache = 2048;


template <typename T, int L>
__global__ void __launch_bounds__(kBlock, 2) grid_kernel(ModelDev* md, float2* partials, unsigned* counters) {
  constexpr int NS = 1 + 3 * L;
  const int k = blockIdx.y;
  __shared__ LeafDev s_leaf[L];
  __shared__ T s_xh[kGridCache], s_xl[kGridCache];
  __shared__ ddf s_red[(kBlock / 32) * NS > kBlock ? (kBlock / 32) * NS : kBlock];
  const CompDev& C = md->comp[k];
  const int nleaf = C.n_leaf;
  if (threadIdx.x < L && threadIdx.x < nleaf) s_leaf[threadIdx.x] = md->leaf[k * kMaxLeaf + threadIdx.x];
  const GridDev& G = md->grid[k];
  const int last = G.ndim - 1;
  const int nlast = G.bins[last];
  const bool cached = nlast <= kGridCache;
  if (cached)
    for (int i = threadIdx.x; i < nlast; i += blockDim.x) grid_coord<T>(G, last, i, s_xh[i], s_xl[i]);
  __syncthreads();
  LeafReg<T> lr[L];
  int dimof[L];
#pragma unroll
  for (int l = 0; l < L; ++l) {
    if (l < nleaf) {
      lr[l] = load_leaf<T>(s_leaf[l]);
      dimof[l] = G.dim_of_col[lr[l].col];
    } else {
      lr[l].op = 0;
      lr[l].col = 0;
      dimof[l] = -1;
    }
  }
  const int nseg = (nlast + kSeg - 1) / kSeg;
  int64_t nrows = 1;
  for (int d = 0; d < last; ++d) nrows *= G.bins[d];
  const int64_t units = nrows * nseg;
  int bins_d[kMaxObs];
#pragma unroll
  for (int d = 0; d < kMaxObs; ++d) bins_d[d] = G.bins[d];

  T acc[NS];
  Kahan acc_s;
#pragma unroll
  for (int s = 0; s < NS; ++s) acc[s] = T(0);
  const T aref = (sizeof(T) == 4) ? T(C.a_ref_hi) : T(C.a_ref);
  const T aref_lo = (sizeof(T) == 4) ? T(C.a_ref_lo) : T(0);
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < units; u += (int64_t)gridDim.x * blockDim.x) {
    int64_t row = u / nseg;
    const int seg = (int)(u - row * nseg);
    // coordinates of the other dimensions (at most three)
    T xo0 = T(0), xo1 = T(0), xo2 = T(0), lo0 = T(0), lo1 = T(0), lo2 = T(0);
#pragma unroll
    for (int d = kMaxObs - 2; d >= 0; --d) {
      if (d < last) {
        const int64_t b = bins_d[d];
        const int64_t idx = row % b;
        row /= b;
        T xv, xl;
        grid_coord<T>(G, d, idx, xv, xl);
        if (d == 0) { xo0 = xv; lo0 = xl; }
        if (d == 1) { xo1 = xv; lo1 = xl; }
        if (d == 2) { xo2 = xv; lo2 = xl; }
      }
    }
    // segment-invariant leaves
    T r_row = T(1), a_row = T(0);
    T d_row[L][3];
#pragma unroll
    for (int l = 0; l < L; ++l) {
      d_row[l][0] = d_row[l][1] = d_row[l][2] = T(0);
      if (dimof[l] >= 0 && dimof[l] != last) {
        const int dd = dimof[l];
        const T xv = dd == 0 ? xo0 : (dd == 1 ? xo1 : xo2);
        const T xl = dd == 0 ? lo0 : (dd == 1 ? lo1 : lo2);
        T lr_, la_;
        leaf_eval<true, true>(lr[l], xv, lr_, la_, d_row[l], xl);
        r_row *= lr_;
        a_row += la_;
      }
    }
    a_row = (a_row - aref) - aref_lo;
    T sumU = T(0);
    T dpt[L][3];
#pragma unroll
    for (int l = 0; l < L; ++l) dpt[l][0] = dpt[l][1] = dpt[l][2] = T(0);
    const int i0 = seg * kSeg;
    const int i1 = min(nlast, i0 + kSeg);
    for (int i = i0; i < i1; ++i) {
      T x, xlo;
      if (cached) {
        x = s_xh[i];
        xlo = s_xl[i];
      } else {
        grid_coord<T>(G, last, i, x, xlo);
      }
      T r = r_row, a = a_row;
      T dl[L][3];
#pragma unroll
      for (int l = 0; l < L; ++l) {
        dl[l][0] = dl[l][1] = dl[l][2] = T(0);
        if (dimof[l] == last) {
          T lr_, la_;
          leaf_eval<true, true>(lr[l], x, lr_, la_, dl[l], xlo);
          r *= lr_;
          a += la_;
        }
      }
      T U;
      if constexpr (sizeof(T) == 4) {
        U = r * expf(a);
      } else {
        U = r * exp(a);
      }
      sumU += U;
#pragma unroll
      for (int l = 0; l < L; ++l)
#pragma unroll
        for (int j = 0; j < 3; ++j) dpt[l][j] += U * dl[l][j];
    }
    if constexpr (sizeof(T) == 4) {
      acc_s.add(sumU);
    } else {
      acc[0] += sumU;
    }
#pragma unroll
    for (int l = 0; l < L; ++l)
#pragma unroll
      for (int j = 0; j < 3; ++j) acc[1 + l * 3 + j] += dpt[l][j] + sumU * d_row[l][j];
  }
  ddf v[NS];
  v[0] = (sizeof(T) == 4) ? acc_s.value() : dd_from_double((double)acc[0]);
#pragma unroll
  for (int s = 1; s < NS; ++s) v[s] = (sizeof(T) == 4) ? ddf{(float)acc[s], 0.f} : dd_from_double((double)acc[s]);
  // partials of product k occupy blocks [k * gridDim.x, (k+1) * gridDim.x)
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
      ddf a = s_red[threadIdx.x];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) a = dd_add(a, s_red[w * NS + threadIdx.x]);
      partials[((size_t)k * nbx + blockIdx.x) * NS + threadIdx.x] = make_float2(a.hi, a.lo);
    }
  }
  // last block over the whole launch combines every product
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = atomicAdd(counters, 1u) == (unsigned)(nbx * gridDim.y - 1);
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  __shared__ double s_tot[kMaxComp][NS];
  for (int lane_id = threadIdx.x; lane_id < (int)gridDim.y * NS; lane_id += blockDim.x) {
    const int kk = lane_id / NS, s = lane_id % NS;
    ddf a = {0.f, 0.f};
    for (int b = 0; b < nbx; ++b) {
      float2 p = __ldcg(partials + ((size_t)kk * nbx + b) * NS + s);
      a = dd_add(a, {p.x, p.y});
    }
    s_tot[kk][s] = dd_to_double(a);
  }
  __syncthreads();
  if (threadIdx.x < (int)gridDim.y) {
    const int kk = threadIdx.x;
    CompDev& Ck = md->comp[kk];
    const GridDev& Gk = md->grid[kk];
    const double S = s_tot[kk][0];
    const double aref_used = (sizeof(T) == 4) ? (double)Ck.a_ref_hi + (double)Ck.a_ref_lo : Ck.a_ref;
    const double logN = log(Gk.cell_volume) + aref_used + log(S);
    Ck.log_norm = logN;
    float oh = (float)(-logN);
    Ck.off_hi = oh;
    Ck.off_lo = (float)(-logN - (double)oh);
    for (int p = 0; p < kMaxParams; ++p) md->dlogN[kk][p] = 0.0;
    for (int l = 0; l < Ck.n_leaf && l < L; ++l) {
      const LeafDev& lf = md->leaf[kk * kMaxLeaf + l];
      for (int j = 0; j < 3; ++j)
        if (lf.par[j] >= 0) md->dlogN[kk][lf.par[j]] += s_tot[kk][1 + l * 3 + j] / S;
    }
  }
  if (threadIdx.x == 0) *counters = 0u;
}

// =======================================================================================
// separable grid normalisation: when every leaf of product k acts on its own observable, the
// midpoint sum over product k's grid factorises exactly into one 1-D midpoint sum per leaf,
//   N_k = prod_l h_l exp(a_l) S_l,  S_l = sum_i U_l(x_i) exp(-a_l)  (a_l: reference exponent),
//   d log N_k / d theta = sum_l D_l / S_l,  D_l = sum_i U_l(x_i) exp(-a_l) d log U_l / d theta,
// so the grid costs the sum of the bins instead of their product.  One block per leaf slot
// (blockIdx.x = l, blockIdx.y = k); each leaf is evaluated at its observable's bin centres in
// the path's precision, exactly as in the event kernel, and summed in FP64 in a fixed order;
// the last block to finish combines the products.
// =======================================================================================
template <typename T>
__global__ void __launch_bounds__(kBlock) grid_sep_kernel(ModelDev* md, double* sums, unsigned* counter) {
  grid_dep_launch();  // the event kernel after this one may start its column copies now
  const int k = blockIdx.y, l = blockIdx.x;
  __shared__ double s_red[kBlock / 32][4];
  __shared__ bool s_last;
  const int nleaf = md->comp[k].n_leaf;
  if (l < nleaf) {  // uniform over the block
    const LeafDev& LD = md->leaf[k * kMaxLeaf + l];
    const LeafReg<T> lr = load_leaf<T>(LD);
    const GridDev& G = md->grid[k];
    const int d = G.dim_of_col[lr.col];
    const int nb = G.bins[d];
    const T aref = (sizeof(T) == 4) ? T(LD.a_ref_hi) : T(LD.a_ref);
    const T aref_lo = (sizeof(T) == 4) ? T(LD.a_ref_lo) : T(0);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
      T x, xlo;
      grid_coord<T>(G, d, i, x, xlo);
      T r, a, dl[3];
      leaf_eval<true, true>(lr, x, r, a, dl, xlo);
      T U;
      if constexpr (sizeof(T) == 4) U = r * expf((a - aref) - aref_lo);
      else U = r * exp(a - aref);
      const double u = (double)U;
      acc[0] += u;
#pragma unroll
      for (int j = 0; j < 3; ++j) acc[1 + j] += u * (double)dl[j];
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
      for (int m = 16; m > 0; m >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], m);
    if ((threadIdx.x & 31) == 0)
#pragma unroll
      for (int j = 0; j < 4; ++j) s_red[threadIdx.x >> 5][j] = acc[j];
    __syncthreads();
    // per leaf, in parallel over the blocks: log(h S) + a_ref and D_j / S
    if (threadIdx.x < 4) {
      double S = 0.0, t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        S += s_red[w][0];
        t += s_red[w][threadIdx.x];
      }
      const double aref_used = (sizeof(T) == 4) ? (double)LD.a_ref_hi + (double)LD.a_ref_lo : LD.a_ref;
      sums[(k * kMaxLeaf + l) * 4 + threadIdx.x] = threadIdx.x == 0 ? log(G.h64[d] * S) + aref_used : t / S;
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(counter, 1u) == gridDim.x * gridDim.y - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // last block: log N_k = sum over leaves; d log N_k / d theta scattered to parameters in
  // shared memory (leaves may share a parameter), then written out in parallel
  __shared__ double s_dlogN[kMaxComp][kMaxParams];
  __shared__ double s_term[kMaxComp * kMaxLeaf * 4];
  __shared__ int s_par[kMaxComp * kMaxLeaf][3];
  const int nK = gridDim.y, P = md->n_params;
  for (int t = threadIdx.x; t < kMaxComp * kMaxParams; t += blockDim.x) s_dlogN[t / kMaxParams][t % kMaxParams] = 0.0;
  for (int t = threadIdx.x; t < nK * kMaxLeaf * 4; t += blockDim.x) s_term[t] = __ldcg(sums + t);
  for (int t = threadIdx.x; t < nK * kMaxLeaf * 3; t += blockDim.x)
    s_par[t / 3][t % 3] = (t / 3) % kMaxLeaf < md->comp[t / 3 / kMaxLeaf].n_leaf ? md->leaf[t / 3].par[t % 3] : -1;
  __syncthreads();
  if (threadIdx.x < nK) {
    const int kk = threadIdx.x;
    const int nl = md->comp[kk].n_leaf;
    double logN = 0.0;
    for (int ll = 0; ll < nl; ++ll) {
      const int slot = kk * kMaxLeaf + ll;
      logN += s_term[slot * 4];
      for (int j = 0; j < 3; ++j)
        if (s_par[slot][j] >= 0) s_dlogN[kk][s_par[slot][j]] += s_term[slot * 4 + 1 + j];
    }
    CompDev& Ck = md->comp[kk];
    Ck.log_norm = logN;
    const float oh = (float)(-logN);
    Ck.off_hi = oh;
    Ck.off_lo = (float)(-logN - (double)oh);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nK * P; t += blockDim.x) md->dlogN[t / P][t % P] = s_dlogN[t / P][t % P];
  if (threadIdx.x == 0) *counter = 0u;
}

// =======================================================================================
// per-event log f (no reduction): the product of the same evaluation as sop_event_kernel
// =======================================================================================
template <typename T, int K, int L>
__global__ void __launch_bounds__(kBlock) sop_logf_kernel(const ModelDev* __restrict__ md, const EvConst<T, K, L> P,
                                                          Cols<T> cols, int64_t n, double* __restrict__ logf) {
  T off_hi[K], off_lo[K];
  load_offsets<T, K>(md, off_hi, off_lo);
  const int nobs = P.nobs;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const T x0 = cols.c[0][i];
    const T x1 = nobs > 1 ? cols.c[1][i] : T(0);
    const T x2 = nobs > 2 ? cols.c[2][i] : T(0);
    const T x3 = nobs > 3 ? cols.c[3][i] : T(0);
    T lf, ck[K], dk[K][L][3];
    const bool ok = eval_event<T, K, L, false>(P, off_hi, off_lo, x0, x1, x2, x3, lf, ck, dk);
    logf[i] = ok ? (double)lf : -HUGE_VAL;
  }
}

// =======================================================================================
// host side
// =======================================================================================
struct Term {
  std::vector<int> leaves;                 // node ids
  std::vector<std::pair<int, int>> facs;   // (add index, child position)
};

static int flatten(const goo_node* nodes, int id, std::vector<int>& add_ids, std::vector<Term>& out) {
  const goo_node& n = nodes[id];
  out.clear();
  switch (n.op) {
    case GOO_OP_GAUSS:
    case GOO_OP_EXPO:
    case GOO_OP_POLY2:
    case GOO_OP_ARGUS: {
      Term t;
      t.leaves.push_back(id);
      out.push_back(t);
      return GOO_OK;
    }
    case GOO_OP_PROD: {
      std::vector<Term> acc(1);
      for (int c = 0; c < n.n_child; ++c) {
        std::vector<Term> sub;
        GOO_TRY(flatten(nodes, n.child[c], add_ids, sub));
        std::vector<Term> next;
        for (auto& a : acc)
          for (auto& b : sub) {
            Term t = a;
            t.leaves.insert(t.leaves.end(), b.leaves.begin(), b.leaves.end());
            t.facs.insert(t.facs.end(), b.facs.begin(), b.facs.end());
            next.push_back(t);
          }
        acc.swap(next);
      }
      out = acc;
      return GOO_OK;
    }
    case GOO_OP_ADD: {
      const int ai = (int)add_ids.size();
      add_ids.push_back(id);
      for (int c = 0; c < n.n_child; ++c) {
        std::vector<Term> sub;
        GOO_TRY(flatten(nodes, n.child[c], add_ids, sub));
        for (auto& t : sub) {
          t.facs.push_back({ai, c});
          out.push_back(t);
        }
      }
      return GOO_OK;
    }
    default:
      return set_error(GOO_ERR_ARG, "goo_model_build: node %d has op %d, not allowed in a sum/product tree", id, n.op);
  }
}

static int leaf_npar(int op) {
  switch (op) {
    case GOO_OP_GAUSS: return 2;
    case GOO_OP_EXPO: return 1;
    case GOO_OP_POLY2: return 2;
    case GOO_OP_ARGUS: return 3;
  }
  return 0;
}

int build_sop_model(goo_ctx* ctx, const goo_node* nodes, int n_nodes, int n_params, int n_obs,
                    const double* lo, const double* hi, goo_model* m) {
  if (n_obs > kMaxObs)
    return set_error(GOO_ERR_UNSUPPORTED, "goo_model_build: a sum/product model has at most %d observables", kMaxObs);
  std::vector<int> add_ids;
  std::vector<Term> terms;
  GOO_TRY(flatten(nodes, n_nodes - 1, add_ids, terms));
  if ((int)terms.size() > kMaxComp)
    return set_error(GOO_ERR_UNSUPPORTED, "goo_model_build: %zu products after flattening (max %d)", terms.size(), kMaxComp);
  if ((int)add_ids.size() > kMaxAdd)
    return set_error(GOO_ERR_UNSUPPORTED, "goo_model_build: %zu ADD nodes (max %d)", add_ids.size(), kMaxAdd);
  ModelDev& h = m->host;
  std::memset(&h, 0, sizeof h);
  h.nK = (int)terms.size();
  h.n_obs = n_obs;
  h.n_params = n_params;
  h.norm_kind = GOO_NORM_ANALYTIC;
  for (int o = 0; o < n_obs; ++o) {
    h.lo[o] = lo[o];
    h.hi[o] = hi[o];
  }
  for (size_t a = 0; a < add_ids.size(); ++a) {
    const goo_node& n = nodes[add_ids[a]];
    if (n.n_child < 2 || n.n_child > GOO_MAX_CHILD)
      return set_error(GOO_ERR_ARG, "goo_model_build: ADD node %d has %d children", add_ids[a], n.n_child);
    h.add[a].n_child = n.n_child;
    for (int j = 0; j < n.n_child - 1; ++j) {
      int p = n.par[j];
      if (j >= 8 || p < 0 || p >= n_params)
        return set_error(GOO_ERR_ARG, "goo_model_build: ADD node %d fraction %d has parameter %d", add_ids[a], j, p);
      h.add[a].frac[j] = p;
    }
  }
  h.n_add = (int)add_ids.size();
  int max_leaf = 0;
  for (int k = 0; k < h.nK; ++k) {
    const Term& t = terms[k];
    if ((int)t.leaves.size() > kMaxLeaf)
      return set_error(GOO_ERR_UNSUPPORTED, "goo_model_build: product %d has %zu leaves (max %d)", k, t.leaves.size(), kMaxLeaf);
    if ((int)t.facs.size() > 8) return set_error(GOO_ERR_UNSUPPORTED, "goo_model_build: ADD nesting deeper than 8");
    CompDev& C = h.comp[k];
    C.n_leaf = (int)t.leaves.size();
    max_leaf = C.n_leaf > max_leaf ? C.n_leaf : max_leaf;
    C.n_fac = (int)t.facs.size();
    for (int f = 0; f < C.n_fac; ++f) {
      C.fac_add[f] = t.facs[f].first;
      C.fac_pos[f] = t.facs[f].second;
    }
    for (int l = 0; l < C.n_leaf; ++l) {
      const goo_node& n = nodes[t.leaves[l]];
      LeafDev& L = h.leaf[k * kMaxLeaf + l];
      L.op = n.op;
      L.col = n.obs[0];
      if (L.col < 0 || L.col >= n_obs)
        return set_error(GOO_ERR_ARG, "goo_model_build: leaf node %d uses observable %d of %d", t.leaves[l], L.col, n_obs);
      for (int j = 0; j < 3; ++j) L.par[j] = -1;
      for (int j = 0; j < leaf_npar(n.op); ++j) {
        if (n.par[j] < 0 || n.par[j] >= n_params)
          return set_error(GOO_ERR_ARG, "goo_model_build: leaf node %d parameter slot %d = %d", t.leaves[l], j, n.par[j]);
        L.par[j] = n.par[j];
      }
    }
  }
  m->max_leaf = max_leaf;
  m->kind = 0;
  if (cudaMalloc(&m->dev, sizeof(ModelDev)) != cudaSuccess || cudaMallocHost(&m->stage, sizeof(ModelDev)) != cudaSuccess) {
    cudaGetLastError();
    return set_error(GOO_ERR_OOM, "goo_model_build: cannot allocate model block");
  }
  GOO_CUDA_TRY(cudaMemcpyAsync(m->dev, &h, sizeof(ModelDev), cudaMemcpyHostToDevice, ctx->stream));
  GOO_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return GOO_OK;
}

// True when every product's leaves act on distinct observables (the grid sum factorises).
static int grid_separable(const ModelDev& h) {
  for (int k = 0; k < h.nK; ++k)
    for (int l = 0; l < h.comp[k].n_leaf; ++l)
      for (int l2 = 0; l2 < l; ++l2)
        if (h.leaf[k * kMaxLeaf + l2].col == h.leaf[k * kMaxLeaf + l].col) return 0;
  return 1;
}

int sop_set_norm(goo_model* m, const goo_norm_spec* spec) {
  ModelDev& h = m->host;
  if (spec->kind == GOO_NORM_ANALYTIC) {
    for (int k = 0; k < h.nK; ++k)
      for (int l = 0; l < h.comp[k].n_leaf; ++l) {
        const LeafDev& L = h.leaf[k * kMaxLeaf + l];
        if (L.op == GOO_OP_ARGUS)
          return set_error(GOO_ERR_UNSUPPORTED, "goo_model_set_norm: the Argus shape has no closed-form integral; use GOO_NORM_GRID");
        for (int l2 = 0; l2 < l; ++l2)
          if (h.leaf[k * kMaxLeaf + l2].col == L.col)
            return set_error(GOO_ERR_UNSUPPORTED,
                             "goo_model_set_norm: product %d has two leaves on observable %d; use GOO_NORM_GRID", k, L.col);
      }
  } else if (spec->kind == GOO_NORM_GRID) {
    for (int o = 0; o < h.n_obs; ++o)
      if (spec->bins[o] < 1 || spec->bins[o] > (1 << 20))
        return set_error(GOO_ERR_ARG, "goo_model_set_norm: bins[%d] = %d", o, spec->bins[o]);
    for (int k = 0; k < h.nK; ++k) {
      GridDev& G = h.grid[k];
      std::memset(&G, 0, sizeof G);
      bool used[kMaxObs] = {false, false, false, false};
      for (int l = 0; l < h.comp[k].n_leaf; ++l) used[h.leaf[k * kMaxLeaf + l].col] = true;
      for (int o = 0; o < kMaxObs; ++o) G.dim_of_col[o] = -1;
      G.cell_volume = 1.0;
      for (int o = 0; o < h.n_obs; ++o) {
        if (!used[o]) continue;
        const int d = G.ndim++;
        G.dim_of_col[o] = d;
        G.bins[d] = spec->bins[o];
        const double step = (h.hi[o] - h.lo[o]) / spec->bins[o];
        G.h64[d] = step;
        G.lo64[d] = h.lo[o];
        float hh = (float)step;
        G.h_hi[d] = hh;
        G.h_lo[d] = (float)(step - (double)hh);
        float lh = (float)h.lo[o];
        G.lo_hi[d] = lh;
        G.lo_lo[d] = (float)(h.lo[o] - (double)lh);
        G.cell_volume *= step;
      }
    }
  } else {
    return set_error(GOO_ERR_UNSUPPORTED, "goo_model_set_norm: MC normalisation needs an amplitude model");
  }
  h.norm_kind = spec->kind;
  h.grid_separable = spec->kind == GOO_NORM_GRID ? grid_separable(h) : 0;
  m->norm = *spec;
  goo_ctx* ctx = m->ctx;
  GOO_CUDA_TRY(cudaMemcpyAsync(m->dev, &h, sizeof(ModelDev), cudaMemcpyHostToDevice, ctx->stream));
  GOO_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return GOO_OK;
}

// ---------------------------------------------------------------------------------------
// launches
// ---------------------------------------------------------------------------------------
template <typename KernelT>
static int blocks_per_sm(KernelT kernel, int* cache) {
  if (*cache > 0) return *cache;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, kBlock, 0) != cudaSuccess || n < 1) {
    cudaGetLastError();
    n = 1;
  }
  *cache = n;
  return n;
}

template <typename T>
static int launch_grid_sep(goo_model* m) {
  goo_ctx* ctx = m->ctx;
  // the per-leaf sums (4 doubles per leaf slot) live in the partials scratch
  GOO_TRY(ensure_partials(ctx, (size_t)kMaxComp * kMaxLeaf * 4));
  {
    LaunchScope ls(ctx, sizeof(T) == 4 ? "grid_norm_f32" : "grid_norm_f64");
    grid_sep_kernel<T><<<dim3(m->max_leaf, m->host.nK), kBlock, 0, ctx->stream>>>(
        m->dev, (double*)ctx->scratch.partials, ctx->scratch.counters);
  }
  GOO_CUDA_TRY(cudaGetLastError());
  return GOO_OK;
}

template <typename T, int L>
static int launch_grid_T(goo_model* m) {
  goo_ctx* ctx = m->ctx;
  static int occ = 0;
  const int bps = blocks_per_sm(grid_kernel<T, L>, &occ);
  const ModelDev& h = m->host;
  int64_t units_max = 1;
  for (int k = 0; k < h.nK; ++k) {
    const GridDev& G = h.grid[k];
    int64_t rows = 1;
    for (int d = 0; d < G.ndim - 1; ++d) rows *= G.bins[d];
    int64_t u = rows * ((G.bins[G.ndim - 1] + kSeg - 1) / kSeg);
    units_max = u > units_max ? u : units_max;
  }
  int64_t need = (units_max + kBlock - 1) / kBlock;
  int64_t cap = ((int64_t)ctx->num_sms * bps + h.nK - 1) / h.nK;
  const int nbx = (int)(need < cap ? (need < 1 ? 1 : need) : cap);
  constexpr int NS = 1 + 3 * L;
  GOO_TRY(ensure_partials(ctx, (size_t)nbx * h.nK * NS));
  dim3 grid(nbx, h.nK);
  {
    LaunchScope ls(ctx, sizeof(T) == 4 ? "grid_norm_f32" : "grid_norm_f64");
    grid_kernel<T, L><<<grid, kBlock, 0, ctx->stream>>>(m->dev, ctx->scratch.partials, ctx->scratch.counters);
  }
  GOO_CUDA_TRY(cudaGetLastError());
  return GOO_OK;
}

// Largest number of 1-D grid bins (summed over the leaves) normalised inside the event kernel.
constexpr int kFusedNormBins = 4096;

bool sop_norm_in_event(const goo_model* m, int precision, bool grad) {
  const ModelDev& h = m->host;
  if (precision != GOO_F32 || h.norm_kind != GOO_NORM_GRID || !h.grid_separable) return false;
  if (grad && !(h.nK <= 2 && m->max_leaf <= 3)) return false;  // the scalar kernel takes that shape
  int64_t bins = 0;
  for (int k = 0; k < h.nK; ++k)
    for (int l = 0; l < h.comp[k].n_leaf; ++l) {
      const GridDev& G = h.grid[k];
      bins += G.bins[G.dim_of_col[h.leaf[k * kMaxLeaf + l].col]];
    }
  return bins <= kFusedNormBins;
}

int sop_prepare(goo_model* m, const double* theta_host, int precision, bool norm_in_event) {
  goo_ctx* ctx = m->ctx;
  ModelDev* stage = m->stage;
  *stage = m->host;
  host_prep(*stage, theta_host, precision);
  // the self-contained event kernel (sop_norm_in_event) takes its constants by value and reads
  // no model block: nothing to upload
  if (norm_in_event) return GOO_OK;
  GOO_CUDA_TRY(cudaMemcpyAsync(m->dev, stage, sizeof(ModelDev), cudaMemcpyHostToDevice, ctx->stream));
  if (m->host.norm_kind == GOO_NORM_GRID && m->host.grid_separable) {
    GOO_TRY((precision == GOO_F32 ? launch_grid_sep<float>(m) : launch_grid_sep<double>(m)));
  } else if (m->host.norm_kind == GOO_NORM_GRID) {
    if (precision == GOO_F32) {
      GOO_TRY((m->max_leaf <= 2 ? launch_grid_T<float, 2>(m)
                                : (m->max_leaf <= 3 ? launch_grid_T<float, 3>(m) : launch_grid_T<float, 4>(m))));
    } else {
      GOO_TRY((m->max_leaf <= 2 ? launch_grid_T<double, 2>(m)
                                : (m->max_leaf <= 3 ? launch_grid_T<double, 3>(m) : launch_grid_T<double, 4>(m))));
    }
  }
  return GOO_OK;
}

// Event-kernel constants from a prepared model block (host_prep already applied).
template <typename T, int K, int L>
static EvConst<T, K, L> make_evconst(const ModelDev& h) {
  EvConst<T, K, L> P;
  std::memset(&P, 0, sizeof P);
  P.nK = h.nK;
  P.nobs = h.n_obs;
  for (int k = 0; k < K; ++k) {
    if (k < h.nK) {
      const CompDev& C = h.comp[k];
      P.w_hi[k] = (sizeof(T) == 4) ? (T)C.w_hi : (T)C.w;
      P.w_lo[k] = (sizeof(T) == 4) ? (T)C.w_lo : T(0);
    }
    for (int l = 0; l < L; ++l) {
      LeafReg<T>& R = P.leaf[k][l];
      if (k >= h.nK || l >= h.comp[k].n_leaf) continue;  // opcode 0: value 1, no derivative
      const LeafDev& LD = h.leaf[k * kMaxLeaf + l];
      R.op = LD.op;
      R.col = LD.col;
      for (int j = 0; j < 6; ++j) R.c[j] = (sizeof(T) == 4) ? (T)LD.f[j] : (T)LD.d[j];
      // base-2 rates of the pair kernel, from the float constants the other leaves' terms use
      constexpr double kLog2e = 1.4426950408889634074;
      if (LD.op == GOO_OP_EXPO) P.b2[k][l] = (float)((double)LD.f[0] * kLog2e);
      if (LD.op == GOO_OP_ARGUS) P.b2[k][l] = (float)((double)LD.f[3] * kLog2e);
    }
  }
  return P;
}

template <typename T, int K, int L, bool GRAD>
static int launch_event_T(goo_model* m, const goo_dataset* ds, int64_t begin, int64_t end, int out_mode,
                          double* result) {
  const T* wcol = sizeof(T) == 4 ? (const T*)(const void*)ds->w32 : (const T*)(const void*)ds->w64;
  goo_ctx* ctx = m->ctx;
  static int occ = 0;
  const int bps = blocks_per_sm(sop_event_kernel<T, K, L, GRAD>, &occ);
  const int nb = grid_blocks(ctx, end - begin, bps);
  constexpr int NS = EventLanes<T, K, L, GRAD>::NS;
  GOO_TRY(ensure_partials(ctx, (size_t)nb * NS));
  Cols<T> cols{};
  for (int c = 0; c < kMaxObs; ++c) {
    if (sizeof(T) == 4) cols.c[c] = (const T*)(c < ds->ncols ? (const void*)ds->d32[c] : (const void*)ds->d32[0]);
    else cols.c[c] = (const T*)(c < ds->ncols ? (const void*)ds->d64[c] : (const void*)ds->d64[0]);
  }
  {
    LaunchScope ls(ctx, sizeof(T) == 4 ? (GRAD ? "sop_nll_grad_f32" : "sop_nll_f32") : (GRAD ? "sop_nll_grad_f64" : "sop_nll_f64"));
    sop_event_kernel<T, K, L, GRAD><<<nb, kBlock, 0, ctx->stream>>>(m->dev, make_evconst<T, K, L>(*m->stage), cols,
                                                                   begin, end, ctx->scratch.partials,
                                                                   ctx->scratch.counters, result, out_mode, wcol);
  }
  GOO_CUDA_TRY(cudaGetLastError());
  return GOO_OK;
}

constexpr int kMaxDevicesEv = 64;

// By-value constants of the self-contained event kernel from a prepared model block.
template <int K, int L, bool GRAD>
static EvNorm<K, L, GRAD> make_evnorm(const ModelDev& h) {
  EvNorm<K, L, GRAD> N;
  std::memset(&N, 0, sizeof N);
  for (int k = 0; k < K; ++k) {
    N.w[k] = k < h.nK ? h.comp[k].w : 0.0;
    for (int l = 0; l < L; ++l) {
      const int sl = k * L + l;
      for (int j = 0; j < 3; ++j) N.par[k][l][j] = -1;
      if (k >= h.nK || l >= h.comp[k].n_leaf) continue;
      const LeafDev& LD = h.leaf[k * kMaxLeaf + l];
      const GridDev& G = h.grid[k];
      const int d = G.dim_of_col[LD.col];
      N.nb[sl] = G.bins[d];
      N.lo_hi[sl] = G.lo_hi[d];
      N.lo_lo[sl] = G.lo_lo[d];
      N.h_hi[sl] = G.h_hi[d];
      N.h_lo[sl] = G.h_lo[d];
      N.h64[sl] = G.h64[d];
      N.aref_hi[sl] = LD.a_ref_hi;
      N.aref_lo[sl] = LD.a_ref_lo;
      for (int j = 0; j < 3; ++j) N.par[k][l][j] = (signed char)LD.par[j];
    }
  }
  N.n_params = h.n_params;
  if constexpr (GRAD)
    for (int k = 0; k < K && k < h.nK; ++k)
      for (int p = 0; p < h.n_params; ++p) N.dw[k][p] = h.dw[k][p];
  return N;
}

template <int K, int L, bool GRAD>
static int launch_event2(goo_model* m, const goo_dataset* ds, int64_t begin, int64_t end, int out_mode,
                         bool fused_norm, double* result) {
  goo_ctx* ctx = m->ctx;
  constexpr int TE = 2 * kPairsPerThread * kBlock;
  // the column tiles, and room for the final block reduction (event_finish_fused), which reuses
  // the tile buffers: every lane of every thread as a double-float
  constexpr size_t red_bytes = (size_t)EventLanes<float, K, L, GRAD>::NS * kBlock * sizeof(ddf);
  const size_t smem = std::max((size_t)kEventStages * m->host.n_obs * TE * sizeof(float), red_bytes);
  // room for the largest column count, so one setting serves every model on this device
  const size_t smem_max = std::max((size_t)kEventStages * kMaxObs * TE * sizeof(float), red_bytes);
  static bool configured[kMaxDevicesEv][2] = {};
  if (ctx->device < 0 || ctx->device >= kMaxDevicesEv) return set_error(GOO_ERR_ARG, "device %d", ctx->device);
  // the kernel for this model, gradient form and column source, resolved on its first
  // evaluation: the one specialised for the model's leaf signature (jit.cu), else the
  // interpreter; host columns (GOO_BORROW_HOST) take the direct-read instantiation
  const bool direct = ds->host_borrowed;
  const int gi = (GRAD ? 1 : 0) + (direct ? 2 : 0);
  if (!m->ev2_fn[gi]) {
    const void* interp = direct ? (const void*)sop_event2_kernel<K, L, GRAD, 0, 0, true>
                                : (const void*)sop_event2_kernel<K, L, GRAD>;
    const void* fn = interp;
    int st = m->jit_mode;
    if (m->jit_mode) {
      unsigned long long sig = 0, colmap = 0;
      for (int k = 0; k < m->host.nK && k < K; ++k)
        for (int l = 0; l < m->host.comp[k].n_leaf && l < L; ++l) {
          const LeafDev& LD = m->host.leaf[k * kMaxLeaf + l];
          sig |= (unsigned long long)(LD.op & 15) << (4 * (k * L + l));
          colmap |= (unsigned long long)(LD.col & 3) << (2 * (k * L + l));
        }
      const void* jf = jit_event2_kernel(ctx->device, K, L, GRAD, sig, colmap, direct, smem_max, &st);
      if (jf) fn = jf;
    }
    if (fn == interp && !configured[ctx->device][direct ? 1 : 0]) {
      GOO_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max));
      configured[ctx->device][direct ? 1 : 0] = true;
    }
    m->ev2_fn[gi] = fn;
    m->ev2_status[gi] = st;
  }
  const void* fn = m->ev2_fn[gi];
  m->jit_status = m->ev2_status[gi];
  const int bps = cached_occupancy(fn, ctx->device, kBlock, smem);
  // every block takes an equal contiguous share of the events (sop_event2_kernel), at most
  // one tile's worth when the range is small
  const int64_t tiles = (end - begin + TE - 1) / TE;
  const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)ctx->num_sms * bps));
  constexpr int NS = EventLanes<float, K, L, GRAD>::NS;
  GOO_TRY(ensure_partials(ctx, (size_t)nb * NS));
  Cols<float> cols{};
  for (int c = 0; c < kMaxObs; ++c) cols.c[c] = ds->d32[c < ds->ncols ? c : 0];
  if (ds->host_borrowed) {
    // read over the host link by the kernel itself, each value checked against the float
    // limits that admit exactly the float values inside the double limits
    for (int c = 0; c < kMaxObs && c < ds->ncols; ++c) {
      float lo = (float)ds->lo[c], hi = (float)ds->hi[c];
      if ((double)lo < ds->lo[c]) lo = std::nextafter(lo, HUGE_VALF);
      if ((double)hi > ds->hi[c]) hi = std::nextafter(hi, -HUGE_VALF);
      cols.lo[c] = lo;
      cols.hi[c] = hi;
    }
  }
  {
    // programmatic dependent launch after a normalisation kernel: the kernel's blocks start
    // (and put their first column tiles in flight) while that kernel finishes.  A kernel that
    // normalises the grid itself depends on no kernel's output but the previous evaluation's
    // counters, which plain stream order covers: it launches without the attribute, since its
    // in-kernel dependency wait cost microseconds per evaluation.
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nb);
    cfg.blockDim = dim3(kBlock);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = fused_norm ? 0 : 1;
    LaunchScope ls(ctx, GRAD ? "sop_nll_grad_f32" : "sop_nll_f32");
    EvNorm<K, L, GRAD> N;
    if (fused_norm) N = make_evnorm<K, L, GRAD>(*m->stage);
    else std::memset(&N, 0, sizeof N);
    // the argument list of sop_event2_kernel, for the interpreter and the specialised kernel
    const ModelDev* md = m->dev;
    EvConst<float, K, L> P = make_evconst<float, K, L>(*m->stage);
    float2* partials = ctx->scratch.partials;
    unsigned* counters = ctx->scratch.counters;
    int fused = (int)fused_norm;
    void* args[] = {&md, &P, &N, &cols, &begin, &end, &partials, &counters, &result, &out_mode, &fused};
    GOO_CUDA_TRY(cudaLaunchKernelExC(&cfg, fn, args));
  }
  GOO_CUDA_TRY(cudaGetLastError());
  return GOO_OK;
}

template <typename T, bool GRAD>
static int launch_event_sel(goo_model* m, const goo_dataset* ds, int64_t begin, int64_t end, int out_mode,
                            bool fused_norm, double* result) {
  if constexpr (sizeof(T) == 4) {
    // packed pairs, except the largest shape with gradient lanes (its pair accumulators do
    // not fit in registers) and weighted datasets (the scalar kernel carries the weights)
    if (!ds->w32) {
      if (m->host.nK <= 2 && m->max_leaf <= 3)
        return launch_event2<2, 3, GRAD>(m, ds, begin, end, out_mode, fused_norm, result);
      if constexpr (!GRAD) return launch_event2<4, 4, GRAD>(m, ds, begin, end, out_mode, fused_norm, result);
    }
  }
  if (ds->host_borrowed)
    return set_error(GOO_ERR_UNSUPPORTED, "a GOO_BORROW_HOST dataset is read by the packed-pair FP32 kernel only "
                                          "(at most 2 products of 3 leaves with the gradient, 4 of 4 without)");
  if (fused_norm) return set_error(GOO_ERR_STATE, "sop_events: in-kernel normalisation needs the pair kernel");
  if (m->host.nK <= 2 && m->max_leaf <= 3) return launch_event_T<T, 2, 3, GRAD>(m, ds, begin, end, out_mode, result);
  return launch_event_T<T, 4, 4, GRAD>(m, ds, begin, end, out_mode, result);
}

int sop_events(goo_model* m, const goo_dataset* ds, int64_t begin, int64_t end, int precision, bool grad, int out_mode,
               bool norm_in_event, double* result) {
  if (!result) result = m->ctx->scratch.result;
  if (end <= begin) {
    // empty range: write a zero result without a kernel
    double z[3 + kMaxParams] = {0};
    GOO_CUDA_TRY(cudaMemcpyAsync(m->ctx->scratch.result, z, sizeof z, cudaMemcpyHostToDevice, m->ctx->stream));
    return GOO_OK;
  }
  if (precision == GOO_F32) {
    return grad ? launch_event_sel<float, true>(m, ds, begin, end, out_mode, norm_in_event, result)
                : launch_event_sel<float, false>(m, ds, begin, end, out_mode, norm_in_event, result);
  }
  if (norm_in_event) return set_error(GOO_ERR_STATE, "sop_events: in-kernel normalisation is FP32 only");
  return grad ? launch_event_sel<double, true>(m, ds, begin, end, out_mode, false, result)
              : launch_event_sel<double, false>(m, ds, begin, end, out_mode, false, result);
}

template <typename T, int K, int L>
static int launch_logf_T(goo_model* m, const goo_dataset* ds, double* logf_dev) {
  goo_ctx* ctx = m->ctx;
  Cols<T> cols{};
  for (int c = 0; c < kMaxObs; ++c) {
    if (sizeof(T) == 4) cols.c[c] = (const T*)(c < ds->ncols ? (const void*)ds->d32[c] : (const void*)ds->d32[0]);
    else cols.c[c] = (const T*)(c < ds->ncols ? (const void*)ds->d64[c] : (const void*)ds->d64[0]);
  }
  const int nb = grid_blocks(ctx, ds->n, 4);
  {
    LaunchScope ls(ctx, "sop_logf");
    sop_logf_kernel<T, K, L><<<nb, kBlock, 0, ctx->stream>>>(m->dev, make_evconst<T, K, L>(*m->stage), cols, ds->n,
                                                             logf_dev);
  }
  GOO_CUDA_TRY(cudaGetLastError());
  return GOO_OK;
}

int sop_eval_logf(goo_model* m, const goo_dataset* ds, int precision, double* logf_dev) {
  if (ds->n == 0) return GOO_OK;
  if (precision == GOO_F32)
    return (m->host.nK <= 2 && m->max_leaf <= 3) ? launch_logf_T<float, 2, 3>(m, ds, logf_dev)
                                                 : launch_logf_T<float, 4, 4>(m, ds, logf_dev);
  return (m->host.nK <= 2 && m->max_leaf <= 3) ? launch_logf_T<double, 2, 3>(m, ds, logf_dev)
                                               : launch_logf_T<double, 4, 4>(m, ds, logf_dev);
}

}  // namespace goo

// =======================================================================================
// goo_nll_grad_static: the sum/product likelihood without any device allocation
//
// For callers that cannot call cudaMalloc: code that runs where another component owns
// all device memory (an application-level pool or a framework allocator that forbids side
// allocations), or where the implicit device synchronisation and latency of cudaMalloc /
// cudaFree cannot be paid on every call.  The caller passes the model description (host),
// its device event columns and host outputs; everything else -- the model block, theta,
// the reduction partials, counters and the result record -- lives in one file-scope
// device array of fixed size.
// =======================================================================================
namespace goo {

constexpr size_t kStaticScratchBytes = size_t(1) << 20;  // 1 MiB per device that loads the library
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Layout of the array: the model block (theta reaches the kernels through it and through
// their by-value constants), the counters, the result record, then the reduction partials.
constexpr size_t kStOffModel = 0;
constexpr size_t kStOffCounters = (sizeof(ModelDev) + 255) / 256 * 256;
constexpr size_t kStOffResult = kStOffCounters + 256;
constexpr size_t kStOffPartials = kStOffResult + (kResultDoubles + 1 + 1) / 2 * 2 * sizeof(double);
constexpr int kStaticMaxParams = 32;  // documented limit of goo_nll_grad_static
constexpr size_t kStPartialsCap = (kStaticScratchBytes - kStOffPartials) / sizeof(float2);
static_assert(kStOffPartials < kStaticScratchBytes, "static scratch too small for the model block");

// With the caller's device current: the device address of the scratch array and the SM
// count.  Looked up on every call (neither query allocates), so nothing is cached across a
// cudaDeviceReset or a new primary context, and concurrent host threads share no host state.
static int static_scratch_lookup(int dev, unsigned char** base, int* sms) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess) return set_error(GOO_ERR_CUDA, "goo_nll_grad_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
  e = cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return set_error(GOO_ERR_CUDA, "goo_nll_grad_static: %s", cudaGetErrorString(e));
  *base = (unsigned char*)p;
  return GOO_OK;
}

// Host plan of a two-level model (leaf | PROD of leaves | ADD of leaves / PRODs), written
// into a caller-stack ModelDev without heap use.
static int static_plan(const goo_node* nodes, int n_nodes, int n_params, int n_obs, const double* lo, const double* hi,
                       const goo_norm_spec* norm, ModelDev& h) {
  std::memset(&h, 0, sizeof h);
  h.n_obs = n_obs;
  h.n_params = n_params;
  for (int o = 0; o < n_obs; ++o) {
    h.lo[o] = lo[o];
    h.hi[o] = hi[o];
  }
  const goo_node& root = nodes[n_nodes - 1];
  int comps[kMaxComp];
  int nK = 0;
  if (root.op == GOO_OP_ADD) {
    if (root.n_child < 2 || root.n_child > kMaxComp)
      return set_error(GOO_ERR_UNSUPPORTED, "goo_nll_grad_static: ADD with %d children (2..%d)", root.n_child, kMaxComp);
    for (int c = 0; c < root.n_child; ++c) comps[nK++] = root.child[c];
    h.n_add = 1;
    h.add[0].n_child = root.n_child;
    for (int j = 0; j < root.n_child - 1; ++j) {
      if (root.par[j] < 0 || root.par[j] >= n_params)
        return set_error(GOO_ERR_ARG, "goo_nll_grad_static: fraction %d has parameter %d", j, root.par[j]);
      h.add[0].frac[j] = root.par[j];
    }
  } else {
    comps[nK++] = n_nodes - 1;
  }
  h.nK = nK;
  for (int k = 0; k < nK; ++k) {
    const goo_node& cn = nodes[comps[k]];
    int leaves[kMaxLeaf];
    int nl = 0;
    if (cn.op == GOO_OP_PROD) {
      if (cn.n_child < 1 || cn.n_child > kMaxLeaf)
        return set_error(GOO_ERR_UNSUPPORTED, "goo_nll_grad_static: product with %d factors (1..%d)", cn.n_child, kMaxLeaf);
      for (int c = 0; c < cn.n_child; ++c) leaves[nl++] = cn.child[c];
    } else {
      leaves[nl++] = comps[k];
    }
    CompDev& C = h.comp[k];
    C.n_leaf = nl;
    if (root.op == GOO_OP_ADD) {
      C.n_fac = 1;
      C.fac_add[0] = 0;
      C.fac_pos[0] = k;
    }
    for (int l = 0; l < nl; ++l) {
      const goo_node& n = nodes[leaves[l]];
      if (n.op < GOO_OP_GAUSS || n.op > GOO_OP_ARGUS)
        return set_error(GOO_ERR_UNSUPPORTED, "goo_nll_grad_static: node %d (op %d) is not a leaf of a two-level "
                         "sum of products", leaves[l], n.op);
      LeafDev& L = h.leaf[k * kMaxLeaf + l];
      L.op = n.op;
      L.col = n.obs[0];
      if (L.col < 0 || L.col >= n_obs) return set_error(GOO_ERR_ARG, "goo_nll_grad_static: observable %d", L.col);
      for (int j = 0; j < 3; ++j) L.par[j] = -1;
      for (int j = 0; j < leaf_npar(n.op); ++j) {
        if (n.par[j] < 0 || n.par[j] >= n_params)
          return set_error(GOO_ERR_ARG, "goo_nll_grad_static: leaf %d parameter %d", leaves[l], n.par[j]);
        L.par[j] = n.par[j];
      }
    }
  }
  if (norm->kind == GOO_NORM_ANALYTIC) {
    for (int k = 0; k < nK; ++k)
      for (int l = 0; l < h.comp[k].n_leaf; ++l) {
        const LeafDev& L = h.leaf[k * kMaxLeaf + l];
        if (L.op == GOO_OP_ARGUS)
          return set_error(GOO_ERR_UNSUPPORTED, "goo_nll_grad_static: Argus needs GOO_NORM_GRID");
        for (int l2 = 0; l2 < l; ++l2)
          if (h.leaf[k * kMaxLeaf + l2].col == L.col)
            return set_error(GOO_ERR_UNSUPPORTED, "goo_nll_grad_static: two leaves on one observable need GOO_NORM_GRID");
      }
  } else if (norm->kind == GOO_NORM_GRID) {
    for (int o = 0; o < n_obs; ++o)
      if (norm->bins[o] < 1 || norm->bins[o] > (1 << 20))
        return set_error(GOO_ERR_ARG, "goo_nll_grad_static: bins[%d] = %d", o, norm->bins[o]);
    for (int k = 0; k < nK; ++k) {
      GridDev& G = h.grid[k];
      bool used[kMaxObs] = {false, false, false, false};
      for (int l = 0; l < h.comp[k].n_leaf; ++l) used[h.leaf[k * kMaxLeaf + l].col] = true;
      for (int o = 0; o < kMaxObs; ++o) G.dim_of_col[o] = -1;
      G.cell_volume = 1.0;
      for (int o = 0; o < n_obs; ++o) {
        if (!used[o]) continue;
        const int d = G.ndim++;
        G.dim_of_col[o] = d;
        G.bins[d] = norm->bins[o];
        const double step = (hi[o] - lo[o]) / norm->bins[o];
        G.h64[d] = step;
        G.lo64[d] = lo[o];
        G.h_hi[d] = (float)step;
        G.h_lo[d] = (float)(step - (double)(float)step);
        G.lo_hi[d] = (float)lo[o];
        G.lo_lo[d] = (float)(lo[o] - (double)(float)lo[o]);
        G.cell_volume *= step;
      }
    }
  } else {
    return set_error(GOO_ERR_UNSUPPORTED, "goo_nll_grad_static: only GOO_NORM_ANALYTIC and GOO_NORM_GRID");
  }
  h.norm_kind = norm->kind;
  h.grid_separable = norm->kind == GOO_NORM_GRID ? grid_separable(h) : 0;
  return GOO_OK;
}

template <typename T, int K, int L>
static int static_launch(const ModelDev& h, int max_leaf, unsigned char* base, int sms, const void* const* cols_dev,
                         int64_t n, int precision, cudaStream_t st) {
  ModelDev* md = (ModelDev*)(base + kStOffModel);
  unsigned* counters = (unsigned*)(base + kStOffCounters);
  double* result = (double*)(base + kStOffResult);
  float2* partials = (float2*)(base + kStOffPartials);
  (void)precision;
  if (h.norm_kind == GOO_NORM_GRID && h.grid_separable) {
    static_assert((size_t)kMaxComp * kMaxLeaf * 4 * sizeof(double) <= kStPartialsCap * sizeof(float2),
                  "static scratch too small for the separable grid sums");
    grid_sep_kernel<T><<<dim3((unsigned)max_leaf, h.nK), kBlock, 0, st>>>(md, (double*)partials, counters);
  } else if (h.norm_kind == GOO_NORM_GRID) {
    constexpr int NSg = 1 + 3 * L;
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, grid_kernel<T, L>, kBlock, 0) != cudaSuccess || bps < 1) {
      cudaGetLastError();
      bps = 1;
    }
    int64_t units_max = 1;
    for (int k = 0; k < h.nK; ++k) {
      const GridDev& G = h.grid[k];
      int64_t rows = 1;
      for (int d = 0; d < G.ndim - 1; ++d) rows *= G.bins[d];
      const int64_t u = rows * ((G.bins[G.ndim - 1] + kSeg - 1) / kSeg);
      units_max = u > units_max ? u : units_max;
    }
    int64_t nbx = (units_max + kBlock - 1) / kBlock;
    const int64_t cap = ((int64_t)sms * bps + h.nK - 1) / h.nK;
    if (nbx > cap) nbx = cap;
    const int64_t fit = (int64_t)(kStPartialsCap / ((size_t)NSg * h.nK));
    if (nbx > fit) nbx = fit;
    if (nbx < 1) return set_error(GOO_ERR_UNSUPPORTED, "goo_nll_grad_static: scratch too small for the grid");
    grid_kernel<T, L><<<dim3((unsigned)nbx, h.nK), kBlock, 0, st>>>(md, partials, counters);
  }
  constexpr int NS = EventLanes<T, K, L, true>::NS;
  int bps = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, sop_event_kernel<T, K, L, true>, kBlock, 0) != cudaSuccess ||
      bps < 1) {
    cudaGetLastError();
    bps = 1;
  }
  int64_t nb = (n + kBlock - 1) / kBlock;
  if (nb > (int64_t)sms * bps) nb = (int64_t)sms * bps;
  if (nb > (int64_t)(kStPartialsCap / NS)) nb = (int64_t)(kStPartialsCap / NS);
  if (nb < 1) nb = 1;
  Cols<T> cols{};
  for (int c = 0; c < kMaxObs; ++c) cols.c[c] = (const T*)cols_dev[c < h.n_obs ? c : 0];
  sop_event_kernel<T, K, L, true><<<(unsigned)nb, kBlock, 0, st>>>(md, make_evconst<T, K, L>(h), cols, 0, n, partials,
                                                                   counters, result, 0, nullptr);
  GOO_CUDA_TRY(cudaGetLastError());
  return GOO_OK;
}

}  // namespace goo

extern "C" int goo_nll_grad_static(const goo_node* nodes, int n_nodes, int n_params, int n_obs, const double* obs_lo,
                                   const double* obs_hi, const goo_norm_spec* norm, const void* const* cols_dev,
                                   int precision, int64_t n_events, const double* theta, void* cuda_stream,
                                   double* nll_out, double* grad_out) {
  using namespace goo;
  if (!nodes || !obs_lo || !obs_hi || !norm || !theta || !nll_out || !grad_out || (n_events > 0 && !cols_dev))
    return set_error(GOO_ERR_ARG, "goo_nll_grad_static: NULL argument");
  if (n_nodes < 1 || n_nodes > 256) return set_error(GOO_ERR_ARG, "goo_nll_grad_static: n_nodes=%d", n_nodes);
  if (n_params < 0 || n_params > kStaticMaxParams)
    return set_error(GOO_ERR_ARG, "goo_nll_grad_static: n_params=%d exceeds the maximum %d", n_params, kStaticMaxParams);
  if (n_obs < 1 || n_obs > kMaxObs) return set_error(GOO_ERR_ARG, "goo_nll_grad_static: n_obs=%d (1..%d)", n_obs, kMaxObs);
  if (n_events < 0) return set_error(GOO_ERR_ARG, "goo_nll_grad_static: n_events=%lld", (long long)n_events);
  if (precision != GOO_F64 && precision != GOO_F32) return set_error(GOO_ERR_ARG, "goo_nll_grad_static: precision");
  for (int i = 0; i < n_nodes; ++i)
    for (int c = 0; c < nodes[i].n_child; ++c)
      if (nodes[i].n_child > GOO_MAX_CHILD || nodes[i].child[c] < 0 || nodes[i].child[c] >= i)
        return set_error(GOO_ERR_ARG, "goo_nll_grad_static: node %d is not in post-order", i);
  for (int p = 0; p < n_params; ++p)
    if (!std::isfinite(theta[p])) return set_error(GOO_ERR_ARG, "goo_nll_grad_static: theta[%d] is not finite", p);
  for (int c = 0; n_events > 0 && c < n_obs; ++c)
    if (!cols_dev[c] || ((uintptr_t)cols_dev[c] & 15))
      return set_error(GOO_ERR_ARG, "goo_nll_grad_static: column %d is NULL or not 16-byte aligned", c);
  ModelDev h;
  GOO_TRY(static_plan(nodes, n_nodes, n_params, n_obs, obs_lo, obs_hi, norm, h));
  int max_leaf = 0;
  for (int k = 0; k < h.nK; ++k) max_leaf = h.comp[k].n_leaf > max_leaf ? h.comp[k].n_leaf : max_leaf;
  int dev = 0, sms = 0;
  GOO_CUDA_TRY(cudaGetDevice(&dev));
  unsigned char* base = nullptr;
  GOO_TRY(static_scratch_lookup(dev, &base, &sms));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (n_events == 0) {
    *nll_out = 0.0;
    for (int p = 0; p < n_params; ++p) grad_out[p] = 0.0;
    return GOO_OK;
  }
  host_prep(h, theta, precision);
  GOO_CUDA_TRY(cudaMemcpyAsync(base + kStOffModel, &h, sizeof(ModelDev), cudaMemcpyHostToDevice, st));
  GOO_CUDA_TRY(cudaMemsetAsync(base + kStOffCounters, 0, 256, st));
  const bool small = h.nK <= 2 && max_leaf <= 3;
  if (precision == GOO_F32) {
    GOO_TRY((small ? static_launch<float, 2, 3>(h, max_leaf, base, sms, cols_dev, n_events, precision, st)
                   : static_launch<float, 4, 4>(h, max_leaf, base, sms, cols_dev, n_events, precision, st)));
  } else {
    GOO_TRY((small ? static_launch<double, 2, 3>(h, max_leaf, base, sms, cols_dev, n_events, precision, st)
                   : static_launch<double, 4, 4>(h, max_leaf, base, sms, cols_dev, n_events, precision, st)));
  }
  double res[2 + kStaticMaxParams];
  GOO_CUDA_TRY(cudaMemcpyAsync(res, base + kStOffResult, (2 + n_params) * sizeof(double), cudaMemcpyDeviceToHost, st));
  GOO_CUDA_TRY(cudaStreamSynchronize(st));
  if (res[1] < 0) {  // a device wait gave up (the event kernel's status word)
    *nll_out = HUGE_VAL;
    for (int p = 0; p < n_params; ++p) grad_out[p] = 0.0;
    return set_error(GOO_ERR_TIMEOUT, "goo_nll_grad_static: a device wait gave up; the result is invalid");
  }
  if (res[1] > 0) {
    *nll_out = HUGE_VAL;
    for (int p = 0; p < n_params; ++p) grad_out[p] = 0.0;
    return set_error(GOO_ERR_NONPOSITIVE_PDF, "goo_nll_grad_static: density <= 0 for %.0f events", res[1]);
  }
  *nll_out = res[0];
  for (int p = 0; p < n_params; ++p) grad_out[p] = res[2 + p];
  return GOO_OK;
}
