// sop_kernels.cuh -- device code of the sum-of-products likelihood: the register-resident
// tree interpreter (scalar FP32 / FP64 and packed FP32 pairs), the in-kernel grid
// normalisation, the last-block finish and the event kernels (see tree.cu for the model
// semantics and the host side).
//
// The packed-pair kernel takes a compile-time leaf signature SIG (4 bits per leaf slot: the
// leaf's opcode, 0 for an empty slot) and column map COLS (2 bits per slot: the leaf's
// observable).  SIG = 0 is the interpreter compiled into the library, which reads each slot's
// opcode and column at run time; a nonzero SIG is instantiated at run time by NVRTC for one
// model (jit.cu), so that every slot's dispatch folds away, leaves on one observable share
// one shared-memory load, and only the gradient lanes its leaf has are accumulated.  This
// header therefore compiles under nvcc and under NVRTC alike.
#pragma once

#include "common.cuh"
#include "model.cuh"

namespace goo {

template <bool C, typename A, typename B>
struct Cond {
  using type = A;
};
template <typename A, typename B>
struct Cond<false, A, B> {
  using type = B;
};

// Opcode of leaf slot `slot` in a compile-time signature (0 when SIG holds none).
__host__ __device__ constexpr int sig_op(unsigned long long sig, int slot) { return (int)((sig >> (4 * slot)) & 15ull); }


// Leaves whose value carries a factor r besides exp(a) (the others have r = 1, so a
// specialised kernel skips their products with r), and whether product k of a signature has
// such a leaf or any leaf at all.
__host__ __device__ constexpr bool leaf_has_r(int op) { return op == GOO_OP_POLY2 || op == GOO_OP_ARGUS; }
__host__ __device__ constexpr bool sig_product_has_r(unsigned long long sig, int k, int L) {
  bool any = false;
  for (int l = 0; l < L; ++l) any = any || leaf_has_r(sig_op(sig, k * L + l));
  return any;
}
__host__ __device__ constexpr bool sig_product_used(unsigned long long sig, int k, int L) {
  bool any = false;
  for (int l = 0; l < L; ++l) any = any || sig_op(sig, k * L + l) != 0;
  return any;
}
// Number of parameters (derivative lanes) of a leaf opcode.
__host__ __device__ constexpr int leaf_nder(int op) {
  return op == GOO_OP_GAUSS ? 2 : op == GOO_OP_EXPO ? 1 : op == GOO_OP_POLY2 ? 2 : op == GOO_OP_ARGUS ? 3 : 0;
}

template <typename T>
struct Cols {
  const T* c[kMaxObs];
  // for the pair kernel's direct form (a GOO_BORROW_HOST dataset: c are device-mapped host
  // columns, read straight into registers): the float limits that admit exactly the values
  // inside the double limits
  float lo[kMaxObs], hi[kMaxObs];
};

template <typename T>
__device__ __forceinline__ T pick(int col, T x0, T x1, T x2, T x3) {
  return col == 0 ? x0 : (col == 1 ? x1 : (col == 2 ? x2 : x3));
}

// =======================================================================================
// register-resident interpreter: before the event loop every thread copies the constants,
// opcode and column of each leaf slot (k, l) into registers (compile-time indices), so the
// per-event work is one uniform dispatch per leaf plus the leaf's arithmetic.  Absent leaf
// slots carry opcode 0 (value 1, no derivative); absent products are excluded by k < nK.
// =======================================================================================
template <typename T>
struct LeafReg {
  int op, col;
  T c[6];
};

template <typename T>
__device__ __forceinline__ LeafReg<T> load_leaf(const LeafDev& L) {
  LeafReg<T> R;
  R.op = L.op;
  R.col = L.col;
#pragma unroll
  for (int j = 0; j < 6; ++j) R.c[j] = (sizeof(T) == 4) ? (T)L.f[j] : (T)L.d[j];
  return R;
}

// Per-call constants of the event kernels, passed by value as a kernel parameter: every
// field is read with compile-time indices after unrolling, so the arithmetic takes it as a
// constant-bank operand and it occupies no registers.  Absent leaf slots carry opcode 0.
template <typename T, int K, int L>
struct EvConst {
  LeafReg<T> leaf[K][L];
  T w_hi[K], w_lo[K];   // w_k (FP64 path: w_hi only)
  int nK, nobs;
  // the pair kernel's exponents are in base 2: the rate of an exponential leaf and the slope
  // of an Argus leaf times log2(e), rounded once from the float constants above
  float b2[K][L];
};

// Value r * exp(a) of one leaf at x (+ xlo, the low part of a double-float coordinate when
// HasLo) and, if GRAD, d log(leaf) / d par_j.
template <bool GRAD, bool HasLo = false>
__device__ __forceinline__ void leaf_eval(const LeafReg<float>& L, float x, float& r, float& a, float* d,
                                          float xlo = 0.f) {
  const float* c = L.c;
  d[0] = d[1] = d[2] = 0.f;
  switch (L.op) {
    case GOO_OP_GAUSS: {
      const float z = (HasLo ? (x - c[0]) + (xlo - c[1]) : (x - c[0]) - c[1]) * c[2];
      r = 1.f;
      a = -0.5f * z * z;
      if (GRAD) {
        d[0] = z * c[2];
        d[1] = z * z * c[2];
      }
      break;
    }
    case GOO_OP_EXPO:
      r = 1.f;
      a = HasLo ? fmaf(c[0], x, c[0] * xlo) : c[0] * x;
      if (GRAD) d[0] = HasLo ? x + xlo : x;
      break;
    case GOO_OP_POLY2: {
      const float xx = HasLo ? x + xlo : x;
      r = fmaf(xx, fmaf(c[1], xx, c[0]), 1.f);
      a = 0.f;
      if (GRAD) {
        const float ir = __fdividef(1.f, r);
        d[0] = xx * ir;
        d[1] = xx * xx * ir;
      }
      break;
    }
    case GOO_OP_ARGUS: {
      const float u = HasLo ? ((c[0] - x) + (c[1] - xlo)) * ((c[0] + x) + (c[1] + xlo)) * c[2]
                            : ((c[0] - x) + c[1]) * ((c[0] + x) + c[1]) * c[2];
      if (u > 0.f) {
        const float lu = __logf(u);
        r = HasLo ? x + xlo : x;
        a = fmaf(c[4], lu, c[3] * u);
        if (GRAD) {
          d[0] = c[5] * (1.f - u) * (__fdividef(c[4], u) + c[3]);
          d[1] = u;
          d[2] = lu;
        }
      } else {
        r = 0.f;
        a = 0.f;
      }
      break;
    }
    default:
      r = 1.f;
      a = 0.f;
  }
}

template <bool GRAD, bool HasLo = false>
__device__ __forceinline__ void leaf_eval(const LeafReg<double>& L, double x, double& r, double& a, double* d,
                                          double xlo = 0.0) {
  const double* c = L.c;
  d[0] = d[1] = d[2] = 0.0;
  switch (L.op) {
    case GOO_OP_GAUSS: {
      const double z = (x - c[0]) * c[1];
      r = 1.0;
      a = -0.5 * z * z;
      if (GRAD) {
        d[0] = z * c[1];
        d[1] = z * z * c[1];
      }
      break;
    }
    case GOO_OP_EXPO:
      r = 1.0;
      a = c[0] * x;
      if (GRAD) d[0] = x;
      break;
    case GOO_OP_POLY2:
      r = 1.0 + x * (c[0] + c[1] * x);
      a = 0.0;
      if (GRAD) {
        d[0] = x / r;
        d[1] = x * x / r;
      }
      break;
    case GOO_OP_ARGUS: {
      const double u = (c[0] - x) * (c[0] + x) * c[1];
      if (u > 0.0) {
        const double lu = log(u);
        r = x;
        a = c[3] * lu + c[2] * u;
        if (GRAD) {
          d[0] = c[4] * (1.0 - u) * (c[3] / u + c[2]);
          d[1] = u;
          d[2] = lu;
        }
      } else {
        r = 0.0;
        a = 0.0;
      }
      break;
    }
    default:
      r = 1.0;
      a = 0.0;
  }
}

// One event: log f (returned through logf) and, if GRAD, the shares c_k and the leaf
// derivatives.  Returns false when f <= 0.
template <typename T, int K, int L, bool GRAD>
__device__ __forceinline__ bool eval_event(const EvConst<T, K, L>& P, const T (&off_hi)[K], const T (&off_lo)[K], T x0,
                                           T x1, T x2, T x3, T& logf, T (&ck)[K], T (&dk)[K][L][3]) {
  T rk[K], ak[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    T r = T(1), a = T(0);
#pragma unroll
    for (int l = 0; l < L; ++l) {
      T lr_, la_;
      leaf_eval<GRAD>(P.leaf[k][l], pick<T>(P.leaf[k][l].col, x0, x1, x2, x3), lr_, la_, dk[k][l]);
      r *= lr_;
      a += la_;
    }
    a = (a + off_hi[k]) + off_lo[k];
    rk[k] = r;
    ak[k] = (k < P.nK && r != T(0)) ? a : T(-1e30);
  }
  T M = ak[0];
#pragma unroll
  for (int k = 1; k < K; ++k) M = ak[k] > M ? ak[k] : M;
  T S = T(0);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if constexpr (sizeof(T) == 4) {
      rk[k] = rk[k] * __expf(ak[k] - M);
      S += fmaf(P.w_hi[k], rk[k], P.w_lo[k] * rk[k]);
    } else {
      rk[k] = rk[k] * exp(ak[k] - M);
      S += P.w_hi[k] * rk[k];
    }
  }
  if (!(S > T(0)) || !(M > T(-1e29))) return false;
  if constexpr (sizeof(T) == 4) logf = M + __logf(S);
  else logf = M + log(S);
  if constexpr (GRAD) {
    T invS;
    if constexpr (sizeof(T) == 4) invS = __fdividef(1.f, S);
    else invS = T(1) / S;
#pragma unroll
    for (int k = 0; k < K; ++k) ck[k] = rk[k] * invS;
  }
  return true;
}

// -log N_k of every product (written by the normalisation step) into registers.
template <typename T, int K>
__device__ __forceinline__ void load_offsets(const ModelDev* __restrict__ md, T (&off_hi)[K], T (&off_lo)[K]) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if constexpr (sizeof(T) == 4) {
      off_hi[k] = md->comp[k].off_hi;
      off_lo[k] = md->comp[k].off_lo;
    } else {
      off_hi[k] = -md->comp[k].log_norm;
      off_lo[k] = 0.0;
    }
  }
}

// =======================================================================================
// fused per-event kernel: evaluate, log, accumulate (and adjoint lanes), reduce
// Lanes: 0 = sum log f; 1..K = C_k; then the leaf-derivative lanes A_{k,l,j}: at
// 1 + K + (k*L + l)*3 + j in the interpreter (SIG = 0); in a kernel specialised for a leaf
// signature only the lanes its leaves have, packed in slot order (a_lane).
// =======================================================================================
// Derivative lanes of the leaves in slots [0, slot) of a signature.
__host__ __device__ constexpr int sig_nder_before(unsigned long long sig, int slot) {
  int n = 0;
  for (int s = 0; s < slot; ++s) n += leaf_nder(sig_op(sig, s));
  return n;
}
// Lane of derivative q of leaf slot (k, l), and whether the kernel carries it.
template <int K, int L, unsigned long long SIG>
__host__ __device__ constexpr int a_lane(int k, int l, int q) {
  return SIG == 0 ? 1 + K + (k * L + l) * 3 + q : 1 + K + sig_nder_before(SIG, k * L + l) + q;
}
template <int K, int L, unsigned long long SIG>
__host__ __device__ constexpr bool a_present(int k, int l, int q) {
  return SIG == 0 || q < leaf_nder(sig_op(SIG, k * L + l));
}
template <typename T, int K, int L, bool GRAD, unsigned long long SIG = 0>
struct EventLanes {
  static constexpr int NS = !GRAD ? 1 : (SIG == 0 ? 1 + K + K * L * 3 : 1 + K + sig_nder_before(SIG, K * L));
};

// Block reduction of the per-thread lanes, last-block reduction over the blocks and the
// final FP64 combination (lanes -> NLL and d NLL / d theta), shared by the event kernels.
// Constants of the self-contained FP32 event kernel, passed by value so that the kernel reads
// no model block: per leaf slot the 1-D grid of its observable (separable grid normalisation)
// and the final combination's weights, parameter map and d w / d theta.
template <int K, int L, bool GRAD>
struct EvNorm {
  float lo_hi[K * L], lo_lo[K * L], h_hi[K * L], h_lo[K * L], aref_hi[K * L], aref_lo[K * L];
  double h64[K * L];
  int nb[K * L];                                   // bins (0: no leaf in the slot)
  double w[K];                                     // w_k
  int n_params;
  signed char par[K][L][3];                        // parameter of leaf constant j (-1: none)
  double dw[GRAD ? K : 1][GRAD ? kMaxParams : 1];  // d w_k / d theta_p
};

// Source of the final combination's constants for the kernels that read the model block in
// device memory (the self-normalising pair kernel has its own finish, event_finish_fused).
struct MdFin {
  const ModelDev* __restrict__ md;
  int nK;
  static constexpr bool kOwnNorm = false;
  __device__ int n_params() const { return md->n_params; }
  __device__ double w(int k) const { return k < nK ? md->comp[k].w : 0.0; }
  __device__ double dw(int k, int p) const { return md->dw[k][p]; }
  __device__ double dlogN(int k, int p) const { return md->dlogN[k][p]; }
  __device__ int par(int k, int l, int j) const {
    return (k < nK && l < md->comp[k].n_leaf) ? md->leaf[k * kMaxLeaf + l].par[j] : -1;
  }
  __device__ double term(int, int, int) const { return 0.0; }
};


// Block reduction, last-block reduction over the blocks and the final FP64 combination
// (lanes -> NLL and d NLL / d theta), shared by the event kernels:
//   d NLL / d theta_p = sum_k [w_k C_k dlogN_kp - C_k dw_kp] - sum_{k,l,j: par = p} w_k A_klj,
// with dlogN_kp = sum_{l,j: par = p} t_klj for a block's own normalisation terms.  Thread p
// takes parameter p and gathers its terms in a fixed order.  The constants are loaded before
// the block's reduction, so that their latency overlaps it; the last block alone combines.
template <int K, int L, bool GRAD, unsigned long long SIG, typename Fin>
__device__ __forceinline__ void event_finish(ddf (&v)[EventLanes<float, K, L, GRAD, SIG>::NS], unsigned bad,
                                             const Fin& F, int nK, float2* partials, unsigned* counters,
                                             double* result, int out_mode, ddf* s_red, unsigned* s_bad) {
  constexpr int NS = EventLanes<float, K, L, GRAD, SIG>::NS;
  __shared__ double s_out[NS];
  __shared__ double s_w[K];
  __shared__ int s_par[K][L][3];
  const int p = threadIdx.x;
  const int P = F.n_params();
  double dwp[GRAD ? K : 1], dlp[GRAD ? K : 1];
  if constexpr (GRAD) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const bool on = p < P && k < nK;
      dwp[k] = on ? F.dw(k, p) : 0.0;
      dlp[k] = (on && !Fin::kOwnNorm) ? F.dlogN(k, p) : 0.0;
    }
    for (int t = threadIdx.x; t < K * L * 3; t += blockDim.x) {
      const int k = t / (L * 3), l = (t / 3) % L, jj = t % 3;
      s_par[k][l][jj] = k < nK ? F.par(k, l, jj) : -1;
    }
    if (threadIdx.x < K) s_w[threadIdx.x] = F.w(threadIdx.x);
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
  // every other block added to these words before its ticket (and a fence): plain L2 reads,
  // issued before the reduction so that their latency overlaps it
  unsigned nbad = 0u, status = 0u, nrange = 0u;
  if (threadIdx.x == 0) {
    nbad = __ldcg(counters + 1);
    status = __ldcg(counters + kStatusWord);
    nrange = __ldcg(counters + kRangeWord);
  }
  reduce_partials(partials, NS, gridDim.x, s_out, s_red, blockDim.x);

  // ---- final combination (last block, FP64) ----
  const int off = out_mode == 0 ? 2 : 3;
  if (p < P) {
    double gp = 0.0;
    if constexpr (GRAD) {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if (k >= nK) break;
        const double Ck = s_out[1 + k];
        gp += s_w[k] * Ck * dlp[k] - Ck * dwp[k];
      }
#pragma unroll
      for (int k = 0; k < K; ++k)
#pragma unroll
        for (int l = 0; l < L; ++l)
#pragma unroll
          for (int jj = 0; jj < 3; ++jj)
            if (a_present<K, L, SIG>(k, l, jj) && s_par[k][l][jj] == p)
              gp += s_w[k] * ((Fin::kOwnNorm ? s_out[1 + k] * F.term(k, l, jj) : 0.0) -
                              s_out[a_lane<K, L, SIG>(k, l, jj)]);
    }
    result[off + p] = gp;
  }
  if (threadIdx.x == 0) {
    counters[0] = 0u;  // the ticket
    counters[1] = 0u;
    counters[kStatusWord] = 0u;
    counters[kRangeWord] = 0u;
    // a device wait that gave up is reported as -1, events outside the observable limits
    // (direct reads of host columns) as -(2 + their count)
    const double nb = nrange ? -2.0 - (double)nrange : status ? -1.0 : (double)nbad;
    result[0] = -s_out[0];
    if (out_mode == 0) {
      result[1] = nb;
    } else {
      result[1] = 0.0;
      result[2] = nb;
    }
  }
  result_complete(result, P > 1 ? P : 1);
}

// Resident blocks per SM the event kernel is compiled for: the FP32 form of the small shape
// fits three 256-thread blocks (<= 80 registers) with its leaf constants in the parameter bank.
template <typename T, int K, int L>
struct EventOcc {
  static constexpr int value = (sizeof(T) == 4 && K * L <= 6) ? 3 : 2;
};

// wcol (nullable): per-event weights w_i (a binned dataset: bin centres with their counts);
// the lanes then sum w_i log f_i and w_i times the gradient terms, and events of weight 0 are
// skipped.
template <typename T, int K, int L, bool GRAD>
__global__ void __launch_bounds__(kBlock, EventOcc<T, K, L>::value) sop_event_kernel(const ModelDev* __restrict__ md, const EvConst<T, K, L> P,
                                                              Cols<T> cols, int64_t begin, int64_t end, float2* partials,
                                                              unsigned* counters, double* result, int out_mode,
                                                              const T* __restrict__ wcol) {
  constexpr int NS = EventLanes<T, K, L, GRAD>::NS;
  __shared__ ddf s_red[(kBlock / 32) * NS > kBlock ? (kBlock / 32) * NS : kBlock];
  __shared__ unsigned s_bad[kBlock / 32];
  T off_hi[K], off_lo[K];
  load_offsets<T, K>(md, off_hi, off_lo);
  const int nK = P.nK;

  // per-thread accumulators: FP32 path -> Kahan for sum log f, plain FP32 for the adjoint
  // lanes; FP64 path -> plain FP64
  using Acc = typename Cond<sizeof(T) == 4, float, double>::type;
  double acc64 = 0.0;
  Kahan acc32;
  Acc Cacc[K];
  Acc Aacc[K][L][3];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    Cacc[k] = Acc(0);
#pragma unroll
    for (int l = 0; l < L; ++l)
#pragma unroll
      for (int j = 0; j < 3; ++j) Aacc[k][l][j] = Acc(0);
  }
  unsigned bad = 0;
  const int nobs = P.nobs;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // software pipelining: the next event's columns are requested before this event is
  // evaluated, so the loads' latency overlaps the arithmetic
  int64_t i = begin + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  T n0 = T(0), n1 = T(0), n2 = T(0), n3 = T(0), nw = T(1);
  if (i < end) {
    n0 = cols.c[0][i];
    n1 = nobs > 1 ? cols.c[1][i] : T(0);
    n2 = nobs > 2 ? cols.c[2][i] : T(0);
    n3 = nobs > 3 ? cols.c[3][i] : T(0);
    if (wcol) nw = wcol[i];
  }
  for (; i < end; i += stride) {
    const T x0 = n0, x1 = n1, x2 = n2, x3 = n3, wi = nw;
    const int64_t inext = i + stride;
    if (inext < end) {
      n0 = cols.c[0][inext];
      n1 = nobs > 1 ? cols.c[1][inext] : T(0);
      n2 = nobs > 2 ? cols.c[2][inext] : T(0);
      n3 = nobs > 3 ? cols.c[3][inext] : T(0);
      if (wcol) nw = wcol[inext];
    }
    if (wcol && wi == T(0)) continue;  // an empty bin
    T logf, ck[K], dk[K][L][3];
    if (eval_event<T, K, L, GRAD>(P, off_hi, off_lo, x0, x1, x2, x3, logf, ck, dk)) {
      if (wcol) {
        logf *= wi;
#pragma unroll
        for (int k = 0; k < K; ++k) ck[k] *= wi;
      }
      if constexpr (sizeof(T) == 4) {
        acc32.add(logf);
      } else {
        acc64 += logf;
      }
      if constexpr (GRAD) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
          Cacc[k] += ck[k];
#pragma unroll
          for (int l = 0; l < L; ++l)
#pragma unroll
            for (int j = 0; j < 3; ++j) Aacc[k][l][j] += ck[k] * dk[k][l][j];
        }
      }
    } else {
      bad++;
    }
  }

  // ---- block reduction ----
  ddf v[NS];
  if constexpr (sizeof(T) == 4) {
    v[0] = acc32.value();
  } else {
    v[0] = dd_from_double(acc64);
  }
  if constexpr (GRAD) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      v[1 + k] = (sizeof(T) == 4) ? ddf{(float)Cacc[k], 0.f} : dd_from_double((double)Cacc[k]);
#pragma unroll
      for (int l = 0; l < L; ++l)
#pragma unroll
        for (int j = 0; j < 3; ++j)
          v[1 + K + (k * L + l) * 3 + j] =
              (sizeof(T) == 4) ? ddf{(float)Aacc[k][l][j], 0.f} : dd_from_double((double)Aacc[k][l][j]);
    }
  }
  event_finish<K, L, GRAD, 0>(v, bad, MdFin{md, nK}, nK, partials, counters, result, out_mode, s_red, s_bad);
}

// =======================================================================================
// FP32 event kernel on packed pairs.  Each thread takes two consecutive events at a time and
// evaluates both with the packed FP32 instructions of sm_100-class GPUs (add / sub / mul /
// fma on .f32x2 register pairs), so the arithmetic, the leaf dispatch and the index work
// each issue once per two events; exp2 / lg2 / rcp stay per lane.  Pairs are aligned to
// even event indices (8-byte column loads); a lane outside [begin, end) is masked.  Each
// lane is rounded exactly as a scalar FP32 evaluation of the same formulas.
// =======================================================================================

namespace pk {
__device__ __forceinline__ float2 pick(int col, float2 x0, float2 x1, float2 x2, float2 x3) {
  return col == 0 ? x0 : (col == 1 ? x1 : (col == 2 ? x2 : x3));
}
}  // namespace pk

// Two events of one leaf, in the pair kernel's base-2 form: the value is r * 2^a2 per lane;
// the leaf adds its a2 to `a` (the product's running exponent) and returns r and, if GRAD, the
// raw derivative terms whose weighted sums the lanes collect.  A lane's sum becomes
// sum_events c_k d log(leaf) / d par_j after one constant factor per lane (pair_lane_scale):
//   Gauss    a2 = -z^2 / (2 ln 2), z = (x - mu) / sigma; raw (z, z^2), factor 1 / sigma;
//   Exp      a2 = (lambda log2 e) x;                      raw x;
//   Poly2    r = 1 + c_0 x + c_1 x^2;                      raw (x / r, x^2 / r), or with
//            PQ (the product's only Poly2: its lanes are weighted by c_k / r instead of c_k,
//            which needs no reciprocal) raw (x, x^2);
//   Argus    u = 1 - x^2 / m0^2, r = x, a2 = (xi log2 e) u + p log2 u;
//            raw ((1 - u)(p / u + xi), u, log2 u), factors (2 / m0, 1, ln 2).
// `op` is the slot's opcode: L.op in the interpreter, a compile-time constant in a
// specialised kernel (the switch then folds to one case).
template <bool GRAD, bool PQ = false>
__device__ __forceinline__ void leaf_eval2(const LeafReg<float>& L, float b2, int op, float2 x, float2& r, float2& a,
                                           float2* d) {
  using namespace pk;
  const float* c = L.c;
  constexpr float kHalfLog2e = -0.72134752f;  // -1 / (2 ln 2)
  d[0] = d[1] = d[2] = splat(0.f);
  switch (op) {
    case GOO_OP_GAUSS: {
      const float2 z = mul(sub(sub(x, splat(c[0])), splat(c[1])), splat(c[2]));
      const float2 zz = mul(z, z);
      r = splat(1.f);
      a = fma(zz, splat(kHalfLog2e), a);
      if (GRAD) {
        d[0] = z;
        d[1] = zz;
      }
      break;
    }
    case GOO_OP_EXPO:
      r = splat(1.f);
      a = fma(splat(b2), x, a);
      if (GRAD) d[0] = x;
      break;
    case GOO_OP_POLY2: {
      r = fma(x, fma(splat(c[1]), x, splat(c[0])), splat(1.f));
      if (GRAD) {
        const float2 xx = mul(x, x);
        if (PQ) {
          d[0] = x;
          d[1] = xx;
        } else {
          const float2 ir = rcp(r);
          d[0] = mul(x, ir);
          d[1] = mul(xx, ir);
        }
      }
      break;
    }
    case GOO_OP_ARGUS: {
      const float2 u = mul(mul(add(sub(splat(c[0]), x), splat(c[1])), add(add(splat(c[0]), x), splat(c[1]))), splat(c[2]));
      // a lane with u <= 0 has value 0 (r = 0); u is replaced by 1 there to keep it finite
      const bool p0 = u.x > 0.f, p1 = u.y > 0.f;
      const float2 us = make_float2(p0 ? u.x : 1.f, p1 ? u.y : 1.f);
      const float2 lu2 = make_float2(lg2(us.x), lg2(us.y));
      r = make_float2(p0 ? x.x : 0.f, p1 ? x.y : 0.f);
      a = fma(splat(c[4]), lu2, fma(splat(b2), us, a));
      if (GRAD) {
        d[0] = mul(sub(splat(1.f), us), fma(splat(c[4]), rcp(us), splat(c[3])));
        d[1] = us;
        d[2] = lu2;
      }
      break;
    }
    default:
      r = splat(1.f);
  }
}

// Leaf slot (k, l) of a signature is a Poly2 leaf that is the only one in its product: the
// pair kernel weights its lanes by c_k / r (see leaf_eval2).
__host__ __device__ constexpr bool sig_poly_q(unsigned long long sig, int k, int l, int L) {
  int n = 0;
  for (int t = 0; t < L; ++t) n += sig_op(sig, k * L + t) == GOO_OP_POLY2 ? 1 : 0;
  return sig != 0 && n == 1 && sig_op(sig, k * L + l) == GOO_OP_POLY2;
}
__host__ __device__ constexpr bool sig_product_poly_q(unsigned long long sig, int k, int L) {
  bool any = false;
  for (int l = 0; l < L; ++l) any = any || sig_poly_q(sig, k, l, L);
  return any;
}

// Two events: log2 f per lane, ok per lane (f > 0) and, if GRAD, c_k, q_k = c_k / r of the
// product's PQ Poly2 leaf (sig_poly_q) and the leaves' raw derivative terms.  xl[k][l] holds
// the observable of leaf l of product k; off_hi + off_lo = -log2 N_k.
template <int K, int L, bool GRAD, unsigned long long SIG = 0>
__device__ __forceinline__ void eval_event2(const EvConst<float, K, L>& P, const float (&off_hi)[K],
                                            const float (&off_lo)[K], const float2 (&xl)[K][L], float2& logf,
                                            bool& ok0, bool& ok1, float2 (&ck)[K], float2 (&qk)[K],
                                            float2 (&dk)[K][L][3]) {
  using namespace pk;
  float2 rk[K], ak[K], rq[K], rp[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    // the exponent starts at the offset's high part; r is the product of the leaves' factors,
    // rq the same without the PQ Poly2 leaf's, rp that leaf's alone
    float2 r = splat(1.f), a = splat(off_hi[k]);
    rq[k] = rp[k] = splat(1.f);
#pragma unroll
    for (int l = 0; l < L; ++l) {
      float2 lr_;
      if constexpr (SIG != 0) {
        constexpr int op_unused = 0;
        if (sig_op(SIG, k * L + l) == op_unused) {  // an empty slot: r = 1, a = 0
          dk[k][l][0] = dk[k][l][1] = dk[k][l][2] = splat(0.f);
          continue;
        }
      }
      const int op = SIG != 0 ? sig_op(SIG, k * L + l) : P.leaf[k][l].op;
      if (sig_poly_q(SIG, k, l, L)) {
        leaf_eval2<GRAD, true>(P.leaf[k][l], P.b2[k][l], op, xl[k][l], lr_, a, dk[k][l]);
        rp[k] = lr_;
      } else {
        leaf_eval2<GRAD, false>(P.leaf[k][l], P.b2[k][l], op, xl[k][l], lr_, a, dk[k][l]);
        if (SIG == 0 || leaf_has_r(op)) rq[k] = mul(rq[k], lr_);
      }
    }
    r = sig_product_poly_q(SIG, k, L) ? mul(rq[k], rp[k]) : rq[k];
    a = add(a, splat(off_lo[k]));
    rk[k] = r;
    const bool on = SIG != 0 ? sig_product_used(SIG, k, L) : k < P.nK;
    ak[k] = make_float2((on && r.x != 0.f) ? a.x : -1e30f, (on && r.y != 0.f) ? a.y : -1e30f);
  }
  float2 M = ak[0];
#pragma unroll
  for (int k = 1; k < K; ++k) M = make_float2(fmaxf(M.x, ak[k].x), fmaxf(M.y, ak[k].y));
  float2 S = splat(0.f);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float2 t = sub(ak[k], M);
    const float2 e = make_float2(ex2(t.x), ex2(t.y));
    if (SIG == 0 || sig_product_has_r(SIG, k, L)) {
      rq[k] = mul(rq[k], e);  // the product's value without its PQ factor
      rk[k] = sig_product_poly_q(SIG, k, L) ? mul(rq[k], rp[k]) : rq[k];
    } else {
      rk[k] = e;
    }
    S = fma(splat(P.w_hi[k]), rk[k], fma(splat(P.w_lo[k]), rk[k], S));
  }
  // S > 0 also excludes an event where no product is present (M = -1e30): every product then
  // has r = 0 or w = 0.  The logarithm of a lane with S <= 0 is not used.
  ok0 = S.x > 0.f;
  ok1 = S.y > 0.f;
  logf = add(M, make_float2(lg2(S.x), lg2(S.y)));
  if constexpr (GRAD) {
    const float2 invS = rcp(S);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      ck[k] = mul(rk[k], invS);
      qk[k] = sig_product_poly_q(SIG, k, L) ? mul(rq[k], invS) : ck[k];
    }
  }
}

// Compensated FP32 accumulator of an event pair (one Kahan sum per lane, packed).
struct Kahan2 {
  float2 s = {0.f, 0.f}, c = {0.f, 0.f};
  __device__ __forceinline__ void add(float2 x) {
    const float2 y = pk::sub(x, c);
    const float2 t = pk::add(s, y);
    c = pk::sub(pk::sub(t, s), y);
    s = t;
  }
};


// Midpoint coordinate of bin idx of a 1-D grid as a double-float (the FP32 path's grid_coord).
__device__ __forceinline__ void grid_coord_f(float lo_hi, float lo_lo, float h_hi, float h_lo, int64_t idx, float& x,
                                             float& xlo) {
  const float off = (float)idx + 0.5f;
  const float p = off * h_hi;
  const float perr = fmaf(off, h_hi, -p) + off * h_lo;
  const ddf xs = dd_add({lo_hi, lo_lo}, dd_make(p, perr));
  x = xs.hi;
  xlo = xs.lo;
}

// Midpoint coordinate of bin idx of grid dimension d (double-float in the FP32 path).
template <typename T>
__device__ __forceinline__ void grid_coord(const GridDev& G, int d, int64_t idx, T& x, T& xlo) {
  if constexpr (sizeof(T) == 4) {
    grid_coord_f(G.lo_hi[d], G.lo_lo[d], G.h_hi[d], G.h_lo[d], idx, x, xlo);
  } else {
    x = G.lo64[d] + ((double)idx + 0.5) * G.h64[d];
    xlo = 0.0;
  }
}

// Separable grid normalisation inside the event kernel.  When every leaf of a product acts on
// its own observable, log N_k = sum_l [log(h_l S_l) + a_l] with one 1-D midpoint sum S_l per
// leaf (as grid_sep_kernel computes it), a few hundred leaf evaluations in all; every block
// evaluates them itself at its start instead of waiting for a normalisation kernel, from
// by-value constants only.  Leaf slot sl goes to warp 7 - sl mod 8 (warp 0 issues the block's
// first tile copies meanwhile); its lanes take the bins in a fixed order, kGridIlp at a time
// evaluated independently and added in bin order, accumulate in double-float (exact products by fma) and reduce by a fixed
// exchanging butterfly, so every block obtains bit-identical sums s_raw[k L + l] =
// {S, D_1, D_2, D_3} (D_j = sum of U d log(leaf) / d c_j).  Only the offsets -log N_k are needed before the
// events: one lane per product forms them in FP32 arithmetic (log_dd).  The ratios D_j / S
// that the gradient needs are formed by the last block alone (event_finish_fused), so that
// the prologue every block pays holds no FP64 arithmetic (GB300's FP64 pipe is 1/64 of FP32
// and its latency dominated this step).
// Bins of one leaf evaluated independently per step of the prologue's loop (their latencies
// overlap; the sums still run in bin order).
constexpr int kGridIlp = 4;

template <int K, int L, bool GRAD>
__device__ __forceinline__ void fused_grid_norm(const EvConst<float, K, L>& P, const EvNorm<K, L, GRAD>& N,
                                                ddf (*s_raw)[4], float (*s_off)[2], float (&off_hi)[K],
                                                float (&off_lo)[K]) {
  constexpr int NW = kBlock / 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // one copy of the loop for every warp (a run-time slot index; the slot's constants are
  // selected from the parameter bank), so that the warps share its instructions
#pragma unroll 1
  for (int sl = NW - 1 - warp; sl < K * L; sl += NW) {
    const int nb = N.nb[sl];
    if (nb == 0) continue;
    LeafReg<float> lr = P.leaf[0][0];
#pragma unroll
    for (int t = 1; t < K * L; ++t)
      if (t == sl) lr = P.leaf[t / L][t % L];
    const float aref = N.aref_hi[sl], aref_lo = N.aref_lo[sl];
    const float lo_hi = N.lo_hi[sl], lo_lo = N.lo_lo[sl], h_hi = N.h_hi[sl], h_lo = N.h_lo[sl];
    ddf acc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    for (int i0 = 0; i0 < nb; i0 += 32 * kGridIlp) {
      float U[kGridIlp], D[kGridIlp][3];
#pragma unroll
      for (int u = 0; u < kGridIlp; ++u) {
        const int i = i0 + 32 * u + lane;
        U[u] = D[u][0] = D[u][1] = D[u][2] = 0.f;
        if (i < nb) {
          float x, xlo, r, a, dl[3];
          grid_coord_f(lo_hi, lo_lo, h_hi, h_lo, i, x, xlo);
          leaf_eval<true, true>(lr, x, r, a, dl, xlo);
          U[u] = r * expf((a - aref) - aref_lo);
#pragma unroll
          for (int jj = 0; jj < 3; ++jj) D[u][jj] = dl[jj];
        }
      }
      // in bin order (an absent bin adds an exact zero)
#pragma unroll
      for (int u = 0; u < kGridIlp; ++u) {
        acc[0] = dd_add(acc[0], ddf{U[u], 0.f});
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) {
          const float pr = U[u] * D[u][jj];
          acc[1 + jj] = dd_add(acc[1 + jj], ddf{pr, fmaf(U[u], D[u][jj], -pr)});
        }
      }
    }
    const ddf tot = dd_warp_sum4(acc);
    if ((lane & 7) == 0) s_raw[sl][lane >> 3] = tot;
  }
  __syncthreads();
  if (warp == 0 && lane < K) {
    // log N_k = log prod_l (h_l S_l) + sum_l a_l, one lane per product, the product in
    // double-float and its logarithm in FP32 with the exponent split off exactly (log_dd):
    // about 3e-8 absolute, i.e. 1e-8 of the NLL of ten million events, with no FP64 latency
    // in the prologue every block pays
    ddf prod = {1.f, 0.f}, aref = {0.f, 0.f};
    bool any = false;
    for (int l = 0; l < L; ++l) {
      const int sl = lane * L + l;
      if (N.nb[sl] == 0) continue;
      prod = dd_mul(prod, dd_mul({N.h_hi[sl], N.h_lo[sl]}, s_raw[sl][0]));
      aref = dd_add(aref, dd_make(N.aref_hi[sl], N.aref_lo[sl]));
      any = true;
    }
    const ddf logN = any ? dd_add(log_dd(prod), aref) : ddf{0.f, 0.f};
    s_off[lane][0] = -logN.hi;
    s_off[lane][1] = -logN.lo;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    off_hi[k] = s_off[k][0];
    off_lo[k] = s_off[k][1];
  }
}

// Block reduction, last-block reduction over the blocks and the final FP64 combination of the
// self-normalising pair kernel:
//   d NLL / d theta_p = - sum_k C_k dw_kp + sum_{k,l,j: par = p} w_k (C_k D_klj / S_kl - A_klj),
// the normalisation terms D_klj / S_kl formed here from the block's own grid sums.  Thread p
// takes parameter p; its terms are formed independently and added by a fixed pairwise tree
// (the combination is bound by FP64 latency, not throughput).  buf: NS * blockDim
// double-floats of shared memory (the tile buffers, idle now) for the block reduction.
template <int K, int L, bool GRAD, unsigned long long SIG>
__device__ __forceinline__ void event_finish_fused(const ddf (&v)[EventLanes<float, K, L, GRAD, SIG>::NS],
                                                   unsigned bad, const EvNorm<K, L, GRAD>& N,
                                                   const ddf (*s_raw)[4], int nK, float2* partials,
                                                   unsigned* counters, double* result, int out_mode, ddf* buf,
                                                   unsigned* s_bad) {
  constexpr int NS = EventLanes<float, K, L, GRAD, SIG>::NS;
  constexpr int NT = GRAD ? K + K * L * 3 : 1;  // terms of one parameter's gradient
  __shared__ double s_out[NS];
  __shared__ double s_w[K];
  __shared__ double s_t[K * L][3];
  __shared__ int s_par[K][L][3];
  __shared__ ddf s_red[kBlock / 32];
  const int p = threadIdx.x;
  const int P = N.n_params;
  double dwp[GRAD ? K : 1];
  if constexpr (GRAD) {
#pragma unroll
    for (int k = 0; k < K; ++k) dwp[k] = (p < P && k < nK) ? N.dw[k][p] : 0.0;
    for (int t = threadIdx.x; t < K * L * 3; t += blockDim.x) {
      const int k = t / (L * 3), l = (t / 3) % L, jj = t % 3;
      s_par[k][l][jj] = k < nK ? N.par[k][l][jj] : -1;
    }
    if (threadIdx.x < K) s_w[threadIdx.x] = N.w[threadIdx.x];
  }
  for (int m = 16; m > 0; m >>= 1) bad += __shfl_xor_sync(0xffffffffu, bad, m);
  if ((threadIdx.x & 31) == 0) s_bad[threadIdx.x >> 5] = bad;
  block_reduce_transpose<NS>(v, partials, buf);
  if (threadIdx.x == 0) {
    unsigned b = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += s_bad[w];
    if (b) atomicAdd(counters + 1, b);
  }
  if (!last_block_ticket(counters, gridDim.x)) return;
  // every other block added to these words before its ticket (and a fence): plain L2 reads,
  // issued before the reduction so that their latency overlaps it
  unsigned nbad = 0u, status = 0u, nrange = 0u;
  if (threadIdx.x == 0) {
    nbad = __ldcg(counters + 1);
    status = __ldcg(counters + kStatusWord);
    nrange = __ldcg(counters + kRangeWord);
  }
  if constexpr (GRAD) {
    // the normalisation terms D_j / S of every leaf slot, from this block's grid sums (the
    // quotient in double-float, then FP64)
    for (int t = threadIdx.x; t < K * L * 3; t += blockDim.x) {
      const int sl = t / 3, jj = t % 3;
      s_t[sl][jj] = N.nb[sl] ? dd_to_double(dd_div(s_raw[sl][1 + jj], s_raw[sl][0])) : 0.0;
    }
  }
  reduce_partials<24>(partials, NS, gridDim.x, s_out, s_red, blockDim.x);

  // ---- final combination (last block, FP64) ----
  const int off = out_mode == 0 ? 2 : 3;
  if (p < P) {
    double tm[NT];
    if constexpr (GRAD) {
#pragma unroll
      for (int k = 0; k < K; ++k) tm[k] = k < nK ? -s_out[1 + k] * dwp[k] : 0.0;
#pragma unroll
      for (int k = 0; k < K; ++k)
#pragma unroll
        for (int l = 0; l < L; ++l)
#pragma unroll
          for (int jj = 0; jj < 3; ++jj) {
            double term = 0.0;
            if (a_present<K, L, SIG>(k, l, jj) && s_par[k][l][jj] == p)
              term = s_w[k] * (s_out[1 + k] * s_t[k * L + l][jj] - s_out[a_lane<K, L, SIG>(k, l, jj)]);
            tm[K + (k * L + l) * 3 + jj] = term;
          }
      // fixed pairwise tree over the NT terms
#pragma unroll
      for (int w = 1; w < NT; w *= 2)
#pragma unroll
        for (int i = 0; i + w < NT; i += 2 * w) tm[i] += tm[i + w];
    } else {
      tm[0] = 0.0;
    }
    result[off + p] = tm[0];
  }
  if (threadIdx.x == 0) {
    counters[0] = 0u;  // the ticket
    counters[1] = 0u;
    counters[kStatusWord] = 0u;
    counters[kRangeWord] = 0u;
    // a device wait that gave up is reported as -1, events outside the observable limits
    // (direct reads of host columns) as -(2 + their count)
    const double nb = nrange ? -2.0 - (double)nrange : status ? -1.0 : (double)nbad;
    result[0] = -s_out[0];
    if (out_mode == 0) {
      result[1] = nb;
    } else {
      result[1] = 0.0;
      result[2] = nb;
    }
  }
  result_complete(result, P > 1 ? P : 1);
}

template <int K, int L, bool GRAD>
struct EventOcc2 {
  static constexpr int value = (K * L <= 6 && !GRAD) ? 3 : 2;
};

// Per-thread accumulators of the pair kernel.
template <int K, int L>
struct PairAcc {
  Kahan2 lf;   // compensated sum of the tiles' subtotals of log2 f
  float2 lt;   // this tile's subtotal (at most kPairsPerThread pairs, plain FP32)
  float2 C[K];
  float2 A[K][L][3];
  unsigned bad;
};

// One event pair: evaluate and accumulate the lanes that are in range (v0, v1) with f > 0.
template <int K, int L, bool GRAD, unsigned long long SIG = 0>
__device__ __forceinline__ void pair_step(const EvConst<float, K, L>& P, const float (&off_hi)[K],
                                          const float (&off_lo)[K], const float2 (&xl)[K][L], bool v0, bool v1,
                                          PairAcc<K, L>& S) {
  float2 logf, ck[K], qk[K], dk[K][L][3];
  bool ok0, ok1;
  eval_event2<K, L, GRAD, SIG>(P, off_hi, off_lo, xl, logf, ok0, ok1, ck, qk, dk);
  const bool m0 = v0 && ok0, m1 = v1 && ok1;
  S.bad += (unsigned)(v0 && !ok0) + (unsigned)(v1 && !ok1);
  if (m0 && m1) {
    S.lt = pk::add(S.lt, logf);
    if constexpr (GRAD) {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        S.C[k] = pk::add(S.C[k], ck[k]);
#pragma unroll
        for (int l = 0; l < L; ++l)
#pragma unroll
          for (int q = 0; q < 3; ++q)
            if (SIG == 0 || q < leaf_nder(sig_op(SIG, k * L + l)))  // a specialised kernel skips absent lanes
              S.A[k][l][q] = pk::fma(sig_poly_q(SIG, k, l, L) ? qk[k] : ck[k], dk[k][l][q], S.A[k][l][q]);
      }
    }
  } else {
    // one lane outside the range or with f <= 0: accumulate the other lane alone
#pragma unroll
    for (int lane = 0; lane < 2; ++lane) {
      if (!(lane ? m1 : m0)) continue;
      (lane ? S.lt.y : S.lt.x) += lane ? logf.y : logf.x;
      if constexpr (GRAD) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const float c = lane ? ck[k].y : ck[k].x;
          const float cq = lane ? qk[k].y : qk[k].x;
          (lane ? S.C[k].y : S.C[k].x) += c;
#pragma unroll
          for (int l = 0; l < L; ++l)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
              if (SIG != 0 && q >= leaf_nder(sig_op(SIG, k * L + l))) continue;
              float& A = lane ? S.A[k][l][q].y : S.A[k][l][q].x;
              A = fmaf(sig_poly_q(SIG, k, l, L) ? cq : c, lane ? dk[k][l][q].y : dk[k][l][q].x, A);
            }
        }
      }
    }
  }
}

// Leaf slot (k, l)'s observable in a compile-time column map COLS (2 bits per slot, slot
// k * L + l), the companion of a nonzero signature SIG.
__host__ __device__ constexpr int cols_col(unsigned long long cols, int slot) { return (int)((cols >> (2 * slot)) & 3ull); }

// Work split.  The events [begin, end) are an 8-aligned core [A, B) plus a head [begin, A) and
// a tail [B, end) of fewer than 8 events each.  Block b takes the contiguous range
// [A + b c, A + (b + 1) c) of the core (c = the core divided by the grid, rounded up to 8
// events), so every block has the same number of events to within one tile's worth at the
// end of the grid; the first block also evaluates the head and the last block the tail,
// reading them from global memory.  A block's range runs in tiles of up to TE =
// 2 * kPairsPerThread * kBlock events (the last tile of a range is shorter; every tile starts
// and ends on 8-event boundaries, so its bulk copies are 16-byte aligned multiples of 16
// bytes), staged in shared memory kEventStages tiles ahead.  Within a tile thread t takes the
// pairs t, t + kBlock, ...
//
// Warps consume tiles independently: each warp waits for a tile's copies on the stage's
// mbarrier, evaluates its pairs and counts itself done with the buffer in s_done[stage]; the
// warp that completes the count refills the buffer with the tile kEventStages ahead.  No
// block barrier separates tiles, so a warp that is fast on one tile runs ahead on the next
// instead of waiting for the slowest warp.
// Dynamic shared memory: kEventStages * n_obs * TE floats.
template <int K, int L, bool GRAD, unsigned long long SIG = 0, unsigned long long COLS = 0, bool DIRECT = false>
__global__ void __launch_bounds__(kBlock, EventOcc2<K, L, GRAD>::value)
    sop_event2_kernel(const ModelDev* __restrict__ md, const EvConst<float, K, L> P,
                      const __grid_constant__ EvNorm<K, L, GRAD> N, Cols<float> cols, int64_t begin, int64_t end,
                      float2* partials, unsigned* counters, double* result, int out_mode, int fused_norm) {
  using namespace pk;
  constexpr int NS = EventLanes<float, K, L, GRAD, SIG>::NS;
  constexpr int PPT = kPairsPerThread;
  constexpr int TE = 2 * PPT * kBlock;
  constexpr int NST = kEventStages;
  constexpr unsigned NWARP = kBlock / 32;
  __shared__ ddf s_red[(kBlock / 32) * NS > kBlock ? (kBlock / 32) * NS : kBlock];
  __shared__ unsigned s_bad[kBlock / 32];
  __shared__ __align__(8) uint64_t s_bar[NST];
  __shared__ unsigned s_done[NST];  // warps done with each stage's buffer, counted over all its tiles
  __shared__ int s_last[NST];       // the last tile issued into each stage (-1: none)
  __shared__ unsigned s_fail;
  __shared__ ddf s_raw[K * L][4];
  __shared__ float s_off[K][2];
  extern __shared__ __align__(128) float s_col[];  // [NST][nobs][TE]
  const int nobs = P.nobs;
  const int lane = threadIdx.x & 31;
  const int64_t A = min(end, (begin + 7) & ~(int64_t)7);
  const int64_t B = max(A, end & ~(int64_t)7);
  const int64_t chunk = ((B - A) + (int64_t)gridDim.x * 8 - 1) / ((int64_t)gridDim.x * 8) * 8;
  const int64_t r0 = min(B, A + (int64_t)blockIdx.x * chunk), r1 = min(B, r0 + chunk);
  const int ntile = (int)((r1 - r0 + TE - 1) / TE);
  auto tile_count = [&](int j) { return (int)min((int64_t)TE, r1 - (r0 + (int64_t)j * TE)); };
  auto buf = [&](int st, int c) { return s_col + ((size_t)st * nobs + c) * TE; };
  const unsigned withhold = withheld_tile(counters);
  // one thread stages tile j in buffer j % NST (a withheld tile's copies are never issued, so
  // its waits run out: the failure-detection test hook)
  auto issue = [&](int j) {
    if (j >= ntile || (withhold && j == (int)withhold - 1)) return;
    const int st = j % NST;
    const unsigned bytes = (unsigned)tile_count(j) * (unsigned)sizeof(float);
    const int64_t t0 = r0 + (int64_t)j * TE;
    s_last[st] = j;
    mbar_arrive_expect_tx(&s_bar[st], (unsigned)nobs * bytes);
    for (int c = 0; c < nobs; ++c) bulk_load(buf(st, c), cols.c[c] + t0, bytes, &s_bar[st]);
  };
  // DIRECT (a GOO_BORROW_HOST dataset): the columns are read straight from host memory, so
  // no copies are staged; a separate instantiation, so that the staged kernel carries none of
  // its code
  constexpr bool direct = DIRECT;
  if (threadIdx.x < 32) {
    // warp 0 stages the first NST tiles: lane 0 initialises the barriers and posts each
    // stage's expected bytes, then the lanes issue one column copy each (none when the
    // columns are read directly)
    if (lane == 0) {
      for (int st = 0; st < NST; ++st) {
        mbar_init(&s_bar[st], 1);
        s_done[st] = 0u;
        s_last[st] = -1;
      }
      s_fail = 0u;
      mbar_init_fence();
      for (int j = 0; j < NST && j < ntile && !direct; ++j) {
        if (withhold && j == (int)withhold - 1) continue;
        s_last[j] = j;
        mbar_arrive_expect_tx(&s_bar[j], (unsigned)nobs * (unsigned)tile_count(j) * (unsigned)sizeof(float));
      }
    }
    __syncwarp();
    for (int q = lane; q < NST * nobs && !direct; q += 32) {
      const int j = q / nobs, c = q % nobs;
      if (j < ntile && !(withhold && j == (int)withhold - 1))
        bulk_load(buf(j, c), cols.c[c] + r0 + (int64_t)j * TE, (unsigned)tile_count(j) * (unsigned)sizeof(float),
                  &s_bar[j]);
    }
  }
  // the column copies above read only the dataset; the normalisation written by the
  // previous kernel in the stream is read after this point
  grid_dep_wait();
  float off_hi[K], off_lo[K];
  const int nK = P.nK;
  if (fused_norm) {
    fused_grid_norm<K, L, GRAD>(P, N, s_raw, s_off, off_hi, off_lo);  // synchronises the block
  } else {
    load_offsets<float, K>(md, off_hi, off_lo);
    __syncthreads();  // barriers initialised before any thread waits on them
  }
  // the pair evaluation's exponents are in base 2: -log2 N_k = -log N_k log2(e), in double-float
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const ddf o = dd_mul(ddf{off_hi[k], off_lo[k]}, ddf{kLog2eHi, kLog2eLo});
    off_hi[k] = o.hi;
    off_lo[k] = o.lo;
  }
  PairAcc<K, L> S;
  S.bad = 0;
  S.lt = splat(0.f);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    S.C[k] = splat(0.f);
#pragma unroll
    for (int l = 0; l < L; ++l)
#pragma unroll
      for (int q = 0; q < 3; ++q) S.A[k][l][q] = splat(0.f);
  }
  // column of leaf slot (k, l): compile-time in a specialised kernel
  auto leaf_col = [&](int k, int l) { return SIG != 0 ? cols_col(COLS, k * L + l) : P.leaf[k][l].col; };
  const long long wlim = tile_wait_limit(counters);
  bool failed = false;
  unsigned nout = 0;  // events outside the observable limits (direct reads)
  auto in_range = [&](float v, int c) { return v >= cols.lo[c] && v <= cols.hi[c]; };  // false for NaN
  for (int j = 0; j < ntile; ++j) {
    const int st = j % NST;
    if (direct) {
      // this thread's pairs of tile j straight from the host columns (over the host link),
      // every load issued before any is used, into its own slots of the stage buffer, which
      // no other thread reads: the evaluation below is the staged path's, unchanged
      const int npair_d = tile_count(j) >> 1;
      const int64_t t0 = r0 + (int64_t)j * TE;
      float2 xd[PPT][kMaxObs];
#pragma unroll
      for (int u = 0; u < PPT; ++u) {
        const int pr = threadIdx.x + u * kBlock;
#pragma unroll
        for (int c = 0; c < kMaxObs; ++c)
          xd[u][c] = (pr < npair_d && c < nobs) ? reinterpret_cast<const float2*>(cols.c[c] + t0)[pr]
                                                : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < PPT; ++u) {
        const int pr = threadIdx.x + u * kBlock;
        if (pr >= npair_d) continue;
        bool ok0 = true, ok1 = true;
#pragma unroll
        for (int c = 0; c < kMaxObs; ++c) {
          if (c >= nobs) continue;
          ok0 = ok0 && in_range(xd[u][c].x, c);
          ok1 = ok1 && in_range(xd[u][c].y, c);
          reinterpret_cast<float2*>(buf(st, c))[pr] = xd[u][c];
        }
        nout += (ok0 ? 0u : 1u) + (ok1 ? 0u : 1u);
      }
    } else if (!__all_sync(0xffffffffu, mbar_wait(&s_bar[st], (unsigned)(j / NST) & 1u, wlim))) {
      // the whole warp agrees on whether the tile arrived in time
      failed = true;
      break;
    }
    const int npair = tile_count(j) >> 1;
    int coff[K][L];
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int l = 0; l < L; ++l) coff[k][l] = (st * nobs + leaf_col(k, l)) * TE;
#pragma unroll 1
    for (int u = 0; u < PPT; ++u) {
      const int pr = threadIdx.x + u * kBlock;
      if (pr >= npair) break;
      // each leaf reads its observable's staged column (an unused slot reads column 0 and is
      // ignored)
      float2 xl[K][L];
#pragma unroll
      for (int k = 0; k < K; ++k)
#pragma unroll
        for (int l = 0; l < L; ++l) xl[k][l] = reinterpret_cast<const float2*>(s_col + coff[k][l])[pr];
      pair_step<K, L, GRAD, SIG>(P, off_hi, off_lo, xl, true, true, S);
    }
    S.lf.add(S.lt);
    S.lt = splat(0.f);
    // this warp is done with buffer st; the warp that completes the count for tile j refills
    // it: every warp's reads of the buffer precede its count (block-scope fences around the
    // shared atomic), and the refilling thread orders them before the asynchronous copy
    __syncwarp();
    if (lane == 0 && !direct) {
      __threadfence_block();
      const unsigned done = atomicAdd(&s_done[st], 1u) + 1u;
      if (done == (unsigned)(j / NST + 1) * NWARP) {
        __threadfence_block();
        fence_proxy_async();
        issue(j + NST);
      }
    }
  }
  // head and tail (fewer than 8 events each) from global memory: pairs at even indices
  auto ragged = [&](int64_t lo, int64_t hi) {
    const int64_t i = (lo & ~(int64_t)1) + 2 * (int64_t)threadIdx.x;
    if (i >= hi) return;
    const bool v0 = i >= lo, v1 = i + 1 < hi;
    float2 x[kMaxObs];
    bool ok0 = true, ok1 = true;
#pragma unroll
    for (int c = 0; c < kMaxObs; ++c) {
      x[c] = splat(0.f);
      if (c < nobs) {
        // plain loads: the columns may be host memory (direct reads)
        if (v0 && v1) x[c] = *reinterpret_cast<const float2*>(cols.c[c] + i);
        else if (v0) x[c].x = cols.c[c][i];
        else x[c].y = cols.c[c][i + 1];
        ok0 = ok0 && in_range(x[c].x, c);
        ok1 = ok1 && in_range(x[c].y, c);
      }
    }
    if (direct) nout += (v0 && !ok0 ? 1u : 0u) + (v1 && !ok1 ? 1u : 0u);
    float2 xl[K][L];
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int l = 0; l < L; ++l) xl[k][l] = pk::pick(leaf_col(k, l), x[0], x[1], x[2], x[3]);
    pair_step<K, L, GRAD, SIG>(P, off_hi, off_lo, xl, v0, v1, S);
  };
  if (!failed) {
    if (blockIdx.x == 0 && A > begin) ragged(begin, A);
    if (blockIdx.x == gridDim.x - 1 && end > B) ragged(B, end);
    S.lf.add(S.lt);
  }
  if (failed && lane == 0) atomicOr(&s_fail, 1u);
  if (direct) {
    // events outside the limits: counted before the ticket, reported by the last block
    for (int m = 16; m > 0; m >>= 1) nout += __shfl_xor_sync(0xffffffffu, nout, m);
    if (lane == 0 && nout) atomicAdd(counters + kRangeWord, nout);
  }
  __syncthreads();
  if (s_fail) {
    // a copy did not arrive in time: record it, then wait (again bounded, with the default
    // limit) for this block's copies still in flight before its shared memory is released;
    // the copies of one stage complete in order, so the last one issued is waited for
    if (threadIdx.x == 0) {
      atomicOr(counters + kStatusWord, 1u);
      for (int st = 0; st < NST; ++st)
        if (s_last[st] >= 0) mbar_wait(&s_bar[st], (unsigned)(s_last[st] / NST) & 1u);
    }
    __syncthreads();
  }
  // lanes: the two Kahan sums as one double-float (log2 f, turned into natural logarithms),
  // the gradient lanes as the lane sums, each times its constant factor (leaf_eval2)
  ddf v[NS];
  v[0] = dd_mul(dd_add(dd_make(S.lf.s.x, -S.lf.c.x), dd_make(S.lf.s.y, -S.lf.c.y)), ddf{kLn2Hi, kLn2Lo});
  if constexpr (GRAD) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      v[1 + k] = dd_add(ddf{S.C[k].x, 0.f}, ddf{S.C[k].y, 0.f});
#pragma unroll
      for (int l = 0; l < L; ++l)
#pragma unroll
        for (int q = 0; q < 3; ++q)
          if (a_present<K, L, SIG>(k, l, q)) {
            const int op = SIG != 0 ? sig_op(SIG, k * L + l) : P.leaf[k][l].op;
            ddf t = dd_add(ddf{S.A[k][l][q].x, 0.f}, ddf{S.A[k][l][q].y, 0.f});
            if (op == GOO_OP_GAUSS && q < 2) t = dd_mul(t, ddf{P.leaf[k][l].c[2], 0.f});
            if (op == GOO_OP_ARGUS && q == 0) t = dd_mul(t, ddf{P.leaf[k][l].c[5], 0.f});
            if (op == GOO_OP_ARGUS && q == 2) t = dd_mul(t, ddf{kLn2Hi, kLn2Lo});
            v[a_lane<K, L, SIG>(k, l, q)] = t;
          }
    }
  }
  if (fused_norm)
    event_finish_fused<K, L, GRAD, SIG>(v, S.bad, N, s_raw, nK, partials, counters, result, out_mode,
                                        reinterpret_cast<ddf*>(s_col), s_bad);
  else
    event_finish<K, L, GRAD, SIG>(v, S.bad, MdFin{md, nK}, nK, partials, counters, result, out_mode, s_red, s_bad);
}

}  // namespace goo
