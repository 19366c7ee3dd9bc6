// serve.cu -- toy-MC pseudo-experiment fits served with continuous batching, and the
// batched NLL + gradient of many independent (model, dataset, theta) triples.
//
// Paper: toy MC generation for multi-body systems, used for integration and signal
// generation in the amplitude analyses (Sec. 5); the FitManager fits a PDF to a dataset
// (Fig. 1).  A toy study repeats "generate a pseudo-experiment, fit it" many times; here
// many such fits of uneven size share the GPU:
//   * admission: a request needs 72 bytes per event (two float32 columns and the float32
//     amplitude cache) from one device arena; requests are admitted in arrival order while
//     a fit slot and arena space are free;
//   * generation (on the device): candidate j of a toy with seed s draws Philox4x64-10
//     (Salmon et al., SC'11) outputs w0..w3 at counter (j,0,0,0), key (s, 0x6f6f67); the top
//     32 bits of w0 pick a cell of an envelope grid over the Dalitz box with probability
//     proportional to the cell's bound on |S|^2 (importance sampling), 24-bit float uniforms
//     from w1, w2 place the point in the cell, and it is accepted when
//     u(w3) * bound < |S(s12, s13)|^2 (truth coefficients); the toy is the first n accepted
//     candidates in candidate order, so it does not depend on how toys are batched;
//   * one batched launch per round evaluates NLL and gradient of every active fit at its
//     current trial point; each fit is split into fixed tiles whose partial sums are
//     reduced per fit in tile order, so a fit's result is bit-identical alone or in a mix;
//   * one thread per fit advances that fit's minimiser (BFGS, line search, then Newton
//     steps on a finite-difference Hessian of the gradient, whose inverse gives the errors)
//     and writes the next trial point; minimiser state stays on the device.
// Control crosses the host/device boundary once per round, not once per fit.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <set>
#include <vector>

#include "common.cuh"
#include "dalitz.cuh"
#include "model.cuh"

namespace goo {

constexpr int kSrvKB = 8;                   // resonance slots of the server kernels
constexpr int kSrvKA = kSrvKB + 1;          // + the fixed reference (non-resonant) amplitude
constexpr int kSrvMaxP = 2 * kSrvKB;        // free coefficient parameters per fit
constexpr int kSrvLanes = 1 + 2 * kSrvKA;   // sum log|S|^2 and 2 lanes per amplitude slot
constexpr int kGenPerThread = 16;
constexpr int kGenBlockCands = kBlock * kGenPerThread;
constexpr uint64_t kToyKey1 = 0x6F6F67ull;
constexpr int kEnvCells = 96;     // default envelope grid: kEnvCells x kEnvCells cells
constexpr int kEnvSub = 6;        // lattice points per cell side of the envelope scan
constexpr float kEnvFactor = 1.2f;  // default bound: factor x the 3 x 3 neighbourhood maximum

// ---------------------------------------------------------------------------------------
// Philox4x64-10
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void philox4x64(uint64_t (&c)[4], uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += W0;
      k1 += W1;
    }
    const uint64_t hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
    const uint64_t hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
    const uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

__device__ __forceinline__ float u24(uint64_t w) { return (float)(uint32_t)(w >> 40) * 5.9604644775390625e-8f; }

// ---------------------------------------------------------------------------------------
// toy generation
// ---------------------------------------------------------------------------------------
// Generator constants.  Proposal: a cell (i, j) of an n12 x n13 grid over the Dalitz box,
// chosen by the top 32 bits of the first Philox word against cumulative thresholds thr[]
// (cell c has probability (thr[c] - thr[c-1]) / 2^32, proportional to its envelope bound), a
// point uniform in the cell, and acceptance u * bound[cell] < |S|^2.
struct GenConst {
  float lo12, lo13, cw12, cw13;  // box corner and cell widths (float)
  float M2, m1s, m2s, m3s;       // squared masses (float) for the inside test
  float cr[kSrvKA], ci[kSrvKA];  // generating coefficients (slots: resonances, then reference)
  int nbw, n12, n13, pad;
  const float* bound;                   // per-cell envelope of |S|^2 (device)
  const unsigned long long* thr;        // per-cell cumulative thresholds (device)
  unsigned long long* viol;             // candidates inside the region with |S|^2 > bound (device)
};

// One toy of a generation pass: candidates [cand0, cand0 + nblocks * kGenBlockCands) in
// blocks of kGenBlockCands; `have` events are already accepted, `n` are wanted.
struct GenToy {
  int64_t cand0, nblocks, have, n;
  uint64_t seed;
  float* s12;
  float* s13;
  float4* cache;
};

// Candidate j of the toy with this seed: its point, its cell's bound and u * bound (the
// acceptance threshold); false when the point lies outside the kinematic region.
__device__ __forceinline__ bool gen_point(const GenConst& g, uint64_t seed, int64_t j, float& s12, float& s13,
                                          float& bnd, float& ub) {
  uint64_t c[4] = {(uint64_t)j, 0ull, 0ull, 0ull};
  philox4x64(c, seed, kToyKey1);
  const unsigned long long top = c[0] >> 32;
  int lo = 0, hi = g.n12 * g.n13 - 1;  // first cell with top < thr[cell]; thr[last] = 2^32
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (top < __ldg(g.thr + mid)) hi = mid;
    else lo = mid + 1;
  }
  const int ci = lo / g.n13, cj = lo - ci * g.n13;
  s12 = __fadd_rn(g.lo12, __fmul_rn(__fadd_rn((float)ci, u24(c[1])), g.cw12));
  s13 = __fadd_rn(g.lo13, __fmul_rn(__fadd_rn((float)cj, u24(c[2])), g.cw13));
  bnd = __ldg(g.bound + lo);
  ub = __fmul_rn(u24(c[3]), bnd);
  // inside the Dalitz region: s13 range at fixed s12 from the energies of particles 1 and 3
  // in the (12) rest frame
  const float r = sqrtf(s12);
  const float e1 = (s12 + g.m1s - g.m2s) / (2.f * r);
  const float e3 = (g.M2 - s12 - g.m3s) / (2.f * r);
  const float p1 = sqrtf(fmaxf(e1 * e1 - g.m1s, 0.f));
  const float p3 = sqrtf(fmaxf(e3 * e3 - g.m3s, 0.f));
  const float es = (e1 + e3) * (e1 + e3);
  return s13 > es - (p1 + p3) * (p1 + p3) && s13 < es - (p1 - p3) * (p1 - p3) && e3 > sqrtf(g.m3s);
}

// Candidate j: point and acceptance; the amplitudes of an accepted candidate are returned in
// (ar, ai).
__device__ __forceinline__ bool gen_candidate(const GenConst& g, const DalitzDev& dd, uint64_t seed, int64_t j,
                                              float& s12, float& s13, float (&ar)[kSrvKB], float (&ai)[kSrvKB]) {
  float bnd, ub;
  if (!gen_point(g, seed, j, s12, s13, bnd, ub)) return false;
  const float s23 = (float)(dd.sumsq - (double)s12 - (double)s13);
  float sr = g.cr[kSrvKB], si = g.ci[kSrvKB];  // reference amplitude A = 1
#pragma unroll
  for (int k = 0; k < kSrvKB; ++k) {
    if (k < g.nbw) {
      bw_amp<float>(dd.bwf[k], s12, s13, s23, ar[k], ai[k]);
      sr += g.cr[k] * ar[k] - g.ci[k] * ai[k];
      si += g.cr[k] * ai[k] + g.ci[k] * ar[k];
    } else {
      ar[k] = ai[k] = 0.f;
    }
  }
  return ub < sr * sr + si * si;
}

// Acceptance of candidate j only (the amplitudes are summed on the fly, not kept); nviol counts
// candidates whose |S|^2 exceeds their cell's bound (the envelope does not bound |S|^2 there).
__device__ __forceinline__ bool gen_accept(const GenConst& g, const DalitzDev& dd, uint64_t seed, int64_t j,
                                           unsigned& nviol) {
  float s12, s13, bnd, ub;
  if (!gen_point(g, seed, j, s12, s13, bnd, ub)) return false;
  const float s23 = (float)(dd.sumsq - (double)s12 - (double)s13);
  float sr = g.cr[kSrvKB], si = g.ci[kSrvKB];
  for (int k = 0; k < g.nbw; ++k) {
    float ar, ai;
    bw_amp<float>(dd.bwf[k], s12, s13, s23, ar, ai);
    sr += g.cr[k] * ar - g.ci[k] * ai;
    si += g.cr[k] * ai + g.ci[k] * ar;
  }
  const float s2 = sr * sr + si * si;
  nviol += s2 > bnd ? 1u : 0u;
  return ub < s2;
}

__device__ __forceinline__ int gen_find_toy(const int64_t* __restrict__ bprefix, int ntoys, int64_t b) {
  int lo = 0, hi = ntoys - 1;  // largest t with bprefix[t] <= b
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (bprefix[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void gen_load_dd(DalitzDev& dd, const DalitzDev* ddp) {
  for (int i = threadIdx.x; i < (int)(sizeof(DalitzDev) / 4); i += blockDim.x) ((int*)&dd)[i] = ((const int*)ddp)[i];
}

// Pass 1: accepted candidates per block (each thread owns kGenPerThread consecutive ones);
// the per-thread accept masks are kept for the write pass.
__global__ void __launch_bounds__(kBlock, 2) toy_count_kernel(const __grid_constant__ GenConst g, const DalitzDev* ddp,
                                                           const GenToy* __restrict__ toys,
                                                           const int64_t* __restrict__ bprefix, int ntoys,
                                                           unsigned* counts, unsigned short* masks) {
  __shared__ DalitzDev dd;
  __shared__ unsigned s_warp[kBlock / 32];
  gen_load_dd(dd, ddp);
  __syncthreads();
  const int t = gen_find_toy(bprefix, ntoys, blockIdx.x);
  const GenToy& T = toys[t];
  const int64_t first = T.cand0 + (int64_t)(blockIdx.x - bprefix[t]) * kGenBlockCands + (int64_t)threadIdx.x * kGenPerThread;
  unsigned mask = 0, nviol = 0;
  for (int r = 0; r < kGenPerThread; ++r)
    if (gen_accept(g, dd, T.seed, first + r, nviol)) mask |= 1u << r;
  masks[(size_t)blockIdx.x * kBlock + threadIdx.x] = (unsigned short)mask;
  if (__any_sync(0xffffffffu, nviol != 0)) {
    for (int m = 16; m > 0; m >>= 1) nviol += __shfl_xor_sync(0xffffffffu, nviol, m);
    if ((threadIdx.x & 31) == 0 && nviol) atomicAdd(g.viol, (unsigned long long)nviol);
  }
  unsigned cnt = __popc(mask);
  for (int m = 16; m > 0; m >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, m);
  if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned tot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += s_warp[w];
    counts[blockIdx.x] = tot;
  }
}

// Pass 2 (one block per toy): exclusive scan of the toy's block counts in candidate order;
// out_base[b] = position of block b's first accepted event, or -1 when the toy is complete
// before it (or the block accepted nothing); accepted[2t] = events of toy t after this pass
// (capped at n), accepted[2t+1] = candidates it accepted in this pass.
__global__ void toy_scan_kernel(const GenToy* __restrict__ toys, const int64_t* __restrict__ bprefix,
                                const unsigned* __restrict__ counts, int* out_base, int64_t* accepted) {
  __shared__ int64_t s_sum[kBlock];
  const GenToy& T = toys[blockIdx.x];
  const int64_t b0 = bprefix[blockIdx.x], nb = T.nblocks;
  int64_t running = T.have;
  for (int64_t c0 = 0; c0 < nb; c0 += blockDim.x) {
    const int64_t b = c0 + threadIdx.x;
    const int64_t v = b < nb ? (int64_t)counts[b0 + b] : 0;
    s_sum[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {  // Hillis-Steele inclusive scan
      const int64_t add = threadIdx.x >= o ? s_sum[threadIdx.x - o] : 0;
      __syncthreads();
      s_sum[threadIdx.x] += add;
      __syncthreads();
    }
    if (b < nb) {
      const int64_t base = running + s_sum[threadIdx.x] - v;
      out_base[b0 + b] = (v > 0 && base < T.n) ? (int)base : -1;
    }
    running += s_sum[blockDim.x - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    accepted[2 * blockIdx.x] = running < T.n ? running : T.n;  // capped at n
    accepted[2 * blockIdx.x + 1] = running - T.have;           // accepted in this pass
  }
}

// Pass 3: accepted candidates (from the count pass's per-thread masks) of blocks with
// out_base >= 0 are re-evaluated and written in candidate order (event columns and the
// amplitude-cache planes).
__global__ void __launch_bounds__(kBlock, 2) toy_write_kernel(const __grid_constant__ GenConst g, const DalitzDev* ddp,
                                                           const GenToy* __restrict__ toys,
                                                           const int64_t* __restrict__ bprefix, int ntoys,
                                                           const int* __restrict__ out_base,
                                                           const unsigned short* __restrict__ masks) {
  __shared__ DalitzDev dd;
  __shared__ unsigned s_warp[kBlock / 32];
  const int ob = out_base[blockIdx.x];
  if (ob < 0) return;  // uniform over the block
  gen_load_dd(dd, ddp);
  __syncthreads();
  const int t = gen_find_toy(bprefix, ntoys, blockIdx.x);
  const GenToy& T = toys[t];
  const int64_t first = T.cand0 + (int64_t)(blockIdx.x - bprefix[t]) * kGenBlockCands + (int64_t)threadIdx.x * kGenPerThread;
  unsigned mask = masks[(size_t)blockIdx.x * kBlock + threadIdx.x];
  const unsigned cnt = __popc(mask);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned incl = cnt;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  unsigned before = 0;
  for (int w = 0; w < warp; ++w) before += s_warp[w];
  int64_t pos = (int64_t)ob + before + (incl - cnt);
  while (mask && pos < T.n) {
    const int r = __ffs(mask) - 1;
    mask &= mask - 1;
    float s12, s13, ar[kSrvKB], ai[kSrvKB];
    gen_candidate(g, dd, T.seed, first + r, s12, s13, ar, ai);
    T.s12[pos] = s12;
    T.s13[pos] = s13;
#pragma unroll
    for (int p = 0; p < kSrvKB / 2; ++p)
      if (2 * p < g.nbw) T.cache[(int64_t)p * T.n + pos] = make_float4(ar[2 * p], ai[2 * p], ar[2 * p + 1], ai[2 * p + 1]);
    ++pos;
  }
}

// ---------------------------------------------------------------------------------------
// batched NLL + gradient over (fit, tile) work items
// ---------------------------------------------------------------------------------------
struct SrvEval {
  const float4* cache;   // amplitude planes of the fit's dataset
  int64_t n;             // events
  int64_t plane;         // plane stride (events of the dataset the cache was built for)
  int64_t begin;         // first event of the fit's range
  float cr[kSrvKA], ci[kSrvKA];  // trial coefficients: resonance slots, then the reference
};

struct SrvResult {
  double nll;
  double gre[kSrvKA], gim[kSrvKA];  // dNLL/dRe c, dNLL/dIm c per slot
  double norm;
  unsigned bad;
  unsigned pad;
};

struct SrvModel {   // shared by every fit of a batch
  double G[kSrvKA * kSrvKA * 2];  // Gram matrix in slot order
  int nbw, has_ref;
};

// tiles[t] = (fit, tile index within the fit); fit_tiles[fit] = (number of tiles, first tile).
// A block takes work items t = blockIdx.x, + gridDim.x, ...; each item is consumed in
// sub-tiles of kSrvSub events whose amplitude planes are staged in shared memory by bulk
// copies (every event is one 16-byte float4 per plane, so any sub-range is a legal copy),
// kSrvStages sub-tiles ahead of the consumers.  Dynamic shared memory:
// kSrvStages * (kSrvKB / 2) * kSrvSub float4.  status[0] is set when a copy wait gave up;
// wait_limit bounds each wait for a sub-tile in SM clocks (the drain before exit allows
// kWaitCycles).
constexpr int kSrvSub = 768;
constexpr int kSrvStages = 2;
constexpr size_t kSrvSmem = (size_t)kSrvStages * (kSrvKB / 2) * kSrvSub * sizeof(float4);

__global__ void __launch_bounds__(kBlock, 2) srv_nll_kernel(const SrvEval* __restrict__ ev, const int2* __restrict__ tiles,
                                                           const int2* __restrict__ fit_tiles, int ntiles,
                                                           int tile_events, const SrvModel* __restrict__ sm,
                                                           float2* tile_partials, unsigned* fit_ticket,
                                                           SrvResult* results, unsigned* status,
                                                           long long wait_limit) {
  __shared__ ddf s_red[(kBlock / 32) * kSrvLanes > kBlock ? (kBlock / 32) * kSrvLanes : kBlock];
  __shared__ unsigned s_bad[kBlock / 32];
  __shared__ bool s_last;
  __shared__ double s_fin[kSrvLanes];
  __shared__ __align__(8) uint64_t s_bar[kSrvStages];
  extern __shared__ __align__(128) float4 s_amp[];  // [kSrvStages][kSrvKB / 2][kSrvSub]
  constexpr int NST = kSrvStages, TE = kSrvSub, NP = kSrvKB / 2;
  __shared__ double s_G[kSrvKA * kSrvKA * 2];
  for (int q = threadIdx.x; q < kSrvKA * kSrvKA * 2; q += blockDim.x) s_G[q] = sm->G[q];
  const int nbw = sm->nbw;
  const int planes = (nbw + 1) / 2;
  // the event range [b0, b1) of work item t
  auto item_range = [&](int t, int64_t& b0, int64_t& b1) {
    const SrvEval& e = ev[tiles[t].x];
    b0 = e.begin + (int64_t)tiles[t].y * tile_events;
    b1 = min(e.begin + e.n, b0 + tile_events);
  };
  auto nsub_of = [&](int t) {
    int64_t b0, b1;
    item_range(t, b0, b1);
    return b1 > b0 ? (int)((b1 - b0 + TE - 1) / TE) : 1;  // an empty item still takes one (empty) step
  };
  // producer cursor (thread 0): work item pt, sub-tile ps, job number pj
  int pt = blockIdx.x, ps = 0, pj = 0;
  auto issue_next = [&]() {
    if (pt >= ntiles) return;
    int64_t b0, b1;
    item_range(pt, b0, b1);
    const SrvEval& e = ev[tiles[pt].x];
    const int64_t lo = b0 + (int64_t)ps * TE, hi = min(b1, lo + TE);
    uint64_t* bar = &s_bar[pj % NST];
    if (hi > lo) {
      mbar_arrive_expect_tx(bar, (unsigned)(planes * (hi - lo) * sizeof(float4)));
      for (int p = 0; p < planes; ++p)
        bulk_load(s_amp + ((size_t)(pj % NST) * NP + p) * TE, e.cache + (int64_t)p * e.plane + lo,
                  (unsigned)((hi - lo) * sizeof(float4)), bar);
    } else {
      mbar_arrive(bar);
    }
    ++pj;
    if (++ps == nsub_of(pt)) {
      ps = 0;
      pt += gridDim.x;
    }
  };
  if (threadIdx.x == 0) {
    for (int st = 0; st < NST; ++st) mbar_init(&s_bar[st], 1);
    mbar_init_fence();
    for (int q = 0; q < NST; ++q) issue_next();
  }
  __syncthreads();  // barriers initialised before any thread waits on them
  int j = 0;  // consumer job number
  bool failed = false;
  for (int t = blockIdx.x; t < ntiles && !failed; t += gridDim.x) {
    const int fit = tiles[t].x;
    const SrvEval& e = ev[fit];
    const int2 ft = fit_tiles[fit];
    int64_t b0, b1;
    item_range(t, b0, b1);
    const int nsub = nsub_of(t);
    float2 cre[kSrvKA], cim[kSrvKA];
#pragma unroll
    for (int k = 0; k < kSrvKA; ++k) {
      cre[k] = pk::splat(e.cr[k]);
      cim[k] = pk::splat(e.ci[k]);
    }
    Kahan acc;
    float2 G1[kSrvKA], G2[kSrvKA];
#pragma unroll
    for (int k = 0; k < kSrvKA; ++k) G1[k] = G2[k] = pk::splat(0.f);
    unsigned bad = 0;
    for (int sub = 0; sub < nsub; ++sub, ++j) {
      const int st = j % NST;
      const bool ok_wait = mbar_wait(&s_bar[st], (unsigned)(j / NST) & 1u, wait_limit);
      const int64_t lo = b0 + (int64_t)sub * TE;
      const int64_t left = b1 - lo;
      const int cnt = left <= 0 ? 0 : (left < TE ? (int)left : TE);
      if (ok_wait) {
        const float4* sb = s_amp + (size_t)st * NP * TE;  // plane p at sb + p * TE
        for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
          float2 amp[kSrvKA];
#pragma unroll
          for (int p = 0; p < NP; ++p) {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (p < planes) v = sb[p * TE + q];
            amp[2 * p] = make_float2(v.x, v.y);
            amp[2 * p + 1] = make_float2(v.z, v.w);
          }
          amp[kSrvKB] = make_float2(1.f, 0.f);
          coh_event_pk<kSrvKA, true>(cre, cim, amp, acc, G1, G2, bad);
        }
      }
      // every thread is done with buffer st (and agrees on whether a wait gave up) before
      // the buffer is refilled
      if (__syncthreads_or(!ok_wait)) {
        failed = true;
        break;
      }
      if (threadIdx.x == 0) {
        fence_proxy_async();
        issue_next();
      }
    }
    if (failed) break;
    float gre[kSrvKA], gim[kSrvKA];
#pragma unroll
    for (int k = 0; k < kSrvKA; ++k) {
      gre[k] = G1[k].x - G2[k].y;
      gim[k] = G1[k].y + G2[k].x;
    }
    ddf v[kSrvLanes];
    v[0] = acc.value();
#pragma unroll
    for (int k = 0; k < kSrvKA; ++k) {
      v[1 + 2 * k] = {gre[k], 0.f};
      v[2 + 2 * k] = {gim[k], 0.f};
    }
    for (int m = 16; m > 0; m >>= 1) bad += __shfl_xor_sync(0xffffffffu, bad, m);
    __syncthreads();  // s_red / s_bad reuse across tiles
    if ((threadIdx.x & 31) == 0) s_bad[threadIdx.x >> 5] = bad;
    {
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
      for (int s = 0; s < kSrvLanes; ++s) {
        const ddf w = dd_warp_sum(v[s]);
        if (lane == 0) s_red[warp * kSrvLanes + s] = w;
      }
      __syncthreads();
      if (threadIdx.x < kSrvLanes) {
        ddf a = s_red[threadIdx.x];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) a = dd_add(a, s_red[w * kSrvLanes + threadIdx.x]);
        tile_partials[(size_t)t * kSrvLanes + threadIdx.x] = make_float2(a.hi, a.lo);
      }
      if (threadIdx.x == kSrvLanes) {
        unsigned bb = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) bb += s_bad[w];
        if (bb) atomicAdd(&results[fit].bad, bb);
      }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&fit_ticket[fit], 1u) == (unsigned)(ft.x - 1);
    __syncthreads();
    if (!s_last) continue;
    __threadfence();
    // last tile of this fit: reduce its tiles in order
    if (threadIdx.x < kSrvLanes) {
      // tiles in index order, eight independent loads in flight at a time
      ddf a = {0.f, 0.f};
      int k = 0;
      for (; k + 8 <= ft.x; k += 8) {
        float2 q[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) q[u] = __ldcg(tile_partials + (size_t)(ft.y + k + u) * kSrvLanes + threadIdx.x);
#pragma unroll
        for (int u = 0; u < 8; ++u) a = dd_add(a, {q[u].x, q[u].y});
      }
      for (; k < ft.x; ++k) {
        const float2 q = __ldcg(tile_partials + (size_t)(ft.y + k) * kSrvLanes + threadIdx.x);
        a = dd_add(a, {q.x, q.y});
      }
      s_fin[threadIdx.x] = dd_to_double(a);
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      // warp 0: N = c^H G c and the per-slot gradients (slot k: lane k)
      const int k = threadIdx.x;
      double vr = 0.0, vi = 0.0, ckr = 0.0, cki = 0.0;
      const bool live = k < kSrvKA && (k < nbw || (k == kSrvKB && sm->has_ref));
      if (live) {
        ckr = (double)cre[k].x;
        cki = (double)cim[k].x;
        for (int l = 0; l < kSrvKA; ++l) {
          const bool lv = l < nbw || (l == kSrvKB && sm->has_ref);
          if (!lv) continue;
          const double gr = s_G[2 * (k * kSrvKA + l)], gi = s_G[2 * (k * kSrvKA + l) + 1];
          const double clr = (double)cre[l].x, cli = (double)cim[l].x;
          vr += gr * clr + gi * cli;
          vi += gi * clr - gr * cli;
        }
      }
      double Nk = live ? ckr * vr - cki * vi : 0.0;
      for (int m = 16; m > 0; m >>= 1) Nk += __shfl_xor_sync(0xffffffffu, Nk, m);
      const double nev = (double)e.n;
      SrvResult& R = results[fit];
      if (k < kSrvKA) {
        R.gre[k] = live ? -2.0 * s_fin[1 + 2 * k] + nev * 2.0 * vr / Nk : 0.0;
        R.gim[k] = live ? 2.0 * s_fin[2 + 2 * k] - nev * 2.0 * vi / Nk : 0.0;
      }
      if (k == 0) {
        R.nll = -s_fin[0] + nev * log(Nk);
        R.norm = Nk;
        fit_ticket[fit] = 0u;
      }
    }
    __syncthreads();
  }
  if (failed && threadIdx.x == 0) {
    // a copy did not arrive in time: record it, then wait (again bounded) for the copies this
    // block still has in flight before its shared memory is released
    atomicOr(status, 1u);
    for (int q = j; q < pj; ++q) mbar_wait(&s_bar[q % NST], (unsigned)(q / NST) & 1u);
  }
}

// ---------------------------------------------------------------------------------------
// device minimiser: one thread per fit
// ---------------------------------------------------------------------------------------
enum SrvPhase { PH_FREE = 0, PH_START = 1, PH_LINE = 2, PH_HESS = 3, PH_NEWTON = 4, PH_DONE = 5 };

struct SrvState {
  int phase, P, it, ls, hj, newton, status, evals;
  double f, ft, alpha, gd, edm, best_edm, ftol_rel;
  int stale, restarts;
  double x[kSrvMaxP], g[kSrvMaxP], d[kSrvMaxP], xt[kSrvMaxP], gt[kSrvMaxP];
  double Hi[kSrvMaxP * kSrvMaxP];   // BFGS inverse Hessian, then inverse FD Hessian
  double Hf[kSrvMaxP * kSrvMaxP];   // FD Hessian under construction
  double gp[kSrvMaxP];              // gradient at x + h e_j
  double c0r[kSrvKB], c0i[kSrvKB];  // start coefficients (free slots)
  double err[kSrvMaxP];
  float ref_r, ref_i;               // fixed reference coefficient
};

struct SrvParams {
  double scale[kSrvMaxP];  // parameter scales (x units)
  double edm_tol;
  int max_iter;
  int nbw;
};

__device__ void srv_set_trial(SrvState& s, const SrvParams& sp, SrvEval& e, const double* x) {
  for (int p = 0; p < s.P; ++p) s.xt[p] = x[p];
  for (int k = 0; k < kSrvKB; ++k) {
    if (k < sp.nbw) {
      e.cr[k] = (float)(s.c0r[k] + x[2 * k] * sp.scale[2 * k]);
      e.ci[k] = (float)(s.c0i[k] + x[2 * k + 1] * sp.scale[2 * k + 1]);
    } else {
      e.cr[k] = e.ci[k] = 0.f;
    }
  }
  e.cr[kSrvKB] = s.ref_r;
  e.ci[kSrvKB] = s.ref_i;
}

// Gauss-Jordan inverse of an n x n matrix (row-major) in place; false if singular.
__device__ bool srv_invert(double* A, double* inv, int n) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) inv[i * n + j] = (i == j) ? 1.0 : 0.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(A[r * n + c]) > fabs(A[piv * n + c])) piv = r;
    if (!(fabs(A[piv * n + c]) > 0)) return false;
    if (piv != c)
      for (int k = 0; k < n; ++k) {
        double t = A[c * n + k];
        A[c * n + k] = A[piv * n + k];
        A[piv * n + k] = t;
        t = inv[c * n + k];
        inv[c * n + k] = inv[piv * n + k];
        inv[piv * n + k] = t;
      }
    const double dinv = 1.0 / A[c * n + c];
    for (int k = 0; k < n; ++k) {
      A[c * n + k] *= dinv;
      inv[c * n + k] *= dinv;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = A[r * n + c];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        A[r * n + k] -= f * A[c * n + k];
        inv[r * n + k] -= f * inv[c * n + k];
      }
    }
  }
  return true;
}

// Cholesky factorisation of a copy of the symmetric n x n matrix A: true if every pivot is
// positive (A positive definite).
__device__ bool srv_positive_definite(const double* A, int n) {
  double L[kSrvMaxP * kSrvMaxP];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j <= i; ++j) {
      double v = A[i * n + j];
      for (int k = 0; k < j; ++k) v -= L[i * n + k] * L[j * n + k];
      if (i == j) {
        if (!(v > 0)) return false;
        L[i * n + i] = sqrt(v);
      } else {
        L[i * n + j] = v / L[j * n + j];
      }
    }
  return true;
}

__device__ double srv_edm(const SrvState& s, const double* g) {
  double e = 0.0;
  for (int a = 0; a < s.P; ++a)
    for (int b = 0; b < s.P; ++b) e += 0.5 * g[a] * s.Hi[a * s.P + b] * g[b];
  return e;
}

constexpr double kHessStep = 1e-3;  // finite-difference step in units of the parameter scale
constexpr int kSrvRestarts = 3;     // returns from the Newton phase to the quasi-Newton phase

__device__ void srv_begin_hessian(SrvState& s, const SrvParams& sp, SrvEval& e) {
  s.phase = PH_HESS;
  s.hj = 0;
  double xp[kSrvMaxP];
  for (int p = 0; p < s.P; ++p) xp[p] = s.x[p];
  xp[0] += kHessStep;
  srv_set_trial(s, sp, e, xp);
}

__device__ void srv_propose(SrvState& s, const SrvParams& sp, SrvEval& e) {
  const int P = s.P;
  double gd = 0.0;
  for (int a = 0; a < P; ++a) {
    double v = 0.0;
    for (int b = 0; b < P; ++b) v -= s.Hi[a * P + b] * s.g[b];
    s.d[a] = v;
    gd += s.g[a] * v;
  }
  if (!(gd < 0)) {
    for (int a = 0; a < P * P; ++a) s.Hi[a] = 0.0;
    gd = 0.0;
    for (int a = 0; a < P; ++a) {
      s.Hi[a * P + a] = 1.0;
      s.d[a] = -s.g[a];
      gd -= s.g[a] * s.g[a];
    }
  }
  s.gd = gd;
  s.edm = -0.5 * gd;
  if (s.edm < 0.5 * s.best_edm) {
    s.best_edm = s.edm;
    s.stale = 0;
  } else {
    s.stale++;
  }
  if (s.edm < sp.edm_tol || s.it >= sp.max_iter || s.stale >= 10) {
    srv_begin_hessian(s, sp, e);
    return;
  }
  double gmax = 0.0;
  for (int a = 0; a < P; ++a) gmax = fmax(gmax, fabs(s.d[a]));
  s.alpha = (s.it == 0 && gmax > 1.0) ? 1.0 / gmax : 1.0;
  s.ls = 0;
  double xt[kSrvMaxP];
  for (int a = 0; a < P; ++a) xt[a] = s.x[a] + s.alpha * s.d[a];
  srv_set_trial(s, sp, e, xt);
  s.phase = PH_LINE;
}

// Back to the quasi-Newton phase from the current point, its inverse Hessian the inverse of
// the finite-difference Hessian where that is positive definite, else the inverse of its
// diagonal magnitudes.  Used when the Newton phase finds the Hessian indefinite or its steps
// stall (a step that does not lower the EDM, or four steps short of the tolerance): on small
// samples the likelihood can be far from quadratic where the quasi-Newton phase stopped, its
// curvature estimate having put the EDM under the tolerance too early.
__device__ void srv_restart(SrvState& s, const SrvParams& sp, SrvEval& e, bool pd) {
  const int P = s.P;
  if (!pd)
    for (int a = 0; a < P; ++a)
      for (int b = 0; b < P; ++b)
        s.Hi[a * P + b] = (a == b) ? 1.0 / fmax(fabs(s.Hf[a * P + a]), 1e-12) : 0.0;
  s.restarts++;
  s.newton = 0;
  s.best_edm = HUGE_VAL;
  s.stale = 0;
  s.status = 0;
  srv_propose(s, sp, e);
}

__global__ void srv_bfgs_kernel(SrvState* states, SrvEval* evals, const SrvResult* results, const SrvParams* spp,
                                const int* slots, int nslots, int* done_list, unsigned* done_count) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nslots) return;
  const int fit = slots[q];
  SrvState& s = states[fit];
  SrvEval& e = evals[fit];
  const SrvParams& sp = *spp;
  const SrvResult& R = results[fit];
  const int P = s.P;
  if (s.phase == PH_FREE || s.phase == PH_DONE) return;
  s.evals++;
  // result at the trial point, in x units
  double gx[kSrvMaxP];
  for (int k = 0; k < P / 2; ++k) {
    gx[2 * k] = R.gre[k] * sp.scale[2 * k];
    gx[2 * k + 1] = R.gim[k] * sp.scale[2 * k + 1];
  }
  const double fx = (R.bad > 0) ? HUGE_VAL : R.nll;
  bool finite = isfinite(fx);
  for (int a = 0; a < P && finite; ++a) finite = isfinite(gx[a]);
  switch (s.phase) {
    case PH_START: {
      if (!finite) {
        s.status = 3;
        s.phase = PH_DONE;
        break;
      }
      s.f = fx;
      for (int a = 0; a < P; ++a) s.g[a] = gx[a];
      for (int a = 0; a < P * P; ++a) s.Hi[a] = 0.0;
      for (int a = 0; a < P; ++a) s.Hi[a * P + a] = 1.0;
      s.best_edm = HUGE_VAL;
      srv_propose(s, sp, e);
      break;
    }
    case PH_LINE: {
      const double ftol = s.ftol_rel * fabs(s.f);
      if (finite && fx <= s.f + 1e-4 * s.alpha * s.gd + ftol) {
        // accept; BFGS update if the curvature condition holds
        double sy = 0.0, yy = 0.0, ss = 0.0;
        double sv[kSrvMaxP], yv[kSrvMaxP];
        for (int a = 0; a < P; ++a) {
          sv[a] = s.xt[a] - s.x[a];
          yv[a] = gx[a] - s.g[a];
          sy += sv[a] * yv[a];
          yy += yv[a] * yv[a];
          ss += sv[a] * sv[a];
        }
        if (s.it == 0 && sy > 0 && yy > 0)
          for (int a = 0; a < P * P; ++a) s.Hi[a] *= sy / yy;
        if (sy > 1e-12 * sqrt(yy * ss)) {
          const double rho = 1.0 / sy;
          double Hy[kSrvMaxP];
          double yHy = 0.0;
          for (int a = 0; a < P; ++a) {
            double v = 0.0;
            for (int b = 0; b < P; ++b) v += s.Hi[a * P + b] * yv[b];
            Hy[a] = v;
            yHy += yv[a] * v;
          }
          for (int a = 0; a < P; ++a)
            for (int b = 0; b < P; ++b)
              s.Hi[a * P + b] += -rho * (Hy[a] * sv[b] + sv[a] * Hy[b]) + (rho * rho * yHy + rho) * sv[a] * sv[b];
        }
        for (int a = 0; a < P; ++a) {
          s.x[a] = s.xt[a];
          s.g[a] = gx[a];
        }
        s.f = fx;
        s.it++;
        srv_propose(s, sp, e);
      } else {
        // shrink the step: secant root of the directional derivative when it changed sign
        double next = 0.5 * s.alpha;
        if (finite) {
          double gdt = 0.0;
          for (int a = 0; a < P; ++a) gdt += gx[a] * s.d[a];
          if (gdt > 0) next = s.alpha * s.gd / (s.gd - gdt);
        }
        s.alpha = fmin(0.5 * s.alpha, fmax(0.1 * s.alpha, next));
        if (++s.ls > 40) {
          s.status = 2;
          srv_begin_hessian(s, sp, e);
          break;
        }
        double xt[kSrvMaxP];
        for (int a = 0; a < P; ++a) xt[a] = s.x[a] + s.alpha * s.d[a];
        srv_set_trial(s, sp, e, xt);
      }
      break;
    }
    case PH_HESS: {
      // trial hj: parameter hj/2 shifted by +h (even) or -h (odd)
      const int j = s.hj / 2;
      if (!finite) {
        s.status = 3;
        s.phase = PH_DONE;
        break;
      }
      if ((s.hj & 1) == 0) {
        for (int a = 0; a < P; ++a) s.gp[a] = gx[a];
      } else {
        for (int a = 0; a < P; ++a) s.Hf[j * P + a] = (s.gp[a] - gx[a]) / (2 * kHessStep);
      }
      s.hj++;
      if (s.hj < 2 * P) {
        double xp[kSrvMaxP];
        for (int p = 0; p < P; ++p) xp[p] = s.x[p];
        xp[s.hj / 2] += (s.hj & 1) ? -kHessStep : kHessStep;
        srv_set_trial(s, sp, e, xp);
        break;
      }
      for (int a = 0; a < P; ++a)
        for (int b = a + 1; b < P; ++b) {
          const double v = 0.5 * (s.Hf[a * P + b] + s.Hf[b * P + a]);
          s.Hf[a * P + b] = s.Hf[b * P + a] = v;
        }
      double A[kSrvMaxP * kSrvMaxP];
      for (int a = 0; a < P * P; ++a) A[a] = s.Hf[a];
      const bool pd = srv_positive_definite(s.Hf, P);
      if (!srv_invert(A, s.Hi, P)) {
        if (s.restarts < kSrvRestarts) {
          srv_restart(s, sp, e, false);
          break;
        }
        s.status = 4;
        s.phase = PH_DONE;
        break;
      }
      s.edm = srv_edm(s, s.g);
      for (int a = 0; a < P; ++a) {
        const double v = s.Hi[a * P + a];
        s.err[a] = v > 0 ? sqrt(v) * sp.scale[a] : NAN;
      }
      if (s.edm < sp.edm_tol && pd) {
        s.status = 0;
        s.phase = PH_DONE;
        break;
      }
      if (s.restarts < kSrvRestarts && (!pd || s.newton >= 4)) {
        srv_restart(s, sp, e, pd);
        break;
      }
      if (s.edm < sp.edm_tol || s.newton >= 4 || !pd) {
        s.status = !pd ? 3 : (s.edm < sp.edm_tol) ? 0 : 1;
        s.phase = PH_DONE;
        break;
      }
      // Newton step on the finite-difference Hessian
      for (int a = 0; a < P; ++a) {
        double v = 0.0;
        for (int b = 0; b < P; ++b) v -= s.Hi[a * P + b] * s.g[b];
        s.d[a] = v;
      }
      s.alpha = 1.0;
      double xt[kSrvMaxP];
      for (int a = 0; a < P; ++a) xt[a] = s.x[a] + s.d[a];
      srv_set_trial(s, sp, e, xt);
      s.phase = PH_NEWTON;
      break;
    }
    case PH_NEWTON: {
      // accept when the gradient-based EDM falls (the NLL value carries rounding noise)
      if (finite && srv_edm(s, gx) < s.edm) {
        for (int a = 0; a < P; ++a) {
          s.x[a] = s.xt[a];
          s.g[a] = gx[a];
        }
        s.f = fx;
        s.newton++;
        srv_begin_hessian(s, sp, e);
      } else if (s.alpha > 0.2) {
        s.alpha *= 0.5;
        double xt[kSrvMaxP];
        for (int a = 0; a < P; ++a) xt[a] = s.x[a] + s.alpha * s.d[a];
        srv_set_trial(s, sp, e, xt);
      } else if (s.restarts < kSrvRestarts) {
        srv_restart(s, sp, e, true);  // the Newton phase was entered with a positive-definite Hessian
      } else {
        s.status = 1;
        s.phase = PH_DONE;
      }
      break;
    }
    default:
      break;
  }
  if (s.phase == PH_DONE) {
    const unsigned k = atomicAdd(done_count, 1u);
    done_list[k] = fit;
  }
}

// ---------------------------------------------------------------------------------------
// envelope of the generator: per cell of the n12 x n13 grid, the largest |S|^2 (float32) on
// a sub x sub lattice of points (cell edges included) inside the kinematic region, and the
// lattice sum of |S|^2 (points outside the region count 0) for the acceptance estimate
// ---------------------------------------------------------------------------------------
__global__ void envelope_cells_kernel(const __grid_constant__ GenConst g, const DalitzDev* ddp, int sub,
                                      unsigned* cell_bits, float* cell_sum) {
  __shared__ DalitzDev dd;
  for (int i = threadIdx.x; i < (int)(sizeof(DalitzDev) / 4); i += blockDim.x) ((int*)&dd)[i] = ((const int*)ddp)[i];
  __syncthreads();
  const int ncell = g.n12 * g.n13, per = sub * sub;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)ncell * per;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int cell = (int)(idx / per), q = (int)(idx % per);
    const int ci = cell / g.n13, cj = cell % g.n13;
    const float s12 = g.lo12 + g.cw12 * (ci + (float)(q / sub) / (sub - 1));
    const float s13 = g.lo13 + g.cw13 * (cj + (float)(q % sub) / (sub - 1));
    const float r = sqrtf(s12);
    const float e1 = (s12 + g.m1s - g.m2s) / (2.f * r), e3 = (g.M2 - s12 - g.m3s) / (2.f * r);
    const float p1 = sqrtf(fmaxf(e1 * e1 - g.m1s, 0.f)), p3 = sqrtf(fmaxf(e3 * e3 - g.m3s, 0.f));
    const float es = (e1 + e3) * (e1 + e3);
    if (!(s13 >= es - (p1 + p3) * (p1 + p3) && s13 <= es - (p1 - p3) * (p1 - p3))) continue;
    const float s23 = (float)(dd.sumsq - (double)s12 - (double)s13);
    float sr = g.cr[kSrvKB], si = g.ci[kSrvKB];
    for (int k = 0; k < g.nbw; ++k) {
      float ar, ai;
      bw_amp<float>(dd.bwf[k], s12, s13, s23, ar, ai);
      sr += g.cr[k] * ar - g.ci[k] * ai;
      si += g.cr[k] * ai + g.ci[k] * ar;
    }
    atomicMax(cell_bits + cell, __float_as_uint(sr * sr + si * si));  // positive floats order as integers
    atomicAdd(cell_sum + cell, sr * sr + si * si);
  }
}

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------
struct ArenaBlock {
  size_t off, size;
};

struct Request {
  int64_t ticket;
  int64_t n;
  uint64_t seed;
  std::vector<double> theta_start;
};

struct Slot {
  int64_t ticket = -1;
  int64_t n = 0;
  uint64_t seed = 0;
  size_t off = 0, bytes = 0;
  std::vector<double> theta_start;
  float* s12 = nullptr;
  float* s13 = nullptr;
  float4* cache = nullptr;
};

struct FitOut {
  std::vector<double> theta, err;
  goo_fit_result res;
};

}  // namespace goo

struct goo_server {
  goo_ctx* ctx = nullptr;
  goo_model* model = nullptr;
  goo::AmpModelInfo info{};
  goo_server_options opt{};
  int P = 0;
  std::vector<double> theta_gen, xscale;
  // device
  unsigned char* arena = nullptr;
  size_t arena_bytes = 0;
  goo::SrvState* d_states = nullptr;
  goo::SrvEval* d_evals = nullptr;
  goo::SrvResult* d_results = nullptr;
  goo::SrvModel* d_model = nullptr;
  goo::SrvParams* d_params = nullptr;
  unsigned* d_tickets = nullptr;
  int2* d_fit_tiles = nullptr;
  int* d_slots = nullptr;
  int* d_done = nullptr;
  unsigned* d_done_count = nullptr;
  bool counted = false;  // included in ctx->live
  float* d_env_bound = nullptr;
  unsigned long long* d_env_thr = nullptr;
  unsigned* d_env_bits = nullptr;      // per-cell lattice maxima (float bits), then sums, then the
                                       // violation counter
  double env_max = 0.0, gen_violations = 0.0;
  int2* d_tiles = nullptr;
  size_t tiles_cap = 0;
  float2* d_tile_partials = nullptr;
  size_t partials_cap = 0;
  goo::GenToy* d_gtoys = nullptr;
  size_t gtoys_cap = 0;
  int64_t* d_bprefix = nullptr;
  size_t bprefix_cap = 0;
  unsigned* d_counts = nullptr;
  size_t counts_cap = 0;
  int* d_outbase = nullptr;
  size_t outbase_cap = 0;
  unsigned short* d_masks = nullptr;
  size_t masks_cap = 0;
  int64_t* d_accepted = nullptr;
  size_t accepted_cap = 0;
  goo::GenConst gen{};
  double gen_eff = 0.03;
  // host
  std::vector<goo::ArenaBlock> free_blocks;
  std::deque<goo::Request> queue;
  std::vector<goo::Slot> slots;
  std::vector<int> free_slots;
  std::vector<int> active;
  bool active_dirty = true;
  std::map<int64_t, goo::FitOut> done;
  std::deque<int64_t> finished;  // tickets that entered `done` and were not yet drained
  std::set<int64_t> fail_alloc;  // tickets whose admission fails its allocation (test hook)
  int64_t next_ticket = 1;
  int64_t rounds = 0, ntiles = 0;
  double eval_ms = 0.0, gen_ms = 0.0, gen_candidates = 0.0, gen_accepted = 0.0;
  int occ_nll = 0;
};

namespace goo {

static size_t al256(size_t b) { return (b + 255) / 256 * 256; }

static int arena_alloc(goo_server* s, size_t bytes, size_t* off) {
  bytes = al256(bytes);
  for (size_t i = 0; i < s->free_blocks.size(); ++i) {
    ArenaBlock& b = s->free_blocks[i];
    if (b.size >= bytes) {
      *off = b.off;
      b.off += bytes;
      b.size -= bytes;
      if (b.size == 0) s->free_blocks.erase(s->free_blocks.begin() + i);
      return GOO_OK;
    }
  }
  return GOO_ERR_OOM;
}

static void arena_free(goo_server* s, size_t off, size_t bytes) {
  s->free_blocks.push_back({off, al256(bytes)});
  std::sort(s->free_blocks.begin(), s->free_blocks.end(),
            [](const ArenaBlock& a, const ArenaBlock& b) { return a.off < b.off; });
  std::vector<ArenaBlock> merged;
  for (auto& b : s->free_blocks) {
    if (!merged.empty() && merged.back().off + merged.back().size == b.off) merged.back().size += b.size;
    else merged.push_back(b);
  }
  s->free_blocks.swap(merged);
}

static size_t fit_bytes(int64_t n, int nbw) {
  return al256((size_t)n * 4) * 2 + al256((size_t)((nbw + 1) / 2) * (size_t)n * sizeof(float4));
}

static int grow(void** p, size_t* cap, size_t need) {
  if (need <= *cap) return GOO_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  const size_t c = need + need / 2 + 4096;
  if (cudaMalloc(p, c) != cudaSuccess) {
    cudaGetLastError();
    return set_error(GOO_ERR_OOM, "server: cannot allocate %zu bytes of work space", c);
  }
  *cap = c;
  return GOO_OK;
}

// Generates the toys of newly admitted slots.  Each pass covers, per toy still short of
// events, enough candidates for the remaining events at the running acceptance estimate;
// count, ordered scan and write run on the device, and only per-toy records cross to the
// host.
static int generate(goo_server* s, const std::vector<int>& new_slots) {
  goo_ctx* ctx = s->ctx;
  const auto t0 = std::chrono::steady_clock::now();
  std::vector<int64_t> have(new_slots.size(), 0), cand(new_slots.size(), 0);
  for (int pass = 0; pass < 256; ++pass) {
    std::vector<GenToy> toys;
    std::vector<int> owner;
    std::vector<int64_t> bprefix(1, 0);
    for (size_t i = 0; i < new_slots.size(); ++i) {
      const Slot& sl = s->slots[new_slots[i]];
      const int64_t need = sl.n - have[i];
      if (need <= 0) continue;
      const int64_t nc = (int64_t)((double)need / s->gen_eff * 1.1) + kGenBlockCands;
      GenToy g{};
      g.cand0 = cand[i];
      g.nblocks = (nc + kGenBlockCands - 1) / kGenBlockCands;
      g.have = have[i];
      g.n = sl.n;
      g.seed = sl.seed;
      g.s12 = sl.s12;
      g.s13 = sl.s13;
      g.cache = sl.cache;
      toys.push_back(g);
      owner.push_back((int)i);
      bprefix.push_back(bprefix.back() + g.nblocks);
    }
    if (toys.empty()) break;
    const int nt = (int)toys.size();
    const int64_t nblocks = bprefix.back();
    if (nblocks > (int64_t)INT32_MAX) return set_error(GOO_ERR_UNSUPPORTED, "toy generation pass too large");
    GOO_TRY(grow((void**)&s->d_gtoys, &s->gtoys_cap, nt * sizeof(GenToy)));
    GOO_TRY(grow((void**)&s->d_bprefix, &s->bprefix_cap, (nt + 1) * sizeof(int64_t)));
    GOO_TRY(grow((void**)&s->d_counts, &s->counts_cap, nblocks * sizeof(unsigned)));
    GOO_TRY(grow((void**)&s->d_outbase, &s->outbase_cap, nblocks * sizeof(int)));
    GOO_TRY(grow((void**)&s->d_masks, &s->masks_cap, (size_t)nblocks * kBlock * sizeof(unsigned short)));
    GOO_TRY(grow((void**)&s->d_accepted, &s->accepted_cap, 2 * nt * sizeof(int64_t)));
    GOO_CUDA_TRY(cudaMemcpyAsync(s->d_gtoys, toys.data(), nt * sizeof(GenToy), cudaMemcpyHostToDevice, ctx->stream));
    GOO_CUDA_TRY(cudaMemcpyAsync(s->d_bprefix, bprefix.data(), (nt + 1) * sizeof(int64_t), cudaMemcpyHostToDevice,
                                 ctx->stream));
    const DalitzDev* dd = (const DalitzDev*)s->info.dalitz_dev;
    {
      LaunchScope ls(ctx, "toy_count");
      toy_count_kernel<<<(unsigned)nblocks, kBlock, 0, ctx->stream>>>(s->gen, dd, s->d_gtoys, s->d_bprefix, nt,
                                                                     s->d_counts, s->d_masks);
    }
    {
      LaunchScope ls(ctx, "toy_scan");
      toy_scan_kernel<<<nt, kBlock, 0, ctx->stream>>>(s->d_gtoys, s->d_bprefix, s->d_counts, s->d_outbase,
                                                      s->d_accepted);
    }
    {
      LaunchScope ls(ctx, "toy_write");
      toy_write_kernel<<<(unsigned)nblocks, kBlock, 0, ctx->stream>>>(s->gen, dd, s->d_gtoys, s->d_bprefix, nt,
                                                                     s->d_outbase, s->d_masks);
    }
    GOO_CUDA_TRY(cudaGetLastError());
    std::vector<int64_t> acc(2 * nt);
    unsigned long long viol = 0;
    GOO_CUDA_TRY(cudaMemcpyAsync(acc.data(), s->d_accepted, 2 * nt * sizeof(int64_t), cudaMemcpyDeviceToHost,
                                 ctx->stream));
    GOO_CUDA_TRY(cudaMemcpyAsync(&viol, s->gen.viol, sizeof viol, cudaMemcpyDeviceToHost, ctx->stream));
    GOO_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    s->gen_violations = (double)viol;
    if (log_level() >= 3) {
      std::vector<unsigned> cnt(nblocks);
      std::vector<int> ob(nblocks);
      cudaMemcpy(cnt.data(), s->d_counts, nblocks * sizeof(unsigned), cudaMemcpyDeviceToHost);
      cudaMemcpy(ob.data(), s->d_outbase, nblocks * sizeof(int), cudaMemcpyDeviceToHost);
      for (int t = 0; t < nt; ++t) {
        std::fprintf(stderr, "[goo] gen pass=%d toy=%d slot=%d seed=%llu cand0=%lld nblocks=%lld have=%lld n=%lld -> %lld (+%lld)\n",
                     pass, t, new_slots[owner[t]], (unsigned long long)toys[t].seed, (long long)toys[t].cand0,
                     (long long)toys[t].nblocks, (long long)toys[t].have, (long long)toys[t].n, (long long)acc[2 * t],
                     (long long)acc[2 * t + 1]);
        for (int64_t b = bprefix[t]; b < bprefix[t + 1] && b < bprefix[t] + 4; ++b)
          std::fprintf(stderr, "[goo]    block %lld count=%u out_base=%d\n", (long long)b, cnt[b], ob[b]);
      }
    }
    double raw = 0.0;
    for (int t = 0; t < nt; ++t) {
      const int i = owner[t];
      have[i] = acc[2 * t];
      raw += (double)acc[2 * t + 1];
      cand[i] = toys[t].cand0 + toys[t].nblocks * kGenBlockCands;
    }
    s->gen_candidates += (double)nblocks * kGenBlockCands;
    s->gen_accepted += raw;
    if (s->gen_accepted > 1000) s->gen_eff = s->gen_accepted / s->gen_candidates;
  }
  for (size_t i = 0; i < have.size(); ++i)
    if (have[i] < s->slots[new_slots[i]].n) return set_error(GOO_ERR_STATE, "toy generation did not converge");
  s->gen_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return GOO_OK;
}

static void init_state(goo_server* s, int slot, SrvState& st, SrvEval& ev) {
  const Slot& sl = s->slots[slot];
  std::memset(&st, 0, sizeof st);
  std::memset(&ev, 0, sizeof ev);
  st.phase = PH_START;
  st.P = s->P;
  st.ftol_rel = 1e-9;
  const AmpModelInfo& I = s->info;
  for (int k = 0; k < I.nbw; ++k) {
    st.c0r[k] = sl.theta_start[I.par_re[k]];
    st.c0i[k] = sl.theta_start[I.par_im[k]];
    ev.cr[k] = (float)st.c0r[k];
    ev.ci[k] = (float)st.c0i[k];
  }
  st.ref_r = (float)sl.theta_start[I.par_re[I.nbw]];
  st.ref_i = (float)sl.theta_start[I.par_im[I.nbw]];
  ev.cr[kSrvKB] = st.ref_r;
  ev.ci[kSrvKB] = st.ref_i;
  ev.cache = sl.cache;
  ev.n = sl.n;
  ev.plane = sl.n;
  ev.begin = 0;
}

// A fit that ends without a minimisation (cancelled, or its allocation failed): its result
// is the start point with zero errors, an infinite NLL and the given status.
static void finish_unfitted(goo_server* s, int64_t ticket, const std::vector<double>& theta_start, int status) {
  FitOut out;
  out.theta = theta_start;
  out.err.assign(theta_start.size(), 0.0);
  std::memset(&out.res, 0, sizeof out.res);
  out.res.nll = HUGE_VAL;
  out.res.status = status;
  s->done[ticket] = out;
  s->finished.push_back(ticket);
}

static int admit(goo_server* s, std::vector<int>& admitted) {
  while (!s->queue.empty() && !s->free_slots.empty()) {
    Request& r = s->queue.front();
    const size_t bytes = fit_bytes(r.n, s->info.nbw);
    size_t off = 0;
    if (s->fail_alloc.count(r.ticket)) {
      // the test hook: this fit's allocation fails; it ends alone, the queue moves on
      s->fail_alloc.erase(r.ticket);
      finish_unfitted(s, r.ticket, r.theta_start, GOO_FIT_ALLOC_FAILED);
      s->queue.pop_front();
      continue;
    }
    if (arena_alloc(s, bytes, &off) != GOO_OK) break;  // wait until memory frees up
    const int slot = s->free_slots.back();
    s->free_slots.pop_back();
    Slot& sl = s->slots[slot];
    sl.ticket = r.ticket;
    sl.n = r.n;
    sl.seed = r.seed;
    sl.off = off;
    sl.bytes = bytes;
    sl.theta_start = r.theta_start;
    sl.s12 = (float*)(s->arena + off);
    sl.s13 = (float*)(s->arena + off + al256((size_t)r.n * 4));
    sl.cache = (float4*)(s->arena + off + 2 * al256((size_t)r.n * 4));
    admitted.push_back(slot);
    s->queue.pop_front();
  }
  return GOO_OK;
}

static int upload_active(goo_server* s) {
  goo_ctx* ctx = s->ctx;
  const int T = s->opt.tile_events;
  std::vector<int2> tiles;
  std::vector<int2> fit_tiles(s->opt.max_fits, make_int2(0, 0));
  for (int slot : s->active) {
    const int64_t n = s->slots[slot].n;
    const int nt = (int)((n + T - 1) / T);
    fit_tiles[slot] = make_int2(nt, (int)tiles.size());
    for (int t = 0; t < nt; ++t) tiles.push_back(make_int2(slot, t));
  }
  s->ntiles = (int64_t)tiles.size();
  GOO_TRY(grow((void**)&s->d_tiles, &s->tiles_cap, std::max<size_t>(1, tiles.size()) * sizeof(int2)));
  GOO_TRY(grow((void**)&s->d_tile_partials, &s->partials_cap,
               std::max<size_t>(1, tiles.size()) * kSrvLanes * sizeof(float2)));
  if (!tiles.empty())
    GOO_CUDA_TRY(cudaMemcpyAsync(s->d_tiles, tiles.data(), tiles.size() * sizeof(int2), cudaMemcpyHostToDevice,
                                 ctx->stream));
  GOO_CUDA_TRY(cudaMemcpyAsync(s->d_fit_tiles, fit_tiles.data(), fit_tiles.size() * sizeof(int2),
                               cudaMemcpyHostToDevice, ctx->stream));
  if (!s->active.empty())
    GOO_CUDA_TRY(cudaMemcpyAsync(s->d_slots, s->active.data(), s->active.size() * sizeof(int), cudaMemcpyHostToDevice,
                                 ctx->stream));
  GOO_CUDA_TRY(cudaStreamSynchronize(ctx->stream));  // host vectors above are temporaries
  s->active_dirty = false;
  return GOO_OK;
}

static int retire(goo_server* s) {
  goo_ctx* ctx = s->ctx;
  unsigned cs[2] = {0u, 0u};  // done count, status word of the evaluation kernel
  GOO_CUDA_TRY(cudaMemcpyAsync(cs, s->d_done_count, sizeof cs, cudaMemcpyDeviceToHost, ctx->stream));
  GOO_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  if (cs[1]) return set_error(GOO_ERR_TIMEOUT, "goo_server_step: a device wait for amplitude data gave up");
  const unsigned nd = cs[0];
  if (nd == 0) return GOO_OK;
  std::vector<int> list(nd);
  GOO_CUDA_TRY(cudaMemcpyAsync(list.data(), s->d_done, nd * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  GOO_CUDA_TRY(cudaMemsetAsync(s->d_done_count, 0, sizeof(unsigned), ctx->stream));
  GOO_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  std::sort(list.begin(), list.end());
  std::vector<SrvState> st(nd);
  for (unsigned i = 0; i < nd; ++i)
    GOO_CUDA_TRY(cudaMemcpyAsync(&st[i], s->d_states + list[i], sizeof(SrvState), cudaMemcpyDeviceToHost, ctx->stream));
  GOO_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  const AmpModelInfo& I = s->info;
  for (unsigned i = 0; i < nd; ++i) {
    const int slot = list[i];
    Slot& sl = s->slots[slot];
    FitOut out;
    out.theta = sl.theta_start;
    out.err.assign(sl.theta_start.size(), 0.0);
    for (int k = 0; k < I.nbw; ++k) {
      out.theta[I.par_re[k]] = st[i].c0r[k] + st[i].x[2 * k] * s->xscale[2 * k];
      out.theta[I.par_im[k]] = st[i].c0i[k] + st[i].x[2 * k + 1] * s->xscale[2 * k + 1];
      out.err[I.par_re[k]] = st[i].err[2 * k];
      out.err[I.par_im[k]] = st[i].err[2 * k + 1];
    }
    std::memset(&out.res, 0, sizeof out.res);
    out.res.nll = st[i].f;
    out.res.edm = st[i].edm;
    out.res.iterations = st[i].it;
    out.res.grad_evals = st[i].evals;
    out.res.status = st[i].status;
    s->done[sl.ticket] = out;
    s->finished.push_back(sl.ticket);
    arena_free(s, sl.off, sl.bytes);
    sl = Slot();
    s->free_slots.push_back(slot);
    s->active.erase(std::find(s->active.begin(), s->active.end(), slot));
  }
  s->active_dirty = true;
  return GOO_OK;
}

}  // namespace goo

using namespace goo;

extern "C" {

int goo_server_create(goo_model* model, const double* theta_gen, const int* free_mask, const double* scale,
                      const goo_server_options* options, goo_server** out) {
  if (!model || !theta_gen || !free_mask || !scale || !out) return set_error(GOO_ERR_ARG, "goo_server_create: NULL argument");
  *out = nullptr;
  goo_ctx* ctx = model->ctx;
  GOO_CUDA_TRY(cudaSetDevice(ctx->device));
  AmpModelInfo info;
  GOO_TRY(dalitz_server_info(model, theta_gen, &info));
  if (info.nbw < 1 || info.nbw > kSrvKB)
    return set_error(GOO_ERR_UNSUPPORTED, "toy server: %d resonances (1..%d)", info.nbw, kSrvKB);
  if (!info.has_nr) return set_error(GOO_ERR_UNSUPPORTED, "toy server: the model needs a non-resonant reference amplitude");
  for (int p = 0; p < model->n_params; ++p) {
    bool coef_free = false;
    for (int k = 0; k < info.nbw; ++k) coef_free = coef_free || p == info.par_re[k] || p == info.par_im[k];
    if ((free_mask[p] != 0) != coef_free)
      return set_error(GOO_ERR_UNSUPPORTED,
                       "toy server fits exactly the resonance coefficients (parameter %d has the wrong free flag)", p);
  }
  goo_server* s = new goo_server();
  s->ctx = ctx;
  s->model = model;
  s->info = info;
  goo_server_options o{};
  if (options) o = *options;
  if (o.max_fits <= 0) o.max_fits = 4096;
  if (o.tile_events <= 0) o.tile_events = 16384;
  if (o.max_iter <= 0) o.max_iter = 200;
  if (!(o.edm_tol > 0)) o.edm_tol = 1e-6;
  if (o.hbm_budget_bytes <= 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    o.hbm_budget_bytes = (int64_t)(fr / 2);
  }
  s->opt = o;
  s->P = 2 * info.nbw;
  s->theta_gen.assign(theta_gen, theta_gen + model->n_params);
  s->xscale.assign(kSrvMaxP, 1.0);
  for (int k = 0; k < info.nbw; ++k) {
    s->xscale[2 * k] = scale[info.par_re[k]];
    s->xscale[2 * k + 1] = scale[info.par_im[k]];
    if (!(s->xscale[2 * k] > 0) || !(s->xscale[2 * k + 1] > 0)) {
      delete s;
      return set_error(GOO_ERR_ARG, "toy server: coefficient scales must be > 0");
    }
  }
  auto fail = [&](const char* what) {
    cudaGetLastError();
    goo_server_free(s);
    return set_error(GOO_ERR_OOM, "goo_server_create: cannot allocate %s", what);
  };
  s->arena_bytes = (size_t)o.hbm_budget_bytes;
  if (cudaMalloc(&s->arena, s->arena_bytes) != cudaSuccess) return fail("the event arena");
  s->free_blocks.push_back({0, s->arena_bytes});
  const int F = o.max_fits;
  if (cudaMalloc(&s->d_states, F * sizeof(SrvState)) != cudaSuccess ||
      cudaMalloc(&s->d_evals, F * sizeof(SrvEval)) != cudaSuccess ||
      cudaMalloc(&s->d_results, F * sizeof(SrvResult)) != cudaSuccess ||
      cudaMalloc(&s->d_model, sizeof(SrvModel)) != cudaSuccess ||
      cudaMalloc(&s->d_params, sizeof(SrvParams)) != cudaSuccess ||
      cudaMalloc(&s->d_tickets, F * sizeof(unsigned)) != cudaSuccess ||
      cudaMalloc(&s->d_fit_tiles, F * sizeof(int2)) != cudaSuccess ||
      cudaMalloc(&s->d_slots, F * sizeof(int)) != cudaSuccess || cudaMalloc(&s->d_done, F * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&s->d_done_count, 2 * sizeof(unsigned)) != cudaSuccess)
    return fail("the fit slots");
  cudaMemsetAsync(s->d_states, 0, F * sizeof(SrvState), ctx->stream);
  cudaMemsetAsync(s->d_tickets, 0, F * sizeof(unsigned), ctx->stream);
  cudaMemsetAsync(s->d_done_count, 0, 2 * sizeof(unsigned), ctx->stream);
  s->slots.resize(F);
  for (int i = F - 1; i >= 0; --i) s->free_slots.push_back(i);
  // shared model block: Gram matrix in slot order (resonances, then the reference)
  SrvModel sm{};
  sm.nbw = info.nbw;
  sm.has_ref = 1;
  std::vector<double> G(2 * info.K * info.K);
  GOO_CUDA_TRY(cudaMemcpy(G.data(), info.gram_dev, G.size() * sizeof(double), cudaMemcpyDeviceToHost));
  auto slot_of = [&](int m) { return m < info.nbw ? m : kSrvKB; };
  for (int a = 0; a < info.K; ++a)
    for (int b = 0; b < info.K; ++b) {
      sm.G[2 * (slot_of(a) * kSrvKA + slot_of(b))] = G[2 * (a * info.K + b)];
      sm.G[2 * (slot_of(a) * kSrvKA + slot_of(b)) + 1] = G[2 * (a * info.K + b) + 1];
    }
  GOO_CUDA_TRY(cudaMemcpy(s->d_model, &sm, sizeof sm, cudaMemcpyHostToDevice));
  SrvParams sp{};
  for (int p = 0; p < kSrvMaxP; ++p) sp.scale[p] = s->xscale[p];
  sp.edm_tol = o.edm_tol;
  sp.max_iter = o.max_iter;
  sp.nbw = info.nbw;
  GOO_CUDA_TRY(cudaMemcpy(s->d_params, &sp, sizeof sp, cudaMemcpyHostToDevice));
  // generator constants
  GenConst& g = s->gen;
  g.lo12 = (float)info.lo12;
  g.lo13 = (float)info.lo13;
  g.M2 = (float)(info.M * info.M);
  g.m1s = (float)(info.m1 * info.m1);
  g.m2s = (float)(info.m2 * info.m2);
  g.m3s = (float)(info.m3 * info.m3);
  g.nbw = info.nbw;
  for (int k = 0; k < info.nbw; ++k) {
    g.cr[k] = (float)theta_gen[info.par_re[k]];
    g.ci[k] = (float)theta_gen[info.par_im[k]];
  }
  g.cr[kSrvKB] = (float)theta_gen[info.par_re[info.nbw]];
  g.ci[kSrvKB] = (float)theta_gen[info.par_im[info.nbw]];
  // generator envelope: given, or kEnvFactor x the 3 x 3 neighbourhood maximum of |S|^2 on a
  // kEnvCells^2 grid of cells (kEnvSub^2 lattice points per cell).  The lattice scan runs for
  // a given envelope too: its per-cell sums estimate the acceptance of the first pass.
  const int n12 = o.envelope ? o.envelope->n12 : kEnvCells, n13 = o.envelope ? o.envelope->n13 : kEnvCells;
  if (n12 < 1 || n13 < 1 || n12 > 1024 || n13 > 1024 || (o.envelope && !o.envelope->bound)) {
    goo_server_free(s);
    return set_error(GOO_ERR_ARG, "goo_server_create: envelope grid %d x %d", n12, n13);
  }
  const int ncell = n12 * n13;
  g.n12 = n12;
  g.n13 = n13;
  g.cw12 = (float)((info.hi12 - info.lo12) / n12);
  g.cw13 = (float)((info.hi13 - info.lo13) / n13);
  const size_t scan_words = 2 * (size_t)ncell + 2;  // maxima, sums, violation counter (8 bytes)
  if (cudaMalloc(&s->d_env_bits, scan_words * sizeof(unsigned)) != cudaSuccess) return fail("the envelope");
  GOO_CUDA_TRY(cudaMemsetAsync(s->d_env_bits, 0, scan_words * sizeof(unsigned), ctx->stream));
  {
    LaunchScope ls(ctx, "toy_envelope");
    envelope_cells_kernel<<<ctx->num_sms * 4, kBlock, 0, ctx->stream>>>(g, (const DalitzDev*)info.dalitz_dev, kEnvSub,
                                                                       s->d_env_bits, (float*)(s->d_env_bits + ncell));
  }
  std::vector<float> cmax(ncell), csum(ncell);
  GOO_CUDA_TRY(cudaMemcpyAsync(cmax.data(), s->d_env_bits, ncell * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
  GOO_CUDA_TRY(cudaMemcpyAsync(csum.data(), s->d_env_bits + ncell, ncell * sizeof(float), cudaMemcpyDeviceToHost,
                               ctx->stream));
  GOO_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  std::vector<float> bound(ncell, 0.f);
  if (o.envelope) {
    for (int c = 0; c < ncell; ++c) bound[c] = o.envelope->bound[c];
  } else {
    for (int i = 0; i < n12; ++i)
      for (int j = 0; j < n13; ++j) {
        float mx = 0.f;
        for (int di = -1; di <= 1; ++di)
          for (int dj = -1; dj <= 1; ++dj) {
            const int ii = i + di, jj = j + dj;
            if (ii >= 0 && ii < n12 && jj >= 0 && jj < n13) mx = std::max(mx, cmax[ii * n13 + jj]);
          }
        bound[i * n13 + j] = kEnvFactor * mx;
      }
  }
  // acceptance estimate: sum over cells of the lattice mean of min(|S|^2, bound) / sum of bounds
  double eff0 = 0.2, sacc = 0.0, sbound = 0.0;
  for (int c = 0; c < ncell; ++c) {
    sacc += std::min((double)csum[c] / (kEnvSub * kEnvSub), (double)bound[c]);
    sbound += (double)bound[c];
  }
  if (sbound > 0 && std::isfinite(sbound) && sacc > 0) eff0 = std::min(0.95, std::max(0.005, 0.97 * sacc / sbound));
  // cumulative thresholds of the cell choice: thr[c] = floor(S_c / W * 2^32), S_c the sum of
  // bound[0..c] and W the total (FP64, in index order), thr[last] = 2^32
  std::vector<unsigned long long> thr(ncell);
  double W = 0.0, fmax_all = 0.0;
  for (int c = 0; c < ncell; ++c) {
    if (!(bound[c] >= 0.f) || !std::isfinite(bound[c])) {
      goo_server_free(s);
      return set_error(GOO_ERR_ARG, "goo_server_create: envelope bound %d is not a finite value >= 0", c);
    }
    W += (double)bound[c];
    fmax_all = std::max(fmax_all, (double)bound[c]);
  }
  if (!(W > 0)) {
    goo_server_free(s);
    return set_error(GOO_ERR_ARG, "goo_server_create: the envelope is zero everywhere");
  }
  double S = 0.0;
  for (int c = 0; c < ncell; ++c) {
    S += (double)bound[c];
    thr[c] = (unsigned long long)std::floor(S / W * 4294967296.0);
  }
  thr[ncell - 1] = 4294967296ull;
  if (cudaMalloc(&s->d_env_bound, ncell * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&s->d_env_thr, ncell * sizeof(unsigned long long)) != cudaSuccess)
    return fail("the envelope");
  GOO_CUDA_TRY(cudaMemcpyAsync(s->d_env_bound, bound.data(), ncell * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  GOO_CUDA_TRY(cudaMemcpyAsync(s->d_env_thr, thr.data(), ncell * sizeof(unsigned long long), cudaMemcpyHostToDevice,
                               ctx->stream));
  g.bound = s->d_env_bound;
  g.thr = s->d_env_thr;
  g.viol = (unsigned long long*)(s->d_env_bits + 2 * (size_t)ncell);
  s->gen_eff = eff0;
  s->env_max = fmax_all;
  GOO_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  s->ctx->live++;
  s->counted = true;
  *out = s;
  return GOO_OK;
}

int goo_server_submit(goo_server* s, int64_t n_events, uint64_t seed, const double* theta_start, int64_t* ticket) {
  if (!s || !ticket) return set_error(GOO_ERR_ARG, "goo_server_submit: NULL argument");
  if (n_events < 1) return set_error(GOO_ERR_ARG, "goo_server_submit: n_events=%lld", (long long)n_events);
  if (theta_start)
    for (int p = 0; p < s->model->n_params; ++p)
      if (!std::isfinite(theta_start[p]))
        return set_error(GOO_ERR_ARG, "goo_server_submit: theta_start[%d] is not finite", p);
  if (fit_bytes(n_events, s->info.nbw) > s->arena_bytes)
    return set_error(GOO_ERR_OOM, "goo_server_submit: %lld events need more than the whole arena", (long long)n_events);
  Request r;
  r.ticket = s->next_ticket++;
  r.n = n_events;
  r.seed = seed;
  r.theta_start.assign(theta_start ? theta_start : s->theta_gen.data(),
                       (theta_start ? theta_start : s->theta_gen.data()) + s->model->n_params);
  s->queue.push_back(r);
  *ticket = r.ticket;
  return GOO_OK;
}

int goo_server_step(goo_server* s, int* n_queued, int* n_active, int* n_done) {
  if (!s) return set_error(GOO_ERR_ARG, "goo_server_step: NULL server");
  goo_ctx* ctx = s->ctx;
  GOO_CUDA_TRY(cudaSetDevice(ctx->device));
  // admission and generation of new fits
  std::vector<int> admitted;
  GOO_TRY(admit(s, admitted));
  if (!admitted.empty()) {
    GOO_TRY(generate(s, admitted));
    std::vector<SrvState> st(admitted.size());
    std::vector<SrvEval> ev(admitted.size());
    for (size_t i = 0; i < admitted.size(); ++i) {
      init_state(s, admitted[i], st[i], ev[i]);
      GOO_CUDA_TRY(cudaMemcpyAsync(s->d_states + admitted[i], &st[i], sizeof(SrvState), cudaMemcpyHostToDevice, ctx->stream));
      GOO_CUDA_TRY(cudaMemcpyAsync(s->d_evals + admitted[i], &ev[i], sizeof(SrvEval), cudaMemcpyHostToDevice, ctx->stream));
      s->active.push_back(admitted[i]);
    }
    GOO_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    s->active_dirty = true;
  }
  if (!s->active.empty()) {
    if (s->active_dirty) GOO_TRY(upload_active(s));
    const auto t0 = std::chrono::steady_clock::now();
    GOO_CUDA_TRY(cudaMemsetAsync(s->d_results, 0, s->opt.max_fits * sizeof(SrvResult), ctx->stream));
    if (s->occ_nll == 0) {
      GOO_CUDA_TRY(cudaFuncSetAttribute(srv_nll_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSrvSmem));
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&s->occ_nll, srv_nll_kernel, kBlock, kSrvSmem) != cudaSuccess ||
          s->occ_nll < 1) {
        cudaGetLastError();
        s->occ_nll = 1;
      }
    }
    const int nb = (int)std::min<int64_t>(s->ntiles, (int64_t)ctx->num_sms * s->occ_nll);
    {
      LaunchScope ls(ctx, "srv_nll_grad");
      srv_nll_kernel<<<nb, kBlock, kSrvSmem, ctx->stream>>>(s->d_evals, s->d_tiles, s->d_fit_tiles, (int)s->ntiles,
                                                            s->opt.tile_events, s->d_model, s->d_tile_partials,
                                                            s->d_tickets, s->d_results, s->d_done_count + 1,
                                                            ctx->wait_limit ? (long long)ctx->wait_limit : kWaitCycles);
    }
    GOO_CUDA_TRY(cudaGetLastError());
    {
      LaunchScope ls(ctx, "srv_bfgs");
      const int na = (int)s->active.size();
      // one thread per fit in blocks of one warp, so that the fits' FP64 work spreads over
      // every SM (blocks of 128 put 4096 fits on 32 SMs: 237 against 168 ms over a study)
      srv_bfgs_kernel<<<(na + 31) / 32, 32, 0, ctx->stream>>>(s->d_states, s->d_evals, s->d_results, s->d_params,
                                                              s->d_slots, na, s->d_done, s->d_done_count);
    }
    GOO_CUDA_TRY(cudaGetLastError());
    GOO_TRY(retire(s));
    s->eval_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    s->rounds++;
  }
  if (n_queued) *n_queued = (int)s->queue.size();
  if (n_active) *n_active = (int)s->active.size();
  if (n_done) *n_done = (int)s->done.size();
  return GOO_OK;
}

int goo_server_cancel(goo_server* s, int64_t ticket) {
  if (!s) return set_error(GOO_ERR_ARG, "goo_server_cancel: NULL server");
  if (s->done.count(ticket)) return set_error(GOO_ERR_STATE, "goo_server_cancel: fit %lld has finished", (long long)ticket);
  for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
    if (it->ticket != ticket) continue;
    finish_unfitted(s, ticket, it->theta_start, GOO_FIT_CANCELLED);
    s->queue.erase(it);
    return GOO_OK;
  }
  for (size_t a = 0; a < s->active.size(); ++a) {
    const int slot = s->active[a];
    Slot& sl = s->slots[slot];
    if (sl.ticket != ticket) continue;
    // between steps no kernel of the server is in flight (each step synchronises): the slot's
    // device state is simply no longer advanced, and its events' memory returns to the arena
    finish_unfitted(s, ticket, sl.theta_start, GOO_FIT_CANCELLED);
    arena_free(s, sl.off, sl.bytes);
    sl = Slot();
    s->free_slots.push_back(slot);
    s->active.erase(s->active.begin() + a);
    s->active_dirty = true;
    return GOO_OK;
  }
  return set_error(GOO_ERR_ARG, "goo_server_cancel: no fit with ticket %lld", (long long)ticket);
}

int goo_server_fail_allocation(goo_server* s, int64_t ticket) {
  if (!s) return set_error(GOO_ERR_ARG, "goo_server_fail_allocation: NULL server");
  for (const Request& r : s->queue)
    if (r.ticket == ticket) {
      s->fail_alloc.insert(ticket);
      return GOO_OK;
    }
  return set_error(GOO_ERR_STATE, "goo_server_fail_allocation: fit %lld is not waiting for admission", (long long)ticket);
}

int goo_server_result(goo_server* s, int64_t ticket, double* theta_out, double* errors_out, goo_fit_result* res) {
  if (!s) return set_error(GOO_ERR_ARG, "goo_server_result: NULL server");
  auto it = s->done.find(ticket);
  if (it == s->done.end()) return GOO_ERR_STATE;
  const FitOut& f = it->second;
  if (theta_out) std::memcpy(theta_out, f.theta.data(), f.theta.size() * sizeof(double));
  if (errors_out) std::memcpy(errors_out, f.err.data(), f.err.size() * sizeof(double));
  if (res) *res = f.res;
  return GOO_OK;
}

int goo_server_finished(goo_server* s, int64_t* tickets, int cap, int* n) {
  if (!s || !n || cap < 0 || (cap > 0 && !tickets)) return set_error(GOO_ERR_ARG, "goo_server_finished: bad arguments");
  int k = 0;
  while (k < cap && !s->finished.empty()) {
    tickets[k++] = s->finished.front();
    s->finished.pop_front();
  }
  *n = k;
  return GOO_OK;
}

int goo_server_stats(const goo_server* s, double* out) {
  if (!s || !out) return set_error(GOO_ERR_ARG, "goo_server_stats: NULL argument");
  out[0] = (double)s->rounds;
  out[1] = s->eval_ms;
  out[2] = s->gen_ms;
  out[3] = s->gen_candidates;
  out[4] = s->gen_accepted;
  out[5] = s->env_max;
  out[6] = (double)s->arena_bytes;
  size_t fr = 0;
  for (auto& b : s->free_blocks) fr += b.size;
  out[7] = (double)(s->arena_bytes - fr);
  out[8] = s->gen_violations;
  return GOO_OK;
}

int goo_server_free(goo_server* s) {
  if (!s) return set_error(GOO_ERR_ARG, "goo_server_free: NULL server");
  cudaSetDevice(s->ctx->device);
  cudaStreamSynchronize(s->ctx->stream);
  void* ptrs[] = {s->arena, s->d_states, s->d_evals, s->d_results, s->d_model, s->d_params, s->d_tickets,
                  s->d_fit_tiles, s->d_slots, s->d_done, s->d_done_count, s->d_tiles, s->d_tile_partials,
                  s->d_gtoys, s->d_bprefix, s->d_counts, s->d_outbase, s->d_accepted, s->d_masks,
                  s->d_env_bound, s->d_env_thr, s->d_env_bits};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (s->counted) s->ctx->live--;
  delete s;
  return GOO_OK;
}

// Toys from the server's generator, all generated in the same passes and written to host
// arrays: toy i (seed seeds[i], n[i] events) goes to s12_out/s13_out at offset sum(n[:i]).
int goo_toys_generate(goo_model* m, const double* theta, const goo_envelope* env, int n_toys, const uint64_t* seeds,
                      const int64_t* n, float* s12_out, float* s13_out) {
  if (!m || !theta || n_toys < 0 || (n_toys > 0 && (!seeds || !n || !s12_out || !s13_out)))
    return set_error(GOO_ERR_ARG, "goo_toys_generate: bad arguments");
  if (n_toys == 0) return GOO_OK;
  goo_ctx* ctx = m->ctx;
  GOO_CUDA_TRY(cudaSetDevice(ctx->device));
  AmpModelInfo info;
  GOO_TRY(dalitz_server_info(m, theta, &info));
  std::vector<int> free_mask(m->n_params, 0);
  std::vector<double> scale(m->n_params, 1.0);
  for (int k = 0; k < info.nbw; ++k) free_mask[info.par_re[k]] = free_mask[info.par_im[k]] = 1;
  goo_server_options o{};
  o.max_fits = n_toys;
  int64_t bytes = 4096;
  for (int i = 0; i < n_toys; ++i) {
    if (n[i] < 1) return set_error(GOO_ERR_ARG, "goo_toys_generate: toy %d has %lld events", i, (long long)n[i]);
    bytes += (int64_t)fit_bytes(n[i], info.nbw);
  }
  o.hbm_budget_bytes = bytes;
  o.envelope = env;
  goo_server* s = nullptr;
  GOO_TRY(goo_server_create(m, theta, free_mask.data(), scale.data(), &o, &s));
  int rc = GOO_OK;
  std::vector<int64_t> tickets(n_toys);
  for (int i = 0; i < n_toys && rc == GOO_OK; ++i) rc = goo_server_submit(s, n[i], seeds[i], theta, &tickets[i]);
  std::vector<int> admitted;
  if (rc == GOO_OK) rc = admit(s, admitted);
  if (rc == GOO_OK && (int)admitted.size() != n_toys) rc = set_error(GOO_ERR_OOM, "goo_toys_generate: not all toys fit");
  if (rc == GOO_OK) rc = generate(s, admitted);
  int64_t off = 0;
  for (int i = 0; i < n_toys && rc == GOO_OK; ++i) {
    const Slot& sl = s->slots[admitted[i]];
    if (cudaMemcpy(s12_out + off, sl.s12, n[i] * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(s13_out + off, sl.s13, n[i] * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = set_error(GOO_ERR_CUDA, "goo_toys_generate: copy failed");
    off += n[i];
  }
  goo_server_free(s);
  return rc;
}

int goo_toy_generate(goo_model* m, const double* theta, const goo_envelope* env, uint64_t seed, int64_t n, float* s12_out,
                     float* s13_out) {
  if (n == 0) return GOO_OK;
  return goo_toys_generate(m, theta, env, 1, &seed, &n, s12_out, s13_out);
}

// Batched NLL + gradient of n_fits (dataset, theta) pairs with one launch (per-fit tiles,
// per-fit reduction in tile order).
int goo_nll_grad_batch(goo_model* m, int n_fits, const goo_dataset* const* ds, const double* theta, int precision,
                       double* nll_out, double* grad_out) {
  if (!m || n_fits < 0 || (n_fits && (!ds || !theta || !nll_out || !grad_out)))
    return set_error(GOO_ERR_ARG, "goo_nll_grad_batch: bad arguments");
  if (precision != GOO_F32) return set_error(GOO_ERR_UNSUPPORTED, "goo_nll_grad_batch: the batched path is FP32");
  if (n_fits == 0) return GOO_OK;
  for (int f = 0; f < n_fits; ++f)
    if (!ds[f] || ds[f]->w64 || ds[f]->host_borrowed)
      return set_error(ds[f] ? GOO_ERR_UNSUPPORTED : GOO_ERR_ARG, "goo_nll_grad_batch: dataset %d is %s", f,
                       !ds[f] ? "NULL" : ds[f]->w64 ? "weighted" : "in host memory (GOO_BORROW_HOST)");
  goo_ctx* ctx = m->ctx;
  GOO_CUDA_TRY(cudaSetDevice(ctx->device));
  const int P = m->n_params;
  AmpModelInfo info;
  GOO_TRY(dalitz_server_info(m, theta, &info));
  if (info.nbw > kSrvKB || !info.has_nr)
    return set_error(GOO_ERR_UNSUPPORTED, "goo_nll_grad_batch: needs <= %d resonances and a reference amplitude", kSrvKB);
  // one Gram matrix serves the batch: every fit must share the lineshape (non-coefficient)
  // parameters
  for (int f = 1; f < n_fits; ++f)
    for (int p = 0; p < P; ++p) {
      bool coef = false;
      for (int k = 0; k < info.K; ++k) coef = coef || p == info.par_re[k] || p == info.par_im[k];
      if (!coef && theta[(size_t)f * P + p] != theta[p])
        return set_error(GOO_ERR_ARG, "goo_nll_grad_batch: fit %d differs from fit 0 in lineshape parameter %d", f, p);
    }
  const int T = 16384;
  std::vector<SrvEval> ev(n_fits);
  std::vector<int2> tiles, fit_tiles(n_fits);
  for (int f = 0; f < n_fits; ++f) {
    const void* cache = nullptr;
    int nres = 0;
    GOO_TRY(dalitz_amplitudes(m, ds[f], theta + (size_t)f * P, GOO_F32, &cache, &nres));
    SrvEval& e = ev[f];
    std::memset(&e, 0, sizeof e);
    e.cache = (const float4*)cache;
    e.n = ds[f]->n;
    e.plane = ds[f]->n;
    for (int k = 0; k < info.nbw; ++k) {
      e.cr[k] = (float)theta[(size_t)f * P + info.par_re[k]];
      e.ci[k] = (float)theta[(size_t)f * P + info.par_im[k]];
    }
    e.cr[kSrvKB] = (float)theta[(size_t)f * P + info.par_re[info.nbw]];
    e.ci[kSrvKB] = (float)theta[(size_t)f * P + info.par_im[info.nbw]];
    const int nt = (int)std::max<int64_t>(1, (e.n + T - 1) / T);
    fit_tiles[f] = make_int2(nt, (int)tiles.size());
    for (int t = 0; t < nt; ++t) tiles.push_back(make_int2(f, t));
  }
  SrvModel sm{};
  sm.nbw = info.nbw;
  sm.has_ref = 1;
  std::vector<double> G(2 * info.K * info.K);
  GOO_CUDA_TRY(cudaMemcpy(G.data(), info.gram_dev, G.size() * sizeof(double), cudaMemcpyDeviceToHost));
  auto slot_of = [&](int a) { return a < info.nbw ? a : kSrvKB; };
  for (int a = 0; a < info.K; ++a)
    for (int b = 0; b < info.K; ++b)
      for (int c = 0; c < 2; ++c) sm.G[2 * (slot_of(a) * kSrvKA + slot_of(b)) + c] = G[2 * (a * info.K + b) + c];
  // one allocation for the work space of this call
  const size_t bytes = sizeof(SrvEval) * n_fits + sizeof(int2) * (tiles.size() + n_fits) + sizeof(SrvModel) +
                       sizeof(SrvResult) * n_fits + sizeof(unsigned) * n_fits + sizeof(float2) * kSrvLanes * tiles.size() +
                       sizeof(unsigned) + 9 * 256;
  unsigned char* w = nullptr;
  if (cudaMalloc(&w, bytes) != cudaSuccess) {
    cudaGetLastError();
    return set_error(GOO_ERR_OOM, "goo_nll_grad_batch: work space");
  }
  size_t o = 0;
  auto take = [&](size_t b) {
    unsigned char* p = w + o;
    o = al256(o + b);
    return p;
  };
  SrvEval* d_ev = (SrvEval*)take(sizeof(SrvEval) * n_fits);
  int2* d_tiles = (int2*)take(sizeof(int2) * tiles.size());
  int2* d_ft = (int2*)take(sizeof(int2) * n_fits);
  SrvModel* d_sm = (SrvModel*)take(sizeof(SrvModel));
  SrvResult* d_res = (SrvResult*)take(sizeof(SrvResult) * n_fits);
  unsigned* d_tk = (unsigned*)take(sizeof(unsigned) * n_fits);
  float2* d_part = (float2*)take(sizeof(float2) * kSrvLanes * tiles.size());
  unsigned* d_status = (unsigned*)take(sizeof(unsigned));
  int rc = GOO_OK;
  unsigned status = 0;
  std::vector<SrvResult> res(n_fits);
  do {
    if (cudaMemcpyAsync(d_ev, ev.data(), sizeof(SrvEval) * n_fits, cudaMemcpyHostToDevice, ctx->stream) ||
        cudaMemcpyAsync(d_tiles, tiles.data(), sizeof(int2) * tiles.size(), cudaMemcpyHostToDevice, ctx->stream) ||
        cudaMemcpyAsync(d_ft, fit_tiles.data(), sizeof(int2) * n_fits, cudaMemcpyHostToDevice, ctx->stream) ||
        cudaMemcpyAsync(d_sm, &sm, sizeof sm, cudaMemcpyHostToDevice, ctx->stream) ||
        cudaMemsetAsync(d_res, 0, sizeof(SrvResult) * n_fits, ctx->stream) ||
        cudaMemsetAsync(d_tk, 0, sizeof(unsigned) * n_fits, ctx->stream) ||
        cudaMemsetAsync(d_status, 0, sizeof(unsigned), ctx->stream)) {
      rc = set_error(GOO_ERR_CUDA, "goo_nll_grad_batch: copy failed");
      break;
    }
    int occ = 0;
    if (cudaFuncSetAttribute(srv_nll_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSrvSmem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, srv_nll_kernel, kBlock, kSrvSmem) != cudaSuccess || occ < 1)
      occ = 1;
    cudaGetLastError();
    const int nb = (int)std::min<size_t>(tiles.size(), (size_t)ctx->num_sms * occ);
    {
      LaunchScope ls(ctx, "srv_nll_grad");
      srv_nll_kernel<<<nb, kBlock, kSrvSmem, ctx->stream>>>(d_ev, d_tiles, d_ft, (int)tiles.size(), T, d_sm, d_part, d_tk,
                                                            d_res, d_status,
                                                            ctx->wait_limit ? (long long)ctx->wait_limit : kWaitCycles);
    }
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(res.data(), d_res, sizeof(SrvResult) * n_fits, cudaMemcpyDeviceToHost, ctx->stream) ||
        cudaMemcpyAsync(&status, d_status, sizeof status, cudaMemcpyDeviceToHost, ctx->stream) ||
        cudaStreamSynchronize(ctx->stream)) {
      rc = set_error(GOO_ERR_CUDA, "goo_nll_grad_batch: kernel failed");
      break;
    }
  } while (false);
  cudaFree(w);
  if (rc != GOO_OK) return rc;
  if (status) return set_error(GOO_ERR_TIMEOUT, "goo_nll_grad_batch: a device wait for amplitude data gave up");
  for (int f = 0; f < n_fits; ++f) {
    double* g = grad_out + (size_t)f * P;
    for (int p = 0; p < P; ++p) g[p] = 0.0;
    nll_out[f] = res[f].bad ? HUGE_VAL : res[f].nll;
    for (int k = 0; k <= info.nbw; ++k) {
      const int sl = slot_of(k);
      g[info.par_re[k]] = res[f].gre[sl];
      g[info.par_im[k]] = res[f].gim[sl];
    }
  }
  return GOO_OK;
}

}  // extern "C"
