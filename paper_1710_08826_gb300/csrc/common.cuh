// common.cuh -- shared infrastructure of the goo library: errors, context, datasets,
// double-float (float hi + float lo) arithmetic and the deterministic block / last-block
// reductions used by every likelihood kernel.
//
// GB300's FP64 pipe runs at 1/64 of the FP32 rate (measured: 6.0e11 FP64 FMA/s against
// 3.75e13 FP32 FMA/s), so cross-thread and cross-block sums are carried in double-float
// (a pair of floats holding ~48 significant bits) rather than in FP64.  Only the final
// combination of a few hundred numbers runs in FP64.
#pragma once

// The device parts of this header (limits, double-float arithmetic, packed FP32, mbarrier
// and bulk-copy helpers, reductions) are also compiled at run time by NVRTC for the
// model-specialised event kernels; the host parts are left out there.
#ifndef __CUDACC_RTC__
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>
#endif

#include "goo.h"

namespace goo {

#ifndef __CUDACC_RTC__
// ---------------------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------------------
int set_error(int code, const char* fmt, ...);
int log_level();

#define GOO_CUDA_TRY(expr)                                                                 \
  do {                                                                                     \
    cudaError_t _e = (expr);                                                               \
    if (_e != cudaSuccess)                                                                 \
      return ::goo::set_error(GOO_ERR_CUDA, "%s failed: %s (%s:%d)", #expr,                \
                              cudaGetErrorString(_e), __FILE__, __LINE__);                 \
  } while (0)

#define GOO_TRY(expr)                                                                      \
  do {                                                                                     \
    int _rc = (expr);                                                                      \
    if (_rc != GOO_OK) return _rc;                                                         \
  } while (0)
#endif

// ---------------------------------------------------------------------------------------
// limits
// ---------------------------------------------------------------------------------------
constexpr int kMaxParams = 128;    // parameters of one model
constexpr int kMaxObs = 4;         // observables of a sum/product model
constexpr int kMaxCols = 8;        // columns of a dataset, observables of any model
constexpr int kMaxComp = 4;        // products in the flattened sum of products
constexpr int kMaxLeaf = 4;        // leaves per product
constexpr int kMaxSlots = 64;      // reduction lanes of one kernel
// Threads per block of the memory-bound coherent kernel, which streams its amplitude tiles
// through shared memory: one block of 16 warps per SM, so that all warps of an SM draw on one
// tile stream and finish together (two co-resident blocks of 8 warps drift apart by ~10 %;
// the compute-bound staged kernels keep two 256-thread blocks, which measured faster).
constexpr int kStagedBlock = 512;
constexpr int kBlock = 256;        // threads per block of the likelihood kernels
// the pair kernel of the sum-of-products models: column tiles in flight per block (bulk
// copies) and event pairs per thread per tile (a tile: 2 * 6 * 256 = 3072 events)
constexpr int kEventStages = 2;
constexpr int kPairsPerThread = 6;
constexpr int kResultDoubles = 4 + kMaxParams + 60;  // result record of one evaluation
constexpr int kPinnedResult = 256;                   // offset of the result in host_pinned
// Completion word after the result record: the kernels set it to 1 once the record is
// written (every result buffer holds kResultDoubles + 1 doubles); a reader that has
// synchronised the stream may test it.
constexpr int kResultFlag = kResultDoubles;
// A record in mapped host memory is polled field by field instead: the host fills it with
// this bit pattern (a signalling NaN that no arithmetic produces) before the launch, the
// kernel writes every field it returns exactly once as one aligned 8-byte store, and a field
// that no longer holds the pattern holds its final value.  No fence orders the fields.
constexpr unsigned long long kResultSentinel = 0x7ff4dead5e171e1aull;

#ifndef __CUDACC_RTC__
// ---------------------------------------------------------------------------------------
// context and datasets
// ---------------------------------------------------------------------------------------
struct Scratch {
  // Per-context device scratch for one likelihood evaluation: per-block partial sums in
  // double-float, the last-block ticket counter, the non-positive-density counter and the
  // result record.  Reused by every call on the context's stream.
  float2* partials = nullptr;
  size_t partials_cap = 0;          // in float2 elements
  // [0]: ticket, [1]: non-positive events, [kStatusWord]: a device wait gave up,
  // [kWaitLimitWord]: the tile-wait limit (goo_set_wait_limit), [kWithholdWord]: the
  // failure-detection test hook (goo_debug_withhold_tile), [5..]: spare
  unsigned* counters = nullptr;
  double* result = nullptr;         // kResultDoubles doubles
  double* theta = nullptr;          // kMaxParams doubles
  double* host_pinned = nullptr;    // pinned staging: [0, 256) theta in, [256, 512) result out
  // result record in mapped pinned host memory (kResultDoubles + 1 doubles, the device writes
  // it over the host link): the sum-of-products path reads its result here without a copy
  double* result_host = nullptr;
  // destination of the amplitude kernels' record for the evaluation in progress: `result`,
  // or `result_host` while dalitz_nll / td4_nll run
  double* result_out = nullptr;
  // goo_nll_grad_streamed: one mapped record per chunk (kStreamChunks records of
  // kResultDoubles + 1 doubles), a second stream for the chunks' copies and an event per chunk
  double* chunk_records = nullptr;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t chunk_events[65] = {};
};
constexpr int kStreamChunks = 64;  // chunks of one goo_nll_grad_streamed call, at most

}  // namespace goo

namespace goo {
// Optional per-kernel timing: CUDA events recorded around each launch on the context's
// stream, folded into per-kernel totals when the table is read.
struct TimedLaunch {
  const char* name;
  cudaEvent_t start, stop;
};
struct KernelStat {
  std::string name;
  int64_t count = 0;
  double ms = 0.0;
};
struct CacheSlot {
  void* ptr = nullptr;
  size_t bytes = 0;
  uint64_t key = 0;
};
}  // namespace goo

struct goo_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool owns_stream = false;
  int num_sms = 0;
  int64_t launches = 0;
  int live = 0;  // datasets, models and servers created on this context and not yet freed
  // limit of the kernels' waits for input tiles in SM clocks (0: the default, about one
  // second); a copy of counters[kWaitLimitWord] for the kernels that take it as an argument
  unsigned wait_limit = 0;
  goo::Scratch scratch;
  bool timing = false;
  std::vector<goo::TimedLaunch> pending;
  std::vector<cudaEvent_t> event_pool;
  std::vector<goo::KernelStat> stats;
};

struct goo_dataset {
  goo_ctx* ctx = nullptr;
  int64_t n = 0;
  int64_t capacity = 0;  // events the owned buffers hold (goo_dataset_update)
  // changes whenever the events change (goo_dataset_update); part of every key of a result
  // cached from this dataset's events (amplitude caches, MC Gram matrices)
  uint64_t epoch = 0;
  int ncols = 0;
  double* d64[goo::kMaxCols] = {};
  float* d32[goo::kMaxCols] = {};
  bool owns64 = true, owns32 = true;
  // per-event weights (null: every event weighs 1), set by goo_dataset_set_weights
  double* w64 = nullptr;
  float* w32 = nullptr;
  // GOO_BORROW_HOST: d32 are device-mapped pinned host columns, read by every evaluation over
  // the host link and range-checked there; no d64
  bool host_borrowed = false;
  double lo[goo::kMaxCols] = {};
  double hi[goo::kMaxCols] = {};
  // amplitude caches attached to this dataset, [0]: float32, [1]: float64, [2], [3]: the
  // same at the exchanged Dalitz point (time-dependent three-body model); built lazily by the
  // amplitude-model path and rebuilt when the model or its lineshapes change
  goo::CacheSlot cache[4];
};

namespace goo {

int ensure_partials(goo_ctx* ctx, size_t n_float2);

// Brackets one kernel launch: counts it and, when timing is on, records CUDA events
// around it on the context's stream.
struct LaunchScope {
  goo_ctx* ctx;
  const char* name;
  cudaEvent_t start = nullptr, stop = nullptr;
  LaunchScope(goo_ctx* c, const char* n);
  ~LaunchScope();
};
int grid_blocks(goo_ctx* ctx, int64_t work_items, int blocks_per_sm);
// Resident blocks per SM of `kernel` (a __global__ function or a run-time compiled kernel
// handle) with `block` threads and `smem` bytes of dynamic shared memory on the current
// device, at least 1.  Cached per (kernel, device, block, smem): the occupancy query is a
// driver call, and the launchers need its answer on every evaluation.
int cached_occupancy(const void* kernel, int device, int block, size_t smem);
// Waits until the first n fields of the record a kernel writes to scratch.result_host no
// longer hold kResultSentinel (polling for up to 2 ms, then waiting on the stream, which also
// reports a failed kernel) and copies them to dst.
int read_result_mapped(goo_ctx* ctx, int n, double* dst);
// Fills the mapped record with kResultSentinel before a launch that writes to it.
void arm_result_mapped(goo_ctx* ctx);
// For the lifetime of the guard, the amplitude kernels write their record to the mapped host
// copy (scratch.result_out = scratch.result_host), armed with kResultSentinel.
struct MappedResult {
  goo_ctx* ctx;
  explicit MappedResult(goo_ctx* c);
  ~MappedResult();
};

#endif  // __CUDACC_RTC__

// ---------------------------------------------------------------------------------------
// double-float arithmetic (Dekker / Knuth two-sum); every operation is exact up to the
// final renormalisation, giving ~2^-48 relative precision.
// ---------------------------------------------------------------------------------------
struct ddf {
  float hi, lo;
};

__device__ __forceinline__ ddf dd_make(float hi, float lo) {
  float s = hi + lo;
  float e = lo - (s - hi);
  return {s, e};
}

__device__ __forceinline__ ddf dd_add(ddf a, ddf b) {
  float s = a.hi + b.hi;
  float v = s - a.hi;
  float e = (a.hi - (s - v)) + (b.hi - v);
  e += a.lo + b.lo;
  float h = s + e;
  return {h, e - (h - s)};
}

__device__ __forceinline__ ddf dd_from_double(double x) {
  float h = (float)x;
  return {h, (float)(x - (double)h)};
}

__device__ __forceinline__ double dd_to_double(ddf a) { return (double)a.hi + (double)a.lo; }

// a b in double-float: the product of the high parts split exactly by an FMA, plus the cross
// terms; about 2^-44 relative.
__device__ __forceinline__ ddf dd_mul(ddf a, ddf b) {
  const float p = a.hi * b.hi;
  return dd_make(p, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, fmaf(a.hi, b.hi, -p))));
}

// a / b in double-float (Dekker's division): a first quotient, the remainder a - q1 b with
// q1 b.hi split exactly by an FMA, and a correction quotient; about 2^-44 relative.
__device__ __forceinline__ ddf dd_div(ddf a, ddf b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const float p = q1 * b.hi;
  const float pe = fmaf(q1, b.hi, -p);  // q1 b.hi = p + pe exactly
  const float r = (((a.hi - p) - pe) + a.lo) - q1 * b.lo;
  return dd_make(q1, __fdiv_rn(r, b.hi));
}

__device__ __forceinline__ ddf dd_shfl_xor(ddf a, int m) {
  return {__shfl_xor_sync(0xffffffffu, a.hi, m), __shfl_xor_sync(0xffffffffu, a.lo, m)};
}

__device__ __forceinline__ ddf dd_warp_sum(ddf v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v = dd_add(v, dd_shfl_xor(v, m));
  return v;
}

// Warp sums of four double-float values at once by an exchanging butterfly: at the first two
// levels each lane keeps half of its quantities and sends the other half, so a lane performs
// six additions instead of twenty.  Afterwards lanes 8q .. 8q + 7 hold the sum of a[q]
// (q = 0..3).  Fixed order, so bitwise repeatable.
__device__ __forceinline__ ddf dd_warp_sum4(const ddf (&a)[4]) {
  const int lane = threadIdx.x & 31;
  const bool h16 = (lane & 16) != 0, h8 = (lane & 8) != 0;
  // level 16: the lower half keeps quantities 0 and 1, the upper half 2 and 3
  ddf k0 = h16 ? a[2] : a[0], k1 = h16 ? a[3] : a[1];
  const ddf s0 = h16 ? a[0] : a[2], s1 = h16 ? a[1] : a[3];
  k0 = dd_add(k0, dd_shfl_xor(s0, 16));
  k1 = dd_add(k1, dd_shfl_xor(s1, 16));
  // level 8: lanes with bit 3 clear keep the first of the two
  ddf k = h8 ? k1 : k0;
  k = dd_add(k, dd_shfl_xor(h8 ? k0 : k1, 8));
#pragma unroll
  for (int m = 4; m > 0; m >>= 1) k = dd_add(k, dd_shfl_xor(k, m));
  return k;
}

// Natural logarithm of a positive double-float as a double-float, in FP32 arithmetic: the
// exponent is split off exactly, x.hi = m 2^e with m in [sqrt(1/2), sqrt(2)), so that
// ln 2 and log2(e) as double-floats (high part: the float nearest; low part: the float
// nearest the remainder)
constexpr float kLn2Hi = 0.693147182464599609375f, kLn2Lo = -1.9046542999577152e-09f;
constexpr float kLog2eHi = 1.44269502162933349609375f, kLog2eLo = 1.925963033500011e-08f;

// log x = e ln 2 + log m + log(1 + x.lo / x.hi) with |log m| < 0.35; logf(m) is within one
// FP32 ulp of 0.35 (3e-8), e ln 2 is formed exactly in double-float and log(1 + r) = r to
// below 1e-14 (|r| <= 2^-24).  About 3e-8 absolute.
__device__ __forceinline__ ddf log_dd(ddf x) {
  int e;
  float m = frexpf(x.hi, &e);  // x.hi = m 2^e, m in [1/2, 1)
  if (m < 0.70710678f) {
    m *= 2.f;
    e -= 1;
  }
  const float fe = (float)e;
  const float ph = fe * kLn2Hi;
  ddf r = dd_make(ph, fmaf(fe, kLn2Hi, -ph) + fe * kLn2Lo);
  r = dd_add(r, {logf(m), 0.f});
  return dd_add(r, {x.lo / x.hi, 0.f});
}

// Kahan-compensated FP32 accumulator (the per-thread NLL lane of the FP32 path).
struct Kahan {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    float y = x - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ ddf value() const { return dd_make(s, -c); }
};

// ---------------------------------------------------------------------------------------
// Packed FP32 arithmetic of sm_100-class GPUs: add / sub / mul / fma on .f32x2 register
// pairs (each lane rounded as the scalar instruction), and the hardware base-2 exponential,
// logarithm and reciprocal (PTX .approx forms, denormals flushed).
// ---------------------------------------------------------------------------------------
namespace pk {
__device__ __forceinline__ float2 splat(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub(float2 a, float2 b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;"
      : "=l"(d)
      : "l"(*reinterpret_cast<const unsigned long long*>(&a)), "l"(*reinterpret_cast<const unsigned long long*>(&b)));
  return *reinterpret_cast<const float2*>(&d);
}
// hardware base-2 exponential / logarithm / reciprocal (PTX .approx forms, denormals flushed)
__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
constexpr float kLn2 = 0.6931471805599453f;
__device__ __forceinline__ float2 rcp(float2 x) { return make_float2(rcp(x.x), rcp(x.y)); }
}  // namespace pk

// ---------------------------------------------------------------------------------------
// Bulk asynchronous copies global -> shared (the non-tensor TMA form, cp.async.bulk) that
// signal an mbarrier with their byte count, and waits on that barrier with a time limit.
// A wait that exceeds its limit in SM clocks gives up and returns false; the caller records
// GOO_ERR_TIMEOUT in the device status word (kStatusWord) and drains.  The limit of the
// waits for input tiles is the context's setting in counters[kWaitLimitWord]
// (goo_set_wait_limit; 0 selects kWaitCycles, about one second); the waits that drain a
// block's own copies before it exits always allow kWaitCycles, so that no block leaves
// while a copy into its shared memory is in flight.
// ---------------------------------------------------------------------------------------
constexpr long long kWaitCycles = 2000000000LL;
constexpr int kStatusWord = 2;     // counters[2]: nonzero after a device wait gave up
constexpr int kWaitLimitWord = 3;  // counters[3]: limit of the tile waits in SM clocks (0: kWaitCycles)
// counters[4]: failure-detection test hook (goo_debug_withhold_tile); 1 + the index of a tile
// whose copies the first block of the staged kernels does not issue, 0: none
constexpr int kWithholdWord = 4;
// counters[5]: events outside the observable limits met by an evaluation that reads its events
// from host memory (GOO_BORROW_HOST); reported as result[nb] = -(2 + count)
constexpr int kRangeWord = 5;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// makes barrier initialisation visible to the asynchronous (TMA) proxy
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n"
      "  .reg .pred p;\n"
      "  mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "  selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Non-blocking probe of the phase with the given parity (test_wait never suspends the thread).
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n"
      "  .reg .pred p;\n"
      "  mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "  selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for the phase with the given parity to complete; false after `limit` SM clocks.  The
// default limit probes with try_wait (which may suspend the thread for a system-dependent
// time); a shorter one (goo_set_wait_limit) probes with test_wait, so that the limit holds
// even where try_wait would have suspended the thread for longer.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, long long limit = kWaitCycles) {
  if (limit >= kWaitCycles) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
      if (clock64() - t0 > limit) return false;
    return true;
  }
  const long long t0 = clock64();
  while (!mbar_test_wait(bar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}

// 1 + the block-local tile whose copies this block withholds (goo_debug_withhold_tile: the
// first block only), 0: none.
__device__ __forceinline__ unsigned withheld_tile(const unsigned* counters) {
  return blockIdx.x == 0 ? __ldcg(counters + kWithholdWord) : 0u;
}

// The tile-wait limit of the evaluation in progress (counters[kWaitLimitWord], 0: kWaitCycles).
__device__ __forceinline__ long long tile_wait_limit(const unsigned* counters) {
  const unsigned w = __ldcg(counters + kWaitLimitWord);
  return w ? (long long)w : kWaitCycles;
}

// orders this thread's earlier generic-proxy shared-memory accesses before later async-proxy
// (bulk copy) accesses of the same memory
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// bytes: a multiple of 16; src and dst 16-byte aligned
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// Programmatic dependent launch: a kernel launched with the programmatic-serialisation
// attribute may start while the previous kernel in the stream runs; grid_dep_wait() blocks
// until that kernel has completed and its writes are visible.  grid_dep_launch() lets the
// dependent kernel start early.  Both are no-ops without such a launch.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---------------------------------------------------------------------------------------
// Block reduction of `nslots` double-float lanes held per thread in `v[]` (compile-time
// count NS, runtime count nslots <= NS).  Lane results of block b go to
// partials[b * nslots + s].  Fixed order: warp xor-tree, then warps in index order.
// ---------------------------------------------------------------------------------------
template <int NS>
__device__ __forceinline__ void block_reduce_to_partials(ddf (&v)[NS], int nslots, float2* partials,
                                                         ddf* smem /* [kBlock/32][NS] */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    if (s < nslots) {
      ddf w = dd_warp_sum(v[s]);
      if (lane == 0) smem[warp * NS + s] = w;
    }
  }
  __syncthreads();
  if (threadIdx.x < nslots) {
    ddf acc = smem[threadIdx.x];
    for (int w = 1; w < nwarps; ++w) acc = dd_add(acc, smem[w * NS + threadIdx.x]);
    partials[(size_t)blockIdx.x * nslots + threadIdx.x] = make_float2(acc.hi, acc.lo);
  }
}

// Block reduction of NS double-float lanes through shared memory: every thread writes its lanes
// to buf[s * blockDim + t], then lane s is summed by G consecutive threads (G the largest
// power of two, at most 32, with G NS <= blockDim), thread g of the group adding rows g,
// g + G, ... in order, and the group combined by an xor tree.  The lane results of block b go
// to partials[b * NS + s].  buf: NS * blockDim double-floats of shared memory no thread uses
// at the call.  Fixed order, so bitwise repeatable; ends with the partials written by the
// groups' first threads (no barrier after).
template <int NS>
__device__ __forceinline__ void block_reduce_transpose(const ddf (&v)[NS], float2* partials, ddf* buf) {
  const int nt = blockDim.x, t = threadIdx.x;
#pragma unroll
  for (int s = 0; s < NS; ++s) buf[s * nt + t] = v[s];
  __syncthreads();
  int G = 32;
  while (G > 1 && G * NS > nt) G >>= 1;
  const int s = t / G, g = t % G;
  ddf acc = {0.f, 0.f};
  if (s < NS)
    for (int i = g; i < nt; i += G) acc = dd_add(acc, buf[s * nt + i]);
  for (int m = G / 2; m > 0; m >>= 1) acc = dd_add(acc, dd_shfl_xor(acc, m));
  if (s < NS && g == 0) partials[(size_t)blockIdx.x * NS + s] = make_float2(acc.hi, acc.lo);
}

// Completion word of a result record (kResultFlag): every thread of the last block calls
// this after its last write to `result`; thread 0 sets the word.  A host that polls a mapped
// record watches its fields (kResultSentinel), so no system-scope fence is needed here (one
// cost about 1.5 us at the end of every evaluation); `writers` is kept for the call sites.
__device__ __forceinline__ void result_complete(double* result, int writers = 1 << 30) {
  (void)writers;
  __syncthreads();
  if (threadIdx.x == 0) *(volatile double*)(result + kResultFlag) = 1.0;
}

// After every block has written its partials: take a ticket.  True in the block that draws
// the last one; every partial is then visible to it.  The caller resets the ticket.  The
// block barrier orders the block's writes before thread 0's ticket, an acquire-release
// atomic at device scope (release: cumulative over the writes the barrier ordered before it;
// acquire: the last block sees every block's released writes, and its barrier passes that on
// to its other threads) - no full fence in every thread.
__device__ __forceinline__ bool last_block_ticket(unsigned* ticket, int nblocks) {
  __shared__ bool is_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned prev;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], 1;" : "=r"(prev) : "l"(ticket) : "memory");
    is_last = prev == (unsigned)(nblocks - 1);
  }
  __syncthreads();
  return is_last;
}

// Lane sums of partials[0 .. nblocks) by threads [0, nthreads) of the block (every thread of
// the block calls it), loads in rounds of U per thread: lane s is summed by `per` consecutive
// threads (per a power of two),
// thread g of the group adding blocks g, g + per, ... (each round of U by a pairwise tree,
// the rounds in order); the group is combined by an
// xor tree (and, for groups wider than a warp, by the warps in index order) into out[s]
// (FP64).  Ends with a block barrier.
template <int U = 16>
__device__ __forceinline__ void reduce_partials(const float2* partials, int nslots, int nblocks, double* out,
                                                ddf* smem, int nthreads) {
  int per = 1;
  while (per * 2 * nslots <= nthreads) per *= 2;
  const int s = threadIdx.x / per, g = threadIdx.x % per;
  ddf acc = {0.f, 0.f};
  if (s < nslots && (int)threadIdx.x < nthreads) {
    // rounds of U independent loads in flight (the last round padded with exact zeros), each
    // round added by a fixed pairwise tree (log2 U dependent additions, not U): one L2 round
    // trip per round
    for (int b = g; b < nblocks; b += U * per) {
      ddf q[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int bb = b + u * per;
        const float2 v = bb < nblocks ? __ldcg(partials + (size_t)bb * nslots + s) : make_float2(0.f, 0.f);
        q[u] = ddf{v.x, v.y};
      }
#pragma unroll
      for (int w = 1; w < U; w *= 2)
#pragma unroll
        for (int i = 0; i + w < U; i += 2 * w) q[i] = dd_add(q[i], q[i + w]);
      acc = dd_add(acc, q[0]);
    }
  }
  const int wper = per < 32 ? per : 32;
  for (int m = wper / 2; m > 0; m >>= 1) acc = dd_add(acc, dd_shfl_xor(acc, m));
  if (per <= 32) {
    if (g == 0 && s < nslots && (int)threadIdx.x < nthreads) out[s] = dd_to_double(acc);
  } else {
    if ((threadIdx.x & 31) == 0) smem[threadIdx.x >> 5] = acc;
    __syncthreads();
    if ((int)threadIdx.x < nslots) {
      const int w0 = threadIdx.x * (per / 32);
      ddf tot = smem[w0];
      for (int k = 1; k < per / 32; ++k) tot = dd_add(tot, smem[w0 + k]);
      out[threadIdx.x] = dd_to_double(tot);
    }
  }
  __syncthreads();
}

// The ticket and the reduction by every thread; returns true in the last block, which also
// resets the ticket.
__device__ __forceinline__ bool last_block_reduce(const float2* partials, int nslots, int nblocks,
                                                  unsigned* ticket, double* out, ddf* smem) {
  if (!last_block_ticket(ticket, nblocks)) return false;
  reduce_partials(partials, nslots, nblocks, out, smem, blockDim.x);
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

}  // namespace goo
