// core.cu -- context, error reporting, dataset upload with the on-device range check,
// and the host combination of shard partials.
//
// Paper: DataSets attach event data to observables (Fig. 1); input is range-checked so
// that users who load data out of range are warned (Sec. 4); MPI runs divide the dataset
// among processes and sum their partial results (Sec. 4).
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <chrono>
#include <map>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "model.cuh"

namespace goo {

static thread_local std::string g_last_error;

int log_level() {
  static int level = [] {
    const char* s = std::getenv("GOO_LOG");
    return s ? std::atoi(s) : 0;
  }();
  return level;
}

int set_error(int code, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  if (log_level() >= 1) std::fprintf(stderr, "[goo] error %d: %s\n", code, buf);
  return code;
}

int ensure_partials(goo_ctx* ctx, size_t n_float2) {
  Scratch& s = ctx->scratch;
  if (n_float2 <= s.partials_cap) return GOO_OK;
  if (s.partials) cudaFree(s.partials);
  s.partials = nullptr;
  s.partials_cap = 0;
  size_t cap = n_float2 < 65536 ? 65536 : n_float2;
  if (cudaMalloc(&s.partials, cap * sizeof(float2)) != cudaSuccess) {
    cudaGetLastError();
    return set_error(GOO_ERR_OOM, "cannot allocate %zu reduction partials", cap);
  }
  s.partials_cap = cap;
  return GOO_OK;
}

static cudaEvent_t pool_event(goo_ctx* ctx) {
  if (!ctx->event_pool.empty()) {
    cudaEvent_t e = ctx->event_pool.back();
    ctx->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

LaunchScope::LaunchScope(goo_ctx* c, const char* n) : ctx(c), name(n) {
  ctx->launches++;
  if (ctx->timing) {
    start = pool_event(ctx);
    stop = pool_event(ctx);
    if (start) cudaEventRecord(start, ctx->stream);
  }
}

LaunchScope::~LaunchScope() {
  if (start && stop) {
    cudaEventRecord(stop, ctx->stream);
    ctx->pending.push_back({name, start, stop});
  }
}

static void fold_timings(goo_ctx* ctx) {
  for (auto& p : ctx->pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.stop) == cudaSuccess && cudaEventElapsedTime(&ms, p.start, p.stop) == cudaSuccess) {
      KernelStat* st = nullptr;
      for (auto& s : ctx->stats)
        if (s.name == p.name) st = &s;
      if (!st) {
        ctx->stats.push_back(KernelStat{p.name, 0, 0.0});
        st = &ctx->stats.back();
      }
      st->count++;
      st->ms += ms;
    }
    cudaGetLastError();
    ctx->event_pool.push_back(p.start);
    ctx->event_pool.push_back(p.stop);
  }
  ctx->pending.clear();
}

// Waits until the first `n` fields of the mapped result record that a kernel writes (armed
// with kResultSentinel before its launch) all hold values, then copies them.  Each field is
// one aligned 8-byte store of the kernel, so a field read without the sentinel is final.  The
// host polls for up to 2 ms, then waits on the stream, which also reports a failed launch.
void arm_result_mapped(goo_ctx* ctx) {
  volatile unsigned long long* rec = reinterpret_cast<volatile unsigned long long*>(ctx->scratch.result_host);
  for (int i = 0; i < kResultDoubles; ++i) rec[i] = kResultSentinel;
  ctx->scratch.result_host[kResultFlag] = 0.0;
}

int read_result_mapped(goo_ctx* ctx, int n, double* dst) {
  volatile unsigned long long* rec = reinterpret_cast<volatile unsigned long long*>(ctx->scratch.result_host);
  const auto t0 = std::chrono::steady_clock::now();
  int i = 0;
  for (unsigned it = 0;; ++it) {
    while (i < n && rec[i] != kResultSentinel) ++i;
    if (i == n) break;
    if ((it & 255u) == 0 && std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(2)) {
      GOO_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
      for (i = 0; i < n; ++i)
        if (rec[i] == kResultSentinel)
          return set_error(GOO_ERR_STATE, "the kernel finished without writing field %d of its result record", i);
      break;
    }
  }
  std::atomic_thread_fence(std::memory_order_acquire);
  std::memcpy(dst, (const double*)ctx->scratch.result_host, n * sizeof(double));
  return GOO_OK;
}

MappedResult::MappedResult(goo_ctx* c) : ctx(c) {
  arm_result_mapped(ctx);
  ctx->scratch.result_out = ctx->scratch.result_host;
}
MappedResult::~MappedResult() { ctx->scratch.result_out = ctx->scratch.result; }

int cached_occupancy(const void* kernel, int device, int block, size_t smem) {
  struct Key {
    const void* k;
    int dev, block;
    size_t smem;
    bool operator<(const Key& o) const {
      if (k != o.k) return k < o.k;
      if (dev != o.dev) return dev < o.dev;
      if (block != o.block) return block < o.block;
      return smem < o.smem;
    }
  };
  static std::mutex mu;
  static std::map<Key, int> cache;
  const Key key{kernel, device, block, smem};
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, block, smem) != cudaSuccess || n < 1) {
    cudaGetLastError();
    n = 1;
  }
  std::lock_guard<std::mutex> lock(mu);
  cache[key] = n;
  return n;
}

int grid_blocks(goo_ctx* ctx, int64_t work_items, int blocks_per_sm) {
  int64_t need = (work_items + kBlock - 1) / kBlock;
  int64_t cap = (int64_t)ctx->num_sms * blocks_per_sm;
  if (need < 1) need = 1;
  return (int)(need < cap ? need : cap);
}

// ---------------------------------------------------------------------------------------
// dataset kernels
// ---------------------------------------------------------------------------------------
// One pass over the events at upload: reads each column in the precision it was given
// (from the dataset's own buffer, or from pinned host memory for a mapped upload), writes the
// other precision (and, for a mapped upload, the given one), and counts events with any
// column outside [lo, hi] (NaN counts as outside).  Four events per thread where every source
// is 16-byte aligned.  One integer atomic per block: the count is exact and order-independent.
struct IngestArgs {
  const void* src[kMaxCols];
  double* d64[kMaxCols];
  float* d32[kMaxCols];
  double lo[kMaxCols], hi[kMaxCols];
  int ncols;
  int store_src;  // also store the source values into the buffer of their own precision
};

template <bool F32>
__device__ __forceinline__ bool ingest_one(const IngestArgs& a, int c, int64_t i) {
  double v;
  if constexpr (F32) {
    const float f = ((const float*)a.src[c])[i];
    if (a.store_src) a.d32[c][i] = f;
    v = (double)f;
    a.d64[c][i] = v;
  } else {
    v = ((const double*)a.src[c])[i];
    if (a.store_src) a.d64[c][i] = v;
    a.d32[c][i] = (float)v;
  }
  return v >= a.lo[c] && v <= a.hi[c];
}

template <bool F32, bool VEC>
__global__ void ingest_kernel(IngestArgs a, int64_t n, unsigned long long* bad) {
  unsigned local = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t tail = 0;
  if constexpr (VEC) {
    const int64_t nq = n / 4;
    tail = nq * 4;
    for (int64_t q = t0; q < nq; q += stride) {
      bool ok[4] = {true, true, true, true};
      for (int c = 0; c < a.ncols; ++c) {
        double v[4];
        if constexpr (F32) {
          const float4 f = ((const float4*)a.src[c])[q];
          if (a.store_src) ((float4*)a.d32[c])[q] = f;
          v[0] = f.x, v[1] = f.y, v[2] = f.z, v[3] = f.w;
          ((double2*)a.d64[c])[2 * q] = make_double2(v[0], v[1]);
          ((double2*)a.d64[c])[2 * q + 1] = make_double2(v[2], v[3]);
        } else {
          const double2 d0 = ((const double2*)a.src[c])[2 * q], d1 = ((const double2*)a.src[c])[2 * q + 1];
          if (a.store_src) {
            ((double2*)a.d64[c])[2 * q] = d0;
            ((double2*)a.d64[c])[2 * q + 1] = d1;
          }
          v[0] = d0.x, v[1] = d0.y, v[2] = d1.x, v[3] = d1.y;
          ((float4*)a.d32[c])[q] = make_float4((float)v[0], (float)v[1], (float)v[2], (float)v[3]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) ok[j] = ok[j] && v[j] >= a.lo[c] && v[j] <= a.hi[c];
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) local += ok[j] ? 0u : 1u;
    }
  }
  for (int64_t i = tail + t0; i < n; i += stride) {
    bool ok = true;
    for (int c = 0; c < a.ncols; ++c) ok = ingest_one<F32>(a, c, i) && ok;
    local += ok ? 0u : 1u;
  }
  for (int m = 16; m > 0; m >>= 1) local += __shfl_xor_sync(0xffffffffu, local, m);
  __shared__ unsigned warp_sum[32];
  if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = local;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += warp_sum[w];
    if (t) atomicAdd(bad, t);
  }
}

static void free_dataset_memory(goo_dataset* ds) {
  for (int c = 0; c < kMaxCols; ++c) {
    if (ds->d64[c] && ds->owns64) cudaFree(ds->d64[c]);
    if (ds->d32[c] && ds->owns32) cudaFree(ds->d32[c]);
    ds->d64[c] = nullptr;
    ds->d32[c] = nullptr;
  }
  if (ds->w64) cudaFree(ds->w64);
  if (ds->w32) cudaFree(ds->w32);
  ds->w64 = nullptr;
  ds->w32 = nullptr;
  for (auto& c : ds->cache) {
    if (c.ptr) cudaFree(c.ptr);
    c.ptr = nullptr;
    c.bytes = 0;
    c.key = 0;
  }
}


// Brings n events of the given columns into the dataset's buffers and range-checks them:
// with mapped == false the columns are already in the buffer of `dtype` (copied or borrowed);
// with mapped == true `cols` are pinned host arrays that the ingest kernel reads itself.
// Waits for the stream and returns the number of out-of-range events in *nb.
static int ingest(goo_dataset* ds, const void* const* cols, int dtype, int64_t n, bool mapped,
                  unsigned long long* nb) {
  goo_ctx* ctx = ds->ctx;
  *nb = 0;
  if (n > 0) {
    IngestArgs a{};
    a.ncols = ds->ncols;
    a.store_src = mapped ? 1 : 0;
    bool aligned = true;
    for (int c = 0; c < ds->ncols; ++c) {
      a.src[c] = mapped ? cols[c] : (dtype == GOO_F32 ? (const void*)ds->d32[c] : (const void*)ds->d64[c]);
      a.d64[c] = ds->d64[c];
      a.d32[c] = ds->d32[c];
      a.lo[c] = ds->lo[c];
      a.hi[c] = ds->hi[c];
      aligned = aligned && ((uintptr_t)a.src[c] & 15) == 0 && ((uintptr_t)a.d64[c] & 15) == 0 &&
                ((uintptr_t)a.d32[c] & 15) == 0;
    }
    unsigned long long* bad = (unsigned long long*)(ctx->scratch.counters + 8);
    GOO_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(unsigned long long), ctx->stream));
    {
      LaunchScope ls(ctx, "ingest");
      const int nb_ = grid_blocks(ctx, aligned ? (n + 3) / 4 : n, 8);
      if (dtype == GOO_F32) {
        if (aligned) ingest_kernel<true, true><<<nb_, kBlock, 0, ctx->stream>>>(a, n, bad);
        else ingest_kernel<true, false><<<nb_, kBlock, 0, ctx->stream>>>(a, n, bad);
      } else {
        if (aligned) ingest_kernel<false, true><<<nb_, kBlock, 0, ctx->stream>>>(a, n, bad);
        else ingest_kernel<false, false><<<nb_, kBlock, 0, ctx->stream>>>(a, n, bad);
      }
      GOO_CUDA_TRY(cudaGetLastError());
    }
    unsigned long long* stage = (unsigned long long*)(ctx->scratch.host_pinned + kPinnedResult);
    GOO_CUDA_TRY(cudaMemcpyAsync(stage, bad, sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx->stream));
    GOO_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    *nb = *stage;
  } else {
    GOO_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  }
  return GOO_OK;
}

// A fresh value for goo_dataset::epoch (unique over the process).
static uint64_t next_dataset_epoch() {
  static std::atomic<uint64_t> counter{1};
  return counter.fetch_add(1);
}

// True when every column is host memory the device can address (pinned / registered).
static bool host_mapped(const void* const* cols, int ncols) {
  for (int c = 0; c < ncols; ++c) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, cols[c]) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    if (at.type != cudaMemoryTypeHost || at.devicePointer != cols[c]) return false;
  }
  return true;
}

}  // namespace goo

using namespace goo;

extern "C" {

const char* goo_last_error(void) { return g_last_error.c_str(); }

const char* goo_version(void) { return "goo-gb300 0.1 (sm_103a)"; }

int64_t goo_launch_count(const goo_ctx* ctx) { return ctx ? ctx->launches : -1; }

int goo_timing_enable(goo_ctx* ctx, int on) {
  if (!ctx) return set_error(GOO_ERR_ARG, "goo_timing_enable: NULL context");
  fold_timings(ctx);
  ctx->timing = on != 0;
  return GOO_OK;
}

int goo_timing_read(goo_ctx* ctx, int max_entries, char* names, int64_t* counts, double* total_ms, int reset) {
  if (!ctx || max_entries < 0 || (max_entries > 0 && (!names || !counts || !total_ms)))
    return set_error(GOO_ERR_ARG, "goo_timing_read: bad arguments");
  fold_timings(ctx);
  const int n = (int)ctx->stats.size();
  for (int i = 0; i < n && i < max_entries; ++i) {
    std::snprintf(names + 64 * i, 64, "%s", ctx->stats[i].name.c_str());
    counts[i] = ctx->stats[i].count;
    total_ms[i] = ctx->stats[i].ms;
  }
  if (reset) ctx->stats.clear();
  return n;
}

int goo_set_wait_limit(goo_ctx* ctx, int64_t cycles) {
  if (!ctx) return set_error(GOO_ERR_ARG, "goo_set_wait_limit: NULL context");
  if (cycles < 0 || cycles > (int64_t)0xffffffffLL)
    return set_error(GOO_ERR_ARG, "goo_set_wait_limit: %lld cycles (0 .. 2^32 - 1)", (long long)cycles);
  GOO_CUDA_TRY(cudaSetDevice(ctx->device));
  const unsigned w = (unsigned)cycles;
  // ordered on the context's stream before every later evaluation; the call returns once the
  // word is on the device, so `w` may leave scope
  GOO_CUDA_TRY(cudaMemcpyAsync(ctx->scratch.counters + kWaitLimitWord, &w, sizeof w, cudaMemcpyHostToDevice,
                               ctx->stream));
  GOO_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  ctx->wait_limit = w;
  return GOO_OK;
}

int goo_debug_withhold_tile(goo_ctx* ctx, int64_t tile) {
  if (!ctx) return set_error(GOO_ERR_ARG, "goo_debug_withhold_tile: NULL context");
  if (tile < -1 || tile > (int64_t)0xfffffffeLL)
    return set_error(GOO_ERR_ARG, "goo_debug_withhold_tile: tile %lld", (long long)tile);
  GOO_CUDA_TRY(cudaSetDevice(ctx->device));
  const unsigned w = (unsigned)(tile + 1);
  GOO_CUDA_TRY(cudaMemcpyAsync(ctx->scratch.counters + kWithholdWord, &w, sizeof w, cudaMemcpyHostToDevice,
                               ctx->stream));
  GOO_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return GOO_OK;
}

int goo_init(int device, void* cuda_stream, goo_ctx** out) {
  if (!out) return set_error(GOO_ERR_ARG, "goo_init: out is NULL");
  *out = nullptr;
  int ndev = 0;
  GOO_CUDA_TRY(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return set_error(GOO_ERR_ARG, "goo_init: device %d of %d", device, ndev);
  GOO_CUDA_TRY(cudaSetDevice(device));
  goo_ctx* ctx = new goo_ctx();
  ctx->device = device;
  GOO_CUDA_TRY(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device));
  if (cuda_stream) {
    ctx->stream = (cudaStream_t)cuda_stream;
  } else {
    GOO_CUDA_TRY(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
    ctx->owns_stream = true;
  }
  Scratch& s = ctx->scratch;
  GOO_CUDA_TRY(cudaMalloc(&s.counters, 64 * sizeof(unsigned)));
  GOO_CUDA_TRY(cudaMemset(s.counters, 0, 64 * sizeof(unsigned)));
  GOO_CUDA_TRY(cudaMalloc(&s.result, (kResultDoubles + 1) * sizeof(double)));
  GOO_CUDA_TRY(cudaHostAlloc(&s.result_host, (kResultDoubles + 1) * sizeof(double), cudaHostAllocMapped));
  std::memset(s.result_host, 0, (kResultDoubles + 1) * sizeof(double));
  s.result_out = s.result;
  GOO_CUDA_TRY(cudaMalloc(&s.theta, 2 * kMaxParams * sizeof(double)));
  GOO_CUDA_TRY(cudaMallocHost(&s.host_pinned, 512 * sizeof(double)));
  int rc = ensure_partials(ctx, 65536);
  if (rc != GOO_OK) {
    goo_finalize(ctx);
    return rc;
  }
  *out = ctx;
  return GOO_OK;
}

int goo_finalize(goo_ctx* ctx) {
  if (!ctx) return set_error(GOO_ERR_ARG, "goo_finalize: NULL context");
  if (ctx->live > 0)
    return set_error(GOO_ERR_STATE, "goo_finalize: %d datasets, models or servers of this context are not freed", ctx->live);
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  Scratch& s = ctx->scratch;
  if (s.partials) cudaFree(s.partials);
  if (s.counters) cudaFree(s.counters);
  if (s.result) cudaFree(s.result);
  if (s.theta) cudaFree(s.theta);
  if (s.host_pinned) cudaFreeHost(s.host_pinned);
  if (s.result_host) cudaFreeHost(s.result_host);
  if (s.chunk_records) cudaFreeHost(s.chunk_records);
  for (cudaEvent_t e : s.chunk_events)
    if (e) cudaEventDestroy(e);
  if (s.copy_stream) cudaStreamDestroy(s.copy_stream);
  fold_timings(ctx);
  for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
  if (ctx->owns_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return GOO_OK;
}

// Copies n events of host columns into the dataset's buffers of `dtype` (copy engine, the
// context's stream).
static int copy_columns(goo_dataset* ds, const void* const* cols, int dtype, int64_t n) {
  const size_t es = dtype == GOO_F32 ? sizeof(float) : sizeof(double);
  for (int c = 0; c < ds->ncols && n > 0; ++c) {
    void* dst = dtype == GOO_F32 ? (void*)ds->d32[c] : (void*)ds->d64[c];
    GOO_CUDA_TRY(cudaMemcpyAsync(dst, cols[c], (size_t)n * es, cudaMemcpyHostToDevice, ds->ctx->stream));
  }
  return GOO_OK;
}

int goo_dataset_upload(goo_ctx* ctx, int ncols, const void* const* cols, int dtype, int64_t n_events,
                       const double* lo, const double* hi, int flags, goo_dataset** out, int64_t* n_bad) {
  if (n_bad) *n_bad = 0;
  if (!ctx || !cols || !lo || !hi || !out) return set_error(GOO_ERR_ARG, "goo_dataset_upload: NULL argument");
  *out = nullptr;
  if (ncols < 1 || ncols > kMaxCols) return set_error(GOO_ERR_ARG, "goo_dataset_upload: ncols=%d (1..%d)", ncols, kMaxCols);
  if (n_events < 0) return set_error(GOO_ERR_ARG, "goo_dataset_upload: n_events=%lld", (long long)n_events);
  if (dtype != GOO_F64 && dtype != GOO_F32) return set_error(GOO_ERR_ARG, "goo_dataset_upload: dtype=%d", dtype);
  if (flags != GOO_COPY && flags != GOO_BORROW_DEVICE && flags != GOO_COPY_MAPPED && flags != GOO_BORROW_HOST)
    return set_error(GOO_ERR_ARG, "goo_dataset_upload: flags=%d", flags);
  if (flags == GOO_BORROW_HOST && dtype != GOO_F32)
    return set_error(GOO_ERR_ARG, "goo_dataset_upload: GOO_BORROW_HOST takes float32 columns (GOO_F32)");
  for (int c = 0; c < ncols; ++c) {
    if (!(lo[c] < hi[c])) return set_error(GOO_ERR_ARG, "goo_dataset_upload: column %d has lo >= hi", c);
    if (n_events > 0 && !cols[c]) return set_error(GOO_ERR_ARG, "goo_dataset_upload: column %d is NULL", c);
    if ((flags == GOO_BORROW_DEVICE || flags == GOO_BORROW_HOST) && ((uintptr_t)cols[c] & 15))
      return set_error(GOO_ERR_ARG, "goo_dataset_upload: borrowed column %d is not 16-byte aligned", c);
  }
  GOO_CUDA_TRY(cudaSetDevice(ctx->device));
  if ((flags == GOO_COPY_MAPPED || flags == GOO_BORROW_HOST) && n_events > 0 && !host_mapped(cols, ncols))
    return set_error(GOO_ERR_ARG, "goo_dataset_upload: %s needs pinned host columns",
                     flags == GOO_COPY_MAPPED ? "GOO_COPY_MAPPED" : "GOO_BORROW_HOST");
  if (flags == GOO_BORROW_HOST) {
    // the columns stay in host memory; evaluations read them through their device mapping
    goo_dataset* ds = new goo_dataset();
    ds->ctx = ctx;
    ds->n = n_events;
    ds->capacity = n_events;
    ds->epoch = next_dataset_epoch();
    ds->ncols = ncols;
    ds->owns64 = ds->owns32 = false;
    ds->host_borrowed = true;
    for (int c = 0; c < ncols; ++c) {
      ds->lo[c] = lo[c];
      ds->hi[c] = hi[c];
      void* dp = nullptr;
      if (n_events > 0 && cudaHostGetDevicePointer(&dp, const_cast<void*>(cols[c]), 0) != cudaSuccess) {
        cudaGetLastError();
        delete ds;
        return set_error(GOO_ERR_ARG, "goo_dataset_upload: column %d has no device mapping", c);
      }
      if ((uintptr_t)dp & 15) {
        delete ds;
        return set_error(GOO_ERR_ARG, "goo_dataset_upload: the device mapping of column %d is not 16-byte aligned", c);
      }
      ds->d32[c] = (float*)dp;
    }
    ctx->live++;
    *out = ds;
    return GOO_OK;
  }
  goo_dataset* ds = new goo_dataset();
  ds->ctx = ctx;
  ds->n = n_events;
  ds->capacity = n_events;
  ds->epoch = next_dataset_epoch();
  ds->ncols = ncols;
  ds->owns64 = !(flags == GOO_BORROW_DEVICE && dtype == GOO_F64);
  ds->owns32 = !(flags == GOO_BORROW_DEVICE && dtype == GOO_F32);
  const size_t n_alloc = (size_t)(n_events > 0 ? n_events : 1) + 4;  // +4: room for vector tails
  auto fail = [&](int code, const char* what) {
    cudaGetLastError();
    free_dataset_memory(ds);
    delete ds;
    return set_error(code, "goo_dataset_upload: %s", what);
  };
  for (int c = 0; c < ncols; ++c) {
    ds->lo[c] = lo[c];
    ds->hi[c] = hi[c];
    if (flags == GOO_BORROW_DEVICE && dtype == GOO_F64) ds->d64[c] = (double*)cols[c];
    else if (cudaMalloc(&ds->d64[c], n_alloc * sizeof(double)) != cudaSuccess) return fail(GOO_ERR_OOM, "out of device memory");
    if (flags == GOO_BORROW_DEVICE && dtype == GOO_F32) ds->d32[c] = (float*)cols[c];
    else if (cudaMalloc(&ds->d32[c], n_alloc * sizeof(float)) != cudaSuccess) return fail(GOO_ERR_OOM, "out of device memory");
  }
  if (flags == GOO_COPY && copy_columns(ds, cols, dtype, n_events) != GOO_OK) return fail(GOO_ERR_CUDA, "host-to-device copy failed");
  unsigned long long nb = 0;
  if (ingest(ds, cols, dtype, n_events, flags == GOO_COPY_MAPPED, &nb) != GOO_OK) return fail(GOO_ERR_CUDA, "range check failed");
  if (nb) {
    if (n_bad) *n_bad = (int64_t)nb;
    free_dataset_memory(ds);
    delete ds;
    return set_error(GOO_ERR_RANGE, "goo_dataset_upload: %llu of %lld events lie outside the observable limits", nb,
                     (long long)n_events);
  }
  ctx->live++;
  *out = ds;
  return GOO_OK;
}

int goo_dataset_update(goo_dataset* ds, const void* const* cols, int dtype, int64_t n_events, int flags,
                       int64_t* n_bad) {
  if (n_bad) *n_bad = 0;
  if (!ds || !cols) return set_error(GOO_ERR_ARG, "goo_dataset_update: NULL argument");
  if (!ds->owns32 || !ds->owns64)
    return set_error(GOO_ERR_STATE, "goo_dataset_update: the dataset borrows its columns%s",
                     ds->host_borrowed ? " (GOO_BORROW_HOST: rewrite the host columns instead)" : "");
  if (n_events < 0 || n_events > ds->capacity)
    return set_error(GOO_ERR_ARG, "goo_dataset_update: n_events=%lld (capacity %lld)", (long long)n_events,
                     (long long)ds->capacity);
  if (dtype != GOO_F64 && dtype != GOO_F32) return set_error(GOO_ERR_ARG, "goo_dataset_update: dtype=%d", dtype);
  if (flags != GOO_COPY && flags != GOO_COPY_MAPPED) return set_error(GOO_ERR_ARG, "goo_dataset_update: flags=%d", flags);
  for (int c = 0; c < ds->ncols; ++c)
    if (n_events > 0 && !cols[c]) return set_error(GOO_ERR_ARG, "goo_dataset_update: column %d is NULL", c);
  GOO_CUDA_TRY(cudaSetDevice(ds->ctx->device));
  if (flags == GOO_COPY_MAPPED && n_events > 0 && !host_mapped(cols, ds->ncols))
    return set_error(GOO_ERR_ARG, "goo_dataset_update: GOO_COPY_MAPPED needs pinned host columns");
  // launches in flight may still read the old events and weights
  GOO_CUDA_TRY(cudaStreamSynchronize(ds->ctx->stream));
  ds->n = 0;
  ds->epoch = next_dataset_epoch();
  if (ds->w64) cudaFree(ds->w64);
  if (ds->w32) cudaFree(ds->w32);
  ds->w64 = nullptr;
  ds->w32 = nullptr;
  for (auto& c : ds->cache) c.key = 0;
  if (flags == GOO_COPY) GOO_TRY(copy_columns(ds, cols, dtype, n_events));
  unsigned long long nb = 0;
  GOO_TRY(ingest(ds, cols, dtype, n_events, flags == GOO_COPY_MAPPED, &nb));
  if (nb) {
    if (n_bad) *n_bad = (int64_t)nb;
    return set_error(GOO_ERR_RANGE, "goo_dataset_update: %llu of %lld events lie outside the observable limits; the "
                     "dataset now holds no events", nb, (long long)n_events);
  }
  ds->n = n_events;
  return GOO_OK;
}

int goo_nll_grad_streamed(goo_model* m, goo_dataset* ds, const float* const* host_cols, int64_t n_events,
                          int n_chunks, const double* theta, double* nll_out, double* grad_out, int64_t* n_bad) {
  if (n_bad) *n_bad = 0;
  if (!m || !ds || !host_cols || !theta || !nll_out) return set_error(GOO_ERR_ARG, "goo_nll_grad_streamed: NULL argument");
  if (m->kind != 0)
    return set_error(GOO_ERR_UNSUPPORTED, "goo_nll_grad_streamed: sum-of-product models only");
  if (ds->ctx != m->ctx) return set_error(GOO_ERR_ARG, "goo_nll_grad_streamed: model and dataset of different contexts");
  if (!ds->owns32 || !ds->owns64) return set_error(GOO_ERR_STATE, "goo_nll_grad_streamed: the dataset borrows its columns");
  if (n_events < 1 || n_events > ds->capacity)
    return set_error(GOO_ERR_ARG, "goo_nll_grad_streamed: n_events=%lld (capacity %lld)", (long long)n_events,
                     (long long)ds->capacity);
  if (n_chunks < 1 || n_chunks > kStreamChunks)
    return set_error(GOO_ERR_ARG, "goo_nll_grad_streamed: n_chunks=%d (1..%d)", n_chunks, kStreamChunks);
  if (ds->ncols < m->n_obs) return set_error(GOO_ERR_ARG, "goo_nll_grad_streamed: dataset has too few columns");
  for (int o = 0; o < m->n_obs; ++o)
    if (ds->lo[o] != m->lo[o] || ds->hi[o] != m->hi[o])
      return set_error(GOO_ERR_ARG, "goo_nll_grad_streamed: observable %d limits differ from the model's", o);
  for (int p = 0; p < m->n_params; ++p)
    if (!std::isfinite(theta[p])) return set_error(GOO_ERR_ARG, "goo_nll_grad_streamed: theta[%d] is not finite", p);
  goo_ctx* ctx = m->ctx;
  GOO_CUDA_TRY(cudaSetDevice(ctx->device));
  if (!host_mapped((const void* const*)host_cols, ds->ncols))
    return set_error(GOO_ERR_ARG, "goo_nll_grad_streamed: the host columns must be pinned");
  Scratch& sc = ctx->scratch;
  if (!sc.copy_stream) GOO_CUDA_TRY(cudaStreamCreateWithFlags(&sc.copy_stream, cudaStreamNonBlocking));
  for (cudaEvent_t& e : sc.chunk_events)
    if (!e) GOO_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  const size_t rec = kResultDoubles + 1;
  if (!sc.chunk_records) {
    GOO_CUDA_TRY(cudaHostAlloc(&sc.chunk_records, (size_t)kStreamChunks * rec * sizeof(double), cudaHostAllocMapped));
    std::memset(sc.chunk_records, 0, (size_t)kStreamChunks * rec * sizeof(double));
  }
  // launches in flight may still read the old events: the copies start after them
  GOO_CUDA_TRY(cudaEventRecord(sc.chunk_events[kStreamChunks], ctx->stream));
  GOO_CUDA_TRY(cudaStreamWaitEvent(sc.copy_stream, sc.chunk_events[kStreamChunks], 0));
  ds->n = 0;
  ds->epoch = next_dataset_epoch();
  if (ds->w64) cudaFree(ds->w64);
  if (ds->w32) cudaFree(ds->w32);
  ds->w64 = nullptr;
  ds->w32 = nullptr;
  for (auto& c : ds->cache) c.key = 0;
  const bool fuse = sop_norm_in_event(m, GOO_F32, true);
  GOO_TRY(sop_prepare(m, theta, GOO_F32, fuse));
  unsigned long long* bad = (unsigned long long*)(sc.counters + 8);
  GOO_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(unsigned long long), ctx->stream));
  // chunk boundaries on multiples of the event kernel's column tile
  constexpr int64_t kTile = 2 * kPairsPerThread * kBlock;
  const int64_t step = ((n_events + n_chunks - 1) / n_chunks + kTile - 1) / kTile * kTile;
  int nc = 0;
  const goo_dataset& dsv = *ds;
  for (int64_t b = 0; b < n_events; b += step, ++nc) {
    const int64_t e = std::min(n_events, b + step);
    for (int c = 0; c < ds->ncols; ++c)
      GOO_CUDA_TRY(cudaMemcpyAsync(ds->d32[c] + b, host_cols[c] + b, (size_t)(e - b) * sizeof(float),
                                   cudaMemcpyHostToDevice, sc.copy_stream));
    GOO_CUDA_TRY(cudaEventRecord(sc.chunk_events[nc], sc.copy_stream));
    GOO_CUDA_TRY(cudaStreamWaitEvent(ctx->stream, sc.chunk_events[nc], 0));
    // the chunk's float64 copy and range count, then its evaluation
    IngestArgs a{};
    a.ncols = ds->ncols;
    a.store_src = 0;
    bool aligned = true;
    for (int c = 0; c < ds->ncols; ++c) {
      a.src[c] = ds->d32[c] + b;
      a.d64[c] = ds->d64[c] + b;
      a.d32[c] = ds->d32[c] + b;
      a.lo[c] = ds->lo[c];
      a.hi[c] = ds->hi[c];
      aligned = aligned && ((uintptr_t)a.src[c] & 15) == 0 && ((uintptr_t)a.d64[c] & 15) == 0;
    }
    {
      LaunchScope ls(ctx, "ingest");
      const int nb_ = grid_blocks(ctx, aligned ? (e - b + 3) / 4 : e - b, 8);
      if (aligned) ingest_kernel<true, true><<<nb_, kBlock, 0, ctx->stream>>>(a, e - b, bad);
      else ingest_kernel<true, false><<<nb_, kBlock, 0, ctx->stream>>>(a, e - b, bad);
      GOO_CUDA_TRY(cudaGetLastError());
    }
    double* r = sc.chunk_records + (size_t)nc * rec;
    r[kResultFlag] = 0.0;
    ds->n = e;  // the event kernel reads [b, e) of the columns
    GOO_TRY(sop_events(m, &dsv, b, e, GOO_F32, true, 1, fuse, r));
  }
  unsigned long long* stage = (unsigned long long*)(sc.host_pinned + kPinnedResult);
  GOO_CUDA_TRY(cudaMemcpyAsync(stage, bad, sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx->stream));
  GOO_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  const unsigned long long nb = *stage;
  if (nb) {
    ds->n = 0;
    *nll_out = HUGE_VAL;
    if (n_bad) *n_bad = (int64_t)nb;
    return set_error(GOO_ERR_RANGE, "goo_nll_grad_streamed: %llu of %lld events lie outside the observable limits; the "
                     "dataset now holds no events", nb, (long long)n_events);
  }
  ds->n = n_events;
  // the chunks' records, added in chunk order with compensation (as goo_combine_partials)
  const int P = m->n_params;
  std::vector<double> parts((size_t)nc * (3 + P));
  double nbad_total = 0.0, status = 0.0;
  for (int c = 0; c < nc; ++c) {
    const double* r = sc.chunk_records + (size_t)c * rec;
    if (r[kResultFlag] == 0.0) return set_error(GOO_ERR_STATE, "goo_nll_grad_streamed: chunk %d wrote no record", c);
    if (r[2] < 0) status = -1.0;
    else nbad_total += r[2];
    double* q = parts.data() + (size_t)c * (3 + P);
    q[0] = r[0];
    q[1] = r[1];
    q[2] = 0.0;
    for (int p = 0; p < P; ++p) q[3 + p] = r[3 + p];
  }
  if (status < 0) {
    *nll_out = HUGE_VAL;
    return set_error(GOO_ERR_TIMEOUT, "goo_nll_grad_streamed: a device wait for event data gave up");
  }
  if (nbad_total > 0) {
    *nll_out = HUGE_VAL;
    if (grad_out)
      for (int p = 0; p < P; ++p) grad_out[p] = 0.0;
    return set_error(GOO_ERR_NONPOSITIVE_PDF, "goo_nll_grad_streamed: density <= 0 for %.0f events", nbad_total);
  }
  std::vector<double> tot(3 + P);
  GOO_TRY(goo_combine_partials(nc, P, parts.data(), tot.data()));
  *nll_out = tot[0] + tot[1];
  if (grad_out)
    for (int p = 0; p < P; ++p) grad_out[p] = tot[3 + p];
  return GOO_OK;
}

int goo_dataset_free(goo_dataset* ds) {
  if (!ds) return set_error(GOO_ERR_ARG, "goo_dataset_free: NULL dataset");
  cudaSetDevice(ds->ctx->device);
  cudaStreamSynchronize(ds->ctx->stream);
  free_dataset_memory(ds);
  ds->ctx->live--;
  delete ds;
  return GOO_OK;
}

int64_t goo_dataset_size(const goo_dataset* ds) { return ds ? ds->n : -1; }

// Per-event weights: checked on the host, then copied to the device in both precisions
// (the float32 copy rounded to nearest).  Replacing or removing them waits for the stream,
// since a launch in flight may read the old arrays.
int goo_dataset_set_weights(goo_dataset* ds, const double* w) {
  if (!ds) return set_error(GOO_ERR_ARG, "goo_dataset_set_weights: NULL dataset");
  if (ds->host_borrowed)
    return set_error(GOO_ERR_UNSUPPORTED, "goo_dataset_set_weights: a GOO_BORROW_HOST dataset takes no weights");
  const int64_t n = ds->n;
  std::vector<float> w32;
  if (w) {
    w32.resize((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
      if (!std::isfinite(w[i]) || w[i] < 0.0)
        return set_error(GOO_ERR_ARG, "goo_dataset_set_weights: weight %lld is %g (finite and >= 0 required)",
                         (long long)i, w[i]);
      w32[(size_t)i] = (float)w[i];
    }
  }
  GOO_CUDA_TRY(cudaSetDevice(ds->ctx->device));
  GOO_CUDA_TRY(cudaStreamSynchronize(ds->ctx->stream));
  if (ds->w64) cudaFree(ds->w64);
  if (ds->w32) cudaFree(ds->w32);
  ds->w64 = nullptr;
  ds->w32 = nullptr;
  if (!w) return GOO_OK;
  const size_t bytes = (size_t)std::max<int64_t>(n, 1);
  double* d64 = nullptr;
  float* d32 = nullptr;
  if (cudaMalloc(&d64, bytes * sizeof(double)) != cudaSuccess || cudaMalloc(&d32, bytes * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    if (d64) cudaFree(d64);
    return set_error(GOO_ERR_OOM, "goo_dataset_set_weights: device allocation of %lld weights failed", (long long)n);
  }
  if (n > 0) {
    GOO_CUDA_TRY(cudaMemcpyAsync(d64, w, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, ds->ctx->stream));
    GOO_CUDA_TRY(cudaMemcpyAsync(d32, w32.data(), (size_t)n * sizeof(float), cudaMemcpyHostToDevice, ds->ctx->stream));
    GOO_CUDA_TRY(cudaStreamSynchronize(ds->ctx->stream));
  }
  ds->w64 = d64;
  ds->w32 = d32;
  return GOO_OK;
}

const void* goo_dataset_column(const goo_dataset* ds, int col, int dtype) {
  if (!ds || col < 0 || col >= ds->ncols) return nullptr;
  return dtype == GOO_F32 ? (const void*)ds->d32[col] : (const void*)ds->d64[col];
}

// Compensated (two-sum) addition of shard records in index order.
int goo_combine_partials(int n_parts, int n_params, const double* parts, double* out) {
  if (n_parts < 0 || n_params < 0 || (n_parts && !parts) || !out)
    return set_error(GOO_ERR_ARG, "goo_combine_partials: bad arguments");
  const int stride = 3 + n_params;
  double s = 0.0, c = 0.0, cnt = 0.0;
  std::vector<double> g(n_params, 0.0), gc(n_params, 0.0);
  auto two_sum = [](double a, double b, double& err) {
    double t = a + b;
    double v = t - a;
    err = (a - (t - v)) + (b - v);
    return t;
  };
  for (int p = 0; p < n_parts; ++p) {
    const double* r = parts + (size_t)p * stride;
    double e1, e2;
    s = two_sum(s, r[0], e1);
    c += e1 + r[1];
    (void)e2;
    cnt += r[2];
    for (int j = 0; j < n_params; ++j) {
      double e;
      g[j] = two_sum(g[j], r[3 + j], e);
      gc[j] += e;
    }
  }
  double e;
  double hi = two_sum(s, c, e);
  out[0] = hi;
  out[1] = e;
  out[2] = cnt;
  for (int j = 0; j < n_params; ++j) out[3 + j] = g[j] + gc[j];
  return GOO_OK;
}

}  // extern "C"
