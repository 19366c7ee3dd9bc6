// jit.cu -- run-time specialisation of the FP32 packed-pair event kernel for one model.
//
// The interpreter compiled into the library reads each leaf slot's opcode at run time: per
// event pair it dispatches every slot and accumulates all three gradient lanes of every
// slot, although a model's leaves are fixed once it is built.  For a model whose FP32
// evaluation runs in the packed-pair kernel, the library compiles that kernel again with the
// model's leaf signature as a template argument (sop_kernels.cuh), using NVRTC on the first
// evaluation, so that the dispatch folds away and only the lanes the leaves have are
// accumulated.  The result is the same computation in the same order up to the rounding
// of fused multiply-adds; the parity tests compare both kernels against the oracle.
//
// Compiled kernels are kept for the life of the process, keyed by shape and signature, and
// shared by every model and device (a CUDA library is context-independent).  If NVRTC fails
// the interpreter runs instead and the failure is reported by goo_model_jit_status.
#include <nvrtc.h>

#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "jit.cuh"
#include "jit_sources.inc"  // kJitHeaderNames / kJitHeaderSources, generated at build time

#ifndef GOO_CUDA_INCLUDE
#define GOO_CUDA_INCLUDE "/usr/local/cuda/include"
#endif

namespace goo {

namespace {

struct JitEntry {
  int state = 0;  // 1: compiled and loaded, -1: failed
  cudaLibrary_t lib = nullptr;
  cudaKernel_t kernel = nullptr;
  bool smem_set[64] = {};
};

std::mutex g_mu;
std::map<std::string, JitEntry> g_cache;

// NVRTC compilation of sop_event2_kernel<K, L, grad, sig, cols, direct> to an sm_103a cubin:
// the image and the kernel's lowered name.  Needs no device.
int compile_event2_cubin(int K, int L, bool grad, unsigned long long sig, unsigned long long cols, bool direct,
                         std::vector<char>& cubin, std::string& kname) {
  const char* src = "#include \"sop_kernels.cuh\"\n";
  const int nh = (int)(sizeof(kJitHeaderNames) / sizeof(kJitHeaderNames[0]));
  nvrtcProgram prog;
  if (nvrtcCreateProgram(&prog, src, "goo_event2_jit.cu", nh, kJitHeaderSources, kJitHeaderNames) != NVRTC_SUCCESS)
    return set_error(GOO_ERR_CUDA, "NVRTC: cannot create the program");
  char name[192];
  std::snprintf(name, sizeof name, "goo::sop_event2_kernel<%d, %d, %s, 0x%llxull, 0x%llxull, %s>", K, L,
                grad ? "true" : "false", sig, cols, direct ? "true" : "false");
  nvrtcAddNameExpression(prog, name);
  const char* opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-default-device", "-lineinfo", "-I" GOO_CUDA_INCLUDE,
                        "-I" GOO_CUDA_INCLUDE "/cccl"};
  const nvrtcResult rc = nvrtcCompileProgram(prog, (int)(sizeof(opts) / sizeof(opts[0])), opts);
  if (rc != NVRTC_SUCCESS) {
    size_t n = 0;
    nvrtcGetProgramLogSize(prog, &n);
    std::string log(n, '\0');
    if (n) nvrtcGetProgramLog(prog, &log[0]);
    nvrtcDestroyProgram(&prog);
    return set_error(GOO_ERR_CUDA, "NVRTC compilation of %s failed: %s\n%.2000s", name, nvrtcGetErrorString(rc),
                     log.c_str());
  }
  const char* lowered = nullptr;
  size_t cubin_size = 0;
  if (nvrtcGetLoweredName(prog, name, &lowered) != NVRTC_SUCCESS || nvrtcGetCUBINSize(prog, &cubin_size) != NVRTC_SUCCESS) {
    nvrtcDestroyProgram(&prog);
    return set_error(GOO_ERR_CUDA, "NVRTC: no kernel image for %s", name);
  }
  kname = lowered;
  cubin.resize(cubin_size);
  nvrtcGetCUBIN(prog, cubin.data());
  nvrtcDestroyProgram(&prog);
  return GOO_OK;
}

int compile_event2(int K, int L, bool grad, unsigned long long sig, unsigned long long cols, bool direct,
                   JitEntry& e) {
  std::vector<char> cubin;
  std::string kname;
  GOO_TRY(compile_event2_cubin(K, L, grad, sig, cols, direct, cubin, kname));
  GOO_CUDA_TRY(cudaLibraryLoadData(&e.lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0));
  GOO_CUDA_TRY(cudaLibraryGetKernel(&e.kernel, e.lib, kname.c_str()));
  return GOO_OK;
}

}  // namespace

const void* jit_event2_kernel(int device, int K, int L, bool grad, unsigned long long sig, unsigned long long cols,
                              bool direct, size_t max_smem, int* status) {
  char key[112];
  std::snprintf(key, sizeof key, "%d:%d:%d:%llx:%llx:%d", K, L, (int)grad, sig, cols, (int)direct);
  std::lock_guard<std::mutex> lock(g_mu);
  JitEntry& e = g_cache[key];
  if (e.state == 0) {
    const int rc = compile_event2(K, L, grad, sig, cols, direct, e);
    e.state = rc == GOO_OK ? 1 : -1;
    if (rc != GOO_OK) {
      cudaGetLastError();
      if (log_level() >= 1) std::fprintf(stderr, "[goo] kernel specialisation unavailable; the interpreter runs\n");
    }
  }
  if (e.state < 0) {
    *status = -1;
    return nullptr;
  }
  if (device >= 0 && device < 64 && !e.smem_set[device]) {
    if (cudaFuncSetAttribute((const void*)e.kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_smem) !=
        cudaSuccess) {
      cudaGetLastError();
      *status = -1;
      return nullptr;
    }
    e.smem_set[device] = true;
  }
  *status = 2;
  return (const void*)e.kernel;
}

}  // namespace goo

extern "C" int goo_jit_check(int K, int L, int grad, unsigned long long sig, unsigned long long cols,
                             int64_t* cubin_bytes) {
  using namespace goo;
  if (K < 1 || K > kMaxComp || L < 1 || L > kMaxLeaf)
    return set_error(GOO_ERR_ARG, "goo_jit_check: shape %d x %d (1..%d x 1..%d)", K, L, kMaxComp, kMaxLeaf);
  std::vector<char> cubin;
  std::string kname;
  GOO_TRY(compile_event2_cubin(K, L, grad != 0, sig, cols, false, cubin, kname));
  if (cubin_bytes) *cubin_bytes = (int64_t)cubin.size();
  return GOO_OK;
}
