// jit.cuh -- run-time specialisation of the FP32 packed-pair event kernel (jit.cu).
#pragma once

#include <cstddef>

namespace goo {

// The packed-pair event kernel sop_event2_kernel<K, L, grad, sig, cols, direct> compiled for
// this model's leaf signature and column map (4 and 2 bits per slot, see sop_kernels.cuh) and
// the column source (direct: host columns read by the kernel itself), with its
// dynamic shared memory limit raised to max_smem on `device`: a handle for the runtime's
// launch and occupancy calls.  Compiles on the first request of a signature.  Returns nullptr
// when NVRTC is unavailable or fails (*status = -1), else *status = 2.
const void* jit_event2_kernel(int device, int K, int L, bool grad, unsigned long long sig, unsigned long long cols,
                              bool direct, size_t max_smem, int* status);

}  // namespace goo
