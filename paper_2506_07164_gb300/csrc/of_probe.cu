// Bandwidth probe: the measured peak that per-kernel L2 figures are divided
// by.  Not part of the detector.
//
// One launch reads `bytes` of a device buffer `reps` times with 16-byte loads
// cached in L2 only (ld.global.cg: no L1 allocation), from a grid of 8 blocks
// of 256 threads per SM, four independent loads in flight per thread.  A
// buffer that fits in L2 is served from L2 after the first pass, so the read
// rate over many passes is the L2 read bandwidth; a buffer far larger than L2
// gives the HBM read bandwidth.  The loaded words are folded into one value
// so the loads cannot be removed; that value is written to *sink.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "ofast.h"

namespace ofk {
void set_last_error(const std::string& msg);
}

namespace {

__global__ void __launch_bounds__(256) k_probe_read(const uint4* __restrict__ p, int64_t n16, int reps,
                                                    uint32_t* __restrict__ sink) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0;
    for (int r = 0; r < reps; ++r) {
        int64_t i = t;
        for (; i + 3 * stride < n16; i += 4 * stride) {
            const uint4 a = __ldcg(p + i), b = __ldcg(p + i + stride), c = __ldcg(p + i + 2 * stride),
                        d = __ldcg(p + i + 3 * stride);
            acc ^= (a.x ^ a.y ^ a.z ^ a.w) + (b.x ^ b.y ^ b.z ^ b.w) + (c.x ^ c.y ^ c.z ^ c.w) +
                   (d.x ^ d.y ^ d.z ^ d.w);
        }
        for (; i < n16; i += stride) {
            const uint4 a = __ldcg(p + i);
            acc ^= a.x ^ a.y ^ a.z ^ a.w;
        }
        acc = acc * 0x9E3779B1u + (uint32_t)r;
    }
    acc ^= __shfl_xor_sync(0xFFFFFFFFu, acc, 16);
    if (acc == 0x5A5A5A5Au) atomicXor(sink, acc);  // data-dependent, practically never taken
}

}  // namespace

extern "C" int of_probe_read(const void* buf, int64_t bytes, int reps, uint32_t* sink, void* stream) {
    if (!buf || !sink || bytes < 16 || reps < 1 || ((uintptr_t)buf & 15) != 0) {
        ofk::set_last_error("of_probe_read: buf 16-byte aligned, bytes >= 16, reps >= 1, sink not NULL");
        return OF_ERR_ARG;
    }
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        sms = 1;
    k_probe_read<<<8 * sms, 256, 0, (cudaStream_t)stream>>>(static_cast<const uint4*>(buf), bytes / 16, reps,
                                                            sink);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        ofk::set_last_error(std::string("of_probe_read: ") + cudaGetErrorString(e));
        return OF_ERR_CUDA;
    }
    return OF_OK;
}
