// sg_probe.cu -- read-bandwidth probe: the measured denominator of the L2
// roofline that the benchmark reports for the simulator kernels.  Not part
// of the paper's method.
#include <cuda_runtime.h>

#include <cstdint>

#include "sg_host.h"
#include "sparrow_gb.h"

namespace {

// `reps` passes over n16 16-byte words with loads that are cached in L2 only
// (ld.global.cg), so that a buffer smaller than L2 is read from L2 on every
// pass after the first; the XOR of everything a CTA read goes to sink.
__global__ void __launch_bounds__(512) k_probe_read(const uint4* __restrict__ buf, long long n16, int reps,
                                                    uint32_t* __restrict__ sink) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  uint32_t acc = 0;
  for (int r = 0; r < reps; ++r) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    // four independent loads in flight per thread
    for (; i + 3 * stride < n16; i += 4 * stride) {
      const uint4 a = __ldcg(buf + i), b = __ldcg(buf + i + stride);
      const uint4 c = __ldcg(buf + i + 2 * stride), d = __ldcg(buf + i + 3 * stride);
      acc ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w ^ c.x ^ c.y ^ c.z ^ c.w ^ d.x ^ d.y ^ d.z ^ d.w;
    }
    for (; i < n16; i += stride) {
      const uint4 a = __ldcg(buf + i);
      acc ^= a.x ^ a.y ^ a.z ^ a.w;
    }
  }
  // one word per CTA (warp-reduced, then one atomic per warp)
  for (int off = 16; off > 0; off >>= 1) acc ^= __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) atomicXor(sink + blockIdx.x, acc);
}

}  // namespace

extern "C" int sg_probe_read(const void* buf_dev, size_t bytes, int32_t reps, uint32_t* sink_dev,
                             int32_t sink_words, sg_stream_t stream) {
  SG_RANGE("sg_probe_read");
  if (!buf_dev || !sink_dev || bytes < 16 || (bytes & 15) || ((uintptr_t)buf_dev & 15) || reps < 1)
    return SG_E_INVAL;
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe_read, 512, 0);
  if (e != cudaSuccess) return sg_set_cuda_error(e, "sg_probe_read");
  const int grid = sms * (per_sm > 0 ? per_sm : 1);
  if (sink_words < grid) return SG_E_INVAL;
  k_probe_read<<<grid, 512, 0, stream>>>(static_cast<const uint4*>(buf_dev), (long long)(bytes / 16), reps,
                                         sink_dev);
  e = cudaGetLastError();
  return e == cudaSuccess ? SG_OK : sg_set_cuda_error(e, "k_probe_read");
}
