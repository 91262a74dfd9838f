// probe.cu -- a measurement kernel, not part of the method: the read
// bandwidth of this GPU's L2 cache, the roof against which the traversal's
// L2 traffic is reported (its node, triangle and plane arrays stay resident
// in L2).
#include "bt_internal.cuh"

namespace bt {

// Every thread sums float4s of an L2-resident buffer in a grid-stride loop,
// `repeats` times over, with loads cached in L2 only (ld.global.cg), so that
// the bytes come from L2 and not from the SM's L1.  One partial sum per
// thread goes to `sink`, so that the loads cannot be dropped.
__global__ void __launch_bounds__(256) k_l2_read(const float4 *buf, int64_t n4, int repeats, float *sink) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  float acc = 0.0f;
  for (int r = 0; r < repeats; r++) {
#pragma unroll 4
    for (int64_t i = i0; i < n4; i += stride) {
      const float4 v = __ldcg(buf + i);
      acc += (v.x + v.y) + (v.z + v.w);
    }
  }
  sink[i0] = acc;
}

cudaError_t launch_l2_read(cudaStream_t st, const float4 *buf, int64_t n4, int repeats, float *sink, int blocks) {
  k_l2_read<<<blocks, 256, 0, st>>>(buf, n4, repeats, sink);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace bt
