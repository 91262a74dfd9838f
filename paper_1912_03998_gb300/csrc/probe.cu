// probe.cu -- measurement kernels, not part of the method: the read
// bandwidth of this GPU's L2 cache, the roof against which the traversal's
// L2 traffic is reported (its node, triangle and plane arrays stay resident
// in L2), and the rate of float64 atomic additions the L2 sustains, the roof
// of a scatter whose accumulators take every contribution as eight atomic
// additions.
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

// Every thread adds 1.0 with float64 atomics (reductions: no value comes
// back) to the eight consecutive doubles of a 64-byte slot, `repeats` times,
// each time at a slot drawn by a per-thread linear congruential sequence
// from an L2-resident buffer of n_slots slots: the access pattern of the
// scatter's band accumulators.
__global__ void __launch_bounds__(256) k_l2_atomics(double *buf, uint32_t n_slots, int repeats) {
  const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  uint32_t h = (uint32_t)tid * 2654435761u + 12345u;
  for (int r = 0; r < repeats; r++) {
    h = h * 1664525u + 1013904223u;
    double *e = buf + (size_t)(h % n_slots) * 8;
#pragma unroll
    for (int b = 0; b < 8; b++) atomicAdd(e + b, 1.0);
  }
}

cudaError_t launch_l2_atomics(cudaStream_t st, double *buf, uint32_t n_slots, int repeats, int blocks) {
  k_l2_atomics<<<blocks, 256, 0, st>>>(buf, n_slots, repeats);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace bt
