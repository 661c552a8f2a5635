// Test-only comparator: raw Philox4x32-10 words from cuRAND's device function,
// called as a black box, for the counters the integrator uses.
#include <cuda_runtime.h>
#include <curand_kernel.h>
#include <stdint.h>

__global__ void k_curand_words(uint64_t seed, uint32_t rep, uint64_t step, uint32_t atom0, int count,
                               uint32_t *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const uint4 c = make_uint4(atom0 + i, rep, (uint32_t)step, (uint32_t)(step >> 32));
    const uint2 k = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    const uint4 w = curand_Philox4x32_10(c, k);
    out[4 * i] = w.x; out[4 * i + 1] = w.y; out[4 * i + 2] = w.z; out[4 * i + 3] = w.w;
}

extern "C" int curand_words(uint64_t seed, uint32_t rep, uint64_t step, uint32_t atom0, int count,
                            uint32_t *host_out) {
    uint32_t *d = nullptr;
    if (cudaMalloc(&d, sizeof(uint32_t) * 4 * count) != cudaSuccess) return 1;
    k_curand_words<<<(count + 255) / 256, 256>>>(seed, rep, step, atom0, count, d);
    cudaError_t e = cudaMemcpy(host_out, d, sizeof(uint32_t) * 4 * count, cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e == cudaSuccess ? 0 : 2;
}
