// Known-answer helper for the GPU Philox stream: cuRAND's Philox4_32_10
// generator (device API, used as a library) writes the four 32-bit words of
// counter block m of subsequence t under key `seed`, i.e. the state after
// curand_init(seed, t, 4 m), for arrays of (t, m).  Built by the test with nvcc.
#include <cstdint>
#include <curand_kernel.h>

__global__ void curand_blocks(uint64_t seed, const uint64_t *t, const uint64_t *m, int64_t n, uint32_t *out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    curandStatePhilox4_32_10_t st;
    curand_init(seed, t[i], 4 * m[i], &st);
    const uint4 w = curand4(&st);
    out[4 * i + 0] = w.x;
    out[4 * i + 1] = w.y;
    out[4 * i + 2] = w.z;
    out[4 * i + 3] = w.w;
}

extern "C" int curand_philox_blocks(uint64_t seed, const uint64_t *t, const uint64_t *m, int64_t n, uint32_t *out) {
    if (n <= 0) return 0;
    curand_blocks<<<(unsigned)((n + 255) / 256), 256>>>(seed, t, m, n, out);
    return cudaDeviceSynchronize() == cudaSuccess ? 0 : 1;
}
