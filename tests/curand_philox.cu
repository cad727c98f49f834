// Test helper: raw Philox4x32-10 words of cuRAND's device generator for a
// list of counters, to pin the oracle's generator against a library.
//
// After curand_init(seed, subsequence, offset) the generator's counter is
// (offset/4 low, offset/4 high, subsequence low, subsequence high) and its key
// (seed low, seed high); the first curand4 returns Philox4x32-10 of that
// counter.  So counter (c0, c1, c2, c3) under key (k0, k1) is reached with
// seed = k0 | k1 << 32, subsequence = c2 | c3 << 32 and
// offset = 4 (c0 | c1 << 32), which needs c1 < 2^30.
#include <curand_kernel.h>

__global__ void k_words(const uint4* ctr, unsigned long long seed, int n, uint4* out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 c = ctr[i];
    curandStatePhilox4_32_10_t st;
    curand_init(seed, (unsigned long long)c.z | ((unsigned long long)c.w << 32),
                4ull * ((unsigned long long)c.x | ((unsigned long long)c.y << 32)), &st);
    out[i] = curand4(&st);
}

extern "C" int curand_philox_words(const unsigned* ctr, unsigned long long seed, int n, unsigned* out)
{
    uint4 *d_c = nullptr, *d_o = nullptr;
    cudaError_t e = cudaMalloc(&d_c, n * sizeof(uint4));
    if (e == cudaSuccess) e = cudaMalloc(&d_o, n * sizeof(uint4));
    if (e == cudaSuccess) e = cudaMemcpy(d_c, ctr, n * sizeof(uint4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_words<<<(n + 127) / 128, 128>>>(d_c, seed, n, d_o);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, d_o, n * sizeof(uint4), cudaMemcpyDeviceToHost);
    cudaFree(d_c);
    cudaFree(d_o);
    return (int)e;
}
