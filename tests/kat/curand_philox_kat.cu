// Test-only known-answer source for the Philox4x32-10 generator: the CUDA toolkit's own device
// routine (curand_Philox4x32_10 from curand_kernel.h) evaluated on caller-given counters and keys.
// It is compiled by tests/test_gpu_philox_kat.py into a separate shared library and is not part of
// the product library; it gives the library's and the oracle's Philox an answer that neither of
// them wrote.
#include <cstdint>
#include <cuda_runtime.h>
#include <curand_kernel.h>

namespace {
__global__ void k_kat(uint32_t seed, uint32_t medium, const uint4 *ctr, long long n, uint4 *out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = curand_Philox4x32_10(ctr[i], make_uint2(seed, medium));
}
}  // namespace

// host ctr [n][4] -> host out [n][4]; returns a cudaError_t value (0 on success)
extern "C" int kat_philox(uint32_t seed, uint32_t medium, const uint32_t *ctr, long long n,
                          uint32_t *out)
{
    if (n <= 0) return 0;
    uint4 *dc = nullptr, *dout = nullptr;
    const size_t bytes = sizeof(uint4) * (size_t)n;
    cudaError_t e = cudaMalloc(&dc, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&dout, bytes);
    if (e == cudaSuccess) e = cudaMemcpy(dc, ctr, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        const long long blocks = (n + 255) / 256;
        k_kat<<<(unsigned)blocks, 256>>>(seed, medium, dc, n, dout);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, bytes, cudaMemcpyDeviceToHost);
    cudaFree(dc);
    cudaFree(dout);
    return (int)e;
}
