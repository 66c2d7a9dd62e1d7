// Test helper: runs cuRAND's device Philox4x32-10 (curand_Philox4x32_10 from
// curand_kernel.h) on given (counter, key) pairs, as the reference the
// engine's and the oracle's Philox are compared with.
#include <cstddef>
#include <curand_kernel.h>

__global__ void k_curand_philox(const uint4* ctr, const uint2* key, uint4* out, size_t n) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = curand_Philox4x32_10(ctr[i], key[i]);
}

extern "C" int curand_philox_batch(const unsigned* ctr, const unsigned* key, unsigned* out, size_t n) {
    uint4 *dc = nullptr, *dout = nullptr;
    uint2* dk = nullptr;
    cudaError_t e = cudaMalloc(&dc, n * 16 + 16);
    if (e == cudaSuccess) e = cudaMalloc(&dk, n * 8 + 8);
    if (e == cudaSuccess) e = cudaMalloc(&dout, n * 16 + 16);
    if (e == cudaSuccess) e = cudaMemcpy(dc, ctr, n * 16, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dk, key, n * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_curand_philox<<<(unsigned)((n + 255) / 256), 256>>>(dc, dk, dout, n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, n * 16, cudaMemcpyDeviceToHost);
    cudaFree(dc);
    cudaFree(dk);
    cudaFree(dout);
    return (int)e;
}
