// cuRAND's Philox4x32-10 (device API, header curand_philox4x32_x.h) for the
// generator cross-check in tests/test_gpu_parity.py.  Built by that test.
#include <curand_philox4x32_x.h>
#include <stdint.h>

__global__ void k_ref(uint2 key, const uint4 *ctr, uint4 *out, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = curand_Philox4x32_10(ctr[i], key);
}

extern "C" int curand_philox_ref(uint32_t k0, uint32_t k1, const uint32_t *ctr, int n,
                                 uint32_t *out)
{
    uint4 *dc = nullptr, *dout = nullptr;
    if (cudaMalloc(&dc, sizeof(uint4) * n) != cudaSuccess) return 1;
    if (cudaMalloc(&dout, sizeof(uint4) * n) != cudaSuccess) return 1;
    cudaMemcpy(dc, ctr, sizeof(uint4) * n, cudaMemcpyHostToDevice);
    k_ref<<<(n + 255) / 256, 256>>>(make_uint2(k0, k1), dc, dout, n);
    cudaError_t e = cudaMemcpy(out, dout, sizeof(uint4) * n, cudaMemcpyDeviceToHost);
    cudaFree(dc);
    cudaFree(dout);
    return e == cudaSuccess ? 0 : 2;
}
