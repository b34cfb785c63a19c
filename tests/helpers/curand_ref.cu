// Test helper: draws from cuRAND's device Philox4_32_10 generator (library
// code) so the library's own Philox can be compared with it.
#include <cstdint>
#include <curand_kernel.h>

__global__ void k_curand_philox(unsigned long long seed, const unsigned long long* subseq,
                                const unsigned long long* offset, int n, uint32_t* out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    curandStatePhilox4_32_10_t s;
    curand_init(seed, subseq[i], offset[i], &s);
    uint4 r = curand4(&s);
    out[4 * i] = r.x;
    out[4 * i + 1] = r.y;
    out[4 * i + 2] = r.z;
    out[4 * i + 3] = r.w;
}

extern "C" int curand_ref_philox(unsigned long long seed, const unsigned long long* d_subseq,
                                 const unsigned long long* d_offset, int n, uint32_t* d_out)
{
    if (n <= 0) return 0;
    k_curand_philox<<<(n + 127) / 128, 128>>>(seed, d_subseq, d_offset, n, d_out);
    return cudaDeviceSynchronize() == cudaSuccess ? 0 : 1;
}
