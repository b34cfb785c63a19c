// Throughput probe of Philox4x32-10 on this GPU (not part of the library).
//
// Every thread draws 8192 blocks along one row (counters (step, 7, tid, g)),
// as the pair tile does, with and without the byte test of the pair tile.
// Prints blocks/s and pair tests/s (16 pairs per block).  Combined with ncu's
// pipe counters it shows which pipe bounds Philox: its 32x32->64 multiplies.
//
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o philox_rate \
//        paper_1208_0961_gb300/csrc/probes/philox_rate.cu && ./philox_rate
#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>

#include "../philox.cuh"

using namespace cuba;

__device__ __forceinline__ uint32_t any_zero_byte(uint4 r)
{
    const uint32_t t = 0x01010101u;
    return (((r.x - t) & ~r.x) | ((r.y - t) & ~r.y) | ((r.z - t) & ~r.z) | ((r.w - t) & ~r.w)) & 0x80808080u;
}

template <int TEST>
__global__ void __launch_bounds__(256) k_rate(uint32_t step, uint32_t nblk, uint32_t* out, uint32_t k0, uint32_t k1)
{
    const PhiloxKey K = philox_schedule(k0, k1);
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0;
    PhiloxRow R;
    R.init(step, 7u, i, K);
    for (uint32_t g = 0; g < nblk; g += 2) {
        const uint4 a = R.block(g, K), b = R.block(g + 1, K);
        if (TEST) {
            acc += __popc(__ballot_sync(0xffffffffu, (any_zero_byte(a) | any_zero_byte(b)) != 0u));
        } else {
            acc ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w;
        }
    }
    out[i] = acc;
}

template <int TEST>
static void run(const char* name, int sms, uint32_t* d)
{
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_rate<TEST>, 256, 0);
    const int grid = sms * per;
    const uint32_t nblk = 8192;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_rate<TEST><<<grid, 256>>>(1, 256, d, 3, 4);
    cudaEventRecord(e0);
    for (int rep = 0; rep < 3; ++rep) k_rate<TEST><<<grid, 256>>>(rep, nblk, d, 3, 4);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double blocks = 3.0 * grid * 256.0 * nblk;
    printf("%-22s blocks/SM=%d  %.3e blocks/s  %.3e pair tests/s\n", name, per, blocks / (ms * 1e-3),
           16.0 * blocks / (ms * 1e-3));
}

int main()
{
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    uint32_t* d = nullptr;
    if (cudaMalloc(&d, (size_t)sms * 8 * 256 * 4) != cudaSuccess) return 1;
    run<0>("philox only", sms, d);
    run<1>("philox + byte test", sms, d);
    cudaError_t e = cudaDeviceSynchronize();
    printf("status %s\n", cudaGetErrorString(e));
    cudaFree(d);
    return e != cudaSuccess;
}
