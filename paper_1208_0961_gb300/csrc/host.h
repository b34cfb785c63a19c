// Host-side helpers shared by the single-simulation and the batch C ABI:
// error reporting, parameter checks, arena allocation, state settling and the
// CUDA-graph replay of a step.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/cuba.h"
#include "engine.cuh"

namespace cuba {
namespace host {

extern thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);

#define CUDA_TRY(call, what)                                          \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return ::cuba::host::cuda_fail(e_, what); \
    } while (0)

// Validate parameters (Sec. 2, Sec. 5) and fill the device descriptor.
int make_desc(const cuba_params* p, SimDesc* S);

template <typename P>
int dalloc(P** ptr, size_t bytes, const char* what)
{
    *ptr = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc((void**)ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(CUBA_ERR_OOM, "cudaMalloc %s (%zu bytes): %s", what, bytes, cudaGetErrorString(e));
    }
    return CUBA_OK;
}

int arena_alloc(Arena& A, int precision, uint32_t pcap, uint32_t ccap, int simcap);
void arena_free(Arena& A);
int enqueue_step(Arena& A, cudaStream_t st);
int split_counts(int64_t n, const cuba_region* R, int nreg, std::vector<int64_t>& counts);
int sample_regions(Arena& A, int sim_index, const SimDesc& S, int64_t n, const cuba_region* regions, int n_regions,
                   const double* L, cudaStream_t st);
int settle_arena(Arena& A, cudaStream_t st, int* realloc);
int read_kernel_errors(Arena& A);
int autotune_arena(Arena& A, int n_steps, cudaStream_t st, int32_t* chosen, double* ms);
int set_small_max(Arena& A, int32_t v);
int set_launch_shape(Arena& A, const cuba_launch_shape* shape);
void get_launch_shape(const Arena& A, cuba_launch_shape* shape);
int autotune_shape(Arena& A, int n_steps, cudaStream_t st, cuba_launch_shape* chosen, double* ms);
// Record the descriptor table's key and acceptance modes for the pair
// kernels (after every upload).
void set_key_param(Arena& A, const SimDesc* table, int n);

// Captured step graphs (one per ping-pong buffer) and what they were
// captured for.
struct StepGraphs {
    cudaGraphExec_t g[2] = {nullptr, nullptr};
    cudaStream_t capture = nullptr;
    uint32_t np = 0, ncells = 0, small_max = 0;
    int one_key = 0, modes = 0;
    uint32_t tile_nb = 0, small_nb = 0;
    uint32_t key0 = 0, key1 = 0;
    const void* acc = nullptr;
    int trace = 0, nsims = 0;
    void drop();
    int run(Arena& A, int n, cudaStream_t st);
    ~StepGraphs();
};

}  // namespace host
}  // namespace cuba
