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

// Device memory of an arena and of the object owning it: from the caller's
// allocator when one was given, else cudaMalloc; every block is recorded and
// returned by arena_dfree or arena_free.
int arena_dalloc_raw(Arena& A, void** ptr, size_t bytes, const char* what);
template <typename P>
int arena_dalloc(Arena& A, P** ptr, size_t bytes, const char* what)
{
    void* p = nullptr;
    int rc = arena_dalloc_raw(A, &p, bytes, what);
    *ptr = static_cast<P*>(p);
    return rc;
}
void arena_dfree(Arena& A, void* ptr);

// Sizes in bytes of the buffers arena_alloc allocates (state and keys and
// permutation counted once per ping-pong copy in total()).
struct ArenaPlan {
    size_t state = 0, keys = 0, perm = 0, cell_start = 0, cell_work = 0, skip_work = 0, acc_count = 0, active = 0;
    size_t radix_hist = 0, scan_tmp = 0, counters = 0, surv = 0, used_bits = 0, nbr_rel = 0, nbr_cs = 0;
    size_t stats = 0, sims = 0;
    uint32_t radix_hist_cap = 0, surv_cap = 0, nbr_cap = 0;
    size_t total() const
    {
        return 2 * state + 2 * keys + 2 * perm + cell_start + cell_work + skip_work + acc_count + active + radix_hist +
               scan_tmp + counters + surv + used_bits + nbr_rel + nbr_cs + stats + sims;
    }
};
ArenaPlan arena_plan(int precision, uint32_t pcap, uint32_t ccap, int simcap);
// Entries of the smallest accepted-pair list settle_arena allocates.
constexpr uint64_t kMinAccEntries = 1ull << 20;
// Observables scratch of a simulation or batch with ccap cells, and the
// totals scratch.
inline size_t obs_scratch_bytes(uint32_t ccap) { return (size_t)ccap * 20 + 64; }
constexpr size_t kTotScratchBytes = 64;
// Bytes an object with this arena allocates at creation plus the smallest
// accepted-pair list.
inline size_t object_bytes(int precision, uint32_t pcap, uint32_t ccap, int simcap)
{
    return arena_plan(precision, pcap, ccap, simcap).total() + obs_scratch_bytes(ccap) + kTotScratchBytes +
           kMinAccEntries * sizeof(unsigned long long);
}

// mem: the caller's allocator, or NULL for cudaMalloc.
int arena_alloc(Arena& A, int precision, uint32_t pcap, uint32_t ccap, int simcap, const cuba_allocator* mem);
void arena_free(Arena& A);
int enqueue_step(Arena& A, cudaStream_t st);
int split_counts(int64_t n, const cuba_region* R, int nreg, std::vector<int64_t>& counts);
int sample_regions(Arena& A, int sim_index, const SimDesc& S, int64_t n, const cuba_region* regions, int n_regions,
                   const double* L, cudaStream_t st);
// member >= 0: only that member's particles are sorted (desc: its
// descriptor); kSettleNoSort: only the list sizing (state already sorted)
constexpr int kSettleNoSort = -2;
int settle_arena(Arena& A, cudaStream_t st, int* realloc, int member = -1, const SimDesc* desc = nullptr);
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
