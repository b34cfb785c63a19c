// Device-side data structures and kernel launchers of the test-particle step.
//
// Several independent simulations can share one arena: simulation s owns the
// particles [p_off, p_off + np) and the global cells [cell_off, cell_off +
// ncells).  Global cell keys are cell_off + local key, so one stable sort of
// the whole arena by global key keeps every simulation inside its own range.
// A single simulation is an arena with one entry.
#pragma once
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>
#include <vector>

#include "philox.cuh"

namespace cuba {

struct SimDesc {
    double L[3];      // box edges, fm
    double dx[3];     // cell edges L / n, fm
    float Lf[3];      // FP32 copies (rounded once)
    float dxf[3];
    double rdx[3];    // RN(1 / dx) and RN(1 / dxf): the fast path of the cell coordinate
    float rdxf[3];
    int32_t n[3];     // cells per axis
    uint32_t ncells;  // n0 n1 n2
    uint32_t cell_off;
    uint32_t p_off;
    uint32_t np;
    uint32_t step;    // index of the next step (first Philox counter word)
    double dt;
    float dtf;
    float Cf;         // FP32 copy of C
    double C;         // sigma dt / (n_test V_cell): P22 = C v_rel
    double norm;      // n_test V_cell: T^00 = sum E / norm
    uint32_t key0, key1;
    uint32_t thr8;    // top byte above thr8 rejects a pair outright; 256 = never
    uint32_t thr16;   // top 16 bits above thr16 reject a pair; 65536 = never
    float gamma_fp64; // FP32 path: CM boosts with gamma above this use FP64
    uint32_t stat_slot; // row of the counters array (stable while the simulation lives)
    // skip-ahead acceptance (skip = 1): P_max = 2.0001 C as a 0.64 fixed-point
    // fraction and rounded to double and float; skipQ[b] = (1 - P_max)^(2^b)
    // in 0.64 fixed point, b = 0 .. 32
    uint32_t skip;
    float pmaxf;
    uint64_t pfix;
    double pmax;
    uint64_t skipQ[33];
    // adaptive time step (kappa > 0): dt_max caps it; sigma, n_test and V
    // enter the rule; time is the sum of the steps taken
    double kappa;
    double dt_max;
    double sigma, n_test, V;
    double time;
    // particle mass (m2 = m^2, m2f its FP32 copy) and the screening mass of
    // the forward-peaked angular distribution (0: isotropic)
    double mass, m2, mu;
    float m2f;
};

// C, its FP32 copy, the byte thresholds and the skip-ahead tables of a
// descriptor from its dt (host and device: the same IEEE operations).
__host__ __device__ inline void derive_step_constants(SimDesc& S)
{
    S.dtf = (float)S.dt;
    S.C = (S.sigma * S.dt) / (S.n_test * S.V);
    S.Cf = (float)S.C;
    // a top byte above thr8 proves u >= (thr8 + 1) / 256 > 2.0001 C >= P22
    const double pb = 2.0001 * S.C;
    S.thr8 = (pb >= 0.5) ? 256u : (uint32_t)floor(pb * 256.0);
    S.thr16 = (pb >= 1.0) ? 65536u : (uint32_t)floor(pb * 65536.0);
    S.pfix = 0;
    S.pmax = 0.0;
    S.pmaxf = 0.f;
    if (S.skip && S.C > 0.0 && pb < 1.0) {
        // P_fix = floor(2.0001 C 2^64) >= 1; q = 1 - P_max; Q[b] = q^(2^b)
        // by truncated 0.64 fixed-point squaring
        uint64_t P = (uint64_t)(pb * 18446744073709551616.0);
        if (P == 0) P = 1;
        S.pfix = P;
        S.pmax = (double)P * 0x1p-64;
        S.pmaxf = (float)S.pmax;
        S.skipQ[0] = (uint64_t)0 - P;
        for (int b = 1; b <= 32; ++b) {
#ifdef __CUDA_ARCH__
            S.skipQ[b] = __umul64hi(S.skipQ[b - 1], S.skipQ[b - 1]);
#else
            S.skipQ[b] = (uint64_t)(((unsigned __int128)S.skipQ[b - 1] * S.skipQ[b - 1]) >> 64);
#endif
        }
    }
}

// Per-simulation counters (unsigned long long for atomics).
enum StatIdx {
    kStatSteps = 0,
    kStatPairTests,
    kStatAccepted,
    kStatExecuted,
    kStatReflections,
    kStatFp64Boosts,
    kStatOverflow,
    kStatCandidates,  // skip-ahead candidates
    kStatCount = 8
};

// Error bits set by kernels.
constexpr uint32_t kErrAccOverflow = 1u;   // accepted list ran out of room
constexpr uint32_t kErrCapacity = 2u;      // list capacity of a step exceeds the allocation
constexpr uint32_t kErrMove = 4u;          // a particle moved more than one cell along an axis

// Radix sort geometry: 256 threads x 16 keys per tile.  11-bit digits for the
// sort inside a step and the settling sort of a new state (one pass up to 2048
// cells, two up to 2^22); 8-bit digits only for the allocation-free binning of
// caller buffers (cuba_bin_noalloc), whose fixed scratch holds 256-bin
// histograms.
constexpr int kRadixBits = 8;
constexpr int kRadixBins = 1 << kRadixBits;
constexpr int kBinBits = 11;
constexpr int kBinBins = 1 << kBinBits;
constexpr int kBinChunks = 512;   // chunks of tiles of the digit-major histogram scan
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;

// Scan geometry: 256 threads x 8 items per block.
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// Pair tile: one warp per item of 32 rows of one cell.
constexpr int kPairRows = 32;
constexpr int kPairThreads = 256;
// Launch shape of the pair kernels: Philox blocks a lane draws per loop
// iteration (tile: 8, 4 or 2, warp-per-small-cell: 2 or 1; chosen at run
// time, by the autotuner) and the register budget.  With one simulation the
// round keys are kernel parameters (constant-bank operands): four blocks run
// uncapped (94 registers in FP32, two blocks of 256 per SM: measured faster
// than 80 registers and three blocks, or 64 and four), eight capped at two
// blocks of 256 per SM (122 registers in FP32).  With several simulations
// each warp holds its cell's round keys in registers, capped at 128 (four or
// eight blocks) or 80 (two).
template <bool kOneKey, int NB>
struct PairShape {
    static constexpr int min_blocks = kOneKey ? (NB >= 8 ? 2 : 1) : (NB >= 4 ? 2 : 3);  // resident blocks per SM
};

// Resolve: per-cell accepted lists up to this size are sorted in shared memory.
constexpr int kResolveThreads = 256;
constexpr int kResolveSmemPairs = 4096;
constexpr int kResolveBitmapWords = 4096;   // cells up to 131072 particles

struct Uint2Add {
    __host__ __device__ uint2 operator()(uint2 a, uint2 b) const { return make_uint2(a.x + b.x, a.y + b.y); }
};

// Locate the simulation that owns global particle g / global cell c.
__device__ __forceinline__ int sim_of_particle(const SimDesc* sims, int nsims, uint32_t g)
{
    int lo = 0, hi = nsims - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (sims[mid].p_off <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int sim_of_cell(const SimDesc* sims, int nsims, uint32_t c)
{
    int lo = 0, hi = nsims - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (sims[mid].cell_off <= c) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Device buffers of one arena.
struct Arena {
    int precision = 1;          // 0 FP32, 1 FP64
    uint32_t pcap = 0, ccap = 0;
    uint32_t np = 0, ncells = 0; // current totals
    int nsims = 0, simcap = 0;
    void* st[2] = {nullptr, nullptr};   // SoA state ping-pong, 6 * pcap elements
    int cur = 0;
    int sorted_buf = 0;                 // which key/idx buffer holds the last sort's result
    uint32_t* key[2] = {nullptr, nullptr};
    uint32_t* idx[2] = {nullptr, nullptr};
    uint32_t* cell_start = nullptr;     // ccap + 1
    uint2* cell_work = nullptr;         // ccap + 1: (pair items, list capacity) -> scanned
    uint32_t* skip_work = nullptr;      // ccap + 1: skip-ahead row blocks per cell -> scanned
    uint32_t* acc_count = nullptr;      // ccap
    unsigned long long* acc = nullptr;  // accepted (i << 32 | j), per-cell segments
    uint64_t acc_capacity = 0;
    // neighbour-move sort: per-direction counts / in-cell offsets (27 rows of
    // nbr_cap cells), the new cell_start; allocated for arenas of more than
    // 2048 cells; nbr_ok: every simulation's dt (or its cap) lies below 0.98
    // of the cell edge on each axis with more than one cell
    uint32_t* nbr_rel = nullptr;
    uint32_t* nbr_cs = nullptr;
    uint32_t nbr_cap = 0;
    int nbr_ok = 0;
    uint4* surv = nullptr;              // survivors of both random-byte filters, counters[3] of them
    uint32_t surv_cap = 0;
    uint32_t* radix_hist = nullptr;     // digit histograms and their scan, 2 kBinBins * tiles
    uint32_t radix_hist_cap = 0;
    void* scan_tmp = nullptr;           // scan partial sums
    size_t scan_tmp_bytes = 0;
    uint32_t* counters = nullptr;       // [0] pair work counter, [1] error bits, [2] active cells, [3] survivors
    uint32_t* active = nullptr;         // ccap: cells with at least one accepted pair
    uint32_t* used_bits = nullptr;      // pcap / 32 + 1: greedy bitmap for cells too big for smem
    unsigned long long* stats = nullptr;  // simcap * kStatCount
    SimDesc* d_sims = nullptr;
    // tracing
    int trace = 0;
    uint32_t* trace_keys = nullptr;     // pcap
    // cells with 2 <= n <= small_max take the warp-per-cell pair and resolve
    // kernels (0: every cell takes the row-block path); at most 1024
    uint32_t small_max = 32;
    // Philox blocks per lane and loop iteration of the pair kernels
    uint32_t tile_nb = 4, small_nb = 2;
    // one simulation: its Philox round keys, passed to the pair kernels as a
    // parameter (set whenever the descriptor table is uploaded)
    int one_key = 0;
    PhiloxKey key_sched = {};
    // which acceptance modes the resident simulations use; any adaptive dt
    int any_all_pairs = 1, any_skip = 0, any_adapt = 0;
    // device memory: every buffer of the arena (and of the object that owns
    // it) comes from mem_alloc — cudaMalloc when none was given — and is
    // recorded in mem_blocks so that it goes back through mem_free
    void* (*mem_alloc)(size_t, void*) = nullptr;
    void (*mem_free)(void*, size_t, void*) = nullptr;
    void* mem_ctx = nullptr;
    struct Block {
        void* ptr;
        size_t bytes;
    };
    std::vector<Block> mem_blocks;
};

// ---- launchers (kernels_sort.cu) ----
int launch_init_thermal(const Arena& A, int sim, const SimDesc& S, const double* d_regions, int nreg,
                        const uint64_t* d_region_first, cudaStream_t st);
int launch_init_hotspot(const Arena& A, const SimDesc& S, double T0, double dT, double width, cudaStream_t st);
int launch_settle_bin(Arena& A, cudaStream_t st);   // present positions -> keys, sorted state, cell_start
int launch_fill_u32(uint32_t* p, uint32_t n, uint32_t v, cudaStream_t st);
int launch_add_u32(uint32_t* p, uint32_t n, uint32_t v, cudaStream_t st);
int scan_u32(uint32_t* data, size_t n, void* tmp, size_t tmp_bytes, cudaStream_t st);

// ---- launchers (kernels_bin.cu) ----
// A1-A4 of a step: streams st[cur] into the sorted st[cur ^ 1] (cur flips),
// cell_start and, when tracing, the keys and the permutation.  after_stream
// (may be null) is recorded once the streaming pass is done.
int launch_step_bin(Arena& A, cudaStream_t st, cudaEvent_t after_stream);
// A1-A4 as a neighbour-move sort (many small cells, dt below the cell edge):
// used instead of launch_step_bin when nbr_path(A)
bool nbr_path(const Arena& A);
int launch_step_nbr(Arena& A, cudaStream_t st, cudaEvent_t after_stream);
int bin_kernels_init();
size_t bin_scan_bytes();   // scratch the histogram scan needs in scan_tmp
int launch_cell_prep(const Arena& A, cudaStream_t st, int count_pairs = 1);
int launch_observables(const Arena& A, int sim, double* T00, double* T0x, int32_t* counts, cudaStream_t st);
int launch_totals(const Arena& A, int sim, double* d_out4, cudaStream_t st);
int launch_advance(const Arena& A, cudaStream_t st);
int launch_adapt_dt(const Arena& A, cudaStream_t st);   // adaptive dt of the coming step
int launch_philox(const uint32_t* ctr, int64_t n, uint64_t key, uint32_t* out, cudaStream_t st);
int launch_bin_raw(const SimDesc& S, int precision, const void* xyz, uint32_t n, uint32_t* key_a, uint32_t* key_b,
                   uint32_t* idx_a, uint32_t* idx_b, uint32_t* hist, void* partials, size_t partial_bytes,
                   uint32_t* perm, uint32_t* cell_start, cudaStream_t st);

// ---- launchers (kernels_pairs.cu) ----
int launch_pair_tile(const Arena& A, cudaStream_t st);
int launch_resolve(const Arena& A, cudaStream_t st);
int kernels_init();   // attributes and launch shapes; call before any capture
int launch_kinematics_check(const SimDesc& S, const float* pin, int64_t npairs, float* pout, int32_t* used64,
                            cudaStream_t st);

// number of radix passes of `digit_bits` bits for keys below ncells
inline int radix_passes(uint32_t ncells, int digit_bits = kRadixBits)
{
    int bits = 0;
    while (bits < 32 && (ncells - 1) >> bits) ++bits;
    return (bits + digit_bits - 1) / digit_bits;
}

int sm_count();

}  // namespace cuba
