// A1-A4 of a step: free streaming with wall reflection, cell keys and the
// stable counting sort by cell, in radix passes over 11-bit digits (one pass
// up to 2048 cells, two up to 2^22).
//
// The state is sorted by cell at the start of a step.  The first kernel
// streams every particle in registers (A1, A2), computes its new cell key
// (A3) and the tile histogram of the key's first digit, writing only the key
// (FP32) or the key and the streamed state in place (FP64).  In FP32 the
// streamed state is recomputed, from the unmodified old state with the same
// IEEE operations and so to the same bits, by the kernel that writes each
// particle into its sorted slot (A4):
//   one pass:  the ranking kernel itself (it reads the old state in order and
//              writes runs of sorted slots, since particles move little);
//              cell_start is the scanned digit histogram;
//   two passes: (key, index) pairs are permuted by both digits, then a gather
//              reads the old state through the permutation, which is nearly
//              monotone, and derives cell_start from the sorted keys.
//
// Digit histograms are stored tile-major (hist[tile][digit]) so that every
// kernel touches them with coalesced accesses; the digit-major exclusive scan
// over them runs in three kernels over chunks of tiles.
//
// Stability: tile t covers elements [4096 t, 4096 (t + 1)); warp w of a tile
// owns the 512 elements from 512 w, processed 32 at a time in order; ranks
// follow (tile, warp, round, lane), which is index order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "engine.cuh"
#include "fp.cuh"
#include "stream.cuh"

namespace cuba {

constexpr int kWarpsPerTile = kSortThreads / 32;
// FP64 streaming is bound by the FP64 divisions and square root (a small
// fraction of the FP32 rate on this GPU), so in FP64 the first kernel writes
// the streamed state back in place and the sorted write copies it instead of
// streaming again; in FP32 re-streaming is cheaper than that extra write.
template <typename T> struct StreamInPlace { static constexpr bool value = sizeof(T) == 8; };
// kStream = false: the same kernels bin a state as it is (the settling sort
// of a new state): no streaming, the sorted write copies.
constexpr int kDigitsPerThread = kBinBins / kSortThreads;
#ifndef CUBA_BIN_MIN_BLOCKS
#define CUBA_BIN_MIN_BLOCKS 4   // resident ranking blocks per SM the register budget targets
#endif

template <typename T>
__device__ __forceinline__ void load_particle(const T* __restrict__ st, uint32_t pcap, uint32_t g, T pos[3], T mom[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        pos[a] = st[(size_t)a * pcap + g];
        mom[a] = st[(size_t)(3 + a) * pcap + g];
    }
}

template <typename T>
__device__ __forceinline__ void store_particle(T* __restrict__ st, uint32_t pcap, uint32_t p, const T pos[3],
                                               const T mom[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        st[(size_t)a * pcap + p] = pos[a];
        st[(size_t)(3 + a) * pcap + p] = mom[a];
    }
}

// Write the tile histogram h (shared) to row blockIdx.x of hist.
__device__ __forceinline__ void store_tile_hist(const uint32_t* h, uint32_t* __restrict__ hist)
{
    uint32_t* row = hist + (size_t)blockIdx.x * kBinBins;
#pragma unroll
    for (int j = 0; j < kDigitsPerThread; ++j) row[threadIdx.x + j * kSortThreads] = h[threadIdx.x + j * kSortThreads];
}

// Pass 0: stream, key, digit histogram of the tile.  The particles of a warp
// are taken four rounds at a time so that their loads overlap.
template <typename T, bool kStream, bool kOne>
__global__ void __launch_bounds__(kSortThreads) k_stream_hist(const SimDesc* __restrict__ sims, int nsims,
                                                              T* __restrict__ st, uint32_t pcap, uint32_t n,
                                                              uint32_t* __restrict__ keys_out, int shift,
                                                              uint32_t* __restrict__ hist,
                                                              unsigned long long* __restrict__ stats)
{
    __shared__ uint32_t h[kBinBins];
    for (int d = threadIdx.x; d < kBinBins; d += blockDim.x) h[d] = 0;
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t base = blockIdx.x * kSortTile + w * (32 * kSortItems);
    uint32_t cur_slot = 0xFFFFFFFFu;
    uint32_t nref = 0;
    SimDesc Sl;  // one simulation: the streaming's descriptor fields, read once
    if (kOne) copy_stream_fields(Sl, sims[0]);
#pragma unroll 4
    for (int r = 0; r < kSortItems; ++r) {
        const uint32_t i = base + r * 32 + lane;
        const bool ok = i < n;
        uint32_t d = 0xFFFFFFFFu;
        if (ok) {
            const SimDesc& S = kOne ? Sl : sims[sim_of_particle(sims, nsims, i)];
            T pos[3], mom[3];
            load_particle<T>(st, pcap, i, pos, mom);
            const int nr = kStream ? stream_one<T>(S, pos, mom) : 0;
            if (kStream && StreamInPlace<T>::value) store_particle<T>(st, pcap, i, pos, mom);
            if (nr) {
                if (S.stat_slot != cur_slot) {
                    if (nref) atomicAdd(&stats[cur_slot * kStatCount + kStatReflections], (unsigned long long)nref);
                    nref = 0;
                    cur_slot = S.stat_slot;
                }
                nref += (uint32_t)nr;
            }
            const uint32_t key = S.cell_off + cell_key<T>(S, pos);
            keys_out[i] = key;
            d = (key >> shift) & (kBinBins - 1);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (ok && lane == __ffs(peers) - 1) atomicAdd(&h[d], (uint32_t)__popc(peers));
    }
    // reflections: one atomic per warp and simulation (a thread reflects at
    // most 3 kSortItems times, so the warp sum fits 32 bits)
    const unsigned peers = __match_any_sync(0xffffffffu, cur_slot);
    const unsigned sum = __reduce_add_sync(peers, nref);
    if (lane == __ffs(peers) - 1 && cur_slot != 0xFFFFFFFFu && sum)
        atomicAdd(&stats[cur_slot * kStatCount + kStatReflections], (unsigned long long)sum);
    __syncthreads();
    store_tile_hist(h, hist);
}

// Streaming and the cell key, one particle per thread, the streamed state
// written back in place: used in FP64 when the arena has fewer 4096-particle
// tiles than SMs, where the histogram kernel's 16 particles per thread would
// run their FP64 divisions and square roots one after another on a few SMs.
template <typename T>
__global__ void __launch_bounds__(256) k_stream_inplace(const SimDesc* __restrict__ sims, int nsims,
                                                        T* __restrict__ st, uint32_t pcap, uint32_t n,
                                                        uint32_t* __restrict__ keys_out,
                                                        unsigned long long* __restrict__ stats)
{
    const uint32_t lane = threadIdx.x & 31;
    uint32_t cur_slot = 0xFFFFFFFFu, nref = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const SimDesc& S = sims[sim_of_particle(sims, nsims, i)];
        T pos[3], mom[3];
        load_particle<T>(st, pcap, i, pos, mom);
        const int nr = stream_one<T>(S, pos, mom);
        store_particle<T>(st, pcap, i, pos, mom);
        keys_out[i] = S.cell_off + cell_key<T>(S, pos);
        if (nr) {
            if (S.stat_slot != cur_slot) {
                if (nref) atomicAdd(&stats[cur_slot * kStatCount + kStatReflections], (unsigned long long)nref);
                nref = 0;
                cur_slot = S.stat_slot;
            }
            nref += (uint32_t)nr;
        }
    }
    const unsigned peers = __match_any_sync(0xffffffffu, cur_slot);
    const unsigned sum = __reduce_add_sync(peers, nref);
    if (lane == __ffs(peers) - 1 && cur_slot != 0xFFFFFFFFu && sum)
        atomicAdd(&stats[cur_slot * kStatCount + kStatReflections], (unsigned long long)sum);
}

// Histogram of a later digit.
__global__ void __launch_bounds__(kSortThreads) k_bin_hist(const uint32_t* __restrict__ keys, uint32_t n, int shift,
                                                           uint32_t* __restrict__ hist)
{
    __shared__ uint32_t h[kBinBins];
    for (int d = threadIdx.x; d < kBinBins; d += blockDim.x) h[d] = 0;
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t base = blockIdx.x * kSortTile + w * (32 * kSortItems);
#pragma unroll 4
    for (int r = 0; r < kSortItems; ++r) {
        const uint32_t i = base + r * 32 + lane;
        const bool ok = i < n;
        const uint32_t d = ok ? (keys[i] >> shift) & (kBinBins - 1) : 0xFFFFFFFFu;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (ok && lane == __ffs(peers) - 1) atomicAdd(&h[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    store_tile_hist(h, hist);
}

// ---------------------------------------------------------------------------
// Digit-major exclusive scan of the tile-major histograms:
// off[t][d] = sum_{d' < d} total[d'] + sum_{t' < t} hist[t'][d].
// Chunk b covers tiles [b ct, min((b + 1) ct, ntiles)).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSortThreads) k_col_reduce(const uint32_t* __restrict__ hist, uint32_t ntiles,
                                                             uint32_t ct, uint32_t* __restrict__ csum)
{
    const uint32_t t0 = blockIdx.x * ct;
    const uint32_t t1 = min(t0 + ct, ntiles);
    uint32_t acc[kDigitsPerThread] = {};
    for (uint32_t t = t0; t < t1; ++t) {
        const uint32_t* row = hist + (size_t)t * kBinBins;
#pragma unroll
        for (int j = 0; j < kDigitsPerThread; ++j) acc[j] += row[threadIdx.x + j * kSortThreads];
    }
#pragma unroll
    for (int j = 0; j < kDigitsPerThread; ++j)
        csum[(size_t)blockIdx.x * kBinBins + threadIdx.x + j * kSortThreads] = acc[j];
}

// Per digit, the exclusive prefix of the chunk sums (coff) and the digit
// total (dtot).  Block b owns digits 32 b + lane; warp w a contiguous range
// of chunks.
__global__ void __launch_bounds__(kSortThreads) k_col_scan(const uint32_t* __restrict__ csum, uint32_t nchunks,
                                                           uint32_t* __restrict__ coff, uint32_t* __restrict__ dtot)
{
    __shared__ uint32_t part[kWarpsPerTile][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t d = blockIdx.x * 32 + lane;
    const uint32_t cw = (nchunks + kWarpsPerTile - 1) / kWarpsPerTile;
    const uint32_t b0 = min(w * cw, nchunks), b1 = min(b0 + cw, nchunks);
    uint32_t s = 0;
#pragma unroll 8
    for (uint32_t b = b0; b < b1; ++b) s += csum[(size_t)b * kBinBins + d];
    part[w][lane] = s;
    __syncthreads();
    uint32_t run = 0, tot = 0;
#pragma unroll
    for (int ww = 0; ww < kWarpsPerTile; ++ww) {
        const uint32_t v = part[ww][lane];
        run += ww < w ? v : 0u;
        tot += v;
    }
    if (w == 0) dtot[d] = tot;
#pragma unroll 8
    for (uint32_t b = b0; b < b1; ++b) {
        coff[(size_t)b * kBinBins + d] = run;
        run += csum[(size_t)b * kBinBins + d];
    }
}

// off rows of chunk b: the digit bases (exclusive scan of dtot, done by every
// block), plus the chunk offset, plus the tiles before in the chunk.  With
// cell_start given (one pass: the digit is the whole key) block 0 writes the
// digit bases there, cell_start[ncells] = n.
__global__ void __launch_bounds__(kSortThreads) k_col_apply(const uint32_t* __restrict__ hist,
                                                            uint32_t* __restrict__ off, uint32_t ntiles, uint32_t ct,
                                                            const uint32_t* __restrict__ coff,
                                                            const uint32_t* __restrict__ dtot,
                                                            uint32_t* __restrict__ cell_start, uint32_t ncells,
                                                            uint32_t n)
{
    __shared__ uint32_t s_base[kBinBins];
    __shared__ uint32_t wsum[kWarpsPerTile];
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    // thread tid scans digits [8 tid, 8 tid + 8)
    uint32_t v[kDigitsPerThread], sum = 0;
#pragma unroll
    for (int j = 0; j < kDigitsPerThread; ++j) {
        v[j] = dtot[kDigitsPerThread * tid + j];
        sum += v[j];
    }
    uint32_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    uint32_t base = inc - sum;
    for (int ww = 0; ww < w; ++ww) base += wsum[ww];
#pragma unroll
    for (int j = 0; j < kDigitsPerThread; ++j) {
        s_base[kDigitsPerThread * tid + j] = base;
        base += v[j];
    }
    __syncthreads();
    if (cell_start && blockIdx.x == 0) {
        for (uint32_t d = tid; d < ncells && d < (uint32_t)kBinBins; d += kSortThreads) cell_start[d] = s_base[d];
        if (tid == 0) cell_start[ncells] = n;
    }
    const uint32_t t0 = blockIdx.x * ct;
    const uint32_t t1 = min(t0 + ct, ntiles);
    uint32_t run[kDigitsPerThread];
#pragma unroll
    for (int j = 0; j < kDigitsPerThread; ++j) {
        const int d = tid + j * kSortThreads;
        run[j] = s_base[d] + coff[(size_t)blockIdx.x * kBinBins + d];
    }
    for (uint32_t t = t0; t < t1; ++t) {
#pragma unroll
        for (int j = 0; j < kDigitsPerThread; ++j) {
            const size_t e = (size_t)t * kBinBins + tid + j * kSortThreads;
            off[e] = run[j];
            run[j] += hist[e];
        }
    }
}

// ---------------------------------------------------------------------------
// Ranking
// ---------------------------------------------------------------------------
// Per-tile ranking state in shared memory: for each warp and digit the
// offset of the warp's first element within the tile's elements of that
// digit (16 bits: a tile holds 4096 elements), and the tile's global offset
// of each digit.
struct RankSmem {
    uint16_t wh[kWarpsPerTile][kBinBins];
    uint32_t off[kBinBins];
};

// Fill RankSmem for the keys k of this thread (rounds r = 0 .. kSortItems-1).
__device__ __forceinline__ void tile_prefix(RankSmem& R, const uint32_t k[kSortItems], uint32_t n, int shift,
                                            const uint32_t* __restrict__ off)
{
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int d = lane; d < kBinBins; d += 32) R.wh[w][d] = 0;
    __syncwarp();
    const uint32_t base = blockIdx.x * kSortTile + w * (32 * kSortItems);
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const bool ok = base + r * 32 + lane < n;
        const uint32_t d = ok ? (k[r] >> shift) & (kBinBins - 1) : 0xFFFFFFFFu;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (ok && lane == __ffs(peers) - 1) R.wh[w][d] += (uint16_t)__popc(peers);
        __syncwarp();
    }
    __syncthreads();
    const uint32_t* row = off + (size_t)blockIdx.x * kBinBins;
#pragma unroll
    for (int j = 0; j < kDigitsPerThread; ++j) {
        const int d = threadIdx.x + j * kSortThreads;
        R.off[d] = row[d];
        uint32_t run = 0;
#pragma unroll
        for (int ww = 0; ww < kWarpsPerTile; ++ww) {
            const uint32_t c = R.wh[ww][d];
            R.wh[ww][d] = (uint16_t)run;
            run += c;
        }
    }
    __syncthreads();
}

// Destination of this lane's element of the current round (the rounds of a
// warp must be taken in order); valid only where ok.
__device__ __forceinline__ uint32_t rank_next(RankSmem& R, uint32_t key, bool ok, int shift)
{
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t d = ok ? (key >> shift) & (kBinBins - 1) : 0xFFFFFFFFu;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    uint32_t pos = 0;
    if (ok) pos = R.off[d] + R.wh[w][d] + (uint32_t)__popc(peers & ((1u << lane) - 1u));
    __syncwarp();
    if (ok && lane == __ffs(peers) - 1) R.wh[w][d] += (uint16_t)__popc(peers);
    __syncwarp();
    return pos;
}

// Permute (key, index) by one digit; idx_in null means the identity.
__global__ void __launch_bounds__(kSortThreads, CUBA_BIN_MIN_BLOCKS)
    k_bin_scatter(const uint32_t* __restrict__ key_in, const uint32_t* __restrict__ idx_in,
                  uint32_t* __restrict__ key_out, uint32_t* __restrict__ idx_out, uint32_t n, int shift,
                  const uint32_t* __restrict__ off)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    RankSmem& R = *reinterpret_cast<RankSmem*>(smem_raw);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t base = blockIdx.x * kSortTile + w * (32 * kSortItems);
    uint32_t k[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const uint32_t i = base + r * 32 + lane;
        k[r] = i < n ? key_in[i] : 0xFFFFFFFFu;
    }
    tile_prefix(R, k, n, shift, off);
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const uint32_t i = base + r * 32 + lane;
        const bool ok = i < n;
        const uint32_t p = rank_next(R, k[r], ok, shift);
        if (ok) {
            key_out[p] = k[r];
            idx_out[p] = idx_in ? idx_in[i] : i;
        }
    }
}

// One pass: rank by the (only) digit, re-stream each particle from the old
// state and write it into its sorted slot; perm (tracing only) receives the
// origin of each slot.  The slots of all rounds come first (they need only
// the keys), then the particles are loaded FinalGroup rounds at a time, so
// that their loads are in flight together: four in FP32 under an
// 80-register budget (three blocks per SM; measured 0.229 against 0.251 ms
// per 16 M-particle step with two rounds and four blocks), one in FP64,
// whose second particle would spill under the 64-register budget.
template <typename T> struct FinalGroup { static constexpr int value = sizeof(T) == 8 ? 1 : 4; };
template <typename T> struct FinalBlocks { static constexpr int value = sizeof(T) == 8 ? CUBA_BIN_MIN_BLOCKS : 3; };

template <typename T, bool kStream, bool kOne>
__global__ void __launch_bounds__(kSortThreads, FinalBlocks<T>::value)
    k_bin_final(const SimDesc* __restrict__ sims, int nsims, const uint32_t* __restrict__ key_in,
                const T* __restrict__ st_old, T* __restrict__ st_new, uint32_t pcap, uint32_t n,
                const uint32_t* __restrict__ off, uint32_t* __restrict__ perm)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    RankSmem& R = *reinterpret_cast<RankSmem*>(smem_raw);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t base = blockIdx.x * kSortTile + w * (32 * kSortItems);
    uint32_t k[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const uint32_t i = base + r * 32 + lane;
        k[r] = i < n ? key_in[i] : 0xFFFFFFFFu;
    }
    tile_prefix(R, k, n, 0, off);
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const uint32_t i = base + r * 32 + lane;
        k[r] = rank_next(R, k[r], i < n, 0);   // the key's register now holds the slot
    }
    constexpr int kG = FinalGroup<T>::value;
#pragma unroll
    for (int r0 = 0; r0 < kSortItems; r0 += kG) {
        T x[kG][3], m[kG][3];
#pragma unroll
        for (int g = 0; g < kG; ++g) {
            const uint32_t i = base + (r0 + g) * 32 + lane;
            if (i < n) load_particle<T>(st_old, pcap, i, x[g], m[g]);
        }
#pragma unroll
        for (int g = 0; g < kG; ++g) {
            const uint32_t i = base + (r0 + g) * 32 + lane;
            if (i < n) {
                if (kStream && !StreamInPlace<T>::value)
                    stream_one<T>(sims[kOne ? 0 : sim_of_particle(sims, nsims, i)], x[g], m[g]);
                store_particle<T>(st_new, pcap, k[r0 + g], x[g], m[g]);
                if (perm) perm[k[r0 + g]] = i;
            }
        }
    }
}

// Two passes: sorted slot k takes particle perm[k], re-streamed from the old
// state; cell_start[c] = first sorted slot with key >= c.
template <typename T, bool kStream>
__global__ void __launch_bounds__(256) k_bin_gather(const SimDesc* __restrict__ sims, int nsims,
                                                    const uint32_t* __restrict__ perm,
                                                    const uint32_t* __restrict__ skey, const T* __restrict__ st_old,
                                                    T* __restrict__ st_new, uint32_t pcap, uint32_t np,
                                                    uint32_t* __restrict__ cell_start, uint32_t ncells)
{
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < np; k += stride) {
        const uint32_t g = perm[k];
        const int s = sim_of_particle(sims, nsims, g);
        T x[3], p[3];
        load_particle<T>(st_old, pcap, g, x, p);
        if (kStream && !StreamInPlace<T>::value) stream_one<T>(sims[s], x, p);
        store_particle<T>(st_new, pcap, k, x, p);
        const uint32_t kk = skey[k];
        const int64_t prev = (k == 0) ? -1 : (int64_t)skey[k - 1];
        for (int64_t c = prev + 1; c <= (int64_t)kk; ++c) cell_start[c] = k;
        if (k == np - 1)
            for (int64_t c = (int64_t)kk + 1; c <= (int64_t)ncells; ++c) cell_start[c] = np;
    }
}

// ---------------------------------------------------------------------------
// Launcher
// ---------------------------------------------------------------------------
static const size_t kBinSmem = sizeof(RankSmem);

template <typename T, bool kStream, bool kOne>
static int final_attr()
{
    return cudaFuncSetAttribute(k_bin_final<T, kStream, kOne>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kBinSmem) == cudaSuccess ? 0 : -1;
}

int bin_kernels_init()
{
    if (cudaFuncSetAttribute(k_bin_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBinSmem) != cudaSuccess)
        return -1;
    int rc = final_attr<float, true, true>() | final_attr<float, true, false>() | final_attr<float, false, true>() |
             final_attr<float, false, false>() | final_attr<double, true, true>() | final_attr<double, true, false>() |
             final_attr<double, false, true>() | final_attr<double, false, false>();
    return rc ? -1 : 0;
}

// The stream/key and ranking kernels of one step, one simulation (kOne: its
// descriptor read once, outside the particle loops) or several.
template <typename T, bool kStream>
static void stream_hist(const Arena& A, uint32_t ntiles, uint32_t* hist, cudaStream_t st)
{
    if (A.nsims == 1)
        k_stream_hist<T, kStream, true><<<ntiles, kSortThreads, 0, st>>>(A.d_sims, A.nsims, (T*)A.st[A.cur], A.pcap,
                                                                         A.np, A.key[0], 0, hist, A.stats);
    else
        k_stream_hist<T, kStream, false><<<ntiles, kSortThreads, 0, st>>>(A.d_sims, A.nsims, (T*)A.st[A.cur], A.pcap,
                                                                          A.np, A.key[0], 0, hist, A.stats);
}

template <typename T, bool kStream>
static void bin_final(const Arena& A, uint32_t ntiles, const uint32_t* off, uint32_t* perm, cudaStream_t st)
{
    if (A.nsims == 1)
        k_bin_final<T, kStream, true><<<ntiles, kSortThreads, kBinSmem, st>>>(
            A.d_sims, A.nsims, A.key[0], (const T*)A.st[A.cur], (T*)A.st[A.cur ^ 1], A.pcap, A.np, off, perm);
    else
        k_bin_final<T, kStream, false><<<ntiles, kSortThreads, kBinSmem, st>>>(
            A.d_sims, A.nsims, A.key[0], (const T*)A.st[A.cur], (T*)A.st[A.cur ^ 1], A.pcap, A.np, off, perm);
}

// scan_tmp layout of the histogram scan: csum, coff (kBinChunks rows each), dtot
size_t bin_scan_bytes() { return ((size_t)2 * kBinChunks + 1) * kBinBins * sizeof(uint32_t); }

// Exclusive digit-major scan of hist (ntiles rows) into off; cell_start as
// k_col_apply.
static int col_scan(const Arena& A, const uint32_t* hist, uint32_t* off, uint32_t ntiles, uint32_t* cell_start,
                    cudaStream_t st)
{
    if (A.scan_tmp_bytes < bin_scan_bytes()) return -1;
    const uint32_t ct = (ntiles + kBinChunks - 1) / kBinChunks;
    const uint32_t nchunks = (ntiles + ct - 1) / ct;
    uint32_t* csum = (uint32_t*)A.scan_tmp;
    uint32_t* coff = csum + (size_t)kBinChunks * kBinBins;
    uint32_t* dtot = coff + (size_t)kBinChunks * kBinBins;
    k_col_reduce<<<nchunks, kSortThreads, 0, st>>>(hist, ntiles, ct, csum);
    k_col_scan<<<kBinBins / 32, kSortThreads, 0, st>>>(csum, nchunks, coff, dtot);
    k_col_apply<<<nchunks, kSortThreads, 0, st>>>(hist, off, ntiles, ct, coff, dtot, cell_start, A.ncells, A.np);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

// A1-A4 of one step for every simulation of the arena: the old state in
// st[cur] is left untouched, the new sorted state goes to st[cur ^ 1] (cur
// flips), cell_start is written; with tracing on, the keys before sorting go
// to trace_keys and the permutation to idx[sorted_buf].
template <bool kStream>
static int step_bin(Arena& A, cudaStream_t st, cudaEvent_t after_stream)
{
    const uint32_t n = A.np;
    if (n == 0) {
        // nothing to move: the state buffer stays where it is
        return launch_fill_u32(A.cell_start, A.ncells + 1, 0u, st);
    }
    int passes = radix_passes(A.ncells, kBinBits);
    if (passes < 1) passes = 1;  // one cell: a single pass on a zero digit
    const uint32_t ntiles = (n + kSortTile - 1) / kSortTile;
    if ((size_t)2 * kBinBins * ntiles > A.radix_hist_cap) return -1;
    uint32_t* hist = A.radix_hist;
    uint32_t* off = A.radix_hist + (size_t)kBinBins * ntiles;
    const bool fp64 = A.precision == 1;
    if (fp64 && kStream && ntiles < (uint32_t)sm_count()) {
        // few tiles: stream and key one particle per thread first (FP64
        // writes the streamed state back in place in either case), then the
        // digit histogram of the keys
        k_stream_inplace<double><<<(n + 255) / 256, 256, 0, st>>>(A.d_sims, A.nsims, (double*)A.st[A.cur], A.pcap, n,
                                                                  A.key[0], A.stats);
        k_bin_hist<<<ntiles, kSortThreads, 0, st>>>(A.key[0], n, 0, hist);
    } else if (fp64) {
        stream_hist<double, kStream>(A, ntiles, hist, st);
    } else {
        stream_hist<float, kStream>(A, ntiles, hist, st);
    }
    if (after_stream) cudaEventRecord(after_stream, st);
    if (A.trace) cudaMemcpyAsync(A.trace_keys, A.key[0], sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st);
    if (passes == 1) {
        if (col_scan(A, hist, off, ntiles, A.cell_start, st)) return -1;
        uint32_t* perm = A.trace ? A.idx[1] : nullptr;
        if (fp64)
            bin_final<double, kStream>(A, ntiles, off, perm, st);
        else
            bin_final<float, kStream>(A, ntiles, off, perm, st);
        A.sorted_buf = 1;
    } else {
        int src = 0;
        for (int p = 0; p < passes; ++p) {
            if (p > 0) k_bin_hist<<<ntiles, kSortThreads, 0, st>>>(A.key[src], n, p * kBinBits, hist);
            if (col_scan(A, hist, off, ntiles, nullptr, st)) return -1;
            k_bin_scatter<<<ntiles, kSortThreads, kBinSmem, st>>>(A.key[src], p == 0 ? nullptr : A.idx[src],
                                                                  A.key[src ^ 1], A.idx[src ^ 1], n, p * kBinBits,
                                                                  off);
            src ^= 1;
        }
        const unsigned g = (unsigned)std::min<uint32_t>((n + 255) / 256, (uint32_t)sm_count() * 8);
        if (fp64)
            k_bin_gather<double, kStream><<<g, 256, 0, st>>>(A.d_sims, A.nsims, A.idx[src], A.key[src],
                                                    (const double*)A.st[A.cur], (double*)A.st[A.cur ^ 1], A.pcap, n,
                                                    A.cell_start, A.ncells);
        else
            k_bin_gather<float, kStream><<<g, 256, 0, st>>>(A.d_sims, A.nsims, A.idx[src], A.key[src],
                                                   (const float*)A.st[A.cur], (float*)A.st[A.cur ^ 1], A.pcap, n,
                                                   A.cell_start, A.ncells);
        A.sorted_buf = src;
    }
    A.cur ^= 1;
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

int launch_step_bin(Arena& A, cudaStream_t st, cudaEvent_t after_stream)
{
    return step_bin<true>(A, st, after_stream);
}

// The settling sort of a state as it is (keys of the present positions,
// stable sort, cell_start), with the same kernels.
int launch_settle_bin(Arena& A, cudaStream_t st)
{
    return step_bin<false>(A, st, nullptr);
}

}  // namespace cuba
