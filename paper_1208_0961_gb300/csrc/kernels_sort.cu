// Particle-parallel kernels: thermal sampling, the per-cell work preparation of
// the pair step, the FP64 observables and totals (A8), the adaptive time step,
// scans, and the LSD radix sort on 8-bit digits that bins caller buffers
// without allocation (the step's own stream, key and sort kernels are in
// kernels_bin.cu and kernels_nbr.cu).
//
// Bit-reproducibility: the streaming, the key and the sampling positions use
// explicitly rounded IEEE operations (__dadd_rn, __fdiv_rn, ...) in the order
// the method states, so that a CPU evaluation of the same expressions gives
// identical bits.  The library is also compiled without multiply-add
// contraction.
#include <cuda_runtime.h>

#include <cstdint>

#include "engine.cuh"
#include "fp.cuh"
#include "stream.cuh"

namespace cuba {

// ---------------------------------------------------------------------------
// Thermal sampling (generation order; sorted afterwards)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double open01(uint32_t r) { return ((double)r + 0.5) * 0x1p-32; }

// Momentum magnitude of a thermal particle at temperature T.  Massless: the
// Gamma(3, T) variate p0.  Massive (m > 0): the Juttner density
// p^2 exp(-sqrt(p^2 + m^2)/T) by rejection from the massless one: try k draws
// the block (STEP_INIT, g, 0, TAG_MASS | k), proposes q = -T ln(u0 u1 u2) and
// keeps it iff u3 < exp(-(m^2 / (sqrt(q^2 + m^2) + q)) / T); after 64
// rejected tries the last proposal is kept.
__device__ __forceinline__ double sample_pmag(const SimDesc& S, const PhiloxKey& K, double T, uint32_t g, double p0)
{
    if (!(S.mass > 0.0)) return p0;
    const double m2 = S.m2;
    double q = p0;
    for (uint32_t k = 0; k < 64; ++k) {
        const uint4 w = philox4x32_10(make_uint4(kStepInit, g, 0u, kTagMass | k), K);
        q = -T * log(open01(w.x) * open01(w.y) * open01(w.z));
        const double acc = exp(-(m2 / (sqrt(q * q + m2) + q)) / T);
        if (open01(w.w) < acc) break;
    }
    return q;
}

template <typename T>
__global__ void __launch_bounds__(256) k_init_thermal(SimDesc S, T* __restrict__ st, uint32_t pcap,
                                                      const double* __restrict__ regions, int nreg,
                                                      const uint64_t* __restrict__ first)
{
    const PhiloxKey K = philox_schedule(S.key0, S.key1);
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < S.np; g += stride) {
        int r = 0;
        while (r + 1 < nreg && first[r + 1] <= g) ++r;
        const double* R = regions + 7 * r;  // lo[3], hi[3], T
        const uint4 a = philox4x32_10(make_uint4(kStepInit, g, 0u, 0u), K);
        const uint4 b = philox4x32_10(make_uint4(kStepInit, g, 0u, 1u), K);
        const uint32_t aw[3] = {a.x, a.y, a.z};
        double pos[3];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax)
            pos[ax] = __dadd_rn(R[ax], __dmul_rn(open01(aw[ax]), __dsub_rn(R[3 + ax], R[ax])));
        const double E = sample_pmag(S, K, R[6], g, -R[6] * log(open01(a.w) * open01(b.x) * open01(b.y)));
        const double ct = 2.0 * open01(b.z) - 1.0;
        const double stt = sqrt((1.0 - ct) * (1.0 + ct));
        const double phi = 2.0 * 3.141592653589793 * open01(b.w);
        double sp, cp;
        sincos(phi, &sp, &cp);
        const double mom[3] = {E * stt * cp, E * stt * sp, E * ct};
        const uint32_t o = S.p_off + g;
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            st[(size_t)ax * pcap + o] = (T)pos[ax];
            st[(size_t)(3 + ax) * pcap + o] = (T)mom[ax];
        }
    }
}

// Hot-spot state: T(r) = T0 + dT exp(-|r - centre|^2 / (2 w^2)), density
// proportional to T(r)^3 by rejection (try k draws the block
// (STEP_INIT, g, 0, 2 + k): a uniform position and the acceptance variate;
// after 64 rejected tries the last position is kept), momentum from the
// thermal blocks (…, 0) and (…, 1) at the local T(r).
template <typename T>
__global__ void __launch_bounds__(256) k_init_hotspot(SimDesc S, T* __restrict__ st, uint32_t pcap, double T0,
                                                      double dT, double width)
{
    const PhiloxKey K = philox_schedule(S.key0, S.key1);
    const double Tmax = T0 + dT;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < S.np; g += stride) {
        double pos[3] = {0.0, 0.0, 0.0};
        double Tl = T0;
        for (uint32_t k = 0; k < 64; ++k) {
            const uint4 t = philox4x32_10(make_uint4(kStepInit, g, 0u, 2u + k), K);
            const uint32_t tw[3] = {t.x, t.y, t.z};
            double r2 = 0.0;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                pos[a] = __dmul_rn(open01(tw[a]), S.L[a]);
                const double d = __dsub_rn(pos[a], __dmul_rn(0.5, S.L[a]));
                r2 = __dadd_rn(r2, __dmul_rn(d, d));
            }
            Tl = T0 + dT * exp(-r2 / (2.0 * width * width));
            const double ratio = Tl / Tmax;
            if (open01(t.w) < ratio * ratio * ratio) break;
        }
        const uint4 a = philox4x32_10(make_uint4(kStepInit, g, 0u, 0u), K);
        const uint4 b = philox4x32_10(make_uint4(kStepInit, g, 0u, 1u), K);
        const double E = sample_pmag(S, K, Tl, g, -Tl * log(open01(a.w) * open01(b.x) * open01(b.y)));
        const double ct = 2.0 * open01(b.z) - 1.0;
        const double stt = sqrt((1.0 - ct) * (1.0 + ct));
        const double phi = 2.0 * 3.141592653589793 * open01(b.w);
        double sp, cp;
        sincos(phi, &sp, &cp);
        const double mom[3] = {E * stt * cp, E * stt * sp, E * ct};
        const uint32_t o = S.p_off + g;
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            st[(size_t)ax * pcap + o] = (T)pos[ax];
            st[(size_t)(3 + ax) * pcap + o] = (T)mom[ax];
        }
    }
}

// ---------------------------------------------------------------------------
// Device-wide exclusive scan (reduce, scan partials, apply)
// ---------------------------------------------------------------------------
template <typename V, typename Op>
__device__ __forceinline__ V warp_incl_scan(V v, Op op)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        V t;
        if constexpr (sizeof(V) == 8) {
            uint2 u = *reinterpret_cast<uint2*>(&v);
            uint2 w;
            w.x = __shfl_up_sync(0xffffffffu, u.x, o);
            w.y = __shfl_up_sync(0xffffffffu, u.y, o);
            t = *reinterpret_cast<V*>(&w);
        } else {
            t = __shfl_up_sync(0xffffffffu, v, o);
        }
        if (lane >= o) v = op(t, v);
    }
    return v;
}

// Block-wide exclusive scan of kScanThreads values; returns the block total.
template <typename V, typename Op>
__device__ __forceinline__ V block_excl_scan(V v, V zero, Op op, V* excl)
{
    __shared__ V warp_tot[kScanThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    V inc = warp_incl_scan(v, op);
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        V t = (lane < kScanThreads / 32) ? warp_tot[lane] : zero;
        t = warp_incl_scan(t, op);
        if (lane < kScanThreads / 32) warp_tot[lane] = t;
    }
    __syncthreads();
    V base = (w > 0) ? warp_tot[w - 1] : zero;
    V total = warp_tot[kScanThreads / 32 - 1];
    // exclusive within warp
    V ex;
    if constexpr (sizeof(V) == 8) {
        uint2 u = *reinterpret_cast<uint2*>(&inc);
        uint2 q;
        q.x = __shfl_up_sync(0xffffffffu, u.x, 1);
        q.y = __shfl_up_sync(0xffffffffu, u.y, 1);
        ex = *reinterpret_cast<V*>(&q);
    } else {
        ex = __shfl_up_sync(0xffffffffu, inc, 1);
    }
    if (lane == 0) ex = zero;
    *excl = op(base, ex);
    __syncthreads();
    return total;
}

template <typename V, typename Op>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const V* __restrict__ in, size_t n, V* __restrict__ partial, V zero, Op op)
{
    const size_t base = (size_t)blockIdx.x * kScanTile + (size_t)threadIdx.x * kScanItems;
    V acc = zero;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) acc = op(acc, in[base + k]);
    V ex;
    V tot = block_excl_scan(acc, zero, op, &ex);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

template <typename V, typename Op>
__global__ void __launch_bounds__(kScanThreads) k_scan_partials(V* __restrict__ partial, size_t nb, V zero, Op op)
{
    V carry = zero;
    for (size_t off = 0; off < nb; off += kScanTile) {
        const size_t base = off + (size_t)threadIdx.x * kScanItems;
        V vals[kScanItems];
        V acc = zero;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            vals[k] = (base + k < nb) ? partial[base + k] : zero;
            acc = op(acc, vals[k]);
        }
        V ex;
        V tot = block_excl_scan(acc, zero, op, &ex);
        V run = op(carry, ex);
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            if (base + k < nb) partial[base + k] = run;
            run = op(run, vals[k]);
        }
        carry = op(carry, tot);
        __syncthreads();
    }
}

template <typename V, typename Op>
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(V* __restrict__ data, size_t n, const V* __restrict__ partial, V zero, Op op)
{
    const size_t base = (size_t)blockIdx.x * kScanTile + (size_t)threadIdx.x * kScanItems;
    V vals[kScanItems];
    V acc = zero;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        vals[k] = (base + k < n) ? data[base + k] : zero;
        acc = op(acc, vals[k]);
    }
    V ex;
    block_excl_scan(acc, zero, op, &ex);
    V run = op(partial[blockIdx.x], ex);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) data[base + k] = run;
        run = op(run, vals[k]);
    }
}

struct U32Add {
    __host__ __device__ uint32_t operator()(uint32_t a, uint32_t b) const { return a + b; }
};

constexpr size_t kScanOneBlockTiles = 2;

template <typename V, typename Op>
static int exclusive_scan(V* data, size_t n, V zero, Op op, void* tmp, size_t tmp_bytes, cudaStream_t st)
{
    if (n == 0) return 0;
    const size_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb <= kScanOneBlockTiles) {
        // short arrays: one block scans them tile by tile (one launch instead
        // of three)
        k_scan_partials<V, Op><<<1, kScanThreads, 0, st>>>(data, n, zero, op);
        return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
    }
    if (nb * sizeof(V) > tmp_bytes) return -1;
    V* partial = reinterpret_cast<V*>(tmp);
    k_scan_reduce<V, Op><<<(unsigned)nb, kScanThreads, 0, st>>>(data, n, partial, zero, op);
    k_scan_partials<V, Op><<<1, kScanThreads, 0, st>>>(partial, nb, zero, op);
    k_scan_apply<V, Op><<<(unsigned)nb, kScanThreads, 0, st>>>(data, n, partial, zero, op);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

int scan_u32(uint32_t* data, size_t n, void* tmp, size_t tmp_bytes, cudaStream_t st)
{
    return exclusive_scan<uint32_t, U32Add>(data, n, 0u, U32Add(), tmp, tmp_bytes, st);
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort of cell keys on 8-bit digits (binning without
// allocation)
// ---------------------------------------------------------------------------
// Tile t covers keys [t * 4096, (t + 1) * 4096); warp w of a tile owns the
// contiguous 512 keys starting at w * 512, processed 32 at a time in order.
// Stability follows from (tile, warp, round, lane) order = index order.

__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t* __restrict__ keys, uint32_t n, int shift,
                                                             uint32_t ntiles, uint32_t* __restrict__ hist)
{
    __shared__ uint32_t h[kRadixBins];
    for (int d = threadIdx.x; d < kRadixBins; d += blockDim.x) h[d] = 0;
    __syncthreads();
    const uint32_t base = blockIdx.x * kSortTile;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int r = 0; r < kSortItems; ++r) {
        const uint32_t i = base + w * (32 * kSortItems) + r * 32 + lane;
        const bool ok = i < n;
        const uint32_t d = ok ? (keys[i] >> shift) & (kRadixBins - 1) : 0xFFFFFFFFu;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (ok && lane == __ffs(peers) - 1) atomicAdd(&h[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadixBins; d += blockDim.x) hist[(size_t)d * ntiles + blockIdx.x] = h[d];
}

__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const uint32_t* __restrict__ key_in, const uint32_t* __restrict__ idx_in,
                                                                uint32_t* __restrict__ key_out, uint32_t* __restrict__ idx_out,
                                                                uint32_t n, int shift, uint32_t ntiles,
                                                                const uint32_t* __restrict__ hist_scanned)
{
    __shared__ uint32_t wh[kSortThreads / 32][kRadixBins];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int d = lane; d < kRadixBins; d += 32) wh[w][d] = 0;
    __syncwarp();
    const uint32_t base = blockIdx.x * kSortTile + w * (32 * kSortItems);
    uint32_t k[kSortItems], v[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const uint32_t i = base + r * 32 + lane;
        const bool ok = i < n;
        k[r] = ok ? key_in[i] : 0xFFFFFFFFu;
        v[r] = ok ? (idx_in ? idx_in[i] : i) : 0u;
        const uint32_t d = ok ? (k[r] >> shift) & (kRadixBins - 1) : 0xFFFFFFFFu;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (ok && lane == __ffs(peers) - 1) wh[w][d] += (uint32_t)__popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit: global tile offset, then warps in order
    for (int d = threadIdx.x; d < kRadixBins; d += blockDim.x) {
        uint32_t run = hist_scanned[(size_t)d * ntiles + blockIdx.x];
#pragma unroll
        for (int ww = 0; ww < kSortThreads / 32; ++ww) {
            const uint32_t c = wh[ww][d];
            wh[ww][d] = run;
            run += c;
        }
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const uint32_t i = base + r * 32 + lane;
        const bool ok = i < n;
        const uint32_t d = ok ? (k[r] >> shift) & (kRadixBins - 1) : 0xFFFFFFFFu;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        uint32_t pos = 0;
        if (ok) {
            pos = wh[w][d] + (uint32_t)__popc(peers & lt);
            key_out[pos] = k[r];
            idx_out[pos] = v[r];
        }
        __syncwarp();
        if (ok && lane == __ffs(peers) - 1) wh[w][d] += (uint32_t)__popc(peers);
        __syncwarp();
    }
}

__global__ void k_fill_u32(uint32_t* p, uint32_t n, uint32_t v)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = v;
}

__global__ void k_add_u32(uint32_t* p, uint32_t n, uint32_t v)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] += v;
}

__global__ void k_iota(uint32_t* p, uint32_t n)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = i;
}

// ---------------------------------------------------------------------------
// Per-cell preparation of the pair step
// ---------------------------------------------------------------------------
// Row blocks of 32 rows (rows 0 .. n-2 have partners); accepted-list room is
// mu + 8 sqrt(mu) + 16 with mu = 2.0001 C n (n - 1) / 2: the accepted count is
// dominated by a binomial with success probability max P22 <= 2 C, so the
// room is exceeded with probability far below 1e-15 per cell and step.
// The value is the FP64 evaluation's; an FP32 evaluation decides it first
// (FP64 square roots are slow on this GPU): for n <= 4096, n (n - 1) / 2 is
// exact in FP32 and the FP32 result r lies within 1e-6 r of the FP64 one, so
// when no integer lies within 2^-16 r + 2^-10 of r both have the same
// ceiling; otherwise, or for larger cells, FP64 decides.
__device__ __forceinline__ uint32_t list_room(double C, float Cf, uint32_t n)
{
    if (n <= 4096u) {
        const float mu = 2.0001f * Cf * (0.5f * (float)n * (float)(n - 1));
        const float r = mu + 8.0f * sqrtf(mu) + 16.0f;
        const float e = r * 0x1p-16f + 0x1p-10f;
        const float lo = ceilf(r - e), hi = ceilf(r + e);
        if (lo == hi && r < 1.0e9f) return (uint32_t)hi;
    }
    const double mu = 2.0001 * C * (0.5 * (double)n * (double)(n - 1));
    const double room = ceil(mu + 8.0 * sqrt(mu) + 16.0);
    return room > 4.0e9 ? 0xFFFFFFFFu : (uint32_t)room;
}

// work[c] = (row-block items of the all-pairs tile, list room); skip_work[c]
// = row blocks of a skip-ahead cell (null when no simulation uses that mode).
__global__ void __launch_bounds__(256) k_cell_prep(const SimDesc* __restrict__ sims, int nsims,
                                                   const uint32_t* __restrict__ cell_start, uint2* __restrict__ work,
                                                   uint32_t* __restrict__ skip_work,
                                                   uint32_t* __restrict__ acc_count, uint32_t ncells, uint32_t small_max,
                                                   uint32_t* __restrict__ counters, unsigned long long* __restrict__ stats,
                                                   int count_pairs)
{
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t t0 = blockIdx.x * blockDim.x + threadIdx.x;
    if (t0 == 0) {
        counters[0] = 0;  // pair work counter
        counters[2] = 0;  // active cells
        counters[3] = 0;  // survivors of the random-byte filters
        work[ncells] = make_uint2(0, 0);
        if (skip_work) skip_work[ncells] = 0;
    }
    // pair tests summed per thread and simulation, flushed on a change
    uint32_t cur_slot = 0xFFFFFFFFu;
    unsigned long long tests = 0;
    for (uint32_t c = t0; c < ncells; c += stride) {
        const int s = sim_of_cell(sims, nsims, c);
        const SimDesc& S = sims[s];
        const uint32_t n = cell_start[c + 1] - cell_start[c];
        uint32_t items = 0, room = 0, skip_items = 0;
        if (n >= 2 && S.C > 0.0) {
            if (S.skip) skip_items = (n - 1 + kPairRows - 1) / kPairRows;
            else if (n > small_max) items = (n - 1 + kPairRows - 1) / kPairRows;
            room = list_room(S.C, S.Cf, n);
            if (count_pairs) {
                if (S.stat_slot != cur_slot) {
                    if (tests) atomicAdd(&stats[cur_slot * kStatCount + kStatPairTests], tests);
                    tests = 0;
                    cur_slot = S.stat_slot;
                }
                tests += (unsigned long long)n * (n - 1) / 2;
            }
        }
        work[c] = make_uint2(items, room);
        if (skip_work) skip_work[c] = skip_items;
        acc_count[c] = 0;
    }
    // one atomic per warp and simulation
    const unsigned mask = __activemask();
    const unsigned peers = __match_any_sync(mask, cur_slot);
    const int leader = __ffs(peers) - 1;
    unsigned long long sum = 0;
    for (unsigned m = peers; m; m &= m - 1) sum += __shfl_sync(peers, tests, __ffs(m) - 1);
    if ((int)(threadIdx.x & 31) == leader && cur_slot != 0xFFFFFFFFu && sum)
        atomicAdd(&stats[cur_slot * kStatCount + kStatPairTests], sum);
}

// ---------------------------------------------------------------------------
// A8: observables (FP64 sums per cell, fixed order) and totals
// ---------------------------------------------------------------------------
__device__ __forceinline__ double block_sum_fixed(double v, double* red)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    }
    __syncthreads();
    return t;
}

// sqrt(e2) to FP64 accuracy for the FP64 sums of A8: one FP64 Newton step
// from the FP32 square root, e0 + (e2 - e0^2) / (2 e0), with the FP32
// reciprocal of e0 (FP64 square roots are slow on this GPU).  The FP32 start
// is within 1e-7 relative, so the step leaves about 1e-14.
__device__ __forceinline__ double energy_sqrt(double e2)
{
    const float s = __fsqrt_rn((float)e2);
    if (!(s > 1e-30f) || !(s < 1e30f)) return sqrt(e2);
    const double e0 = (double)s;
    const double r = fma(-e0, e0, e2);
    return fma(r, 0.5 * (double)__frcp_rn(s), e0);
}

template <typename T>
__global__ void __launch_bounds__(256) k_observables(SimDesc S, const T* __restrict__ st, uint32_t pcap,
                                                     const uint32_t* __restrict__ cell_start, double* __restrict__ T00,
                                                     double* __restrict__ T0x, int32_t* __restrict__ counts)
{
    __shared__ double red[8];
    for (uint32_t c = blockIdx.x; c < S.ncells; c += gridDim.x) {
        const uint32_t b = cell_start[S.cell_off + c], e = cell_start[S.cell_off + c + 1];
        double se = 0.0, sx = 0.0;
        for (uint32_t k = b + threadIdx.x; k < e; k += blockDim.x) {
            const double qx = st[3 * (size_t)pcap + k], qy = st[4 * (size_t)pcap + k], qz = st[5 * (size_t)pcap + k];
            se += energy_sqrt(((qx * qx + qy * qy) + qz * qz) + S.m2);
            sx += qx;
        }
        const double te = block_sum_fixed(se, red);
        const double tx = block_sum_fixed(sx, red);
        if (threadIdx.x == 0) {
            T00[c] = te / S.norm;
            T0x[c] = tx / S.norm;
            counts[c] = (int32_t)(e - b);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_totals_partial(SimDesc S, const T* __restrict__ st, uint32_t pcap,
                                                        double* __restrict__ part)
{
    __shared__ double red[8];
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < S.np; k += stride) {
        const uint32_t g = S.p_off + k;
        const double qx = st[3 * (size_t)pcap + g], qy = st[4 * (size_t)pcap + g], qz = st[5 * (size_t)pcap + g];
        a[0] += energy_sqrt(((qx * qx + qy * qy) + qz * qz) + S.m2);
        a[1] += qx;
        a[2] += qy;
        a[3] += qz;
    }
    for (int q = 0; q < 4; ++q) {
        const double t = block_sum_fixed(a[q], red);
        if (threadIdx.x == 0) part[blockIdx.x * 4 + q] = t;
    }
}

__global__ void k_totals_final(const double* __restrict__ part, int nb, double* __restrict__ out)
{
    if (threadIdx.x < 4) {
        double t = 0.0;
        for (int b = 0; b < nb; ++b) t += part[b * 4 + threadIdx.x];
        out[threadIdx.x] = t;
    }
}

__global__ void k_advance(SimDesc* sims, int nsims, unsigned long long* stats)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < nsims) {
        sims[s].step += 1;
        sims[s].time += sims[s].dt;
        stats[sims[s].stat_slot * kStatCount + kStatSteps] += 1;
    }
}

// Adaptive time step of the coming step (one block per simulation): the most
// populated cell n_max of the sorted state, dt = ((kappa N_test) V_cell) /
// (sigma (n_max - 1)) capped by dt_max (the cap without collisions), and the
// constants that follow from dt.
__global__ void __launch_bounds__(256) k_adapt_dt(SimDesc* __restrict__ sims, const uint32_t* __restrict__ cell_start)
{
    __shared__ uint32_t red[8];
    SimDesc& S = sims[blockIdx.x];
    if (!(S.kappa > 0.0)) return;
    uint32_t m = 0;
    for (uint32_t c = threadIdx.x; c < S.ncells; c += blockDim.x) {
        const uint32_t g = S.cell_off + c;
        m = max(m, cell_start[g + 1] - cell_start[g]);
    }
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = max(m, red[w]);
        double dt = S.dt_max;
        if (S.sigma > 0.0 && m >= 2) {
            const double a = __ddiv_rn(__dmul_rn(__dmul_rn(S.kappa, S.n_test), S.V), __dmul_rn(S.sigma, (double)(m - 1)));
            dt = a < S.dt_max ? a : S.dt_max;
        }
        S.dt = dt;
        derive_step_constants(S);
    }
}

__global__ void k_philox(const uint32_t* __restrict__ ctr, int64_t n, uint32_t k0, uint32_t k1, uint32_t* __restrict__ out)
{
    const PhiloxKey K = philox_schedule(k0, k1);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
        const uint4 r = philox4x32_10(c, K);
        out[4 * i] = r.x;
        out[4 * i + 1] = r.y;
        out[4 * i + 2] = r.z;
        out[4 * i + 3] = r.w;
    }
}

// Cell keys of caller-owned positions (SoA x, y, z of one simulation).
template <typename T>
__global__ void __launch_bounds__(256) k_keys_raw(SimDesc S, const T* __restrict__ xyz, uint32_t n,
                                                  uint32_t* __restrict__ keys)
{
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < n; g += stride) {
        T pos[3] = {xyz[g], xyz[(size_t)n + g], xyz[2 * (size_t)n + g]};
        keys[g] = cell_key<T>(S, pos);
    }
}

// cell_start[c] = first sorted position with key >= c (keys sorted), for
// c = 0 .. ncells: one lower-bound search per cell, so empty cells cost one
// search each wherever they lie (no serial fill of runs of empty cells).
__global__ void __launch_bounds__(256) k_cell_bounds(const uint32_t* __restrict__ skey, uint32_t np,
                                                     uint32_t* __restrict__ cell_start, uint32_t ncells)
{
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c <= ncells; c += stride) {
        uint32_t lo = 0, hi = np;
        while (lo < hi) {
            const uint32_t mid = lo + ((hi - lo) >> 1);
            if (skey[mid] < c) lo = mid + 1; else hi = mid;
        }
        cell_start[c] = lo;
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
int sm_count()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

static unsigned grid_for(uint64_t n, int threads, int per_sm)
{
    uint64_t need = (n + threads - 1) / threads;
    uint64_t cap = (uint64_t)sm_count() * per_sm;
    if (need < 1) need = 1;
    return (unsigned)(need < cap ? need : cap);
}

static int last_err() { return cudaPeekAtLastError() == cudaSuccess ? 0 : -1; }

int launch_init_thermal(const Arena& A, int sim, const SimDesc& S, const double* d_regions, int nreg,
                        const uint64_t* d_first, cudaStream_t st)
{
    (void)sim;
    if (S.np == 0) return 0;
    const unsigned g = grid_for(S.np, 256, 8);
    if (A.precision == 1)
        k_init_thermal<double><<<g, 256, 0, st>>>(S, (double*)A.st[A.cur], A.pcap, d_regions, nreg, d_first);
    else
        k_init_thermal<float><<<g, 256, 0, st>>>(S, (float*)A.st[A.cur], A.pcap, d_regions, nreg, d_first);
    return last_err();
}

int launch_init_hotspot(const Arena& A, const SimDesc& S, double T0, double dT, double width, cudaStream_t st)
{
    if (S.np == 0) return 0;
    const unsigned g = grid_for(S.np, 256, 8);
    if (A.precision == 1)
        k_init_hotspot<double><<<g, 256, 0, st>>>(S, (double*)A.st[A.cur], A.pcap, T0, dT, width);
    else
        k_init_hotspot<float><<<g, 256, 0, st>>>(S, (float*)A.st[A.cur], A.pcap, T0, dT, width);
    return last_err();
}

int launch_fill_u32(uint32_t* p, uint32_t n, uint32_t v, cudaStream_t st)
{
    if (n == 0) return 0;
    k_fill_u32<<<grid_for(n, 256, 4), 256, 0, st>>>(p, n, v);
    return last_err();
}

int launch_add_u32(uint32_t* p, uint32_t n, uint32_t v, cudaStream_t st)
{
    if (n == 0) return 0;
    k_add_u32<<<grid_for(n, 256, 4), 256, 0, st>>>(p, n, v);
    return last_err();
}

int launch_cell_prep(const Arena& A, cudaStream_t st, int count_pairs)
{
    const unsigned g = grid_for(A.ncells, 256, 8);
    uint32_t* skip_work = A.any_skip ? A.skip_work : nullptr;
    k_cell_prep<<<g, 256, 0, st>>>(A.d_sims, A.nsims, A.cell_start, A.cell_work, skip_work, A.acc_count, A.ncells,
                                   A.small_max, A.counters, A.stats, count_pairs);
    if (last_err()) return -1;
    if (exclusive_scan<uint2, Uint2Add>(A.cell_work, (size_t)A.ncells + 1, make_uint2(0, 0), Uint2Add(), A.scan_tmp,
                                        A.scan_tmp_bytes, st))
        return -1;
    if (skip_work && exclusive_scan<uint32_t, U32Add>(skip_work, (size_t)A.ncells + 1, 0u, U32Add(), A.scan_tmp,
                                                      A.scan_tmp_bytes, st))
        return -1;
    return 0;
}

int launch_observables(const Arena& A, int sim, double* T00, double* T0x, int32_t* counts, cudaStream_t st)
{
    SimDesc S;
    if (cudaMemcpy(&S, A.d_sims + sim, sizeof(SimDesc), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
    const unsigned g = grid_for((uint64_t)S.ncells * 256, 256, 16);
    if (A.precision == 1)
        k_observables<double><<<g, 256, 0, st>>>(S, (const double*)A.st[A.cur], A.pcap, A.cell_start, T00, T0x, counts);
    else
        k_observables<float><<<g, 256, 0, st>>>(S, (const float*)A.st[A.cur], A.pcap, A.cell_start, T00, T0x, counts);
    return last_err();
}

int launch_totals(const Arena& A, int sim, double* d_out4, cudaStream_t st)
{
    SimDesc S;
    if (cudaMemcpy(&S, A.d_sims + sim, sizeof(SimDesc), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
    const int nb = 256;
    double* part = reinterpret_cast<double*>(A.scan_tmp);
    if (A.scan_tmp_bytes < nb * 4 * sizeof(double)) return -1;
    if (A.precision == 1)
        k_totals_partial<double><<<nb, 256, 0, st>>>(S, (const double*)A.st[A.cur], A.pcap, part);
    else
        k_totals_partial<float><<<nb, 256, 0, st>>>(S, (const float*)A.st[A.cur], A.pcap, part);
    k_totals_final<<<1, 32, 0, st>>>(part, nb, d_out4);
    return last_err();
}

int launch_adapt_dt(const Arena& A, cudaStream_t st)
{
    if (A.nsims == 0) return 0;
    k_adapt_dt<<<A.nsims, 256, 0, st>>>(A.d_sims, A.cell_start);
    return last_err();
}

int launch_advance(const Arena& A, cudaStream_t st)
{
    k_advance<<<(A.nsims + 127) / 128, 128, 0, st>>>(A.d_sims, A.nsims, A.stats);
    return last_err();
}

// Keys and stable counting sort of caller-owned positions with caller-given
// scratch (no allocation): key_a/key_b/idx_a/idx_b hold n words each, hist
// 256 * ceil(n / 4096) words, partials partial_bytes.  perm and cell_start
// are outputs.
int launch_bin_raw(const SimDesc& S, int precision, const void* xyz, uint32_t n, uint32_t* key_a, uint32_t* key_b,
                   uint32_t* idx_a, uint32_t* idx_b, uint32_t* hist, void* partials, size_t partial_bytes,
                   uint32_t* perm, uint32_t* cell_start, cudaStream_t st)
{
    if (n == 0) {
        k_fill_u32<<<grid_for((uint64_t)S.ncells + 1, 256, 4), 256, 0, st>>>(cell_start, S.ncells + 1, 0u);
        return last_err();
    }
    const unsigned g = grid_for(n, 256, 8);
    if (precision == 1)
        k_keys_raw<double><<<g, 256, 0, st>>>(S, (const double*)xyz, n, key_a);
    else
        k_keys_raw<float><<<g, 256, 0, st>>>(S, (const float*)xyz, n, key_a);
    const int passes = radix_passes(S.ncells);
    const uint32_t ntiles = (n + kSortTile - 1) / kSortTile;
    uint32_t* keys[2] = {key_a, key_b};
    uint32_t* idx[2] = {idx_a, idx_b};
    int src = 0;
    for (int p = 0; p < passes; ++p) {
        const int shift = p * kRadixBits;
        k_radix_hist<<<ntiles, kSortThreads, 0, st>>>(keys[src], n, shift, ntiles, hist);
        if (exclusive_scan<uint32_t, U32Add>(hist, (size_t)kRadixBins * ntiles, 0u, U32Add(), partials, partial_bytes, st))
            return -1;
        k_radix_scatter<<<ntiles, kSortThreads, 0, st>>>(keys[src], p == 0 ? nullptr : idx[src], keys[src ^ 1],
                                                         idx[src ^ 1], n, shift, ntiles, hist);
        src ^= 1;
    }
    if (passes == 0)
        k_iota<<<grid_for(n, 256, 4), 256, 0, st>>>(perm, n);
    else if (cudaMemcpyAsync(perm, idx[src], sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return -1;
    k_cell_bounds<<<grid_for((uint64_t)S.ncells + 1, 256, 8), 256, 0, st>>>(keys[src], n, cell_start, S.ncells);
    return last_err();
}

int launch_philox(const uint32_t* ctr, int64_t n, uint64_t key, uint32_t* out, cudaStream_t st)
{
    if (n <= 0) return 0;
    const unsigned g = grid_for((uint64_t)n, 256, 8);
    k_philox<<<g, 256, 0, st>>>(ctr, n, (uint32_t)key, (uint32_t)(key >> 32), out);
    return last_err();
}

}  // namespace cuba
