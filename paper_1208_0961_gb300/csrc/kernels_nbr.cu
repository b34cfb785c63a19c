// A1-A4 of a step for arenas with many small cells: the stable counting sort
// by cell as a neighbour-move sort.
//
// At the start of a step the state is sorted by cell and cell_start describes
// it.  A particle moves by |p/E| dt <= dt in a step, so when dt is below the
// cell edge on every axis (with a margin), its new cell is one of the 27
// cells around its old one: direction d = (dx+1) + 3 (dy+1) + 9 (dz+1), with
// d_a the change of its cell coordinate along axis a.  The stable sort by
// new cell then needs no radix passes:
//   count:   every particle is streamed (A1, A2) and written back to its
//            slot; its old cell is the key of its position before streaming,
//            its direction that of its new cell (A3), kept as c << 5 | d;
//            rel[d][c] counts the particles of old cell c moving in
//            direction d (one atomic per group of a warp's 32 particles);
//   offsets: one thread per new cell c visits its 27 possible source cells in
//            increasing key order (decreasing d: the source is c - delta_d,
//            delta_d = d_x + n_x (d_y + n_y d_z)), replacing each count by the
//            number of earlier particles of c, and writes c's total;
//   scan:    the totals give the new cell_start;
//   scatter: every streamed particle is moved into slot cell_start[c'] +
//            rel[d][c] + (rank among its old cell's earlier particles of the
//            same direction), the rank carried along each warp's 128
//            particles; the stream arithmetic runs once per step.
// Within a new cell the particles come source cell by source cell in key
// order and, inside a source cell, in their old order: the stable order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "engine.cuh"
#include "fp.cuh"
#include "stream.cuh"

namespace cuba {

constexpr int kNbrDirs = 27;
constexpr int kNbrThreads = 256;
constexpr int kNbrWarps = kNbrThreads / 32;
constexpr unsigned kNbrFull = 0xffffffffu;
constexpr int kNbrGroup = 4;   // scatter rounds whose loads are issued together
// The scatter's warps take 128 particles each (4 rounds of 32, all loaded
// together): more, shorter ranges than the count pass's 512 keep more loads
// in flight across the GPU (1.07 against 1.16 ms per step of the 64 M hot spot;
// 2 or 8 rounds measured 1.09 and 1.08).
constexpr int kScatRounds = 4;
constexpr int kScatTile = kNbrThreads * kScatRounds;

template <typename T>
__device__ __forceinline__ void nbr_load(const T* __restrict__ st, uint32_t pcap, uint32_t g, T pos[3], T mom[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        pos[a] = st[(size_t)a * pcap + g];
        mom[a] = st[(size_t)(3 + a) * pcap + g];
    }
}

// Old cell (global key) and direction of a particle: the old cell from its
// position before streaming (the key the last sort used), the direction from
// the cell coordinates after streaming.  Returns false if it moved more than
// one cell along an axis.
// The same with the old cell's coordinates io given.
template <typename T>
__device__ __forceinline__ bool nbr_move_from(const SimDesc& S, const uint32_t io[3], T pos[3], T mom[3], int& d,
                                              uint32_t& key_new, uint32_t& nref)
{
    uint32_t in[3];
    nref += (uint32_t)stream_one<T>(S, pos, mom);
    cell_coords<T>(S, pos, in);
    const uint32_t n0 = (uint32_t)S.n[0], n1 = (uint32_t)S.n[1];
    key_new = S.cell_off + in[0] + n0 * (in[1] + n1 * in[2]);
    const int32_t m0 = (int32_t)in[0] - (int32_t)io[0], m1 = (int32_t)in[1] - (int32_t)io[1],
                  m2 = (int32_t)in[2] - (int32_t)io[2];
    if (m0 < -1 || m0 > 1 || m1 < -1 || m1 > 1 || m2 < -1 || m2 > 1) return false;
    d = (m0 + 1) + 3 * (m1 + 1) + 9 * (m2 + 1);
    return true;
}

template <typename T>
__device__ __forceinline__ bool nbr_move(const SimDesc& S, T pos[3], T mom[3], uint32_t& c_old, int& d,
                                         uint32_t& key_new, uint32_t& nref)
{
    uint32_t io[3];
    cell_coords<T>(S, pos, io);
    c_old = S.cell_off + io[0] + (uint32_t)S.n[0] * (io[1] + (uint32_t)S.n[1] * io[2]);
    return nbr_move_from<T>(S, io, pos, mom, d, key_new, nref);
}

// Count pass, 4096 particles per block (512 per warp, 32 at a time): rel[d][c]
// += particles of old cell c moving in direction d (rel zeroed before), one
// atomic per (cell, direction) group of a warp's 32 particles; trace keys;
// reflections.  The streamed particle goes back to its slot (positions, and
// the momentum when it reflected) and keys[i] = c << 5 | d (all ones for a
// move of more than one cell), so that the scatter pass only moves data.
// One simulation (kOne): the old cell of particle i is read off cell_start
// (the state is sorted by cell): the range's first particle's cell from its
// position, then each lane walks the cell boundaries up to its particle,
// carrying the cell's coordinates, instead of dividing three coordinates.
template <typename T> struct NbrCountBlocks { static constexpr int value = sizeof(T) == 4 ? 5 : 3; };

template <typename T, bool kOne>
__global__ void __launch_bounds__(kNbrThreads, NbrCountBlocks<T>::value) k_nbr_count(const SimDesc* __restrict__ sims, int nsims,
                                                           T* __restrict__ st, uint32_t pcap, uint32_t n,
                                                           const uint32_t* __restrict__ cs,
                                                           uint32_t* __restrict__ rel, size_t rel_stride,
                                                           uint32_t* __restrict__ keys,
                                                           uint32_t* __restrict__ trace_keys,
                                                           uint32_t* __restrict__ counters,
                                                           unsigned long long* __restrict__ stats)
{
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t base = blockIdx.x * kSortTile + w * (32 * kSortItems);
    uint32_t cur_slot = 0xFFFFFFFFu, nref = 0;
    SimDesc Sl;  // one simulation: the streaming's descriptor fields, read once
    if (kOne) copy_stream_fields(Sl, sims[0]);
    // kOne: cell (global key) of the last particle of the previous round and
    // its coordinates
    uint32_t cur = 0, cx = 0, cy = 0, cz = 0;
    const uint32_t nx = (uint32_t)sims[0].n[0], ny = (uint32_t)sims[0].n[1];
    if (kOne && base < n) {
        T p0[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) p0[a] = st[(size_t)a * pcap + base];
        uint32_t io[3];
        cell_coords<T>(sims[0], p0, io);
        cx = io[0];
        cy = io[1];
        cz = io[2];
        cur = sims[0].cell_off + cx + nx * (cy + ny * cz);
    }
#pragma unroll 4
    for (int r = 0; r < kSortItems; ++r) {
        const uint32_t i = base + r * 32 + lane;
        uint32_t key = 0xFFFFFFFFu, c = 0;
        int d = 0;
        uint32_t io[3] = {cx, cy, cz};
        if (kOne) {
            c = cur;
            if (i < n)
                while (cs[c + 1] <= i) {
                    ++c;
                    if (++io[0] == nx) {
                        io[0] = 0;
                        if (++io[1] == ny) {
                            io[1] = 0;
                            ++io[2];
                        }
                    }
                }
            const uint32_t r_lo = base + r * 32;
            const int last = r_lo < n ? (int)min(31u, n - 1 - r_lo) : 0;
            cur = __shfl_sync(kNbrFull, c, last);
            cx = __shfl_sync(kNbrFull, io[0], last);
            cy = __shfl_sync(kNbrFull, io[1], last);
            cz = __shfl_sync(kNbrFull, io[2], last);
        }
        if (i < n) {
            const SimDesc& S = kOne ? Sl : sims[sim_of_particle(sims, nsims, i)];
            if (S.stat_slot != cur_slot) {
                if (nref) atomicAdd(&stats[cur_slot * kStatCount + kStatReflections], (unsigned long long)nref);
                nref = 0;
                cur_slot = S.stat_slot;
            }
            T pos[3], mom[3];
            nbr_load<T>(st, pcap, i, pos, mom);
            uint32_t kn;
            const uint32_t r0 = nref;
            if (kOne ? nbr_move_from<T>(S, io, pos, mom, d, kn, nref) : nbr_move<T>(S, pos, mom, c, d, kn, nref))
                key = (c << 5) | (uint32_t)d;
            else
                atomicOr(&counters[1], kErrMove);
#pragma unroll
            for (int a = 0; a < 3; ++a) st[(size_t)a * pcap + i] = pos[a];
            if (nref != r0) {
#pragma unroll
                for (int a = 0; a < 3; ++a) st[(size_t)(3 + a) * pcap + i] = mom[a];
            }
            keys[i] = key;
            if (trace_keys) trace_keys[i] = kn;
        }
        const unsigned peers = __match_any_sync(kNbrFull, key);
        if (key != 0xFFFFFFFFu && lane == __ffs(peers) - 1)
            atomicAdd(&rel[(size_t)d * rel_stride + c], (uint32_t)__popc(peers));
    }
    const unsigned peers = __match_any_sync(kNbrFull, cur_slot);
    const unsigned sum = __reduce_add_sync(peers, nref);
    if (lane == __ffs(peers) - 1 && cur_slot != 0xFFFFFFFFu && sum)
        atomicAdd(&stats[cur_slot * kStatCount + kStatReflections], (unsigned long long)sum);
}

// Scatter pass over 128-particle warp ranges (kScatRounds): moves the streamed
// particles (the count pass wrote them back in place, with their keys
// c << 5 | d).  A particle's slot is cell_start_new[new cell] + rel[d][old
// cell] (earlier source cells of the new cell) + its rank among the earlier
// particles of its old cell with the same direction.  Within a warp range the
// rank is carried from round to round for the cell that spans them (run[d]);
// the keys of the first cell's particles before the range are counted first.
template <typename T, bool kOne>
__global__ void __launch_bounds__(kNbrThreads) k_nbr_scatter(const SimDesc* __restrict__ sims, int nsims,
                                                             const T* __restrict__ st_old, T* __restrict__ st_new,
                                                             uint32_t pcap, uint32_t n, uint32_t ncells,
                                                             const uint32_t* __restrict__ cs_old,
                                                             const uint32_t* __restrict__ keys,
                                                             const uint32_t* __restrict__ rel, size_t rel_stride,
                                                             const uint32_t* __restrict__ cs_new,
                                                             uint32_t* __restrict__ perm,
                                                             uint32_t* __restrict__ counters)
{
    __shared__ uint32_t run[kNbrWarps][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t base = blockIdx.x * kScatTile + w * (32 * kScatRounds);
    if (base >= n) return;
    run[w][lane] = 0;
    // one simulation: the key offsets of the 27 directions are kernel-wide
    const int32_t nx1 = sims[0].n[0], nxy1 = sims[0].n[0] * sims[0].n[1];
    // the first cell of the range (a move error leaves an all-ones key: the
    // cell is clamped so that every read stays in bounds) and the ranks of
    // its particles before the range
    uint32_t carry = min(keys[base] >> 5, ncells - 1u);
    __syncwarp();
    for (uint32_t k = cs_old[carry]; k < base; k += 32) {
        const uint32_t j = k + lane;
        const uint32_t key = j < base ? keys[j] : 0xFFFFFFFFu;
        const unsigned peers = __match_any_sync(kNbrFull, key);
        if (key != 0xFFFFFFFFu && lane == __ffs(peers) - 1) run[w][key & 31u] += (uint32_t)__popc(peers);
        __syncwarp();
    }
    // rounds are taken kNbrGroup at a time: their loads and the gathers of
    // their slot bases are issued together, the rank carry is then applied
    // round by round
    for (int r0 = 0; r0 < kScatRounds; r0 += kNbrGroup) {
        if (base + r0 * 32 >= n) break;
        uint32_t key[kNbrGroup], sb[kNbrGroup];
        T pos[kNbrGroup][3], mom[kNbrGroup][3];
#pragma unroll
        for (int k = 0; k < kNbrGroup; ++k) {
            const uint32_t i = base + (r0 + k) * 32 + lane;
            key[k] = i < n ? keys[i] : 0xFFFFFFFFu;
            if (key[k] != 0xFFFFFFFFu) nbr_load<T>(st_old, pcap, i, pos[k], mom[k]);
        }
#pragma unroll
        for (int k = 0; k < kNbrGroup; ++k) {
            sb[k] = 0;
            if (key[k] != 0xFFFFFFFFu) {
                const uint32_t c = key[k] >> 5, d = key[k] & 31u;
                int32_t nx = nx1, nxy = nxy1;
                if (!kOne) {
                    const SimDesc& S = sims[sim_of_cell(sims, nsims, c)];
                    nx = S.n[0];
                    nxy = S.n[0] * S.n[1];
                }
                const int32_t dx = (int32_t)(d % 3u) - 1, dy = (int32_t)((d / 3u) % 3u) - 1, dz = (int32_t)(d / 9u) - 1;
                const uint32_t dest = c + (uint32_t)(dx + nx * dy + nxy * dz);
                sb[k] = cs_new[dest] + rel[(size_t)d * rel_stride + c];
            }
        }
#pragma unroll
        for (int k = 0; k < kNbrGroup; ++k) {
            const uint32_t r_lo = base + (r0 + k) * 32;
            if (r_lo >= n) break;
            const uint32_t i = r_lo + lane;
            const uint32_t c = key[k] == 0xFFFFFFFFu ? 0xFFFFFFFFu : key[k] >> 5, d = key[k] & 31u;
            const unsigned peers = __match_any_sync(kNbrFull, key[k]);
            if (key[k] != 0xFFFFFFFFu) {
                const uint32_t slot = sb[k] + (c == carry ? run[w][d] : 0u) + (uint32_t)__popc(peers & lt);
                if (slot < n) {
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        st_new[(size_t)a * pcap + slot] = pos[k][a];
                        st_new[(size_t)(3 + a) * pcap + slot] = mom[k][a];
                    }
                    if (perm) perm[slot] = i;
                } else {
                    atomicOr(&counters[1], kErrMove);
                }
            }
            // the cell of the round's last particle carries into the next round
            const uint32_t last_lane = min(31u, n - 1 - r_lo);
            const uint32_t last = __shfl_sync(kNbrFull, c, (int)last_lane);
            __syncwarp();
            if (last != carry) {
                run[w][lane] = 0;
                carry = last;
            }
            __syncwarp();
            if (key[k] != 0xFFFFFFFFu && c == carry && lane == __ffs(peers) - 1)
                run[w][d] += (uint32_t)__popc(peers);
            __syncwarp();
        }
    }
}

// One thread per new cell: in-cell offsets of its source blocks (in place in
// rel) and its particle count (cnt[c]; cnt[ncells] = 0 for the scan).  The 27
// counts are read before any offset is written.
__global__ void __launch_bounds__(256) k_nbr_offsets(const SimDesc* __restrict__ sims, int nsims,
                                                     uint32_t* __restrict__ rel, size_t rel_stride, uint32_t ncells,
                                                     uint32_t* __restrict__ cnt)
{
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c <= ncells; c += stride) {
        if (c == ncells) {
            cnt[c] = 0;
            continue;
        }
        const SimDesc& S = sims[sim_of_cell(sims, nsims, c)];
        const uint32_t lc = c - S.cell_off;
        const uint32_t n0 = (uint32_t)S.n[0], n1 = (uint32_t)S.n[1];
        const int32_t ic[3] = {(int32_t)(lc % n0), (int32_t)((lc / n0) % n1), (int32_t)(lc / (n0 * n1))};
        uint32_t src[kNbrDirs], v[kNbrDirs];
#pragma unroll
        for (int d = 0; d < kNbrDirs; ++d) {
            const int32_t s0 = ic[0] - (d % 3 - 1), s1 = ic[1] - ((d / 3) % 3 - 1), s2 = ic[2] - (d / 9 - 1);
            const bool ok = s0 >= 0 && s0 < S.n[0] && s1 >= 0 && s1 < S.n[1] && s2 >= 0 && s2 < S.n[2];
            src[d] = ok ? S.cell_off + (uint32_t)s0 + n0 * ((uint32_t)s1 + n1 * (uint32_t)s2) : 0xFFFFFFFFu;
            v[d] = ok ? rel[(size_t)d * rel_stride + src[d]] : 0u;
        }
        uint32_t acc = 0;
#pragma unroll
        for (int d = kNbrDirs - 1; d >= 0; --d) {
            if (src[d] != 0xFFFFFFFFu) rel[(size_t)d * rel_stride + src[d]] = acc;
            acc += v[d];
        }
        cnt[c] = acc;
    }
}

bool nbr_path(const Arena& A)
{
    return A.nbr_rel && A.nbr_ok && A.ncells > (uint32_t)kBinBins && A.ncells <= A.nbr_cap &&
           (uint64_t)A.np <= 64ull * A.ncells;
}

// The count and scatter passes for one simulation (kOne: its descriptor read
// once, outside the particle loops) or several.
template <typename T>
static void nbr_count(const Arena& A, uint32_t ntiles, uint32_t* tk, cudaStream_t st)
{
    if (A.nsims == 1)
        k_nbr_count<T, true><<<ntiles, kNbrThreads, 0, st>>>(A.d_sims, A.nsims, (T*)A.st[A.cur], A.pcap, A.np,
                                                             A.cell_start, A.nbr_rel, A.nbr_cap, A.key[0], tk,
                                                             A.counters, A.stats);
    else
        k_nbr_count<T, false><<<ntiles, kNbrThreads, 0, st>>>(A.d_sims, A.nsims, (T*)A.st[A.cur], A.pcap, A.np,
                                                              A.cell_start, A.nbr_rel, A.nbr_cap, A.key[0], tk,
                                                              A.counters, A.stats);
}

template <typename T>
static void nbr_scatter(const Arena& A, uint32_t* perm, cudaStream_t st)
{
    const uint32_t ntiles = (A.np + kScatTile - 1) / kScatTile;
    if (A.nsims == 1)
        k_nbr_scatter<T, true><<<ntiles, kNbrThreads, 0, st>>>(A.d_sims, A.nsims, (const T*)A.st[A.cur],
                                                               (T*)A.st[A.cur ^ 1], A.pcap, A.np, A.ncells,
                                                               A.cell_start, A.key[0], A.nbr_rel, A.nbr_cap,
                                                               A.nbr_cs, perm, A.counters);
    else
        k_nbr_scatter<T, false><<<ntiles, kNbrThreads, 0, st>>>(A.d_sims, A.nsims, (const T*)A.st[A.cur],
                                                                (T*)A.st[A.cur ^ 1], A.pcap, A.np, A.ncells,
                                                                A.cell_start, A.key[0], A.nbr_rel, A.nbr_cap,
                                                                A.nbr_cs, perm, A.counters);
}

int launch_step_nbr(Arena& A, cudaStream_t st, cudaEvent_t after_stream)
{
    const uint32_t n = A.np, nc = A.ncells;
    const size_t rs = A.nbr_cap;
    const uint32_t ntiles = (n + kSortTile - 1) / kSortTile;
    uint32_t* perm = A.trace ? A.idx[1] : nullptr;
    uint32_t* tk = A.trace ? A.trace_keys : nullptr;
    cudaMemsetAsync(A.nbr_rel, 0, (size_t)kNbrDirs * rs * sizeof(uint32_t), st);
    if (ntiles) {
        if (A.precision == 1)
            nbr_count<double>(A, ntiles, tk, st);
        else
            nbr_count<float>(A, ntiles, tk, st);
    }
    if (after_stream) cudaEventRecord(after_stream, st);
    const unsigned g2 = (unsigned)std::min<uint32_t>((nc + 256) / 256, (uint32_t)sm_count() * 16);
    k_nbr_offsets<<<g2, 256, 0, st>>>(A.d_sims, A.nsims, A.nbr_rel, rs, nc, A.nbr_cs);
    if (scan_u32(A.nbr_cs, (size_t)nc + 1, A.scan_tmp, A.scan_tmp_bytes, st)) return -1;
    if (ntiles) {
        if (A.precision == 1)
            nbr_scatter<double>(A, perm, st);
        else
            nbr_scatter<float>(A, perm, st);
    }
    cudaMemcpyAsync(A.cell_start, A.nbr_cs, ((size_t)nc + 1) * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st);
    A.sorted_buf = 1;
    A.cur ^= 1;
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace cuba
