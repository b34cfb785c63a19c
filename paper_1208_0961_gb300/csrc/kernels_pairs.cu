// Cell-parallel kernels of the collision step.
//
// k_pair_tile (A5): every pair i < j of every cell is tested against
// P22 = C v_rel (Eq. 3).  The uniform u_ij = r_ij 2^-32 of a pair is built
// from three Philox streams: its top byte from the block (step, cell, i, j/16)
// — one block serves sixteen pairs of a row — its next byte from the block
// (step, cell, i, TAG_MID | j/16), its low 16 bits from the block
// (step, cell, i, TAG_FINE | j).  Because P22 <= 2 C (1 + tiny) for every pair,
// a top byte above thr8 = floor(2.0001 C 256) already proves u_ij >= P22, and
// so does a 16-bit prefix above thr16 = floor(2.0001 C 65536): 255/256 of the
// pairs are rejected from the first block alone, without momenta, and most of
// the rest by the second; only the rare survivors draw the third block and
// evaluate P22.  The decision is the same as testing every pair in full.
// Work unit: one warp takes 32 rows of one cell (lane = row) and walks the
// row's column blocks; blocks with a small byte are queued per warp in shared
// memory and resolved together, one block per lane.  Survivors of both bytes
// are collected per warp and evaluated by k_pair_finish, one per thread.
// Accepted pairs go to the cell's segment of the list.
//
// k_resolve (A6, A7): per cell with accepted pairs — sort the list
// lexicographically (bitonic network in shared memory), take the greedy
// matching in that order (a particle collides at most once per step), then
// apply the centre-of-mass kinematics to every executed pair in parallel.
#include <cuda_runtime.h>

#include <cstdint>

#include "engine.cuh"
#include "fp.cuh"

namespace cuba {

constexpr unsigned kFull = 0xffffffffu;
constexpr unsigned long long kExecFlag = 1ull << 63;

// u = r 2^-32 in the state's precision (FP32: r rounded to nearest float).
template <typename T> __device__ __forceinline__ T unit_u(uint32_t r);
template <> __device__ __forceinline__ double unit_u<double>(uint32_t r) { return __dmul_rn((double)r, 0x1p-32); }
template <> __device__ __forceinline__ float unit_u<float>(uint32_t r) { return __fmul_rn(__uint2float_rn(r), 0x1p-32f); }

// Unit direction p / E of a massless particle (zero vector if p = 0).
template <typename T>
__device__ __forceinline__ void unit_dir(const T* __restrict__ st, uint32_t pcap, uint32_t g, T u[3])
{
    const T px = st[3 * (size_t)pcap + g], py = st[4 * (size_t)pcap + g], pz = st[5 * (size_t)pcap + g];
    const T E = sqrt_rn(add_rn(add_rn(mul_rn(px, px), mul_rn(py, py)), mul_rn(pz, pz)));
    const bool ok = E > T(0);
    u[0] = ok ? div_rn(px, E) : T(0);
    u[1] = ok ? div_rn(py, E) : T(0);
    u[2] = ok ? div_rn(pz, E) : T(0);
}

// P22 = C v_rel with v_rel = s / (2 E_i E_j) = |n_i - n_j|^2 / 2 (massless).
template <typename T>
__device__ __forceinline__ T p22_of_units(T C, const T ui[3], const T uj[3])
{
    const T d0 = sub_rn(ui[0], uj[0]), d1 = sub_rn(ui[1], uj[1]), d2 = sub_rn(ui[2], uj[2]);
    const T v = mul_rn(T(0.5), add_rn(add_rn(mul_rn(d0, d0), mul_rn(d1, d1)), mul_rn(d2, d2)));
    return mul_rn(C, v);
}

// Massive particles (m2 = m^2 > 0): v_rel is the Moller velocity
// sqrt((p_i.p_j)^2 - m^4) / (E_i E_j), p_i.p_j = E_i E_j - p_i.p_j (3-vectors),
// written sqrt((F - m^2)(F + m^2)) / (E_i E_j), 0 where rounding gives F < m^2.
template <typename T>
__device__ __forceinline__ T p22_massive(T C, T m2, const T mi[3], const T mj[3])
{
    const T Ei = sqrt_rn(add_rn(add_rn(add_rn(mul_rn(mi[0], mi[0]), mul_rn(mi[1], mi[1])), mul_rn(mi[2], mi[2])), m2));
    const T Ej = sqrt_rn(add_rn(add_rn(add_rn(mul_rn(mj[0], mj[0]), mul_rn(mj[1], mj[1])), mul_rn(mj[2], mj[2])), m2));
    const T dot = add_rn(add_rn(mul_rn(mi[0], mj[0]), mul_rn(mi[1], mj[1])), mul_rn(mi[2], mj[2]));
    const T EE = mul_rn(Ei, Ej);
    const T F = sub_rn(EE, dot);
    const T a = sub_rn(F, m2);
    if (!(a > T(0))) return T(0);
    return mul_rn(C, div_rn(sqrt_rn(mul_rn(a, add_rn(F, m2))), EE));
}

template <typename T>
__device__ __forceinline__ void load_mom(const T* __restrict__ st, uint32_t pcap, uint32_t g, T m[3])
{
    m[0] = st[3 * (size_t)pcap + g];
    m[1] = st[4 * (size_t)pcap + g];
    m[2] = st[5 * (size_t)pcap + g];
}

template <typename T>
__device__ __forceinline__ T pair_p22(T C, T m2, const T* __restrict__ st, uint32_t pcap, uint32_t gi, uint32_t gj)
{
    if (m2 > T(0)) {
        T mi[3], mj[3];
        load_mom<T>(st, pcap, gi, mi);
        load_mom<T>(st, pcap, gj, mj);
        return p22_massive<T>(C, m2, mi, mj);
    }
    T ui[3], uj[3];
    unit_dir<T>(st, pcap, gi, ui);
    unit_dir<T>(st, pcap, gj, uj);
    return p22_of_units<T>(C, ui, uj);
}

// Exact per-byte test of one word: bit b of the result (b = 0..3) is set iff
// byte b <= thr.  With bit 7 of every byte forced on, subtracting m cannot
// borrow across bytes; a byte is below m iff the difference drops bit 7 and
// the byte itself had bit 7 clear.  The four flags are then gathered by one
// multiply (their shifted copies land on distinct bit positions).
__device__ __forceinline__ uint32_t word_le_mask(uint32_t x, uint32_t thr)
{
    const uint32_t t = 0x01010101u * (thr + 1u);
    const uint32_t lt = ~((x | 0x80808080u) - t) & ~x & 0x80808080u;
    return (((lt >> 7) * 0x00204081u) >> 21) & 0xFu;
}

// 16-bit mask of the bytes <= thr of a block (bit 4 w + b = byte b of word w).
__device__ __forceinline__ uint32_t block_le_mask(uint4 r, uint32_t thr)
{
    if (thr >= 128u) return 0xFFFFu;
    return word_le_mask(r.x, thr) | (word_le_mask(r.y, thr) << 4) | (word_le_mask(r.z, thr) << 8) |
           (word_le_mask(r.w, thr) << 12);
}

// Columns j = 16 g + b of row i that are real pairs (i < j < n), as a mask.
__device__ __forceinline__ uint32_t valid_cols(uint32_t g, uint32_t i, uint32_t n)
{
    const int base = (int)(16u * g);
    int lo = (int)i + 1 - base;
    int hi = (int)n - base;
    lo = lo < 0 ? 0 : (lo > 16 ? 16 : lo);
    hi = hi < 0 ? 0 : (hi > 16 ? 16 : hi);
    if (hi <= lo) return 0u;
    return ((1u << hi) - 1u) & ~((1u << lo) - 1u);
}

__device__ __forceinline__ uint32_t block_byte(uint4 r, uint32_t bit)
{
    const uint32_t w = (bit >> 2) == 0 ? r.x : (bit >> 2) == 1 ? r.y : (bit >> 2) == 2 ? r.z : r.w;
    return (w >> (8u * (bit & 3u))) & 0xFFu;
}

// Could some pair of a block survive both random-byte filters?  The 16
// prefixes r16 = (top byte << 8) | middle byte of the block r and its
// middle-byte block mb, as 16-bit fields (byte_perm), are tested against
// thr16 all at once: a field below t = thr16 + 1 <= 0x8000 drops bit 15 in
// (f | 0x8000) - t without a borrow into the next field.  r16 <= thr16
// implies top byte <= thr8, so a false answer is exact; thr16 >= 0x7FFF
// (2.0001 C >= 1/2) always answers true.
__device__ __forceinline__ bool prefix16_any(uint4 r, uint4 mb, uint32_t thr16)
{
    if (thr16 >= 0x7FFFu) return true;
    const uint32_t t16 = 0x00010001u * (thr16 + 1u);
    const uint32_t rw[4] = {r.x, r.y, r.z, r.w}, mw[4] = {mb.x, mb.y, mb.z, mb.w};
    uint32_t any = 0;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const uint32_t lo = __byte_perm(mw[w], rw[w], 0x5140);   // fields (r0 m0), (r1 m1)
        const uint32_t hi = __byte_perm(mw[w], rw[w], 0x7362);   // fields (r2 m2), (r3 m3)
        any |= ~((lo | 0x80008000u) - t16) & ~lo;
        any |= ~((hi | 0x80008000u) - t16) & ~hi;
    }
    return (any & 0x80008000u) != 0;
}

struct CellCtx {
    uint32_t c;       // global cell
    uint32_t lc;      // cell index inside its simulation
    uint32_t cbase;   // first particle of the cell
    uint32_t n;       // particles in the cell
    uint32_t list0;   // first slot of the cell's accepted-list segment
    uint32_t room;    // slots in the segment
    int s;            // simulation
    uint32_t slot;    // its counters row
};

// Append accepted pair (i, j) to its cell's list; kMark: the cell's first
// accepted pair enters it in the active-cell list.
template <bool kMark>
__device__ __forceinline__ void append_accepted(const CellCtx& cc, uint32_t i, uint32_t j,
                                                uint32_t* __restrict__ acc_count,
                                                unsigned long long* __restrict__ acc, uint64_t acc_cap,
                                                uint32_t* __restrict__ counters, uint32_t* __restrict__ active,
                                                unsigned long long* __restrict__ stats)
{
    const uint32_t slot = atomicAdd(&acc_count[cc.c], 1u);
    if (kMark && slot == 0) active[atomicAdd(&counters[2], 1u)] = cc.c;
    if (slot < cc.room && (uint64_t)cc.list0 + slot < acc_cap) {
        acc[(size_t)cc.list0 + slot] = ((unsigned long long)i << 32) | j;
    } else {
        atomicOr(&counters[1], kErrAccOverflow);
        atomicAdd(&stats[cc.slot * kStatCount + kStatOverflow], 1ull);
    }
}

// Survivors of both random-byte filters (r16 <= thr16, about one pair in
// 2^16) need their low 16 random bits and the momenta: they are collected
// per warp in shared memory and written in bulk to a global list, which
// k_pair_finish evaluates with one thread per survivor, so that no warp of
// the pair tile waits on their momentum loads.  A record is (cell, i, j,
// r16 | kMark << 31).  Where a buffer is full the survivor is evaluated in
// place: the decisions are the same either way.
constexpr uint32_t kSurvBuf = 64;     // per-warp shared-memory survivors
constexpr uint32_t kSurvFlush = 32;   // flushed to the global list from this many

template <typename T, bool kMark>
__device__ __forceinline__ void eval_survivor(const CellCtx& cc, const PhiloxKey& K, uint32_t step, T C, T m2,
                                              const T* __restrict__ st, uint32_t pcap, uint32_t i, uint32_t j,
                                              uint32_t r16, uint32_t* __restrict__ acc_count,
                                              unsigned long long* __restrict__ acc, uint64_t acc_cap,
                                              uint32_t* __restrict__ counters, uint32_t* __restrict__ active,
                                              unsigned long long* __restrict__ stats)
{
    // u = unit_u(r16 << 16 | fine >> 16) lies between the values of the
    // lowest and the highest 16 low bits (the conversion rounds monotonically
    // and the scaling by 2^-32 is exact), so the low bits are drawn only when
    // P22 falls between those two: the same decision as u < P22 in every case.
    const T P = pair_p22<T>(C, m2, st, pcap, cc.cbase + i, cc.cbase + j);
    if (!(P > unit_u<T>(r16 << 16))) return;
    bool acc_it = unit_u<T>((r16 << 16) | 0xFFFFu) < P;
    if (!acc_it) {
        const uint32_t fine = philox4x32_10(make_uint4(step, cc.lc, i, kTagFine | j), K).x;
        acc_it = unit_u<T>((r16 << 16) | (fine >> 16)) < P;
    }
    if (acc_it) append_accepted<kMark>(cc, i, j, acc_count, acc, acc_cap, counters, active, stats);
}

// A survivor record evaluated on its own (its cell's context reloaded).
template <typename T, bool kOneKey>
__device__ __forceinline__ void finish_survivor(uint4 e, const SimDesc* __restrict__ sims, int nsims,
                                                const T* __restrict__ st, uint32_t pcap,
                                                const uint32_t* __restrict__ cell_start,
                                                const uint2* __restrict__ work, uint32_t* __restrict__ acc_count,
                                                unsigned long long* __restrict__ acc, uint64_t acc_cap,
                                                uint32_t* __restrict__ counters, uint32_t* __restrict__ active,
                                                unsigned long long* __restrict__ stats, const PhiloxKey& Kp)
{
    CellCtx cc;
    cc.c = e.x;
    cc.s = sim_of_cell(sims, nsims, e.x);
    const SimDesc& S = sims[cc.s];
    cc.slot = S.stat_slot;
    cc.lc = e.x - S.cell_off;
    cc.cbase = cell_start[e.x];
    cc.n = cell_start[e.x + 1] - cc.cbase;
    const uint2 w0 = work[e.x], w1 = work[e.x + 1];
    cc.list0 = w0.y;
    cc.room = w1.y - w0.y;
    const PhiloxKey Kl = kOneKey ? PhiloxKey{} : philox_schedule(S.key0, S.key1);
    const PhiloxKey& K = kOneKey ? Kp : Kl;
    if (e.w >> 31)
        eval_survivor<T, true>(cc, K, S.step, sim_C<T>(S), sim_m2<T>(S), st, pcap, e.y, e.z, e.w & 0xFFFFu, acc_count,
                               acc, acc_cap, counters, active, stats);
    else
        eval_survivor<T, false>(cc, K, S.step, sim_C<T>(S), sim_m2<T>(S), st, pcap, e.y, e.z, e.w & 0xFFFFu,
                                acc_count, acc, acc_cap, counters, active, stats);
}

// The warp's buffer count gets this bit once the global list is full: every
// later push then finds pos >= kSurvBuf and evaluates in place, and the
// records left in the buffer are evaluated when the warp finishes.
constexpr uint32_t kSurvFull = 0x80000000u;

// Warp-collective: move the warp's buffered survivors to the global list
// (counters[3] counts them).  Records past its capacity stay at the front of
// the buffer, *left of them, and the buffer is marked full.
__device__ __forceinline__ void flush_survivors(uint4* sv, uint32_t* svn, uint32_t* left, uint4* __restrict__ surv,
                                                uint32_t surv_cap, uint32_t* __restrict__ counters)
{
    const uint32_t lane = threadIdx.x & 31;
    __syncwarp();
    const uint32_t v = *svn;
    if (v == 0 || (v & kSurvFull)) return;
    const uint32_t n = min(v, kSurvBuf);
    uint32_t base = 0;
    if (lane == 0) {
        // once the list is full the counter stops growing (no 32-bit wrap
        // however many survivors a step has)
        const uint32_t cur = *reinterpret_cast<volatile uint32_t*>(&counters[3]);
        base = cur >= surv_cap ? surv_cap : atomicAdd(&counters[3], n);
    }
    base = __shfl_sync(kFull, base, 0);
    const uint32_t fit = base >= surv_cap ? 0u : min(n, surv_cap - base);
    uint4 e0 = make_uint4(0, 0, 0, 0), e1 = e0;
    if (lane < n) e0 = sv[lane];
    if (lane + 32 < n) e1 = sv[lane + 32];
    __syncwarp();
    if (lane < n) {
        if (lane < fit) surv[base + lane] = e0; else sv[lane - fit] = e0;
    }
    if (lane + 32 < n) {
        if (lane + 32 < fit) surv[base + lane + 32] = e1; else sv[lane + 32 - fit] = e1;
    }
    __syncwarp();
    if (lane == 0) {
        *svn = fit < n ? kSurvFull : 0u;
        *left = n - fit;
    }
    __syncwarp();
}

// Warp-collective, when the warp has no more work: flush, then evaluate in
// place whatever the full global list could not take.
template <typename T, bool kOneKey>
__device__ __forceinline__ void drain_survivors(uint4* sv, uint32_t* svn, uint32_t* left, uint4* __restrict__ surv,
                                                uint32_t surv_cap, const SimDesc* __restrict__ sims, int nsims,
                                                const T* __restrict__ st, uint32_t pcap,
                                                const uint32_t* __restrict__ cell_start,
                                                const uint2* __restrict__ work, uint32_t* __restrict__ acc_count,
                                                unsigned long long* __restrict__ acc, uint64_t acc_cap,
                                                uint32_t* __restrict__ counters, uint32_t* __restrict__ active,
                                                unsigned long long* __restrict__ stats, const PhiloxKey& Kp)
{
    flush_survivors(sv, svn, left, surv, surv_cap, counters);
    const uint32_t n = *left;
    for (uint32_t k = threadIdx.x & 31; k < n; k += 32)
        finish_survivor<T, kOneKey>(sv[k], sims, nsims, st, pcap, cell_start, work, acc_count, acc, acc_cap, counters,
                                    active, stats, Kp);
}

// Resolve one queued block r of row i, group g: the bytes <= thr8 at real
// pairs j (i < j < n) are refined by the pair's middle byte, drawn from the
// block (step, cell, i, TAG_MID | g) shared by the 16 pairs of the group: a
// 16-bit prefix above thr16 also proves u_ij >= P22.  Only the rare
// survivors draw their low 16 bits (block (step, cell, i, TAG_FINE | j)),
// load momenta and evaluate P22 (in the warp's survivor buffer, or here when
// it is full); accepted pairs are appended to the cell's list.
template <typename T, bool kMark>
__device__ __forceinline__ void resolve_block(const CellCtx& cc, const PhiloxKey& K, uint32_t step, uint32_t thr8,
                                              uint32_t thr16, T C, T m2, const T* __restrict__ st, uint32_t pcap,
                                              uint4 r, uint32_t i, uint32_t g, uint4* sv, uint32_t* svn,
                                              uint32_t* __restrict__ acc_count,
                                              unsigned long long* __restrict__ acc, uint64_t acc_cap,
                                              uint32_t* __restrict__ counters, uint32_t* __restrict__ active,
                                              unsigned long long* __restrict__ stats)
{
    const uint4 mb = philox4x32_10(make_uint4(step, cc.lc, i, kTagMid | g), K);
    // the exact per-byte walk runs only for blocks with a flagged prefix (at
    // thr8 = thr16 = 0 about one pushed block in 250)
    if (!prefix16_any(r, mb, thr16)) return;
    uint32_t m = block_le_mask(r, thr8) & valid_cols(g, i, cc.n);
    while (m) {
        const uint32_t bit = (uint32_t)__ffs(m) - 1u;
        m &= m - 1u;
        const uint32_t r16 = (block_byte(r, bit) << 8) | block_byte(mb, bit);
        if (r16 > thr16) continue;
        const uint32_t j = 16u * g + bit;
        const uint32_t pos = atomicAdd(svn, 1u);
        if (pos < kSurvBuf)
            sv[pos] = make_uint4(cc.c, i, j, r16 | (kMark ? 0x80000000u : 0u));
        else
            eval_survivor<T, kMark>(cc, K, step, C, m2, st, pcap, i, j, r16, acc_count, acc, acc_cap, counters,
                                    active, stats);
    }
}

// Per-lane rings of the 32-row item kernel: lane L keeps the Philox blocks
// of its row that hold a byte <= thr8 (about one block in 16 at thr8 = 0) in
// its column of the ring, entry k at r[k][0][L] (the block) and r[k][1][L].x
// (its first-round word Z1 = A ^ group), so that a push is two predicated
// shared stores and one address increment per block, with no warp-wide vote.
// The warp drains the rings when a lane could not take NB more entries, and
// at the end of its rows.
constexpr int kRingDepth = 12;
struct __align__(16) PairRing {
    uint4 r[kRingDepth][2][32];   // [k][0][L]: the block, [k][1][L].x: its Z1
};
constexpr uint32_t kRingRowBytes = 2u * 32u * sizeof(uint4);  // r[k + 1][0][L] - r[k][0][L]
constexpr uint32_t kRingZOff = 32u * sizeof(uint4);          // r[k][1][L] - r[k][0][L]

// Push block r (first-round word z) onto this lane's ring iff its test word x
// has a bit of 0x80808080 set; ra: shared address of the lane's next entry.
__device__ __forceinline__ void ring_push(uint32_t x, uint32_t& ra, uint4 r, uint32_t z)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t.reg .b32 t;\n\t"
        "and.b32 t, %1, 0x80808080;\n\t"
        "setp.ne.u32 p, t, 0;\n\t"
        "@p st.shared.v4.u32 [%0], {%2, %3, %4, %5};\n\t"
        "@p st.shared.u32 [%0+%7], %6;\n\t"
        "@p add.u32 %0, %0, %8;\n\t}"
        : "+r"(ra)
        : "r"(x), "r"(r.x), "r"(r.y), "r"(r.z), "r"(r.w), "r"(z), "n"(kRingZOff), "n"(kRingRowBytes)
        : "memory");
}

// Warp-collective: resolve the cnt entries of every lane's ring (rows
// 32 rb + L), one entry per lane in compacted order: entry e of the warp
// belongs to the lane L with pre[L] <= e < pre[L + 1] (pre: exclusive prefix
// of the counts), found by a binary search over the lanes' prefixes.
template <typename T, bool kMark>
__device__ __forceinline__ void drain_ring(const CellCtx& cc, uint32_t rb, const PhiloxKey& K, uint32_t step,
                                           uint32_t thr8, uint32_t thr16, T C, T m2, const T* __restrict__ st,
                                           uint32_t pcap, const PairRing& ring, uint32_t A, uint32_t cnt, uint4* sv,
                                           uint32_t* svn, uint32_t* __restrict__ acc_count,
                                           unsigned long long* __restrict__ acc, uint64_t acc_cap,
                                           uint32_t* __restrict__ counters, uint32_t* __restrict__ active,
                                           unsigned long long* __restrict__ stats)
{
    const uint32_t lane = threadIdx.x & 31;
    uint32_t inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(kFull, inc, o);
        if (lane >= (uint32_t)o) inc += v;
    }
    const uint32_t pre = inc - cnt;
    const uint32_t total = __shfl_sync(kFull, inc, 31);
    __syncwarp();
    for (uint32_t base = 0; base < total; base += 32) {
        const uint32_t e = base + lane;
        uint32_t L = 0;
#pragma unroll
        for (uint32_t s = 16; s >= 1; s >>= 1) {
            const uint32_t pc = __shfl_sync(kFull, pre, L + s);
            if (pc <= e) L += s;
        }
        const uint32_t pL = __shfl_sync(kFull, pre, L);
        if (e < total) {
            const uint32_t k = e - pL;
            resolve_block<T, kMark>(cc, K, step, thr8, thr16, C, m2, st, pcap, ring.r[k][0][L], rb * kPairRows + L,
                                    ring.r[k][1][L].x ^ A, sv, svn, acc_count, acc, acc_cap, counters, active, stats);
        }
    }
    __syncwarp();
}

// All pairs (i, j), i < j, of the rows [32 rb, 32 rb + 32) of one cell: one
// lane per row walks the row's 16-pair Philox blocks NB at a time (2, 4 or 8,
// by the launch shape); blocks holding a byte <= thr8 go to the lane's ring
// and are resolved when the warp drains it.  kMark: the first accepted pair of
// the cell appends it to the active-cell list (the small-cell path finds its
// cells by scanning).
template <typename T, bool kMark, int NB>
__device__ __forceinline__ void pair_rows(const CellCtx& cc, uint32_t rb, uint32_t step, uint32_t thr8, uint32_t thr16,
                                          T C, T m2, const PhiloxKey& K, const T* __restrict__ st, uint32_t pcap,
                                          PairRing& ring, uint4* sv, uint32_t* svn,
                                          uint32_t* __restrict__ acc_count,
                                          unsigned long long* __restrict__ acc, uint64_t acc_cap,
                                          uint32_t* __restrict__ counters, uint32_t* __restrict__ active,
                                          unsigned long long* __restrict__ stats)
{
    static_assert(NB <= kRingDepth, "a lane pushes up to NB blocks per iteration");
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t i = rb * kPairRows + lane;
    const bool row_ok = i + 1 < cc.n;
    PhiloxRow R;
    R.init(step, cc.lc, i, K);
    const uint32_t gfirst = (rb * kPairRows + 1) >> 4;
    const uint32_t glast = (cc.n - 1) >> 4;
    // Some byte of a word x is below m = thr8 + 1 <= 128 iff (x - m 0x01010101)
    // & ~x has a bit 7 set (a borrow only adds flags above a true one, so the
    // "any" answer is exact).  Rows without partners test against m = 0,
    // which flags nothing; thr8 >= 128 flags every block of a row with
    // partners.  Blocks of pairs outside i < j < n (before the row's diagonal
    // or past the cell's end) may be pushed: the resolve drops their columns.
    const uint32_t t8 = row_ok ? 0x01010101u * (thr8 + 1u) : 0u;
    const uint32_t x0 = (row_ok && thr8 >= 128u) ? 0x80000000u : 0u;
    const uint32_t ra0 = (uint32_t)__cvta_generic_to_shared(&ring.r[0][0][lane]);
    // past ra_full a lane could not take NB more entries
    const uint32_t ra_full = ra0 + kRingRowBytes * (uint32_t)(kRingDepth - NB);
    uint32_t ra = ra0;
    // groups are walked from a multiple of NB, so that group g + b = g | b and
    // the first-round word of its block is (A ^ g) ^ b; blocks before the
    // row's first group are drawn and dropped by the resolve
    for (uint32_t g = gfirst & ~(uint32_t)(NB - 1); g <= glast; g += NB) {
        if (__any_sync(kFull, ra > ra_full)) {
            drain_ring<T, kMark>(cc, rb, K, step, thr8, thr16, C, m2, st, pcap, ring, R.A, (ra - ra0) / kRingRowBytes,
                                 sv, svn, acc_count, acc, acc_cap, counters, active, stats);
            ra = ra0;
        }
        const uint32_t Ag = R.A ^ g;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const uint32_t z = Ag ^ (uint32_t)b;
            const uint4 r = R.block_z(z, K);
            const uint32_t x = ((r.x - t8) & ~r.x) | ((r.y - t8) & ~r.y) | ((r.z - t8) & ~r.z) |
                               ((r.w - t8) & ~r.w) | x0;
            ring_push(x, ra, r, z);
        }
    }
    if (__any_sync(kFull, ra != ra0))
        drain_ring<T, kMark>(cc, rb, K, step, thr8, thr16, C, m2, st, pcap, ring, R.A, (ra - ra0) / kRingRowBytes, sv,
                             svn, acc_count, acc, acc_cap, counters, active, stats);
}

// Per-lane rings of the small-cell kernel: entry k of lane L holds the block
// at r[k][0][L] and its tag (row i, cell, (n << 8) | group, simulation) at
// r[k][1][L].  Same entry layout as PairRing, so a push is two predicated
// shared stores and one address increment.
constexpr int kSmallRingDepth = 7;
struct __align__(16) SmallRing {
    uint4 r[kSmallRingDepth][2][32];
};

__device__ __forceinline__ void small_ring_push(uint32_t x, uint32_t& ra, uint4 r, uint4 tag)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t.reg .b32 t;\n\t"
        "and.b32 t, %1, 0x80808080;\n\t"
        "setp.ne.u32 p, t, 0;\n\t"
        "@p st.shared.v4.u32 [%0], {%2, %3, %4, %5};\n\t"
        "@p st.shared.v4.u32 [%0+%10], {%6, %7, %8, %9};\n\t"
        "@p add.u32 %0, %0, %11;\n\t}"
        : "+r"(ra)
        : "r"(x), "r"(r.x), "r"(r.y), "r"(r.z), "r"(r.w), "r"(tag.x), "r"(tag.y), "r"(tag.z), "r"(tag.w),
          "n"(kRingZOff), "n"(kRingRowBytes)
        : "memory");
}

// Step, cell offset and thresholds of a one-simulation arena, kernel-wide.
struct OneSim {
    uint32_t step, cell_off, thr8, thr16;
};

// Resolve one ringed block of a small cell: the bytes <= thr8 at real pairs
// j (i < j < n, n carried in the tag) are found first; only a block with one
// draws its middle-byte block (step, cell, i, TAG_MID | g), and the pairs
// whose 16-bit prefix is <= thr16 become survivors (the warp's buffer, or
// evaluated here when it is full).
template <typename T, bool kOneKey>
__device__ __forceinline__ void resolve_small(uint4 r, uint4 tag, const OneSim& one,
                                              const SimDesc* __restrict__ sims, const T* __restrict__ st,
                                              uint32_t pcap, const uint32_t* __restrict__ cell_start,
                                              const uint2* __restrict__ work, uint4* sv, uint32_t* svn,
                                              uint32_t* __restrict__ acc_count, unsigned long long* __restrict__ acc,
                                              uint64_t acc_cap, uint32_t* __restrict__ counters,
                                              uint32_t* __restrict__ active, unsigned long long* __restrict__ stats,
                                              const PhiloxKey& Kp)
{
    const uint32_t i = tag.x, c = tag.y, g = tag.z & 0xFFu, n = tag.z >> 8;
    uint32_t step = one.step, off_c = one.cell_off, thr8 = one.thr8, thr16 = one.thr16;
    if (!kOneKey) {
        const SimDesc& S = sims[tag.w];
        step = S.step;
        off_c = S.cell_off;
        thr8 = S.thr8;
        thr16 = S.thr16;
    }
    uint32_t m = block_le_mask(r, thr8) & valid_cols(g, i, n);
    if (!m) return;
    PhiloxKey Kl;
    if (!kOneKey) Kl = philox_schedule(sims[tag.w].key0, sims[tag.w].key1);
    const PhiloxKey& K = kOneKey ? Kp : Kl;
    const uint4 mb = philox4x32_10(make_uint4(step, c - off_c, i, kTagMid | g), K);
    while (m) {
        const uint32_t bit = (uint32_t)__ffs(m) - 1u;
        m &= m - 1u;
        const uint32_t r16 = (block_byte(r, bit) << 8) | block_byte(mb, bit);
        if (r16 > thr16) continue;
        const uint32_t j = 16u * g + bit;
        const uint32_t pos = atomicAdd(svn, 1u);
        if (pos < kSurvBuf) {
            sv[pos] = make_uint4(c, i, j, r16);
        } else {
            const int s = kOneKey ? 0 : (int)tag.w;
            const SimDesc& S = sims[s];
            CellCtx cc;
            cc.c = c;
            cc.s = s;
            cc.slot = S.stat_slot;
            cc.lc = c - off_c;
            cc.cbase = cell_start[c];
            cc.n = n;
            const uint2 w0 = work[c], w1 = work[c + 1];
            cc.list0 = w0.y;
            cc.room = w1.y - w0.y;
            eval_survivor<T, false>(cc, K, step, sim_C<T>(S), sim_m2<T>(S), st, pcap, i, j, r16, acc_count, acc,
                                    acc_cap, counters, active, stats);
        }
    }
}

// Warp-collective: resolve the cnt entries of every lane's ring, one entry
// per lane in compacted order (the owner of entry e found by a binary search
// over the lanes' exclusive prefixes, as in drain_ring).
template <typename T, bool kOneKey>
__device__ __forceinline__ void drain_small(const SmallRing& ring, uint32_t cnt, const OneSim& one,
                                            const SimDesc* __restrict__ sims, const T* __restrict__ st,
                                            uint32_t pcap, const uint32_t* __restrict__ cell_start,
                                            const uint2* __restrict__ work, uint4* sv, uint32_t* svn,
                                            uint32_t* __restrict__ acc_count, unsigned long long* __restrict__ acc,
                                            uint64_t acc_cap, uint32_t* __restrict__ counters,
                                            uint32_t* __restrict__ active, unsigned long long* __restrict__ stats,
                                            const PhiloxKey& Kp)
{
    const uint32_t lane = threadIdx.x & 31;
    uint32_t inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(kFull, inc, o);
        if (lane >= (uint32_t)o) inc += v;
    }
    const uint32_t pre = inc - cnt;
    const uint32_t total = __shfl_sync(kFull, inc, 31);
    __syncwarp();
    for (uint32_t base = 0; base < total; base += 32) {
        const uint32_t e = base + lane;
        uint32_t L = 0;
#pragma unroll
        for (uint32_t s = 16; s >= 1; s >>= 1) {
            const uint32_t pc = __shfl_sync(kFull, pre, L + s);
            if (pc <= e) L += s;
        }
        const uint32_t pL = __shfl_sync(kFull, pre, L);
        if (e < total) {
            const uint32_t k = e - pL;
            resolve_small<T, kOneKey>(ring.r[k][0][L], ring.r[k][1][L], one, sims, st, pcap, cell_start, work, sv,
                                      svn, acc_count, acc, acc_cap, counters, active, stats, Kp);
        }
    }
    __syncwarp();
}

// ---------------------------------------------------------------------------
// A5, skip-ahead mode
// ---------------------------------------------------------------------------
// Gap of the skip-ahead mode: with M columns left after the last candidate,
// the largest G < 2^(bt+1), bt = ceil(log2 M), whose 0.64 fixed-point power
// q^G — built greedily from bit bt down with the table Q[b] = q^(2^b) — is
// still >= U.  P(G >= k) = q^k up to rounding: the inverse CDF of the
// geometric distribution of the gap between Bernoulli(1 - q) candidates.
// G >= M means no candidate is left in the row.
__device__ __forceinline__ uint64_t skip_gap(const uint64_t* __restrict__ Q, uint64_t U, uint32_t M)
{
    const int bt = M <= 1u ? 0 : 32 - __clz(M - 1u);
    uint64_t G = 0, Qc = ~0ull;
    for (int b = bt; b >= 0; --b) {
        const uint64_t t = __umul64hi(Qc, Q[b]);
        if (t >= U) {
            Qc = t;
            G += 1ull << b;
            if (G >= M) break;  // G only grows: the row has ended
        }
    }
    return G;
}

template <typename T> __device__ __forceinline__ T skip_pmax(const SimDesc& S);
template <> __device__ __forceinline__ double skip_pmax<double>(const SimDesc& S) { return S.pmax; }
template <> __device__ __forceinline__ float skip_pmax<float>(const SimDesc& S) { return S.pmaxf; }

// Rows [32 rb, 32 rb + 32) of one cell in the skip-ahead mode, one row per
// lane: the k-th draw of row i is the Philox block (step, cell, i,
// TAG_SKIP | k) — words 0 and 1 the 64-bit uniform of the gap, word 2 the
// thinning uniform; candidate j is kept iff (w 2^-32) P_max < P22 in the
// state's precision, i.e. with probability P22 / P_max.
// Returns this lane's number of candidates.
template <typename T, bool kMark>
__device__ __forceinline__ uint32_t skip_rows(const CellCtx& cc, uint32_t rb, const SimDesc& S, T C,
                                              const PhiloxKey& K, const T* __restrict__ st, uint32_t pcap,
                                              uint32_t* __restrict__ acc_count, unsigned long long* __restrict__ acc,
                                              uint64_t acc_cap, uint32_t* __restrict__ counters,
                                              uint32_t* __restrict__ active, unsigned long long* __restrict__ stats)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t i = rb * kPairRows + lane;
    uint32_t cand = 0;
    if (i + 1 < cc.n) {
        const T m2 = sim_m2<T>(S);
        T ui[3], mi[3];
        if (m2 > T(0)) load_mom<T>(st, pcap, cc.cbase + i, mi);
        else unit_dir<T>(st, pcap, cc.cbase + i, ui);  // row particle, loaded once (coalesced over the lanes)
        PhiloxRow R;
        R.init(S.step, cc.lc, i, K);
        const T pm = skip_pmax<T>(S);
        uint32_t pos = i;
        for (uint32_t k = 0;; ++k) {
            const uint32_t M = cc.n - 1u - pos;
            if (M == 0) break;
            const uint4 w = R.block(kTagSkip | k, K);
            const uint64_t G = skip_gap(S.skipQ, ((uint64_t)w.x << 32) | w.y, M);
            if (G >= M) break;
            const uint32_t j = pos + 1u + (uint32_t)G;
            ++cand;
            const T u = mul_rn(unit_u<T>(w.z), pm);
            T P;
            if (m2 > T(0)) {
                T mj[3];
                load_mom<T>(st, pcap, cc.cbase + j, mj);
                P = p22_massive<T>(C, m2, mi, mj);
            } else {
                T uj[3];
                unit_dir<T>(st, pcap, cc.cbase + j, uj);
                P = p22_of_units<T>(C, ui, uj);
            }
            if (u < P) append_accepted<kMark>(cc, i, j, acc_count, acc, acc_cap, counters, active, stats);
            pos = j;
        }
    }
    return cand;
}

// Skip-ahead cells (A5 in the skip-ahead mode): one warp per 32-row block,
// blocks taken grid-stride from the scanned per-cell counts skip_work (no
// work counter: the rows cost about the same).  Cells above small_max enter
// the active list (the per-cell resolve), smaller ones are found by the
// warp-per-cell resolve.  Candidates are summed per warp and simulation.
template <typename T, bool kOneKey>
__global__ void __launch_bounds__(kPairThreads, 4)
    k_pair_skip(const SimDesc* __restrict__ sims, int nsims, const T* __restrict__ st, uint32_t pcap,
                const uint32_t* __restrict__ cell_start, const uint2* __restrict__ work,
                const uint32_t* __restrict__ skip_work, uint32_t ncells, uint32_t small_max,
                uint32_t* __restrict__ acc_count, unsigned long long* __restrict__ acc, uint64_t acc_cap,
                uint32_t* __restrict__ counters, uint32_t* __restrict__ active, unsigned long long* __restrict__ stats,
                const PhiloxKey Kp)
{
    if ((uint64_t)work[ncells].y > acc_cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&counters[1], kErrCapacity);
        return;
    }
    const uint32_t total = skip_work[ncells];
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    // a contiguous range of row blocks per warp: consecutive rows of a cell
    const uint32_t per = (total + nw - 1) / nw;
    const uint32_t i0 = min(total, gw * per), i1 = min(total, i0 + per);
    uint32_t cur_slot = 0xFFFFFFFFu, cand = 0;
    uint32_t c = 0;
    if (i0 < i1) {
        // cell of the first item: the last c with skip_work[c] <= i0
        uint32_t lo = 0, hi = ncells - 1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (skip_work[mid] <= i0) lo = mid; else hi = mid - 1;
        }
        c = lo;
    }
    for (uint32_t item = i0; item < i1; ++item) {
        while (skip_work[c + 1] <= item) ++c;
        CellCtx cc;
        cc.c = c;
        cc.s = sim_of_cell(sims, nsims, c);
        const SimDesc& S = sims[cc.s];
        cc.slot = S.stat_slot;
        cc.lc = c - S.cell_off;
        cc.cbase = cell_start[c];
        cc.n = cell_start[c + 1] - cc.cbase;
        const uint2 w0 = work[c], w1 = work[c + 1];
        cc.list0 = w0.y;
        cc.room = w1.y - w0.y;
        if (cc.slot != cur_slot) {
            const unsigned tot = __reduce_add_sync(kFull, cand);
            if (lane == 0 && tot) atomicAdd(&stats[cur_slot * kStatCount + kStatCandidates], (unsigned long long)tot);
            cand = 0;
            cur_slot = cc.slot;
        }
        const PhiloxKey Kl = kOneKey ? PhiloxKey{} : philox_schedule(S.key0, S.key1);
        const PhiloxKey& K = kOneKey ? Kp : Kl;
        const uint32_t rb = item - skip_work[c];
        if (cc.n > small_max)
            cand += skip_rows<T, true>(cc, rb, S, sim_C<T>(S), K, st, pcap, acc_count, acc, acc_cap, counters,
                                       active, stats);
        else
            cand += skip_rows<T, false>(cc, rb, S, sim_C<T>(S), K, st, pcap, acc_count, acc, acc_cap, counters,
                                        active, stats);
    }
    const unsigned tot = __reduce_add_sync(kFull, cand);
    if (lane == 0 && tot) atomicAdd(&stats[cur_slot * kStatCount + kStatCandidates], (unsigned long long)tot);
}

// kOneKey: every cell belongs to one simulation whose round keys come as the
// kernel parameter Kp (constant-bank operands, no registers); otherwise each
// cell's key schedule is derived from its descriptor.
template <typename T, bool kOneKey, int NB>
__global__ void __launch_bounds__(kPairThreads, PairShape<kOneKey, NB>::min_blocks)
    k_pair_tile(const SimDesc* __restrict__ sims, int nsims, const T* __restrict__ st, uint32_t pcap,
                const uint32_t* __restrict__ cell_start, const uint2* __restrict__ work, uint32_t ncells,
                uint32_t* __restrict__ acc_count, unsigned long long* __restrict__ acc, uint64_t acc_cap,
                uint32_t* __restrict__ counters, uint32_t* __restrict__ active, unsigned long long* __restrict__ stats,
                uint4* __restrict__ surv, uint32_t surv_cap, const PhiloxKey Kp)
{
    constexpr int kWarps = kPairThreads / 32;
    extern __shared__ __align__(16) unsigned char pair_smem[];
    PairRing* ring = reinterpret_cast<PairRing*>(pair_smem);
    __shared__ uint4 s_v[kWarps][kSurvBuf];
    __shared__ uint32_t s_vn[kWarps], s_left[kWarps];
    const int w = threadIdx.x >> 5;
    const uint32_t lane = threadIdx.x & 31;
    if (lane == 0) s_vn[w] = s_left[w] = 0;
    __syncwarp();
    const uint32_t total = work[ncells].x;
    if ((uint64_t)work[ncells].y > acc_cap) {
        // the lists of this step do not fit the allocation: report, do nothing
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&counters[1], kErrCapacity);
        return;
    }
    uint32_t c = 0;  // search hint: items are handed out in increasing order

    for (;;) {
        uint32_t item = 0;
        if (lane == 0) item = atomicAdd(&counters[0], 1u);
        item = __shfl_sync(kFull, item, 0);
        if (item >= total) break;
        // cell of the item: the last c with work[c].x <= item.  Gallop from
        // the previous cell (work[c].x <= item holds there), then bisect.
        {
            uint32_t lo = c, stride = 1, hi = c + 1;
            while (hi < ncells && work[hi].x <= item) {
                lo = hi;
                stride <<= 1;
                hi = lo + stride;
            }
            uint32_t b = (hi < ncells ? hi : ncells) - 1;
            while (lo < b) {
                const uint32_t mid = (lo + b + 1) >> 1;
                if (work[mid].x <= item) lo = mid; else b = mid - 1;
            }
            c = lo;
        }
        CellCtx cc;
        cc.c = c;
        cc.s = sim_of_cell(sims, nsims, c);
        const SimDesc& S = sims[cc.s];
        cc.slot = S.stat_slot;
        const uint2 w0 = work[c], w1 = work[c + 1];
        cc.lc = c - S.cell_off;
        cc.cbase = cell_start[c];
        cc.n = cell_start[c + 1] - cc.cbase;
        cc.list0 = w0.y;
        cc.room = w1.y - w0.y;
        const uint32_t rb = item - w0.x;
        const PhiloxKey Kl = kOneKey ? PhiloxKey{} : philox_schedule(S.key0, S.key1);
        const PhiloxKey& K = kOneKey ? Kp : Kl;
        pair_rows<T, true, NB>(cc, rb, S.step, S.thr8, S.thr16, sim_C<T>(S), sim_m2<T>(S), K, st, pcap, ring[w],
                               s_v[w], &s_vn[w], acc_count, acc, acc_cap, counters, active, stats);
        __syncwarp();
        if (s_vn[w] - kSurvFlush < kSurvFull - kSurvFlush)
            flush_survivors(s_v[w], &s_vn[w], &s_left[w], surv, surv_cap, counters);
    }
    drain_survivors<T, kOneKey>(s_v[w], &s_vn[w], &s_left[w], surv, surv_cap, sims, nsims, st, pcap, cell_start, work,
                                acc_count, acc, acc_cap, counters, active, stats, Kp);
}

// Small cells (2 <= n <= small_max): each warp takes 32 cells at a time
// (grid-stride), one per lane.  Row i of a cell with G = (n - 1) >> 4 draws
// the blocks of groups (i + 1) >> 4 .. G: rows of one band h = (i + 1) >> 4
// draw m = G + 1 - h blocks each.  The warp walks m = 1, 2, ... and for each
// m takes the band with m blocks per row of each of its cells as one flat
// row list, 32 rows per round, one per lane: every lane draws exactly m
// blocks in a round (no lane waits for a longer row) and builds its row's
// Philox constants once for them.  Lane L's row is the (t + L)-th of the
// list: its cell comes from the cells whose band starts inside the round
// (one bit each, OR-reduced over the warp) and the rank of the cell holding
// the row before the round.  Blocks with a byte <= thr8 go to the lane's ring
// (dynamic shared memory, one SmallRing per warp), drained when some lane
// could not take NB more entries.
template <typename T, bool kOneKey, int NB>
__global__ void __launch_bounds__(kPairThreads, 3) k_pair_small(const SimDesc* __restrict__ sims, int nsims,
                                                             const T* __restrict__ st, uint32_t pcap,
                                                             const uint32_t* __restrict__ cell_start,
                                                             const uint2* __restrict__ work, uint32_t ncells,
                                                             uint32_t small_max, uint32_t* __restrict__ acc_count,
                                                             unsigned long long* __restrict__ acc, uint64_t acc_cap,
                                                             uint32_t* __restrict__ counters,
                                                             uint32_t* __restrict__ active,
                                                             unsigned long long* __restrict__ stats,
                                                             uint4* __restrict__ surv, uint32_t surv_cap,
                                                             const PhiloxKey Kp)
{
    constexpr int kWarps = kPairThreads / 32;
    extern __shared__ __align__(16) unsigned char small_smem[];
    __shared__ uint4 s_v[kWarps][kSurvBuf];
    __shared__ uint4 s_band[kWarps][32];  // (cell, first row in the list, first row i | n << 16, simulation)
    __shared__ uint32_t s_vn[kWarps], s_left[kWarps];
    const int w = threadIdx.x >> 5;
    const uint32_t lane = threadIdx.x & 31;
    SmallRing& ring = reinterpret_cast<SmallRing*>(small_smem)[w];
    if (lane == 0) s_vn[w] = s_left[w] = 0;
    __syncwarp();
    if ((uint64_t)work[ncells].y > acc_cap) return;  // reported by k_pair_tile
    // one simulation: its step, cell offset and thresholds are kernel-wide
    const OneSim one{sims[0].step, sims[0].cell_off, sims[0].thr8, sims[0].thr16};
    if (kOneKey && (!(sims[0].C > 0.0) || sims[0].skip)) return;  // skip-ahead cells: k_pair_skip
    const uint32_t lt = (1u << lane) - 1u, le = lt | (1u << lane);
    const uint32_t nwarps = gridDim.x * kWarps;
    const uint32_t ra0 = (uint32_t)__cvta_generic_to_shared(&ring.r[0][0][lane]);
    const uint32_t ra_lim = ra0 + (uint32_t)(kSmallRingDepth - NB) * kRingRowBytes;  // room for NB more
    uint32_t ra = ra0;
    for (uint32_t c0 = (blockIdx.x * kWarps + w) * 32u; c0 < ncells; c0 += nwarps * 32u) {
        const uint32_t cl = c0 + lane;
        const uint32_t my_n = cl < ncells ? cell_start[cl + 1] - cell_start[cl] : 0u;
        bool ok = cl < ncells && my_n >= 2 && my_n <= small_max;
        int s = 0;
        if (!kOneKey && ok) {
            s = sim_of_cell(sims, nsims, cl);
            ok = sims[s].C > 0.0 && !sims[s].skip;
        }
        const uint32_t G = ok ? (my_n - 1u) >> 4 : 0u;
        const uint32_t mmax = __reduce_max_sync(kFull, ok ? G + 1u : 0u);
        for (uint32_t m = 1; m <= mmax; ++m) {
            // this cell's band with m blocks per row: h = G + 1 - m, rows
            // max(16 h - 1, 0) .. min(16 h + 14, n - 2)
            const bool in = ok && m <= G + 1u;
            const uint32_t h = G + 1u - m;
            const uint32_t lo = h ? 16u * h - 1u : 0u;
            const uint32_t hi = min(16u * h + 14u, my_n - 2u);
            const uint32_t cnt = in ? hi - lo + 1u : 0u;
            uint32_t E = cnt;  // inclusive prefix of the band sizes
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t v = __shfl_up_sync(kFull, E, d);
                if (lane >= (uint32_t)d) E += v;
            }
            const uint32_t total = __shfl_sync(kFull, E, 31);
            if (total == 0) continue;
            const uint32_t first = E - cnt;
            const unsigned has = __ballot_sync(kFull, cnt != 0);
            __syncwarp();
            if (cnt) s_band[w][__popc(has & lt)] = make_uint4(cl, first, lo | (my_n << 16), (uint32_t)s);
            __syncwarp();
            uint32_t rank_prev = ~0u;  // rank of the band holding the row before the round
            for (uint32_t t = 0; t < total; t += 32u) {
                const uint32_t off = first - t;  // wraps above 31 for bands starting before the round
                const uint32_t M = __reduce_or_sync(kFull, (cnt != 0 && off < 32u) ? 1u << off : 0u);
                // lanes past the list keep the last band's rank (no band starts there)
                const uint32_t rank = min(rank_prev + (uint32_t)__popc(M & le), 31u);
                rank_prev += (uint32_t)__popc(M);
                const uint32_t k = t + lane;
                const bool act = k < total;
                const uint4 be = s_band[w][rank];
                const uint32_t c = be.x;
                const uint32_t i = (be.z & 0xFFFFu) + (k - be.y);
                const uint32_t g0 = (i + 1u) >> 4;
                uint32_t step = one.step, off_c = one.cell_off, thr8 = one.thr8;
                PhiloxKey Kl;
                if (!kOneKey) {
                    const SimDesc& S = sims[be.w];
                    step = S.step;
                    off_c = S.cell_off;
                    thr8 = S.thr8;
                    Kl = philox_schedule(S.key0, S.key1);
                }
                const PhiloxKey& K = kOneKey ? Kp : Kl;
                PhiloxRow R;
                R.init(step, c - off_c, i, K);
                const uint32_t t8 = act ? 0x01010101u * (thr8 + 1u) : 0u;
                const uint32_t x0 = (act && thr8 >= 128u) ? 0x80000000u : 0u;
                const uint32_t tag_n = (be.z >> 16) << 8;
                for (uint32_t b = 0; b < m; b += NB) {
                    if (__any_sync(kFull, ra > ra_lim)) {
                        drain_small<T, kOneKey>(ring, (ra - ra0) / kRingRowBytes, one, sims, st, pcap, cell_start,
                                                work, s_v[w], &s_vn[w], acc_count, acc, acc_cap, counters, active,
                                                stats, Kp);
                        ra = ra0;
                        if (s_vn[w] - kSurvFlush < kSurvFull - kSurvFlush)
                            flush_survivors(s_v[w], &s_vn[w], &s_left[w], surv, surv_cap, counters);
                    }
#pragma unroll
                    for (int bb = 0; bb < NB; ++bb) {
                        if (bb > 0 && b + (uint32_t)bb >= m) break;  // warp-uniform
                        const uint32_t g = g0 + b + (uint32_t)bb;
                        const uint4 r = R.block(g, K);
                        const uint32_t x = ((r.x - t8) & ~r.x) | ((r.y - t8) & ~r.y) | ((r.z - t8) & ~r.z) |
                                           ((r.w - t8) & ~r.w) | x0;
                        small_ring_push(x, ra, r, make_uint4(i, c, tag_n | g, be.w));
                    }
                }
            }
        }
        __syncwarp();
        if (s_vn[w] - kSurvFlush < kSurvFull - kSurvFlush)
            flush_survivors(s_v[w], &s_vn[w], &s_left[w], surv, surv_cap, counters);
    }
    if (__any_sync(kFull, ra != ra0))
        drain_small<T, kOneKey>(ring, (ra - ra0) / kRingRowBytes, one, sims, st, pcap, cell_start, work, s_v[w],
                                &s_vn[w], acc_count, acc, acc_cap, counters, active, stats, Kp);
    drain_survivors<T, kOneKey>(s_v[w], &s_vn[w], &s_left[w], surv, surv_cap, sims, nsims, st, pcap, cell_start, work,
                                acc_count, acc, acc_cap, counters, active, stats, Kp);
}

// The survivors the pair kernels collected: one thread per record.
template <typename T, bool kOneKey>
__global__ void __launch_bounds__(256) k_pair_finish(const SimDesc* __restrict__ sims, int nsims,
                                                     const T* __restrict__ st, uint32_t pcap,
                                                     const uint32_t* __restrict__ cell_start,
                                                     const uint2* __restrict__ work, uint32_t ncells,
                                                     uint32_t* __restrict__ acc_count,
                                                     unsigned long long* __restrict__ acc, uint64_t acc_cap,
                                                     uint32_t* __restrict__ counters, uint32_t* __restrict__ active,
                                                     unsigned long long* __restrict__ stats,
                                                     const uint4* __restrict__ surv, uint32_t surv_cap,
                                                     const PhiloxKey Kp)
{
    if ((uint64_t)work[ncells].y > acc_cap) return;  // reported by k_pair_tile
    const uint32_t n = min(counters[3], surv_cap);
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
        finish_survivor<T, kOneKey>(surv[k], sims, nsims, st, pcap, cell_start, work, acc_count, acc, acc_cap,
                                    counters, active, stats, Kp);
}

// ---------------------------------------------------------------------------
// A6-A7
// ---------------------------------------------------------------------------

// Sorting network for m keys in place, ascending; positions >= m behave as
// +infinity and are never touched (flip/half-cleaner form of bitonic sort).
__device__ void bitonic_sort(unsigned long long* L, uint32_t m)
{
    uint32_t p2 = 1;
    while (p2 < m) p2 <<= 1;
    for (uint32_t k = 2; k <= p2; k <<= 1) {
        const uint32_t half = k >> 1;
        for (uint32_t t = threadIdx.x; t < p2 / 2; t += blockDim.x) {
            const uint32_t blk = t / half, off = t - blk * half;
            const uint32_t a = blk * k + off, b = blk * k + k - 1 - off;
            if (b < m) {
                const unsigned long long x = L[a], y = L[b];
                if (x > y) { L[a] = y; L[b] = x; }
            }
        }
        __syncthreads();
        for (uint32_t j = k >> 2; j >= 1; j >>= 1) {
            for (uint32_t t = threadIdx.x; t < p2 / 2; t += blockDim.x) {
                const uint32_t blk = t / j, off = t - blk * j;
                const uint32_t a = blk * 2 * j + off, b = a + j;
                if (b < m) {
                    const unsigned long long x = L[a], y = L[b];
                    if (x > y) { L[a] = y; L[b] = x; }
                }
            }
            __syncthreads();
        }
    }
}

template <typename R> __device__ __forceinline__ R word_unit(uint32_t w);
template <> __device__ __forceinline__ double word_unit<double>(uint32_t w) { return (double)w * 0x1p-32; }
template <> __device__ __forceinline__ float word_unit<float>(uint32_t w) { return __uint2float_rn(w) * 0x1p-32f; }
__device__ __forceinline__ void sincos_t(double x, double* s, double* c) { sincos(x, s, c); }
__device__ __forceinline__ void sincos_t(float x, float* s, float* c) { sincosf(x, s, c); }

// Invariant mass squared s of a pair of particles of mass m (m2 = m^2):
// massless 2 E_i E_j v_rel with v_rel in the unit-vector form, massive
// 2 m^2 + 2 (E_i E_j - p_i.p_j).  Ei, Ej receive the energies.
template <typename R>
__device__ __forceinline__ R pair_s(R m2, const R mi[3], const R mj[3], R& Ei, R& Ej)
{
    Ei = sqrt(((mi[0] * mi[0] + mi[1] * mi[1]) + mi[2] * mi[2]) + m2);
    Ej = sqrt(((mj[0] * mj[0] + mj[1] * mj[1]) + mj[2] * mj[2]) + m2);
    if (m2 > R(0)) {
        const R F = Ei * Ej - ((mi[0] * mj[0] + mi[1] * mj[1]) + mi[2] * mj[2]);
        return R(2) * m2 + R(2) * F;
    }
    R ui[3], uj[3];
    for (int a = 0; a < 3; ++a) {
        ui[a] = (Ei > R(0)) ? mi[a] / Ei : R(0);
        uj[a] = (Ej > R(0)) ? mj[a] / Ej : R(0);
    }
    const R d0 = ui[0] - uj[0], d1 = ui[1] - uj[1], d2 = ui[2] - uj[2];
    return ((R(2) * Ei) * Ej) * (R(0.5) * ((d0 * d0 + d1 * d1) + d2 * d2));
}

// Lorentz factor of the pair's centre-of-mass frame, gamma = E_t / sqrt(s).
template <typename R>
__device__ __forceinline__ R pair_gamma(R m2, const R mi[3], const R mj[3])
{
    R Ei, Ej;
    const R s = pair_s<R>(m2, mi, mj, Ei, Ej);
    if (!(Ei > R(0)) || !(Ej > R(0))) return R(0);
    return (s > R(4) * m2) ? (Ei + Ej) / sqrt(s) : R(0);
}

// Executed pair (Sec. 2): boost to the CM frame, direction from the Philox
// block (step, cell, i, TAG_ANGLE | j), boost back.  In the CM frame both
// particles carry E* = sqrt(s)/2 and momenta +-p*, |p*| = sqrt(E*^2 - m^2);
// p' = p* + beta (gamma^2 / (gamma + 1) (beta . p*) + gamma E*).  Isotropic
// (mu = 0): cos t = 2 u1 - 1 about the z axis.  Screened (mu > 0):
// dsigma/dt ~ 1/(t - mu^2)^2, t = -2 |p*|^2 (1 - cos t), x = 1 - cos t from
// the closed-form inverse CDF with a = 2 |p*|^2, A = 1/mu^2, B = 1/(2a + mu^2):
// x = (1/(A - u1 (A - B)) - mu^2) / a, measured from particle i's incoming
// CM direction, azimuth about it in the basis e1 = unit(h x e), e2 = e x e1
// (h = x^ if |e_x| < 0.9, else y^).
template <typename R>
__device__ __forceinline__ bool collide_pair(const PhiloxKey& K, uint32_t step, uint32_t lc, uint32_t i, uint32_t j,
                                             R m, R mu, R mi[3], R mj[3])
{
    const R m2 = m * m;
    R Ei, Ej;
    const R s = pair_s<R>(m2, mi, mj, Ei, Ej);
    if (!(s > R(4) * m2)) return false;
    const R rs = sqrt(s);
    const R Es = R(0.5) * rs;
    const R pm = m2 > R(0) ? sqrt((Es - m) * (Es + m)) : Es;
    const R Et = Ei + Ej;
    const R beta[3] = {(mi[0] + mj[0]) / Et, (mi[1] + mj[1]) / Et, (mi[2] + mj[2]) / Et};
    const R gamma = Et / rs;
    const R a = (gamma * gamma) / (gamma + R(1));
    const uint4 w = philox4x32_10(make_uint4(step, lc, i, kTagAngle | j), K);
    const R u1 = word_unit<R>(w.x), u2 = word_unit<R>(w.y);
    R sp, cp;
    sincos_t(R(2) * R(3.141592653589793) * u2, &sp, &cp);
    R ps[3];
    if (!(mu > R(0))) {
        const R ct = R(2) * u1 - R(1);
        const R stt = sqrt((R(1) - ct) * (R(1) + ct));
        ps[0] = pm * (stt * cp);
        ps[1] = pm * (stt * sp);
        ps[2] = pm * ct;
    } else {
        const R bpi = (beta[0] * mi[0] + beta[1] * mi[1]) + beta[2] * mi[2];
        const R fin = a * bpi - gamma * Ei;
        R e[3] = {mi[0] + beta[0] * fin, mi[1] + beta[1] * fin, mi[2] + beta[2] * fin};
        const R en = sqrt((e[0] * e[0] + e[1] * e[1]) + e[2] * e[2]);
        for (int q = 0; q < 3; ++q) e[q] = e[q] / en;
        R h[3] = {R(0), R(0), R(0)};
        if (fabs(e[0]) < R(0.9)) h[0] = R(1); else h[1] = R(1);
        R e1[3] = {h[1] * e[2] - h[2] * e[1], h[2] * e[0] - h[0] * e[2], h[0] * e[1] - h[1] * e[0]};
        const R n1 = sqrt((e1[0] * e1[0] + e1[1] * e1[1]) + e1[2] * e1[2]);
        for (int q = 0; q < 3; ++q) e1[q] = e1[q] / n1;
        const R e2[3] = {e[1] * e1[2] - e[2] * e1[1], e[2] * e1[0] - e[0] * e1[2], e[0] * e1[1] - e[1] * e1[0]};
        const R aa = R(2) * (pm * pm);
        const R mu2 = mu * mu;
        const R A = R(1) / mu2, B = R(1) / (R(2) * aa + mu2);
        R x = (R(1) / (A - u1 * (A - B)) - mu2) / aa;
        x = x < R(0) ? R(0) : (x > R(2) ? R(2) : x);
        const R ct = R(1) - x;
        const R stt = sqrt(x * (R(2) - x));
        for (int q = 0; q < 3; ++q) ps[q] = pm * (ct * e[q] + stt * (cp * e1[q] + sp * e2[q]));
    }
    const R bp = (beta[0] * ps[0] + beta[1] * ps[1]) + beta[2] * ps[2];
    const R fi = a * bp + gamma * Es;
    const R fj = -a * bp + gamma * Es;
    for (int q = 0; q < 3; ++q) {
        mi[q] = ps[q] + beta[q] * fi;
        mj[q] = -ps[q] + beta[q] * fj;
    }
    return true;
}

template <typename T>
__device__ __forceinline__ int collide_state(const SimDesc& S, const PhiloxKey& K, uint32_t lc, uint32_t i, uint32_t j,
                                             T* __restrict__ st, uint32_t pcap, uint32_t gi, uint32_t gj);

template <>
__device__ __forceinline__ int collide_state<double>(const SimDesc& S, const PhiloxKey& K, uint32_t lc, uint32_t i,
                                                     uint32_t j, double* __restrict__ st, uint32_t pcap, uint32_t gi,
                                                     uint32_t gj)
{
    double mi[3], mj[3];
    for (int a = 0; a < 3; ++a) {
        mi[a] = st[(size_t)(3 + a) * pcap + gi];
        mj[a] = st[(size_t)(3 + a) * pcap + gj];
    }
    if (collide_pair<double>(K, S.step, lc, i, j, S.mass, S.mu, mi, mj)) {
        for (int a = 0; a < 3; ++a) {
            st[(size_t)(3 + a) * pcap + gi] = mi[a];
            st[(size_t)(3 + a) * pcap + gj] = mj[a];
        }
    }
    return 0;
}

// FP32 state: FP32 kinematics unless the CM Lorentz factor exceeds the
// simulation's threshold, where the boost cancels badly and FP64 is used
// (always FP64 with the screened angular distribution).
template <>
__device__ __forceinline__ int collide_state<float>(const SimDesc& S, const PhiloxKey& K, uint32_t lc, uint32_t i,
                                                    uint32_t j, float* __restrict__ st, uint32_t pcap, uint32_t gi,
                                                    uint32_t gj)
{
    float mi[3], mj[3];
    for (int a = 0; a < 3; ++a) {
        mi[a] = st[(size_t)(3 + a) * pcap + gi];
        mj[a] = st[(size_t)(3 + a) * pcap + gj];
    }
    const float gam = pair_gamma<float>(S.m2f, mi, mj);
    int used64 = 0;
    bool ok;
    // the screened direction is taken from the incoming CM momentum, whose
    // boost cancels at every gamma: FP64 for every such collision
    if (gam > S.gamma_fp64 || !(gam > 0.0f) || S.mu > 0.0) {
        double di[3], dj[3];
        for (int a = 0; a < 3; ++a) { di[a] = mi[a]; dj[a] = mj[a]; }
        ok = collide_pair<double>(K, S.step, lc, i, j, S.mass, S.mu, di, dj);
        for (int a = 0; a < 3; ++a) { mi[a] = (float)di[a]; mj[a] = (float)dj[a]; }
        used64 = 1;
    } else {
        ok = collide_pair<float>(K, S.step, lc, i, j, (float)S.mass, (float)S.mu, mi, mj);
    }
    if (ok) {
        for (int a = 0; a < 3; ++a) {
            st[(size_t)(3 + a) * pcap + gi] = mi[a];
            st[(size_t)(3 + a) * pcap + gj] = mj[a];
        }
    }
    return used64;
}

template <typename T>
__global__ void __launch_bounds__(kResolveThreads) k_resolve(const SimDesc* __restrict__ sims, int nsims, T* __restrict__ st,
                                                             uint32_t pcap, const uint32_t* __restrict__ cell_start,
                                                             const uint2* __restrict__ work,
                                                             const uint32_t* __restrict__ acc_count,
                                                             unsigned long long* __restrict__ acc,
                                                             const uint32_t* __restrict__ counters,
                                                             const uint32_t* __restrict__ active,
                                                             uint64_t acc_cap, uint32_t* __restrict__ used_global,
                                                             unsigned long long* __restrict__ stats)
{
    extern __shared__ unsigned long long smem[];
    unsigned long long* list_s = smem;
    uint32_t* bits_s = reinterpret_cast<uint32_t*>(smem + kResolveSmemPairs);
    __shared__ uint32_t s_nexe, s_n64;
    const uint32_t nact = counters[2];
    for (uint32_t a = blockIdx.x; a < nact; a += gridDim.x) {
        const uint32_t c = active[a];
        const uint2 w0 = work[c], w1 = work[c + 1];
        const uint32_t room = w1.y - w0.y;
        const uint32_t cnt = acc_count[c];
        uint32_t m = cnt < room ? cnt : room;
        if ((uint64_t)w0.y + m > acc_cap) m = (w0.y < acc_cap) ? (uint32_t)(acc_cap - w0.y) : 0u;
        const int s = sim_of_cell(sims, nsims, c);
        const SimDesc& S = sims[s];
        const uint32_t cbase = cell_start[c], n = cell_start[c + 1] - cbase;
        const uint32_t lc = c - S.cell_off;
        unsigned long long* gl = acc + w0.y;
        const bool in_smem = m <= (uint32_t)kResolveSmemPairs;
        const bool bits_in_smem = n <= 32u * kResolveBitmapWords;
        unsigned long long* L = in_smem ? list_s : gl;
        if (threadIdx.x == 0) { s_nexe = 0; s_n64 = 0; }
        if (in_smem)
            for (uint32_t k = threadIdx.x; k < m; k += blockDim.x) L[k] = gl[k];
        if (bits_in_smem)
            for (uint32_t k = threadIdx.x; k < (n + 31) / 32; k += blockDim.x) bits_s[k] = 0u;
        __syncthreads();
        bitonic_sort(L, m);
        // A6: greedy matching in lexicographic order
        if (threadIdx.x == 0) {
            uint32_t ne = 0;
            for (uint32_t k = 0; k < m; ++k) {
                const unsigned long long v = L[k];
                const uint32_t i = (uint32_t)(v >> 32), j = (uint32_t)v;
                if (bits_in_smem) {
                    const uint32_t bi = (bits_s[i >> 5] >> (i & 31)) & 1u;
                    const uint32_t bj = (bits_s[j >> 5] >> (j & 31)) & 1u;
                    if (bi | bj) continue;
                    bits_s[i >> 5] |= 1u << (i & 31);
                    bits_s[j >> 5] |= 1u << (j & 31);
                } else {
                    const uint32_t gi = cbase + i, gj = cbase + j;
                    const uint32_t bi = (atomicOr(&used_global[gi >> 5], 0u) >> (gi & 31)) & 1u;
                    const uint32_t bj = (atomicOr(&used_global[gj >> 5], 0u) >> (gj & 31)) & 1u;
                    if (bi | bj) continue;
                    atomicOr(&used_global[gi >> 5], 1u << (gi & 31));
                    atomicOr(&used_global[gj >> 5], 1u << (gj & 31));
                }
                L[k] = v | kExecFlag;
                ++ne;
            }
            s_nexe = ne;
        }
        __syncthreads();
        // A7: kinematics of the executed pairs (disjoint, so in parallel)
        const PhiloxKey K = philox_schedule(S.key0, S.key1);
        uint32_t n64 = 0;
        for (uint32_t k = threadIdx.x; k < m; k += blockDim.x) {
            const unsigned long long v = L[k];
            if (!(v & kExecFlag)) continue;
            const uint32_t i = (uint32_t)(v >> 32) & 0x7FFFFFFFu, j = (uint32_t)v;
            n64 += (uint32_t)collide_state<T>(S, K, lc, i, j, st, pcap, cbase + i, cbase + j);
            if (!bits_in_smem) {
                atomicAnd(&used_global[(cbase + i) >> 5], ~(1u << ((cbase + i) & 31)));
                atomicAnd(&used_global[(cbase + j) >> 5], ~(1u << ((cbase + j) & 31)));
            }
        }
        if (n64) atomicAdd(&s_n64, n64);
        if (in_smem)
            for (uint32_t k = threadIdx.x; k < m; k += blockDim.x) gl[k] = L[k];
        __syncthreads();
        if (threadIdx.x == 0) {
            const uint32_t slot = S.stat_slot;
            atomicAdd(&stats[slot * kStatCount + kStatAccepted], (unsigned long long)cnt);
            atomicAdd(&stats[slot * kStatCount + kStatExecuted], (unsigned long long)s_nexe);
            if (s_n64) atomicAdd(&stats[slot * kStatCount + kStatFp64Boosts], (unsigned long long)s_n64);
        }
        __syncthreads();
    }
}

// A6-A7 for small cells (n <= small_max <= 1024) with at most kLaneList
// accepted pairs: one lane per cell, 32 consecutive cells per warp (their
// counts and bounds read in one coalesced round).  A lane walks its cell's
// list in increasing (i, j) order (the lists are tiny: repeated minimum
// search) and takes the greedy matching on a list of used particles; the
// executed pairs of the 32 cells go to a per-warp shared-memory queue and
// their kinematics run one pair per lane (executed pairs share no particle,
// so their order does not matter).  Cells with longer lists are handed to the
// block path through the active-cell list.  Counters are summed per lane and
// flushed per simulation (one atomic per warp and simulation).
constexpr uint32_t kLaneList = 8;
constexpr uint32_t kResolveQueue = 32 * kLaneList;  // executed pairs of 32 cells at most

__device__ __forceinline__ void flush_resolve_stats(uint32_t slot, unsigned long long& a_acc,
                                                    unsigned long long& a_exe,
                                                    unsigned long long* __restrict__ stats)
{
    const uint32_t lane = threadIdx.x & 31;
    const unsigned peers = __match_any_sync(kFull, slot);
    const int leader = __ffs(peers) - 1;
    unsigned long long sa = 0, se = 0;
    for (unsigned m = peers; m; m &= m - 1) {
        sa += __shfl_sync(peers, a_acc, __ffs(m) - 1);
        se += __shfl_sync(peers, a_exe, __ffs(m) - 1);
    }
    if ((int)lane == leader && slot != 0xFFFFFFFFu) {
        if (sa) atomicAdd(&stats[slot * kStatCount + kStatAccepted], sa);
        if (se) atomicAdd(&stats[slot * kStatCount + kStatExecuted], se);
    }
    a_acc = a_exe = 0;
}

template <typename T>
__global__ void __launch_bounds__(256, 4) k_resolve_small(const SimDesc* __restrict__ sims, int nsims, T* __restrict__ st,
                                                       uint32_t pcap, const uint32_t* __restrict__ cell_start,
                                                       const uint2* __restrict__ work, uint32_t ncells,
                                                       uint32_t small_max, const uint32_t* __restrict__ acc_count,
                                                       unsigned long long* __restrict__ acc, uint64_t acc_cap,
                                                       uint32_t* __restrict__ counters, uint32_t* __restrict__ active,
                                                       unsigned long long* __restrict__ stats)
{
    constexpr int kWarps = 8;
    __shared__ uint4 q[kWarps][kResolveQueue];  // (cell, i, j, first particle of the cell)
    __shared__ uint32_t qn[kWarps];
    const int w = threadIdx.x >> 5;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t nwarps = gridDim.x * kWarps;
    uint32_t cur_slot = 0xFFFFFFFFu;
    unsigned long long a_acc = 0, a_exe = 0;
    for (uint32_t c0 = (blockIdx.x * kWarps + w) * 32u; c0 < ncells; c0 += nwarps * 32u) {
        if (lane == 0) qn[w] = 0;
        __syncwarp();
        const uint32_t c = c0 + lane;
        uint32_t cnt = 0, cbase = 0, n = 0, m = 0, list0 = 0;
        bool mine = false;
        if (c < ncells) {
            cnt = acc_count[c];
            if (cnt) {
                cbase = cell_start[c];
                n = cell_start[c + 1] - cbase;
                if (n >= 2 && n <= small_max) {
                    const uint2 w0 = work[c], w1 = work[c + 1];
                    const uint32_t room = w1.y - w0.y;
                    m = cnt < room ? cnt : room;
                    if ((uint64_t)w0.y + m > acc_cap) m = (w0.y < acc_cap) ? (uint32_t)(acc_cap - w0.y) : 0u;
                    list0 = w0.y;
                    if (m > kLaneList) active[atomicAdd(&counters[2], 1u)] = c;
                    else mine = true;
                }
            }
        }
        uint32_t slot = 0xFFFFFFFFu;
        if (mine) slot = sims[sim_of_cell(sims, nsims, c)].stat_slot;
        if (__any_sync(kFull, mine && slot != cur_slot && cur_slot != 0xFFFFFFFFu)) flush_resolve_stats(cur_slot, a_acc, a_exe, stats);
        if (mine) {
            cur_slot = slot;
            // greedy in lexicographic order: repeatedly the smallest unvisited
            // entry; the list is written back sorted, executed pairs flagged.
            // The entries and the particles taken so far stay in registers
            // (every index below is a compile-time constant): a visited entry
            // becomes ~0, above every real (i << 32 | j).
            unsigned long long* gl = acc + list0;
            unsigned long long v[kLaneList];
#pragma unroll
            for (uint32_t k = 0; k < kLaneList; ++k) v[k] = k < m ? gl[k] : ~0ull;
            uint32_t used[2 * kLaneList];
#pragma unroll
            for (uint32_t u = 0; u < 2 * kLaneList; ++u) used[u] = 0xFFFFFFFFu;
            uint32_t nused = 0;
            for (uint32_t r = 0; r < m; ++r) {
                unsigned long long best = v[0];
                uint32_t kb = 0;
#pragma unroll
                for (uint32_t k = 1; k < kLaneList; ++k)
                    if (v[k] < best) {
                        best = v[k];
                        kb = k;
                    }
#pragma unroll
                for (uint32_t k = 0; k < kLaneList; ++k)
                    if (k == kb) v[k] = ~0ull;
                const uint32_t i = (uint32_t)(best >> 32), j = (uint32_t)best;
                bool free_ij = true;
#pragma unroll
                for (uint32_t u = 0; u < 2 * kLaneList; ++u) free_ij &= (used[u] != i) & (used[u] != j);
                if (free_ij) {
#pragma unroll
                    for (uint32_t u = 0; u < 2 * kLaneList; ++u) {
                        if (u == nused) used[u] = i;
                        if (u == nused + 1) used[u] = j;
                    }
                    nused += 2;
                    best |= kExecFlag;
                    const uint32_t qs = atomicAdd(&qn[w], 1u);
                    q[w][qs] = make_uint4(c, i, j, cbase);
                }
                gl[r] = best;
            }
            a_acc += cnt;
            a_exe += nused / 2;
        }
        __syncwarp();
        const uint32_t ne = qn[w];
        for (uint32_t k = lane; k < ne; k += 32) {
            const uint4 e = q[w][k];
            const SimDesc& S = sims[sim_of_cell(sims, nsims, e.x)];
            const PhiloxKey K = philox_schedule(S.key0, S.key1);
            const int u64 = collide_state<T>(S, K, e.x - S.cell_off, e.y, e.z, st, pcap, e.w + e.y, e.w + e.z);
            if (u64) atomicAdd(&stats[S.stat_slot * kStatCount + kStatFp64Boosts], 1ull);
        }
        __syncwarp();
    }
    flush_resolve_stats(cur_slot, a_acc, a_exe, stats);
}

// Kinematics of pairs (2k, 2k+1) of cell 0 in the FP32 path with a given FP64
// threshold, on caller-given momenta (verification of the threshold).
__global__ void k_kinematics_check(SimDesc S, const float* __restrict__ pin, int64_t npairs, float* __restrict__ pout,
                                   int32_t* __restrict__ used64)
{
    const PhiloxKey K = philox_schedule(S.key0, S.key1);
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < npairs; k += (int64_t)gridDim.x * blockDim.x) {
        // scratch state of two particles laid out as the SoA state (pcap = 2)
        float st[12];
        for (int a = 0; a < 3; ++a) {
            st[0 + a * 2] = 0.f;
            st[1 + a * 2] = 0.f;
            st[6 + a * 2] = pin[6 * k + a];
            st[7 + a * 2] = pin[6 * k + 3 + a];
        }
        const int u = collide_state<float>(S, K, 0u, (uint32_t)(2 * k), (uint32_t)(2 * k + 1), st, 2u, 0u, 1u);
        for (int a = 0; a < 3; ++a) {
            pout[6 * k + a] = st[6 + a * 2];
            pout[6 * k + 3 + a] = st[7 + a * 2];
        }
        used64[k] = u;
    }
}

int launch_kinematics_check(const SimDesc& S, const float* pin, int64_t npairs, float* pout, int32_t* used64,
                            cudaStream_t st)
{
    if (npairs <= 0) return 0;
    k_kinematics_check<<<(unsigned)((npairs + 255) / 256 < 4096 ? (npairs + 255) / 256 : 4096), 256, 0, st>>>(
        S, pin, npairs, pout, used64);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
static int last_err() { return cudaPeekAtLastError() == cudaSuccess ? 0 : -1; }

// dynamic shared memory of the item kernel: one ring per warp
constexpr size_t kPairRingSmem = (kPairThreads / 32) * sizeof(PairRing);

template <typename T, bool kOneKey, int NB>
static unsigned pair_grid()
{
    static unsigned g = 0;
    if (!g) {
        cudaFuncSetAttribute(k_pair_tile<T, kOneKey, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kPairRingSmem);
        int per = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pair_tile<T, kOneKey, NB>, kPairThreads,
                                                      kPairRingSmem);
        if (per < 1) per = 1;
        g = (unsigned)(per * sm_count());
    }
    return g;
}

// dynamic shared memory of the small-cell kernel: one ring per warp
constexpr size_t kSmallRingSmem = (kPairThreads / 32) * sizeof(SmallRing);

template <typename T, bool kOneKey, int NB>
static unsigned small_grid()
{
    static unsigned g = 0;
    if (!g) {
        cudaFuncSetAttribute(k_pair_small<T, kOneKey, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kSmallRingSmem);
        int per = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pair_small<T, kOneKey, NB>, kPairThreads,
                                                      kSmallRingSmem);
        if (per < 1) per = 1;
        g = (unsigned)(per * sm_count());
    }
    return g;
}

template <typename T, bool kOneKey>
static unsigned skip_grid()
{
    static unsigned g = 0;
    if (!g) {
        int per = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pair_skip<T, kOneKey>, kPairThreads, 0);
        if (per < 1) per = 1;
        g = (unsigned)(per * sm_count());
    }
    return g;
}

template <typename T, bool kOneKey, int NB>
static void launch_small(const Arena& A, cudaStream_t st)
{
    k_pair_small<T, kOneKey, NB><<<small_grid<T, kOneKey, NB>(), kPairThreads, kSmallRingSmem, st>>>(
        A.d_sims, A.nsims, (const T*)A.st[A.cur], A.pcap, A.cell_start, A.cell_work, A.ncells, A.small_max,
        A.acc_count, A.acc, A.acc_capacity, A.counters, A.active, A.stats, A.surv, A.surv_cap, A.key_sched);
}

template <typename T, bool kOneKey, int NB>
static void launch_tile(const Arena& A, cudaStream_t st)
{
    k_pair_tile<T, kOneKey, NB><<<pair_grid<T, kOneKey, NB>(), kPairThreads, kPairRingSmem, st>>>(
        A.d_sims, A.nsims, (const T*)A.st[A.cur], A.pcap, A.cell_start, A.cell_work, A.ncells, A.acc_count, A.acc,
        A.acc_capacity, A.counters, A.active, A.stats, A.surv, A.surv_cap, A.key_sched);
}

template <typename T, bool kOneKey>
static void launch_finish(const Arena& A, cudaStream_t st)
{
    k_pair_finish<T, kOneKey><<<(unsigned)(sm_count() * 4), 256, 0, st>>>(
        A.d_sims, A.nsims, (const T*)A.st[A.cur], A.pcap, A.cell_start, A.cell_work, A.ncells, A.acc_count, A.acc,
        A.acc_capacity, A.counters, A.active, A.stats, A.surv, A.surv_cap, A.key_sched);
}

template <typename T, bool kOneKey>
static void launch_pairs(const Arena& A, cudaStream_t st)
{
    if (A.any_skip)
        k_pair_skip<T, kOneKey><<<skip_grid<T, kOneKey>(), kPairThreads, 0, st>>>(
            A.d_sims, A.nsims, (const T*)A.st[A.cur], A.pcap, A.cell_start, A.cell_work, A.skip_work, A.ncells,
            A.small_max, A.acc_count, A.acc, A.acc_capacity, A.counters, A.active, A.stats, A.key_sched);
    if (!A.any_all_pairs) return;
    if (A.small_max) {
        if (A.small_nb == 1)
            launch_small<T, kOneKey, 1>(A, st);
        else
            launch_small<T, kOneKey, 2>(A, st);
    }
    if (A.tile_nb == 2)
        launch_tile<T, kOneKey, 2>(A, st);
    else if (A.tile_nb == 4)
        launch_tile<T, kOneKey, 4>(A, st);
    else
        launch_tile<T, kOneKey, 8>(A, st);
    launch_finish<T, kOneKey>(A, st);
}

int launch_pair_tile(const Arena& A, cudaStream_t st)
{
    if (A.ncells == 0) return 0;
    if (A.precision == 1) {
        if (A.one_key) launch_pairs<double, true>(A, st); else launch_pairs<double, false>(A, st);
    } else {
        if (A.one_key) launch_pairs<float, true>(A, st); else launch_pairs<float, false>(A, st);
    }
    return last_err();
}

static const size_t kResolveSmemBytes =
    kResolveSmemPairs * sizeof(unsigned long long) + kResolveBitmapWords * sizeof(uint32_t);

// Kernel attributes and launch shapes, set once before any stream capture.
int kernels_init()
{
    static bool done = false;
    if (done) return 0;
    if (cudaFuncSetAttribute(k_resolve<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kResolveSmemBytes) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_resolve<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kResolveSmemBytes) !=
            cudaSuccess)
        return -1;
    if (bin_kernels_init()) return -1;
    pair_grid<double, false, 8>();
    pair_grid<float, false, 8>();
    pair_grid<double, true, 8>();
    pair_grid<float, true, 8>();
    pair_grid<double, false, 4>();
    pair_grid<float, false, 4>();
    pair_grid<double, true, 4>();
    pair_grid<float, true, 4>();
    pair_grid<double, false, 2>();
    pair_grid<float, false, 2>();
    pair_grid<double, true, 2>();
    pair_grid<float, true, 2>();
    small_grid<double, false, 2>();
    small_grid<float, false, 2>();
    small_grid<double, true, 2>();
    small_grid<float, true, 2>();
    small_grid<double, false, 1>();
    small_grid<float, false, 1>();
    small_grid<double, true, 1>();
    small_grid<float, true, 1>();
    skip_grid<double, false>();
    skip_grid<float, false>();
    skip_grid<double, true>();
    skip_grid<float, true>();
    sm_count();
    done = true;
    return 0;
}

int launch_resolve(const Arena& A, cudaStream_t st)
{
    if (A.ncells == 0) return 0;
    const size_t smem = kResolveSmemBytes;
    const unsigned g = (unsigned)(sm_count() * 4);
    if (A.small_max) {
        const unsigned gs = (unsigned)(sm_count() * 8);
        if (A.precision == 1)
            k_resolve_small<double><<<gs, 256, 0, st>>>(A.d_sims, A.nsims, (double*)A.st[A.cur], A.pcap, A.cell_start,
                                                         A.cell_work, A.ncells, A.small_max, A.acc_count, A.acc,
                                                         A.acc_capacity, A.counters, A.active, A.stats);
        else
            k_resolve_small<float><<<gs, 256, 0, st>>>(A.d_sims, A.nsims, (float*)A.st[A.cur], A.pcap, A.cell_start,
                                                        A.cell_work, A.ncells, A.small_max, A.acc_count, A.acc,
                                                        A.acc_capacity, A.counters, A.active, A.stats);
    }
    if (A.precision == 1)
        k_resolve<double><<<g, kResolveThreads, smem, st>>>(A.d_sims, A.nsims, (double*)A.st[A.cur], A.pcap,
                                                           A.cell_start, A.cell_work, A.acc_count, A.acc, A.counters,
                                                           A.active, A.acc_capacity, A.used_bits, A.stats);
    else
        k_resolve<float><<<g, kResolveThreads, smem, st>>>(A.d_sims, A.nsims, (float*)A.st[A.cur], A.pcap,
                                                          A.cell_start, A.cell_work, A.acc_count, A.acc, A.counters,
                                                          A.active, A.acc_capacity, A.used_bits, A.stats);
    return last_err();
}

}  // namespace cuba
