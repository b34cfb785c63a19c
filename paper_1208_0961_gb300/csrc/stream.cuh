// Per-particle arithmetic of A1-A3 shared by the streaming kernels: free
// streaming with wall reflection and the cell key, in explicitly rounded IEEE
// operations so that a CPU evaluation of the same expressions gives the same
// bits.
#pragma once
#include <cstdint>

#include "engine.cuh"
#include "fp.cuh"

namespace cuba {

// Margin of the fast path of floor_quot: 2^-20 (FP32) and 2^-49 (FP64), four
// times the largest distance between q and the rounded quotient.
template <typename T> __device__ __forceinline__ T quot_margin();
template <> __device__ __forceinline__ float quot_margin<float>() { return 0x1p-20f; }
template <> __device__ __forceinline__ double quot_margin<double>() { return 0x1p-49; }

// floor(RN(x / dx)), the floor of the correctly rounded quotient, without a
// division in all but rare cases.  q = RN(x rdx) with rdx = RN(1 / dx) carries
// two roundings of relative size 2^-24 (FP32; 2^-53 in FP64) and RN(x / dx)
// one, so |q - RN(x / dx)| < 2^-22 |q| (2^-51 |q|).  When the fraction
// f = q - floor(q) (exact: Sterbenz) keeps m = max(|q|, 1) 2^-20 (2^-49) from
// both 0 and 1, RN(x / dx) lies strictly between the same two integers as q
// and floor(q) is the answer; otherwise (x within a few ulps of a cell face)
// the quotient is rounded correctly and floored.
template <typename T>
__device__ __forceinline__ T floor_quot(T x, T dx, T rdx)
{
    const T q = mul_rn(x, rdx);
    const T k = floor_t(q);
    const T f = sub_rn(q, k);
    const T aq = q < T(0) ? -q : q;
    const T m = mul_rn(aq > T(1) ? aq : T(1), quot_margin<T>());
    if (f >= m && f <= sub_rn(T(1), m)) return k;
    return floor_t(div_rn(x, dx));
}

// Cell coordinates: i_a = clamp(floor(x_a / dx_a), 0, n_a - 1) with the
// quotient rounded correctly: in FP64 by floor_quot (an FP64 division costs
// far more than its fast path on this GPU), in FP32 by the division itself
// (measured cheaper than floor_quot's checks); an axis with one cell needs
// none.
template <typename T>
__device__ __forceinline__ void cell_coords(const SimDesc& S, const T pos[3], uint32_t id[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (S.n[a] == 1) {
            id[a] = 0;
            continue;
        }
        T c;
        if constexpr (sizeof(T) == 8)
            c = floor_quot(pos[a], sim_dx<T>(S, a), sim_rdx<T>(S, a));
        else
            c = floor_t(div_rn(pos[a], sim_dx<T>(S, a)));
        uint32_t ic;
        if (c < T(0)) ic = 0;
        else if (c >= (T)S.n[a]) ic = (uint32_t)(S.n[a] - 1);
        else ic = (uint32_t)c;
        id[a] = ic;
    }
}

// Cell key: key = ix + nx (iy + ny iz).
template <typename T>
__device__ __forceinline__ uint32_t cell_key(const SimDesc& S, const T pos[3])
{
    uint32_t id[3];
    cell_coords<T>(S, pos, id);
    return id[0] + (uint32_t)S.n[0] * (id[1] + (uint32_t)S.n[1] * id[2]);
}

// Free streaming x <- x + (p/E) dt (Eq. 2, c = 1, E = sqrt(|p|^2 + m^2)) and elastic
// reflection: beyond a wall the position is mirrored and that momentum
// component flips (selected, not branched on: the same values without
// divergence).  Returns the number of reflections.
template <typename T>
__device__ __forceinline__ int stream_one(const SimDesc& S, T pos[3], T mom[3])
{
    const T E = sqrt_rn(
        add_rn(add_rn(add_rn(mul_rn(mom[0], mom[0]), mul_rn(mom[1], mom[1])), mul_rn(mom[2], mom[2])), sim_m2<T>(S)));
    const T dt = sim_dt<T>(S);
    int nref = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const T L = sim_L<T>(S, a);
        const T v = (E > T(0)) ? div_rn(mom[a], E) : T(0);
        const T x = add_rn(pos[a], mul_rn(v, dt));
        const bool lo = x < T(0), out = lo || x > L;
        const T xr = lo ? -x : sub_rn(add_rn(L, L), x);
        pos[a] = out ? xr : x;
        mom[a] = out ? -mom[a] : mom[a];
        nref += out ? 1 : 0;
    }
    return nref;
}


// The fields of a descriptor that the streaming and the cell key read, copied
// into a local descriptor once per thread (one simulation), so that the
// particle loops take them from registers.
__device__ __forceinline__ void copy_stream_fields(SimDesc& d, const SimDesc& s)
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        d.L[a] = s.L[a];
        d.Lf[a] = s.Lf[a];
        d.dx[a] = s.dx[a];
        d.dxf[a] = s.dxf[a];
        d.rdx[a] = s.rdx[a];
        d.rdxf[a] = s.rdxf[a];
        d.n[a] = s.n[a];
    }
    d.cell_off = s.cell_off;
    d.dt = s.dt;
    d.dtf = s.dtf;
    d.m2 = s.m2;
    d.m2f = s.m2f;
    d.stat_slot = s.stat_slot;
}

}  // namespace cuba
