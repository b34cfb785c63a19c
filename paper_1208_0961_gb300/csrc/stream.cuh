// Per-particle arithmetic of A1-A3 shared by the streaming kernels: free
// streaming with wall reflection and the cell key, in explicitly rounded IEEE
// operations so that a CPU evaluation of the same expressions gives the same
// bits.
#pragma once
#include <cstdint>

#include "engine.cuh"
#include "fp.cuh"

namespace cuba {

// Cell coordinates: i_a = clamp(floor(x_a / dx_a), 0, n_a - 1).
template <typename T>
__device__ __forceinline__ void cell_coords(const SimDesc& S, const T pos[3], uint32_t id[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const T c = floor_t(div_rn(pos[a], sim_dx<T>(S, a)));
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
// component flips.  Returns the number of reflections.
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
        T x = add_rn(pos[a], mul_rn(v, dt));
        if (x < T(0)) {
            x = -x;
            mom[a] = -mom[a];
            ++nref;
        } else if (x > L) {
            x = sub_rn(add_rn(L, L), x);
            mom[a] = -mom[a];
            ++nref;
        }
        pos[a] = x;
    }
    return nref;
}

}  // namespace cuba
