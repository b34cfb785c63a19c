// Explicitly rounded IEEE arithmetic shared by the kernels of both state
// precisions, and the per-simulation constants in the state's precision.
#pragma once
#include <cstdint>

#include "engine.cuh"

namespace cuba {

__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double div_rn(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float div_rn(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double sqrt_rn(double a) { return __dsqrt_rn(a); }
__device__ __forceinline__ float sqrt_rn(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ double floor_t(double a) { return floor(a); }
__device__ __forceinline__ float floor_t(float a) { return floorf(a); }

template <typename T> __device__ __forceinline__ T sim_dt(const SimDesc& S);
template <> __device__ __forceinline__ double sim_dt<double>(const SimDesc& S) { return S.dt; }
template <> __device__ __forceinline__ float sim_dt<float>(const SimDesc& S) { return S.dtf; }
template <typename T> __device__ __forceinline__ T sim_L(const SimDesc& S, int a);
template <> __device__ __forceinline__ double sim_L<double>(const SimDesc& S, int a) { return S.L[a]; }
template <> __device__ __forceinline__ float sim_L<float>(const SimDesc& S, int a) { return S.Lf[a]; }
template <typename T> __device__ __forceinline__ T sim_m2(const SimDesc& S);
template <> __device__ __forceinline__ double sim_m2<double>(const SimDesc& S) { return S.m2; }
template <> __device__ __forceinline__ float sim_m2<float>(const SimDesc& S) { return S.m2f; }
template <typename T> __device__ __forceinline__ T sim_dx(const SimDesc& S, int a);
template <> __device__ __forceinline__ double sim_dx<double>(const SimDesc& S, int a) { return S.dx[a]; }
template <> __device__ __forceinline__ float sim_dx<float>(const SimDesc& S, int a) { return S.dxf[a]; }

template <typename T> __device__ __forceinline__ T sim_rdx(const SimDesc& S, int a);
template <> __device__ __forceinline__ double sim_rdx<double>(const SimDesc& S, int a) { return S.rdx[a]; }
template <> __device__ __forceinline__ float sim_rdx<float>(const SimDesc& S, int a) { return S.rdxf[a]; }

template <typename T> __device__ __forceinline__ T sim_C(const SimDesc& S);
template <> __device__ __forceinline__ double sim_C<double>(const SimDesc& S) { return S.C; }
template <> __device__ __forceinline__ float sim_C<float>(const SimDesc& S) { return S.Cf; }

}  // namespace cuba
