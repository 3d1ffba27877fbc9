// lbm_store.cuh -- conversions between the stored population format and arithmetic.
//
//   LBM_F64   stores f in FP64, arithmetic on f in FP64.
//   LBM_F32   stores h = f - w in FP32 (w the exact lattice weight, so the stored value
//             is O(u) rather than O(w)), arithmetic on h in FP32. Rounding h instead of
//             f shrinks the per-step storage error by the ratio |h| / w (about 1e-3 in
//             slow flows), which is what keeps steady states close to the FP64 ones.
//   LBM_F16S  stores half(h * 2^12); arithmetic on h in FP32. The equilibrium-weight
//             shift keeps the stored values small (Skordos, PRE 48, 1993, "Initial and
//             boundary conditions for the lattice Boltzmann method"; the same shift
//             underlies Lehmann et al., PRE 106, 2022, on FP16 storage).
// The density of a shifted node is rho = 1 + sum_i h_i, since sum_i w_i = 1.
#pragma once
#include "lbm_internal.cuh"

namespace lbm {

template <int DT> __device__ __forceinline__ typename Store<DT>::T nan_value();
template <> __device__ __forceinline__ double nan_value<LBM_F64>() { return __longlong_as_double(0x7ff8000000000000ll); }
template <> __device__ __forceinline__ float nan_value<LBM_F32>() { return __int_as_float(0x7fc00000); }
template <> __device__ __forceinline__ __half nan_value<LBM_F16S>() { return __ushort_as_half((unsigned short)0x7e00); }

// stored value -> f in FP64 (exports, reductions)
template <int DT> __device__ __forceinline__ double to_f64(typename Store<DT>::T v, int i);
template <> __device__ __forceinline__ double to_f64<LBM_F64>(double v, int) { return v; }
template <> __device__ __forceinline__ double to_f64<LBM_F32>(float v, int i) { return wgt(i) + (double)v; }
template <> __device__ __forceinline__ double to_f64<LBM_F16S>(__half v, int i) {
    return wgt(i) + (double)__half2float(v) * (double)F16_INV_SCALE;
}

// f in FP64 -> stored value (initialisation, imports), round to nearest
template <int DT> __device__ __forceinline__ typename Store<DT>::T from_f64(double f, int i);
template <> __device__ __forceinline__ double from_f64<LBM_F64>(double f, int) { return f; }
template <> __device__ __forceinline__ float from_f64<LBM_F32>(double f, int i) { return (float)(f - wgt(i)); }
template <> __device__ __forceinline__ __half from_f64<LBM_F16S>(double f, int i) {
    return __double2half((f - wgt(i)) * (double)F16_SCALE);
}

// stored value -> arithmetic variable (f for F64, h for the shifted formats)
template <int DT> __device__ __forceinline__ typename Store<DT>::R to_arith(typename Store<DT>::T v, int i);
template <> __device__ __forceinline__ double to_arith<LBM_F64>(double v, int) { return v; }
template <> __device__ __forceinline__ float to_arith<LBM_F32>(float v, int) { return v; }
template <> __device__ __forceinline__ float to_arith<LBM_F16S>(__half v, int) { return __half2float(v) * F16_INV_SCALE; }

// arithmetic variable -> stored value, round to nearest even
template <int DT> __device__ __forceinline__ typename Store<DT>::T to_store(typename Store<DT>::R v, int i);
template <> __device__ __forceinline__ double to_store<LBM_F64>(double v, int) { return v; }
template <> __device__ __forceinline__ float to_store<LBM_F32>(float v, int) { return v; }
template <> __device__ __forceinline__ __half to_store<LBM_F16S>(float v, int) { return __float2half_rn(v * F16_SCALE); }

// per-node x force of the tile-major field
template <int DT> __device__ __forceinline__ double gfield_at(const void* g, int64_t idx) {
    return DT == LBM_F64 ? ((const double*)g)[idx] : (double)((const float*)g)[idx];
}

}  // namespace lbm
