// lbm_store.cuh -- conversions between the stored population format and arithmetic.
//
//   LBM_F64   stores f in FP64, arithmetic on f in FP64.
//   LBM_F32   stores f in FP32, arithmetic on h = f - w_f in FP32 (w_f the FP32-rounded
//             weight), which keeps the O(u) deviations free of the cancellation that
//             forming moments of O(1/36) values in FP32 would cause.
//   LBM_F16S  stores half(h * 2^12) with h = f - w_f; arithmetic on h in FP32. The
//             equilibrium-weight shift keeps the stored values small (Skordos, PRE 48,
//             1993, "Initial and boundary conditions for the lattice Boltzmann method";
//             the same shift underlies Lehmann et al., PRE 106, 2022, on FP16 storage).
#pragma once
#include "lbm_internal.cuh"

namespace lbm {

__host__ __device__ constexpr float wf(int i) { return (float)wgt(i); }
// sum_i w_f(i) - 1 (about 1.49e-8): density offset of the FP32-rounded weights, so that
// rho = 1 + (sum h + WF_BIAS) is the density of the stored f = w_f + h.
constexpr double WF_BIAS = (double)(float)(1.0 / 3.0) + 6.0 * (double)(float)(1.0 / 18.0) +
                           12.0 * (double)(float)(1.0 / 36.0) - 1.0;

template <int DT> __device__ __forceinline__ typename Store<DT>::T nan_value();
template <> __device__ __forceinline__ double nan_value<LBM_F64>() { return __longlong_as_double(0x7ff8000000000000ll); }
template <> __device__ __forceinline__ float nan_value<LBM_F32>() { return __int_as_float(0x7fc00000); }
template <> __device__ __forceinline__ __half nan_value<LBM_F16S>() { return __ushort_as_half((unsigned short)0x7e00); }

// stored value -> f in FP64 (exports, reductions)
template <int DT> __device__ __forceinline__ double to_f64(typename Store<DT>::T v, int i);
template <> __device__ __forceinline__ double to_f64<LBM_F64>(double v, int) { return v; }
template <> __device__ __forceinline__ double to_f64<LBM_F32>(float v, int) { return (double)v; }
template <> __device__ __forceinline__ double to_f64<LBM_F16S>(__half v, int i) {
    return (double)wf(i) + (double)__half2float(v) * (double)F16_INV_SCALE;
}

// f in FP64 -> stored value (initialisation, imports), round to nearest
template <int DT> __device__ __forceinline__ typename Store<DT>::T from_f64(double f, int i);
template <> __device__ __forceinline__ double from_f64<LBM_F64>(double f, int) { return f; }
template <> __device__ __forceinline__ float from_f64<LBM_F32>(double f, int) { return (float)f; }
template <> __device__ __forceinline__ __half from_f64<LBM_F16S>(double f, int i) {
    return __double2half((f - (double)wf(i)) * (double)F16_SCALE);
}

// stored value -> arithmetic variable (f for F64, h for the shifted formats)
template <int DT> __device__ __forceinline__ typename Store<DT>::R to_arith(typename Store<DT>::T v, int i);
template <> __device__ __forceinline__ double to_arith<LBM_F64>(double v, int) { return v; }
template <> __device__ __forceinline__ float to_arith<LBM_F32>(float v, int i) { return v - wf(i); }
template <> __device__ __forceinline__ float to_arith<LBM_F16S>(__half v, int) { return __half2float(v) * F16_INV_SCALE; }

// arithmetic variable -> stored value, round to nearest even
template <int DT> __device__ __forceinline__ typename Store<DT>::T to_store(typename Store<DT>::R v, int i);
template <> __device__ __forceinline__ double to_store<LBM_F64>(double v, int) { return v; }
template <> __device__ __forceinline__ float to_store<LBM_F32>(float v, int i) { return wf(i) + v; }
template <> __device__ __forceinline__ __half to_store<LBM_F16S>(float v, int) { return __float2half_rn(v * F16_SCALE); }

// per-node x force of the tile-major field
template <int DT> __device__ __forceinline__ double gfield_at(const void* g, int64_t idx) {
    return DT == LBM_F64 ? ((const double*)g)[idx] : (double)((const float*)g)[idx];
}

}  // namespace lbm
