// ddsg_eval.cuh -- declarations shared by the evaluation kernels (device code
// only): launch parameters, per-precision operand types, the per-thread result
// holder (FP64, or FP32 partials folded into a Kahan total) and the exact
// conversion of fixed-point hat values.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ddsg_internal.h"

namespace ddsg {

__device__ __forceinline__ float pow2m_f(int e) {  // 2^-e, 0 <= e < 126
    return __int_as_float((127 - e) << 23);
}

// phi = N * 2^-e as a double, N < 2^63, built from the bits (truncated to 53
// significant bits; the exact value is N * 2^-e).
__device__ __forceinline__ double basis_to_f64(uint64_t N, int e) {
    if (N == 0) return 0.0;
    const int lz = __clzll((long long)N);
    const uint64_t mant = (N << lz) >> 11;        // 53 bits, leading one at bit 52
    const int64_t ex = (int64_t)(63 - lz) - e + 1023;
    return __longlong_as_double((long long)(((uint64_t)ex << 52) | (mant & ((1ull << 52) - 1))));
}

// phi = N * 2^-e as a float with 32 significant bits kept before rounding.
// For l >= 2, e = 63 - l (l >= 3) or 61 (l == 2): N >> (e - 31) < 2^32.
__device__ __forceinline__ float basis_to_f32(uint64_t N, int e) {
    if (e <= 31) return __uint2float_rn((uint32_t)N) * pow2m_f(e);
    return __uint2float_rn((uint32_t)(N >> (e - 31))) * pow2m_f(31);
}

template <typename W>
__device__ __forceinline__ W basis_val(const Basis1D &o);
template <>
__device__ __forceinline__ double basis_val<double>(const Basis1D &o) { return basis_to_f64(o.N, o.e); }
template <>
__device__ __forceinline__ float basis_val<float>(const Basis1D &o) { return basis_to_f32(o.N, o.e); }

struct EvalParams {
    DevTables t;
    int d, m;
    int64_t n;
    const uint64_t *X;
    const int32_t *flags;
    double *y;
    uint64_t *hash;
    int32_t *count;
    int form;
    unsigned long long *err;
    int issue_end;         // staging copies issued for processed components < issue_end only
                           // (INT_MAX unless a failure-path test withholds them)
};

template <int PREC>
struct Types;
template <>
struct Types<DDSG_F64> {
    using W = double;
    using V = double2;
    static constexpr int VW = 2;
    static __device__ __forceinline__ const double *alpha(const DevTables &t) { return t.alpha64; }
    static __device__ __forceinline__ int stride(const DevTables &t) { return t.mp64; }
};
template <>
struct Types<DDSG_F32C> {
    using W = float;
    using V = float4;
    static constexpr int VW = 4;
    static __device__ __forceinline__ const float *alpha(const DevTables &t) { return t.alpha32; }
    static __device__ __forceinline__ int stride(const DevTables &t) { return t.mp32; }
};

// Final per-thread result holder: FP64 accumulates directly; FP32 folds each
// component's plain-FP32 partial sum into a Kahan-compensated total.
template <int PREC, int MC>
struct Result;
template <int MC>
struct Result<DDSG_F64, MC> {
    double s[MC];
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int o = 0; o < MC; ++o) s[o] = 0.0;
    }
    __device__ __forceinline__ double (&partial())[MC] { return s; }
    __device__ __forceinline__ void fold() {}
    __device__ __forceinline__ double value(int o) const { return s[o]; }
};
template <int MC>
struct Result<DDSG_F32C, MC> {
    float p[MC], s[MC], c[MC];
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int o = 0; o < MC; ++o) p[o] = s[o] = c[o] = 0.0f;
    }
    __device__ __forceinline__ float (&partial())[MC] { return p; }
    __device__ __forceinline__ void fold() {
#pragma unroll
        for (int o = 0; o < MC; ++o) {
            const float yk = __fsub_rn(p[o], c[o]);
            const float tk = __fadd_rn(s[o], yk);
            c[o] = __fsub_rn(__fsub_rn(tk, s[o]), yk);
            s[o] = tk;
            p[o] = 0.0f;
        }
    }
    __device__ __forceinline__ double value(int o) const { return (double)s[o] - (double)c[o]; }
};

}  // namespace ddsg
