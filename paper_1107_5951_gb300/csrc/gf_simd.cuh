// gf_simd.cuh -- small device helpers shared by the evaluation kernels:
// packed FP32 pair arithmetic, compensated sums, and the packed L2P sum with
// its recursion coefficients.  Everything sits in an unnamed namespace, so
// every translation unit that includes this header has its own copy of the
// coefficient tables and uploads it with its own upload_l2p_coefs().
#pragma once

#include <cmath>

#include "gf_internal.cuh"

namespace gf {
namespace {

template <class T>
struct __align__(16) Vec4 {
    T x, y, z, w;
};

template <class T>
__device__ __forceinline__ T rsqrt_t(T x);
template <>
__device__ __forceinline__ float rsqrt_t<float>(float x) {
    return rsqrtf(x);
}
template <>
__device__ __forceinline__ double rsqrt_t<double>(double x) {
    return rsqrt(x);
}

// Packed pairs of FP32 values (f32x2 arithmetic of sm_100 and later: one
// instruction does two FP32 operations, halving the issue slots of the
// near-field loop).
__device__ __forceinline__ uint64_t pk2(float lo, float hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void up2(uint64_t v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
// 1/sqrt(x) on the special-function unit, subnormal inputs read as zero
__device__ __forceinline__ float rsqrt_ftz(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

template <class T>
__device__ __forceinline__ void two_sum(T &hi, T &lo, T x) {
    const T s = hi + x;
    const T bp = s - hi;
    lo += (hi - (s - bp)) + (x - bp);
    hi = s;
}

// Coefficients of the regular-harmonic recursion of the L2P sums (the
// recursion of fmm_math.cuh), for m < n < kMaxP at t = n (n + 1) / 2 + m:
//   c_ra[t] = (2n - 1) / sqrt((n + m)(n - m)),
//   c_rb[t] = sqrt((n - 1 + m)(n - 1 - m)) / sqrt((n + m)(n - m))  (0 for n = m + 1),
// and c_rf[m] = -sqrt((2m - 1) / (2m)) for the sectoral step, so that the
// FP32 evaluation needs no square roots or divisions.
__constant__ float c_ra[kMaxP * (kMaxP + 1) / 2], c_rb[kMaxP * (kMaxP + 1) / 2], c_rf[kMaxP];

// sum_{n<p, m} D_n^m conj(R_n^m(X)) for the gradient expansions of
// l2p_sum (fmm_math.cuh), for two points at once (packed pairs X, Y, Z).
// D holds each coefficient as a duplicated pair {d, d}, with the factor 2
// of the m > 0 terms folded in.
__device__ __forceinline__ void l2p_sum2(int p, const float2 *Dx, const float2 *Dy, const float2 *Dz, uint64_t X,
                                         uint64_t Y, uint64_t Z, uint64_t &gx, uint64_t &gy, uint64_t &gz) {
    const uint64_t r2 = fma2(Z, Z, fma2(Y, Y, mul2(X, X)));
    uint64_t sr = pk2(1.f, 1.f), si = 0;
    uint64_t ax = 0, ay = 0, az = 0;
    auto ld = [](const float2 *d, int k) { return *reinterpret_cast<const uint64_t *>(d + k); };
    for (int m = 0; m < p; ++m) {
        if (m > 0) {
            const float f = c_rf[m];
            const uint64_t XF = mul2(X, pk2(f, f)), YF = mul2(Y, pk2(f, f)), YN = mul2(Y, pk2(-f, -f));
            const uint64_t nr = fma2(XF, sr, mul2(YN, si));
            const uint64_t ni = fma2(XF, si, mul2(YF, sr));
            sr = nr;
            si = ni;
        }
        uint64_t r1 = sr, i1 = si, r0 = 0, i0 = 0;
        for (int n = m; n < p; ++n) {
            uint64_t cr = sr, ci = si;
            if (n > m) {
                const int t = n * (n + 1) / 2 + m;
                const float av = c_ra[t], bv = c_rb[t];
                const uint64_t AZ = mul2(Z, pk2(av, av)), BN = mul2(r2, pk2(-bv, -bv));
                cr = fma2(AZ, r1, mul2(BN, r0));
                ci = fma2(AZ, i1, mul2(BN, i0));
                r0 = r1;
                i0 = i1;
                r1 = cr;
                i1 = ci;
            }
            if (m == 0) {
                const int k = n * n;
                ax = fma2(ld(Dx, k), cr, ax);
                ay = fma2(ld(Dy, k), cr, ay);
                az = fma2(ld(Dz, k), cr, az);
            } else {
                const int k = n * n + 2 * m - 1;
                ax = fma2(ld(Dx, k), cr, fma2(ld(Dx, k + 1), ci, ax));
                ay = fma2(ld(Dy, k), cr, fma2(ld(Dy, k + 1), ci, ay));
                az = fma2(ld(Dz, k), cr, fma2(ld(Dz, k + 1), ci, az));
            }
        }
    }
    gx = ax;
    gy = ay;
    gz = az;
}


// l2p_sum2 for two packed pairs of points at once (four points): the
// recursion coefficients and every coefficient of D are loaded once for both.
__device__ __forceinline__ void l2p_sum2x2(int p, const float2 *Dx, const float2 *Dy, const float2 *Dz,
                                           uint64_t X0, uint64_t Y0, uint64_t Z0, uint64_t X1, uint64_t Y1,
                                           uint64_t Z1, uint64_t g0[3], uint64_t g1[3]) {
    const uint64_t q0 = fma2(Z0, Z0, fma2(Y0, Y0, mul2(X0, X0)));
    const uint64_t q1 = fma2(Z1, Z1, fma2(Y1, Y1, mul2(X1, X1)));
    uint64_t sr0 = pk2(1.f, 1.f), si0 = 0, sr1 = sr0, si1 = 0;
    uint64_t ax0 = 0, ay0 = 0, az0 = 0, ax1 = 0, ay1 = 0, az1 = 0;
    auto ld = [](const float2 *d, int k) { return *reinterpret_cast<const uint64_t *>(d + k); };
    for (int m = 0; m < p; ++m) {
        if (m > 0) {
            const float f = c_rf[m];
            const uint64_t F = pk2(f, f), FN = pk2(-f, -f);
            uint64_t nr = fma2(mul2(X0, F), sr0, mul2(mul2(Y0, FN), si0));
            uint64_t ni = fma2(mul2(X0, F), si0, mul2(mul2(Y0, F), sr0));
            sr0 = nr;
            si0 = ni;
            nr = fma2(mul2(X1, F), sr1, mul2(mul2(Y1, FN), si1));
            ni = fma2(mul2(X1, F), si1, mul2(mul2(Y1, F), sr1));
            sr1 = nr;
            si1 = ni;
        }
        uint64_t r10 = sr0, i10 = si0, r00 = 0, i00 = 0;
        uint64_t r11 = sr1, i11 = si1, r01 = 0, i01 = 0;
        for (int n = m; n < p; ++n) {
            uint64_t cr0 = sr0, ci0 = si0, cr1 = sr1, ci1 = si1;
            if (n > m) {
                const int t = n * (n + 1) / 2 + m;
                const float av = c_ra[t], bv = c_rb[t];
                const uint64_t A = pk2(av, av), BN = pk2(-bv, -bv);
                const uint64_t AZ0 = mul2(Z0, A), BQ0 = mul2(q0, BN), AZ1 = mul2(Z1, A), BQ1 = mul2(q1, BN);
                cr0 = fma2(AZ0, r10, mul2(BQ0, r00));
                ci0 = fma2(AZ0, i10, mul2(BQ0, i00));
                cr1 = fma2(AZ1, r11, mul2(BQ1, r01));
                ci1 = fma2(AZ1, i11, mul2(BQ1, i01));
                r00 = r10;
                i00 = i10;
                r10 = cr0;
                i10 = ci0;
                r01 = r11;
                i01 = i11;
                r11 = cr1;
                i11 = ci1;
            }
            if (m == 0) {
                const int k = n * n;
                const uint64_t dx = ld(Dx, k), dy = ld(Dy, k), dz = ld(Dz, k);
                ax0 = fma2(dx, cr0, ax0);
                ay0 = fma2(dy, cr0, ay0);
                az0 = fma2(dz, cr0, az0);
                ax1 = fma2(dx, cr1, ax1);
                ay1 = fma2(dy, cr1, ay1);
                az1 = fma2(dz, cr1, az1);
            } else {
                const int k = n * n + 2 * m - 1;
                const uint64_t dxr = ld(Dx, k), dxi = ld(Dx, k + 1), dyr = ld(Dy, k), dyi = ld(Dy, k + 1),
                               dzr = ld(Dz, k), dzi = ld(Dz, k + 1);
                ax0 = fma2(dxr, cr0, fma2(dxi, ci0, ax0));
                ay0 = fma2(dyr, cr0, fma2(dyi, ci0, ay0));
                az0 = fma2(dzr, cr0, fma2(dzi, ci0, az0));
                ax1 = fma2(dxr, cr1, fma2(dxi, ci1, ax1));
                ay1 = fma2(dyr, cr1, fma2(dyi, ci1, ay1));
                az1 = fma2(dzr, cr1, fma2(dzi, ci1, az1));
            }
        }
    }
    g0[0] = ax0;
    g0[1] = ay0;
    g0[2] = az0;
    g1[0] = ax1;
    g1[1] = ay1;
    g1[2] = az1;
}

// The recursion coefficients of l2p_sum2 for the current device.
inline gf_status upload_l2p_coefs() {
    constexpr int NT = kMaxP * (kMaxP + 1) / 2;
    float ra[NT] = {}, rb[NT] = {}, rf[kMaxP] = {};
    for (int n = 1; n < kMaxP; ++n)
        for (int m = 0; m < n; ++m) {
            const int t = n * (n + 1) / 2 + m;
            const double inv = 1.0 / std::sqrt((double)((n + m) * (n - m)));
            ra[t] = (float)((2 * n - 1) * inv);
            rb[t] = n - 1 > m ? (float)(std::sqrt((double)((n - 1 + m) * (n - 1 - m))) * inv) : 0.f;
        }
    for (int m = 1; m < kMaxP; ++m) rf[m] = (float)-std::sqrt((2.0 * m - 1.0) / (2.0 * m));
    GF_CUDA(cudaMemcpyToSymbol(c_ra, ra, sizeof(ra)));
    GF_CUDA(cudaMemcpyToSymbol(c_rb, rb, sizeof(rb)));
    GF_CUDA(cudaMemcpyToSymbol(c_rf, rf, sizeof(rf)));
    return GF_OK;
}

// ---------------------------------------------------------------- FP64 without the FP64 pipe
// FP64 arithmetic and conversions run at a small fraction of the FP32 rate
// on this GPU; these conversions use integer operations only.
// Sign, exponent and the top 23 mantissa bits of a double repacked as a
// float (truncation: relative error below 2^-23), integer operations only;
// false when the value is outside the normal FP32 range (zero excepted).
__device__ __forceinline__ bool trunc_f32(double x, float &f) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ff) - 1023;
    if (e < -126 || e > 127) {
        f = 0.f;
        return (b << 1) == 0;
    }
    f = __uint_as_float((unsigned)((b >> 32) & 0x80000000ull) | ((unsigned)(e + 127) << 23) |
                        (unsigned)((b >> 29) & 0x7fffffull));
    return true;
}

// trunc(x 2^k) for |x 2^k| < 2^62, integer operations only.
__device__ __forceinline__ long long to_fix(double x, int k) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ff);
    if (e == 0) return 0;
    const unsigned long long m = (b & 0xfffffffffffffull) | (1ull << 52);
    const int sh = e - 1075 + k;
    const long long v = sh >= 0 ? (long long)(m << sh) : (sh > -64 ? (long long)(m >> -sh) : 0);
    return (b >> 63) ? -v : v;
}

// |v| < 2^63 as a float, truncating, integer operations only.
__device__ __forceinline__ float fix_to_f32(long long v) {
    if (v == 0) return 0.f;
    const unsigned long long a = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
    const int lz = __clzll((long long)a);
    const unsigned long long n = a << lz;   // leading one at bit 63
    return __uint_as_float((v < 0 ? 0x80000000u : 0u) | ((unsigned)(63 - lz + 127) << 23) |
                           (unsigned)((n >> 40) & 0x7fffffull));
}

// v 2^-k as a double (|v| < 2^63; exact for |v| < 2^53, else truncated).
__device__ __forceinline__ double fix_to_f64(long long v, int k) {
    if (v == 0) return 0.0;
    const unsigned long long a = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
    const int lz = __clzll((long long)a);
    const unsigned long long n = a << lz;   // leading one at bit 63
    const long long e = 63 - lz - k + 1023;
    return __longlong_as_double((long long)((v < 0 ? 0x8000000000000000ull : 0ull) |
                                            ((unsigned long long)e << 52) | ((n >> 11) & 0xfffffffffffffull)));
}

// trunc(f 2^k) for a float f with |f 2^k| < 2^62.
__device__ __forceinline__ long long f32_to_fix(float f, int k) {
    const unsigned b = __float_as_uint(f);
    const int e = (int)((b >> 23) & 0xff);
    if (e == 0) return 0;
    const long long m = (long long)((b & 0x7fffffu) | 0x800000u);
    const int sh = e - 150 + k;
    const long long v = sh >= 0 ? (m << sh) : (sh > -32 ? (m >> -sh) : 0);
    return (b >> 31) ? -v : v;
}

// A float as a double (subnormals read as zero; infinities and NaNs kept).
__device__ __forceinline__ double f32_to_f64(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned e = (b >> 23) & 0xff;
    if (e == 0) return 0.0;
    if (e == 0xff)   // infinity or NaN
        return __longlong_as_double((long long)(((unsigned long long)(b >> 31) << 63) | 0x7ff0000000000000ull |
                                                ((unsigned long long)(b & 0x7fffffu) << 29)));
    return __longlong_as_double((long long)(((unsigned long long)(b >> 31) << 63) |
                                            ((unsigned long long)(e - 127 + 1023) << 52) |
                                            ((unsigned long long)(b & 0x7fffffu) << 29)));
}

}  // namespace
}  // namespace gf
