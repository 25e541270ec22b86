// gf_sum_an.cuh -- arithmetic of closed-form (SUM-AN, Sec. 2.1) voxels used
// by the kernels, host-callable so that CPU tests can check it against the
// oracle.
//
// Corner function, with (u, v, w) = corner minus observer and R = |(u,v,w)|,
// from Eq. 1 by integrating along one axis and then over the other two:
//   F_x = v ln(w + R) + w ln(v + R) - u atan(v w / (u R))
//   F_y = w ln(u + R) + u ln(w + R) - v atan(w u / (v R))
//   F_z = u ln(v + R) + v ln(u + R) - w atan(u v / (w R))
// The field of a voxel of density rho is G rho sum_c s_c F(c - r) over its
// eight corners, s_c = +1 at the corners reached from the lower corner
// through an odd number of upper limits, -1 at the others.  A logarithm
// ln(a + R) whose argument would cancel (a < 0) is evaluated as
// ln(q / (R - a)), q = R^2 - a^2 formed as the sum of the other two squares;
// terms whose coefficient is zero are dropped, so F is finite everywhere.
#pragma once

#include <math.h>

namespace gf {

__host__ __device__ __forceinline__ double an_ln(double x) { return log(x); }
__host__ __device__ __forceinline__ float an_ln(float x) { return logf(x); }
__host__ __device__ __forceinline__ double an_atan(double x) { return atan(x); }
__host__ __device__ __forceinline__ float an_atan(float x) { return atanf(x); }
__host__ __device__ __forceinline__ double an_sqrt(double x) { return sqrt(x); }
__host__ __device__ __forceinline__ float an_sqrt(float x) { return sqrtf(x); }
__host__ __device__ __forceinline__ double an_floor(double x) { return floor(x); }
__host__ __device__ __forceinline__ float an_floor(float x) { return floorf(x); }
__host__ __device__ __forceinline__ int an_imax(int a, int b) { return a > b ? a : b; }
__host__ __device__ __forceinline__ int an_imin(int a, int b) { return a < b ? a : b; }

// ln(a + R) with R = sqrt(a^2 + q), q > 0.
template <class T>
__host__ __device__ __forceinline__ T an_log(T a, T q, T R) {
    return a >= T(0) ? an_ln(a + R) : an_ln(q / (R - a));
}

// All three components of the corner function at (u, v, w).
template <class T>
__host__ __device__ __forceinline__ void an_corner(T u, T v, T w, T &fx, T &fy, T &fz) {
    const T u2 = u * u, v2 = v * v, w2 = w * w;
    const T R = an_sqrt(u2 + v2 + w2);
    fx = fy = fz = T(0);
    if (R == T(0)) return;
    const T qu = v2 + w2, qv = u2 + w2, qw = u2 + v2;
    const T Lu = qu > T(0) ? an_log(u, qu, R) : T(0);
    const T Lv = qv > T(0) ? an_log(v, qv, R) : T(0);
    const T Lw = qw > T(0) ? an_log(w, qw, R) : T(0);
    fx = v * Lw + w * Lv - (u != T(0) ? u * an_atan((v * w) / (u * R)) : T(0));
    fy = w * Lu + u * Lw - (v != T(0) ? v * an_atan((w * u) / (v * R)) : T(0));
    fz = u * Lv + v * Lu - (w != T(0) ? w * an_atan((u * v) / (w * R)) : T(0));
}

// The vertical component alone (two logarithms, one arctangent).
template <class T>
__host__ __device__ __forceinline__ T an_corner_z(T u, T v, T w) {
    const T u2 = u * u, v2 = v * v, w2 = w * w;
    const T R = an_sqrt(u2 + v2 + w2);
    if (R == T(0)) return T(0);
    const T qu = v2 + w2, qv = u2 + w2;
    const T Lu = qu > T(0) ? an_log(u, qu, R) : T(0);
    const T Lv = qv > T(0) ? an_log(v, qv, R) : T(0);
    return u * Lv + v * Lu - (w != T(0) ? w * an_atan((u * v) / (w * R)) : T(0));
}

// Neumaier-compensated running sum.
template <class T>
struct AnSum {
    T s = T(0), c = T(0);
    __host__ __device__ __forceinline__ void add(T x) {
        const T t = s + x;
        c += ((s < T(0) ? -s : s) >= (x < T(0) ? -x : x)) ? ((s - t) + x) : ((x - t) + s);
        s = t;
    }
    __host__ __device__ __forceinline__ T value() const { return s + c; }
};

// Near field (without the factor G h) at one observer of the voxels of an
// nb^3 block, in voxel units (h = 1): rho[(k nb + j) nb + i] is the density
// of voxel [i, i+1) x [j, j+1) x [k, k+1), t the observer's position in the
// block.  Voxels within Chebyshev distance rad (2 in FP32) of the
// observer's voxel are integrated in closed form, on their corner lattice
// ((2 rad + 2)^3 corners, each
// weighted by the signed sum of the densities of the included voxels that
// share it); the others take the midpoint rule plus the l = 4 term of a
// uniform cube, whose potential is m [1/R - (7/192)(sum R_i^4 - 3/5 R^4)/R^9]
// up to l = 6 (a cube has no quadrupole), so their error falls like
// (h/d)^6 from two voxels away.  FP32 arithmetic gives about 1e-5 of the
// block's field (the closed form's cancellation grows like (d/h)^3, which is
// why it stops at distance 2).  Rows of the block are summed plainly and
// merged into compensated totals.
template <class T>
__host__ __device__ inline void an_near_block(const T *rho, int nb, T tx, T ty, T tz, T g[3], int rad = 2) {
    const int vi = (int)an_floor(tx), vj = (int)an_floor(ty), vk = (int)an_floor(tz);
    AnSum<T> Sx, Sy, Sz;
    for (int k = 0; k < nb; ++k)
        for (int j = 0; j < nb; ++j) {
            T gx = T(0), gy = T(0), gz = T(0);
            for (int i = 0; i < nb; ++i) {
                const int di = i - vi, dj = j - vj, dk = k - vk;
                const int sh = an_imax(an_imax(di < 0 ? -di : di, dj < 0 ? -dj : dj), dk < 0 ? -dk : dk);
                const T m = rho[(k * nb + j) * nb + i];
                if (sh <= rad || m == T(0)) continue;
                const T Rx = tx - (T(i) + T(0.5)), Ry = ty - (T(j) + T(0.5)), Rz = tz - (T(k) + T(0.5));
                const T r2 = Rx * Rx + Ry * Ry + Rz * Rz;
                const T ri = T(1) / an_sqrt(r2), ri2 = ri * ri;
                const T ri3 = ri * ri2, ri9 = ri3 * ri3 * ri3, ri11 = ri9 * ri2;
                const T S4 = Rx * Rx * Rx * Rx + Ry * Ry * Ry * Ry + Rz * Rz * Rz * Rz;
                const T q = T(9) * (S4 - T(0.6) * r2 * r2) * ri11;
                const T c = T(7) / T(192);
                gx += m * (Rx * ri3 + c * ((T(4) * Rx * Rx - T(2.4) * r2) * Rx * ri9 - q * Rx));
                gy += m * (Ry * ri3 + c * ((T(4) * Ry * Ry - T(2.4) * r2) * Ry * ri9 - q * Ry));
                gz += m * (Rz * ri3 + c * ((T(4) * Rz * Rz - T(2.4) * r2) * Rz * ri9 - q * Rz));
            }
            Sx.add(gx);
            Sy.add(gy);
            Sz.add(gz);
        }
    // closed form: voxels [lo, hi] (clipped to the block) around the observer's voxel
    const int ilo = an_imax(vi - rad, 0), ihi = an_imin(vi + rad, nb - 1);
    const int jlo = an_imax(vj - rad, 0), jhi = an_imin(vj + rad, nb - 1);
    const int klo = an_imax(vk - rad, 0), khi = an_imin(vk + rad, nb - 1);
    for (int K = klo; K <= khi + 1; ++K)
        for (int J = jlo; J <= jhi + 1; ++J) {
            T gx = T(0), gy = T(0), gz = T(0);
            for (int I = ilo; I <= ihi + 1; ++I) {
                T D = T(0);
                for (int e = 0; e < 2; ++e)
                    for (int f = 0; f < 2; ++f)
                        for (int a = 0; a < 2; ++a) {
                            const int i = I - a, j = J - f, k = K - e;
                            if (i < ilo || i > ihi || j < jlo || j > jhi || k < klo || k > khi) continue;
                            const T r = rho[(k * nb + j) * nb + i];
                            D += ((a + f + e) & 1) ? r : -r;
                        }
                if (D == T(0)) continue;
                T fx, fy, fz;
                an_corner(T(I) - tx, T(J) - ty, T(K) - tz, fx, fy, fz);
                gx += D * fx;
                gy += D * fy;
                gz += D * fz;
            }
            Sx.add(gx);
            Sy.add(gy);
            Sz.add(gz);
        }
    g[0] = Sx.value();
    g[1] = Sy.value();
    g[2] = Sz.value();
}

}  // namespace gf
