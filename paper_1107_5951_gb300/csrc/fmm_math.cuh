// fmm_math.cuh -- solid-harmonic expansions of the Laplace kernel and the
// translation operators of the FMM (Sec. 2.3: ME/LE of Eq. 9, P2M, M2M, M2L,
// L2L, L2P of Fig. 3), as host/device functions shared by the table
// generator and the evaluation kernels of this library.
//
// Harmonics.  For x = (x, y, z), r = |x|, the normalised regular and
// irregular solid harmonics R_n^m, I_n^m (n >= 0, |m| <= n) obey
//
//   R_0^0 = 1,            R_n^n = -sqrt((2n-1)/(2n)) (x + i y) R_{n-1}^{n-1}
//   R_n^m = [(2n-1) z R_{n-1}^m - sqrt((n-1+m)(n-1-m)) r^2 R_{n-2}^m]
//           / sqrt((n+m)(n-m))
//   I_0^0 = 1/r,          I_n^n = -sqrt((2n-1)/(2n)) (x + i y) / r^2 I_{n-1}^{n-1}
//   I_n^m = [(2n-1) z I_{n-1}^m - sqrt((n-1+m)(n-1-m)) I_{n-2}^m]
//           / (r^2 sqrt((n+m)(n-m)))
//
// with X_n^{-m} = (-1)^m conj(X_n^m); |R_n^m| <= r^n, |I_n^m| <= r^{-n-1}.
// In this normalisation the addition theorem reads
//
//   1/|x - y| = sum_{n,m} conj(R_n^m(y)) I_n^m(x)        (|y| < |x|)
//
// which is the factorisation of Eq. 9: the kernel splits into terms that
// depend on the source only and terms that depend on the target only.
//
// Expansions.  A box of side s centred at c holds its expansions in units
// of s (so one set of operator tables serves every level):
//   ME  M_n^m = sum_i q_i conj(R_n^m((x_i - c)/s))
//       phi(x) = (1/s) sum_{n,m} M_n^m I_n^m((x - c)/s) * w_n^m
//   LE  phi(x) = (1/s) sum_{n,m} L_n^m conj(R_n^m((x - c)/s))
// Real storage: K = (p+1)^2 reals per expansion, for each degree n:
//   [Re X_n^0, Re X_n^1, Im X_n^1, ..., Re X_n^n, Im X_n^n]
// i.e. index n^2 for m = 0 and n^2 + 2m - 1 (Re), n^2 + 2m (Im) for m > 0;
// the m < 0 half follows from the symmetry above.
#pragma once

#include <math.h>
#include <stdint.h>

#if defined(__CUDACC__)
#define GF_HD __host__ __device__ __forceinline__
#else
#define GF_HD inline
#endif

namespace gf {

GF_HD int tri(int n, int m) { return n * (n + 1) / 2 + m; }   // m >= 0
GF_HD int kidx_re(int n, int m) { return m == 0 ? n * n : n * n + 2 * m - 1; }
GF_HD int kidx_im(int n, int m) { return n * n + 2 * m; }       // m > 0

// Regular harmonics R_n^m (m >= 0) up to degree P into re/im[tri(n,m)].
template <class T>
GF_HD void regular_harmonics(int P, T x, T y, T z, T *re, T *im) {
    const T r2 = x * x + y * y + z * z;
    re[0] = T(1);
    im[0] = T(0);
    for (int n = 1; n <= P; ++n) {  // sectoral
        const T f = -sqrt(T(2 * n - 1) / T(2 * n));
        const T pr = re[tri(n - 1, n - 1)], pi = im[tri(n - 1, n - 1)];
        re[tri(n, n)] = f * (x * pr - y * pi);
        im[tri(n, n)] = f * (x * pi + y * pr);
    }
    for (int m = 0; m < P; ++m) {
        // n = m + 1
        {
            const int n = m + 1;
            const T a = T(2 * n - 1) / sqrt(T((n + m) * (n - m)));
            re[tri(n, m)] = a * z * re[tri(n - 1, m)];
            im[tri(n, m)] = a * z * im[tri(n - 1, m)];
        }
        for (int n = m + 2; n <= P; ++n) {
            const T inv = T(1) / sqrt(T((n + m) * (n - m)));
            const T a = T(2 * n - 1) * inv;
            const T b = sqrt(T((n - 1 + m) * (n - 1 - m))) * inv * r2;
            re[tri(n, m)] = a * z * re[tri(n - 1, m)] - b * re[tri(n - 2, m)];
            im[tri(n, m)] = a * z * im[tri(n - 1, m)] - b * im[tri(n - 2, m)];
        }
    }
}

// Irregular harmonics I_n^m (m >= 0) up to degree P.
template <class T>
GF_HD void irregular_harmonics(int P, T x, T y, T z, T *re, T *im) {
    const T r2 = x * x + y * y + z * z;
    const T ir2 = T(1) / r2;
    re[0] = sqrt(ir2);
    im[0] = T(0);
    for (int n = 1; n <= P; ++n) {
        const T f = -sqrt(T(2 * n - 1) / T(2 * n)) * ir2;
        const T pr = re[tri(n - 1, n - 1)], pi = im[tri(n - 1, n - 1)];
        re[tri(n, n)] = f * (x * pr - y * pi);
        im[tri(n, n)] = f * (x * pi + y * pr);
    }
    for (int m = 0; m < P; ++m) {
        {
            const int n = m + 1;
            const T a = T(2 * n - 1) / sqrt(T((n + m) * (n - m))) * ir2;
            re[tri(n, m)] = a * z * re[tri(n - 1, m)];
            im[tri(n, m)] = a * z * im[tri(n - 1, m)];
        }
        for (int n = m + 2; n <= P; ++n) {
            const T inv = T(1) / sqrt(T((n + m) * (n - m)));
            const T a = T(2 * n - 1) * inv * ir2;
            const T b = sqrt(T((n - 1 + m) * (n - 1 - m))) * inv * ir2;
            re[tri(n, m)] = a * z * re[tri(n - 1, m)] - b * re[tri(n - 2, m)];
            im[tri(n, m)] = a * z * im[tri(n - 1, m)] - b * im[tri(n - 2, m)];
        }
    }
}

// X_n^m for any |m| <= n from the m >= 0 table (X^{-m} = (-1)^m conj X^m).
template <class T>
GF_HD void harm_get(const T *re, const T *im, int n, int m, T &xr, T &xi) {
    if (m >= 0) {
        xr = re[tri(n, m)];
        xi = im[tri(n, m)];
    } else {
        const T s = (m & 1) ? T(-1) : T(1);
        xr = s * re[tri(n, -m)];
        xi = -s * im[tri(n, -m)];
    }
}

// Logarithms of factorials up to kLogFactN - 1, for the binomial factors of
// the translation operators in the normalised basis.
constexpr int kLogFactN = 72;

// sqrt( C(a, b) * C(c, d) ) from log-factorials lf[k] = ln k!.
GF_HD double sqrt_binom2(const double *lf, int a, int b, int c, int d) {
    return exp(0.5 * (lf[a] - lf[b] - lf[a - b] + lf[c] - lf[d] - lf[c - d]));
}

// ---------------------------------------------------------------- operators
// Operator kinds for the table generator.
enum OpKind { OP_M2M = 0, OP_M2L = 1, OP_L2L = 2 };

// Complex coefficient of input component X_{l'}^{k'} (any sign of k') in
// output component Y_n^m (m >= 0) of one translation operator, given the
// harmonic table (R for M2M/L2L at the shift d, I for M2L at the offset o).
//   M2M: Y_n^m = sum_{l,k} 2^{l-n} sqrt(C(n-m, l-k) C(n+m, l+k))
//                conj(R_l^k(d)) X_{n-l}^{m-k}
//   M2L: Y_n^m = sum_{l,k} (-1)^l sqrt(C(n+l-m-k, n-m) C(n+l+m+k, n+m))
//                I_{n+l}^{m+k}(o) X_l^k
//   L2L: Y_j^i = 2^{-(j+1)} sum_{l,k} sqrt(C(j+l-i-k, j-i) C(j+l+i+k, j+i))
//                conj(R_l^k(d)) X_{j+l}^{i+k}
// d is the child centre minus the parent centre in units of the parent side
// (M2M), or the child centre minus the parent centre in parent units (L2L);
// o is the source box centre minus the target box centre in box units.
GF_HD void op_coef(int kind, int p, int n, int m, int lp, int kp, const double *hre,
                   const double *him, const double *lf, double &cr, double &ci) {
    cr = 0.0;
    ci = 0.0;
    if (kind == OP_M2M) {
        const int l = n - lp, k = m - kp;
        if (l < 0 || k < -l || k > l) return;
        double hr, hi;
        harm_get(hre, him, l, k, hr, hi);
        const double f = ldexp(1.0, l - n) * sqrt_binom2(lf, n - m, l - k, n + m, l + k);
        cr = f * hr;
        ci = -f * hi;
    } else if (kind == OP_M2L) {
        const int l = lp, k = kp;
        if (l > p) return;
        const int N = n + l, Mm = m + k;
        double hr, hi;
        harm_get(hre, him, N, Mm, hr, hi);
        const double s = (l & 1) ? -1.0 : 1.0;
        const double f = s * sqrt_binom2(lf, N - Mm, n - m, N + Mm, n + m);
        cr = f * hr;
        ci = f * hi;
    } else {
        const int j = n, i = m;
        const int l = lp - j, k = kp - i;
        if (l < 0 || k < -l || k > l) return;
        double hr, hi;
        harm_get(hre, him, l, k, hr, hi);
        const double f = ldexp(1.0, -(j + 1)) * sqrt_binom2(lf, j + l - i - k, j - i, j + l + i + k, j + i);
        cr = f * hr;
        ci = -f * hi;
    }
}

// Real K x K operator entry: output real component `row`, input real
// component `col` (layout above).  The unit input at (l', k' > 0, Re) is
// X^{k'} = 1, X^{-k'} = (-1)^{k'}; at (l', k' > 0, Im) it is X^{k'} = i,
// X^{-k'} = -(-1)^{k'} i; at (l', 0) it is X^0 = 1.
GF_HD double op_entry(int kind, int p, int row, int col, const double *hre, const double *him,
                      const double *lf) {
    int n = (int)sqrt((double)row);
    while (n * n > row) --n;
    while ((n + 1) * (n + 1) <= row) ++n;
    const int ro = row - n * n;
    const int m = (ro + 1) / 2;
    const bool out_im = ro > 0 && (ro % 2 == 0);
    int l = (int)sqrt((double)col);
    while (l * l > col) --l;
    while ((l + 1) * (l + 1) <= col) ++l;
    const int co = col - l * l;
    const int k = (co + 1) / 2;
    const bool in_im = co > 0 && (co % 2 == 0);
    double yr = 0.0, yi = 0.0;
    double cr, ci;
    if (k == 0) {
        op_coef(kind, p, n, m, l, 0, hre, him, lf, cr, ci);
        yr = cr;
        yi = ci;
    } else {
        const double sg = (k & 1) ? -1.0 : 1.0;
        double c2r, c2i;
        op_coef(kind, p, n, m, l, k, hre, him, lf, cr, ci);
        op_coef(kind, p, n, m, l, -k, hre, him, lf, c2r, c2i);
        if (!in_im) {  // X^k = 1, X^-k = sg
            yr = cr + sg * c2r;
            yi = ci + sg * c2i;
        } else {       // X^k = i, X^-k = -sg i
            yr = -ci + sg * c2i;
            yi = cr - sg * c2r;
        }
    }
    return out_im ? yi : yr;
}


// ---------------------------------------------------------------- L2P
// Gradient of a local expansion.  With phi(x) = (1/s) sum L_n^m conj(R_n^m(X)),
// X = (x - c)/s, the derivative rules of the normalised regular harmonics
//   d/dz R_n^m = sqrt((n-m)(n+m)) R_{n-1}^m
//   d/dx R_n^m = (-a_{n,m} R_{n-1}^{m-1} + b_{n,m} R_{n-1}^{m+1}) / 2
//   d/dy R_n^m = -i (a_{n,m} R_{n-1}^{m-1} + b_{n,m} R_{n-1}^{m+1}) / 2
//   a_{n,m} = sqrt((n+m)(n+m-1)),  b_{n,m} = sqrt((n-m)(n-m-1))
// give s^2 d(phi)/dx_a = sum_{n<p, m} D^a_n^m conj(R_n^m(X)), with
//   D^z_n^m = sqrt((n+1-m)(n+1+m)) L_{n+1}^m
//   D^x_n^m = (-a_{n+1,m+1} L_{n+1}^{m+1} + b_{n+1,m-1} L_{n+1}^{m-1}) / 2
//   D^y_n^m = i (a_{n+1,m+1} L_{n+1}^{m+1} + b_{n+1,m-1} L_{n+1}^{m-1}) / 2
// stored in the real layout of degree p-1 (p^2 reals each).
template <class T>
GF_HD void lget(const T *L, int n, int m, T &r, T &i) {   // L_n^m, any sign of m
    if (m > n || -m > n) {
        r = T(0);
        i = T(0);
        return;
    }
    if (m == 0) {
        r = L[n * n];
        i = T(0);
    } else if (m > 0) {
        r = L[n * n + 2 * m - 1];
        i = L[n * n + 2 * m];
    } else {
        const T s = ((-m) & 1) ? T(-1) : T(1);
        r = s * L[n * n - 2 * m - 1];
        i = -s * L[n * n - 2 * m];
    }
}

// One real component (index `idx` in the degree-(p-1) layout) of the three
// gradient expansions D^x, D^y, D^z of the local expansion L (degree p).
template <class T>
GF_HD void grad_coeff(const T *L, int idx, T &dx, T &dy, T &dz) {
    int n = (int)sqrtf((float)idx);   // corrected below (idx < 2^24)
    while (n * n > idx) --n;
    while ((n + 1) * (n + 1) <= idx) ++n;
    const int ro = idx - n * n;
    const int m = (ro + 1) / 2;
    const bool want_im = ro > 0 && (ro % 2 == 0);
    const int N = n + 1;
    T lr, li, pr, pi, mr, mi;
    lget(L, N, m, lr, li);
    lget(L, N, m + 1, pr, pi);
    lget(L, N, m - 1, mr, mi);
    const T cz = sqrt(T((N - m) * (N + m)));
    const T a = sqrt(T((N + m + 1) * (N + m)));       // a_{N, m+1}
    const T b = sqrt(T((N - m + 1) * (N - m)));       // b_{N, m-1}
    const T xr = T(0.5) * (-a * pr + b * mr), xi = T(0.5) * (-a * pi + b * mi);
    const T sr = T(0.5) * (a * pr + b * mr), si = T(0.5) * (a * pi + b * mi);
    // D^y = i * (sr + i si) = -si + i sr
    if (!want_im) {
        dx = xr;
        dy = -si;
        dz = cz * lr;
    } else {
        dx = xi;
        dy = sr;
        dz = cz * li;
    }
}

// sum_{n<p, m} D_n^m conj(R_n^m(X)) for the three expansions at once,
// sweeping the harmonics column by column (m fixed, n rising) so that only
// two previous degrees are live.  D* are in the degree-(p-1) real layout.
template <class T>
GF_HD void l2p_sum(int p, const T *Dx, const T *Dy, const T *Dz, T X, T Y, T Z, T &gx, T &gy,
                   T &gz) {
    const T r2 = X * X + Y * Y + Z * Z;
    T sr = T(1), si = T(0);  // sectoral R_m^m
    gx = gy = gz = T(0);
    for (int m = 0; m < p; ++m) {
        if (m > 0) {
            const T f = -sqrt(T(2 * m - 1) / T(2 * m));
            const T nr = f * (X * sr - Y * si), ni = f * (X * si + Y * sr);
            sr = nr;
            si = ni;
        }
        T r1 = sr, i1 = si, r0 = T(0), i0 = T(0);  // R_{n-1}, R_{n-2}
        for (int n = m; n < p; ++n) {
            T cr, ci;
            if (n == m) {
                cr = sr;
                ci = si;
            } else {
                const T inv = T(1) / sqrt(T((n + m) * (n - m)));
                const T a = T(2 * n - 1) * inv;
                const T b = (n - 1 > m) ? sqrt(T((n - 1 + m) * (n - 1 - m))) * inv * r2 : T(0);
                cr = a * Z * r1 - b * r0;
                ci = a * Z * i1 - b * i0;
                r0 = r1;
                i0 = i1;
                r1 = cr;
                i1 = ci;
            }
            if (m == 0) {
                const int k = n * n;
                gx += Dx[k] * cr;
                gy += Dy[k] * cr;
                gz += Dz[k] * cr;
            } else {
                const int k = n * n + 2 * m - 1;
                gx += T(2) * (Dx[k] * cr + Dx[k + 1] * ci);
                gy += T(2) * (Dy[k] * cr + Dy[k + 1] * ci);
                gz += T(2) * (Dz[k] * cr + Dz[k + 1] * ci);
            }
        }
    }
}

}  // namespace gf
