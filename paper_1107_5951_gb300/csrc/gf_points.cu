// gf_points.cu -- weighted point sources: the quadrature points of deformed
// hexahedral cells (the general SUM-G1 of Sec. 2.1, integrated in reference
// coordinates with the Jacobian of each cell's map) and scattered density
// points with their volumes (Sec. 4: the FMM takes a random point
// distribution once each point carries the volume of its Voronoi cell).
//
// Source s sits at x_s with volume weight a_s and samples density c(s) =
// s / per_cell; its mass is rho_{c(s)} a_s and the field is Eq. 7 over the
// sources,
//
//   g(r) = G sum_s rho_{c(s)} a_s (r - x_s) / |r - x_s|^3,
//
// by direct summation (FP64 with compensated tile sums; mixed precision with
// positions split into an exact integer part and a fraction of a fixed
// quantum) or by the FMM.  The FMM's tree is uniform: the leaf side is chosen
// from the sources' extent so that about kPointsPerLeaf sources share a leaf
// when they fill it; the sources are sorted by the linear index of their leaf
// in the dense block of source leaves, and every leaf records its first
// sorted source.  The observer tree, M2M, M2L, L2L and L2P are those of the
// voxel FMM (in leaf units: the plan's length unit is the leaf side), so
// only the P2M (harmonics of each point) and the near field (each
// neighbour leaf's points) are specific to points.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <new>
#include <vector>

#include "fmm_math.cuh"
#include "gf_fmm.cuh"
#include "gf_prim.cuh"
#include "gf_simd.cuh"

namespace gf {
namespace {

constexpr int kPtTile = 256;
constexpr double kPointsPerLeaf = 48.0;

// ---------------------------------------------------------------- hexahedra
// Quadrature point q of cell c: the trilinear image of the reference node
// xi_q, and its volume weight 8 (w_q / sum w) |det dx/dxi| (corner a = i +
// 2 j + 4 k of the cell at reference signs (2i - 1, 2j - 1, 2k - 1)).
__global__ void hex_sources_kernel(const double *__restrict__ verts, int64_t ncell, QuadRule qr,
                                   double *__restrict__ x, double *__restrict__ a) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= ncell * qr.nq) return;
    const int64_t c = s / qr.nq;
    const int q = (int)(s - c * qr.nq);
    const double *X = verts + 24 * c;
    const double e0 = qr.xi[q][0], e1 = qr.xi[q][1], e2 = qr.xi[q][2];
    double p[3] = {0.0, 0.0, 0.0};
    double J[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const double s0 = (k & 1) ? 1.0 : -1.0, s1 = (k & 2) ? 1.0 : -1.0, s2 = (k & 4) ? 1.0 : -1.0;
        const double f0 = 1.0 + s0 * e0, f1 = 1.0 + s1 * e1, f2 = 1.0 + s2 * e2;
        const double N = 0.125 * f0 * f1 * f2;
        const double d0 = 0.125 * s0 * f1 * f2, d1 = 0.125 * f0 * s1 * f2, d2 = 0.125 * f0 * f1 * s2;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double v = X[3 * k + d];
            p[d] += N * v;
            J[d][0] += d0 * v;
            J[d][1] += d1 * v;
            J[d][2] += d2 * v;
        }
    }
    const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                       J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    for (int d = 0; d < 3; ++d) x[3 * s + d] = p[d];
    a[s] = 8.0 * qr.wn[q] * fabs(det);
}

// The same in FP32 relative to the cell's first corner, for mixed-precision
// plans.  The corners are read as 64-bit fixed point with k fractional bits
// (k from the cell's largest coordinate), so the corner differences are
// exact integers; the trilinear image of each node and its Jacobian are
// evaluated on those differences in FP32 as tensor products (along xi,
// then eta, then zeta), and the image is added back to the first corner in
// fixed point.  Integer operations replace every FP64 one.  One thread per
// cell.
struct HexRuleF {
    int nq;
    float xi[kMaxQuad][3];
    float w8[kMaxQuad];   // 8 w_q / sum(w)
};

__global__ void hex_sources_fix(const double *__restrict__ verts, int64_t ncell, HexRuleF qr, double *__restrict__ x,
                                double *__restrict__ a) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const double *X = verts + 24 * c;
    // fixed-point scale: |coordinate| 2^k < 2^62 for every corner
    unsigned emax = 0;
#pragma unroll
    for (int v = 0; v < 24; ++v)
        emax = max(emax, (unsigned)((__double_as_longlong(X[v]) >> 52) & 0x7ff));
    const int k = min(80, 61 - ((int)emax - 1022));
    long long X0[3];
    float D[8][3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        X0[d] = to_fix(X[d], k);
        D[0][d] = 0.f;
    }
    const float inv2k = __int_as_float((127 - k) << 23);   // 2^-k (k <= 80)
#pragma unroll
    for (int v = 1; v < 8; ++v)
#pragma unroll
        for (int d = 0; d < 3; ++d) D[v][d] = fix_to_f32(to_fix(X[3 * v + d], k) - X0[d]) * inv2k;
    for (int q = 0; q < qr.nq; ++q) {
        const float u = qr.xi[q][0], w = qr.xi[q][1], t = qr.xi[q][2];
        const float f0 = 0.5f * (1.f - u), f1 = 0.5f * (1.f + u);
        const float g0 = 0.5f * (1.f - w), g1 = 0.5f * (1.f + w);
        const float h0 = 0.5f * (1.f - t), h1 = 0.5f * (1.f + t);
        float p[3], J[3][3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            // along xi: e_jk and d/dxi for the four (eta, zeta) corners
            float e[4], ex[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                e[r] = f0 * D[2 * r][d] + f1 * D[2 * r + 1][d];
                ex[r] = 0.5f * (D[2 * r + 1][d] - D[2 * r][d]);
            }
            // along eta (r = j + 2 k)
            const float e0 = g0 * e[0] + g1 * e[1], e1 = g0 * e[2] + g1 * e[3];
            const float ex0 = g0 * ex[0] + g1 * ex[1], ex1 = g0 * ex[2] + g1 * ex[3];
            const float ey0 = 0.5f * (e[1] - e[0]), ey1 = 0.5f * (e[3] - e[2]);
            // along zeta
            p[d] = h0 * e0 + h1 * e1;
            J[d][0] = h0 * ex0 + h1 * ex1;
            J[d][1] = h0 * ey0 + h1 * ey1;
            J[d][2] = 0.5f * (e1 - e0);
        }
        const float det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                          J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                          J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        const int64_t s = c * qr.nq + q;
#pragma unroll
        for (int d = 0; d < 3; ++d) x[3 * s + d] = fix_to_f64(X0[d] + f32_to_fix(p[d], k), k);
        a[s] = f32_to_f64(qr.w8[q] * fabsf(det));
    }
}

// ---------------------------------------------------------------- direct
__device__ __forceinline__ void neumaier_p(double &s, double &c, double x) {
    const double t = s + x;
    c += (fabs(s) >= fabs(x)) ? ((s - t) + x) : ((x - t) + s);
    s = t;
}

__device__ __forceinline__ double load_rho_p(const void *rho, int f32, int64_t i) {
    return f32 ? (double)__ldg(reinterpret_cast<const float *>(rho) + i) : __ldg(reinterpret_cast<const double *>(rho) + i);
}

// One thread per observer; sources staged kPtTile at a time per block with
// their masses rho_{c(s)} a_s of batch member blockIdx.y.
__global__ void __launch_bounds__(kPtTile)
direct_points_f64(const double *__restrict__ obs, int64_t M, const double *__restrict__ src,
                  const double *__restrict__ wt, int64_t S, int per_cell, int64_t ncell, const void *__restrict__ rho,
                  int rho_f32, double G, double *__restrict__ g, double *__restrict__ gz, int *__restrict__ status) {
    __shared__ double sx[kPtTile], sy[kPtTile], sz[kPtTile], sm[kPtTile];
    const int b = blockIdx.y;
    const int64_t j = (int64_t)blockIdx.x * kPtTile + threadIdx.x;
    const bool active = j < M;
    const double rx = active ? obs[3 * j] : 0.0, ry = active ? obs[3 * j + 1] : 0.0, rz = active ? obs[3 * j + 2] : 0.0;
    double s0 = 0, c0 = 0, s1 = 0, c1 = 0, s2 = 0, c2 = 0;
    bool bad = false;
    for (int64_t t0 = 0; t0 < S; t0 += kPtTile) {
        const int64_t s = t0 + threadIdx.x;
        __syncthreads();
        if (s < S) {
            sx[threadIdx.x] = src[3 * s];
            sy[threadIdx.x] = src[3 * s + 1];
            sz[threadIdx.x] = src[3 * s + 2];
            const double r = load_rho_p(rho, rho_f32, (int64_t)b * ncell + s / per_cell);
            bad |= !isfinite(r);
            sm[threadIdx.x] = r * wt[s];
        } else {
            sx[threadIdx.x] = sy[threadIdx.x] = sz[threadIdx.x] = sm[threadIdx.x] = 0.0;
        }
        __syncthreads();
        const int cnt = (S - t0) < kPtTile ? (int)(S - t0) : kPtTile;
        double px = 0, py = 0, pz = 0;
#pragma unroll 4
        for (int u = 0; u < cnt; ++u) {
            const double dx = rx - sx[u], dy = ry - sy[u], dz = rz - sz[u];
            const double r2 = dx * dx + dy * dy + dz * dz;
            const double ri = rsqrt(r2);
            const double k3 = (r2 > 0.0) ? sm[u] * (ri * ri * ri) : 0.0;
            px = fma(k3, dx, px);
            py = fma(k3, dy, py);
            pz = fma(k3, dz, pz);
        }
        neumaier_p(s0, c0, px);
        neumaier_p(s1, c1, py);
        neumaier_p(s2, c2, pz);
    }
    if (bad && status && blockIdx.x == 0) atomicOr(status, 1);
    if (active) {
        const double vx = G * (s0 + c0), vy = G * (s1 + c1), vz = G * (s2 + c2);
        if (g) {
            double *o = g + ((int64_t)b * M + j) * 3;
            o[0] = vx;
            o[1] = vy;
            o[2] = vz;
        }
        if (gz) gz[(int64_t)b * M + j] = vz;
    }
}

// Positions in units of the quantum q from the corner lo, split into an
// integer part (exact in FP32 below 2^24) and the fraction.
__global__ void split_points(const double *__restrict__ x, int64_t n, double lo0, double lo1, double lo2,
                             double inv_q, float *__restrict__ xi, float *__restrict__ xf) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const double lo[3] = {lo0, lo1, lo2};
    for (int a = 0; a < 3; ++a) {
        const double u = (x[3 * j + a] - lo[a]) * inv_q;
        const double fl = floor(u);
        xi[3 * j + a] = (float)fl;
        xf[3 * j + a] = (float)(u - fl);
    }
}

// Mixed precision: the separation (ri - si) + (rf - sf) in quanta is an exact
// integer difference plus one rounding; FP32 kernel, FP64 sum of the tiles.
__global__ void __launch_bounds__(kPtTile)
direct_points_mixed(const float *__restrict__ oi, const float *__restrict__ of, int64_t M,
                    const float *__restrict__ si, const float *__restrict__ sf, const double *__restrict__ wt,
                    int64_t S, int per_cell, int64_t ncell, const void *__restrict__ rho, int rho_f32, float q,
                    double Gq, double *__restrict__ g, double *__restrict__ gz, int *__restrict__ status) {
    __shared__ float ti[kPtTile][3], tf[kPtTile][3], tm[kPtTile];
    const int b = blockIdx.y;
    const int64_t j = (int64_t)blockIdx.x * kPtTile + threadIdx.x;
    const bool active = j < M;
    float ri[3] = {0.f, 0.f, 0.f}, rf[3] = {0.f, 0.f, 0.f};
    if (active)
        for (int a = 0; a < 3; ++a) {
            ri[a] = oi[3 * j + a];
            rf[a] = of[3 * j + a];
        }
    double ax = 0, ay = 0, az = 0;
    bool bad = false;
    const double inv_q3 = 1.0 / ((double)q * (double)q * (double)q);
    for (int64_t t0 = 0; t0 < S; t0 += kPtTile) {
        const int64_t s = t0 + threadIdx.x;
        __syncthreads();
        if (s < S) {
            for (int a = 0; a < 3; ++a) {
                ti[threadIdx.x][a] = si[3 * s + a];
                tf[threadIdx.x][a] = sf[3 * s + a];
            }
            const double r = load_rho_p(rho, rho_f32, (int64_t)b * ncell + s / per_cell);
            bad |= !isfinite(r);
            tm[threadIdx.x] = (float)(r * wt[s] * inv_q3);   // mass in quantum units
        } else {
            for (int a = 0; a < 3; ++a) ti[threadIdx.x][a] = tf[threadIdx.x][a] = 0.f;
            tm[threadIdx.x] = 0.f;
        }
        __syncthreads();
        const int cnt = (S - t0) < kPtTile ? (int)(S - t0) : kPtTile;
        float px = 0.f, py = 0.f, pz = 0.f;
#pragma unroll 4
        for (int u = 0; u < cnt; ++u) {
            const float dx = (ri[0] - ti[u][0]) + (rf[0] - tf[u][0]);
            const float dy = (ri[1] - ti[u][1]) + (rf[1] - tf[u][1]);
            const float dz = (ri[2] - ti[u][2]) + (rf[2] - tf[u][2]);
            const float r2 = dx * dx + dy * dy + dz * dz;
            const float rinv = rsqrtf(r2);
            const float k3 = (r2 > 0.f) ? tm[u] * (rinv * rinv * rinv) : 0.f;
            px = fmaf(k3, dx, px);
            py = fmaf(k3, dy, py);
            pz = fmaf(k3, dz, pz);
        }
        ax += (double)px;
        ay += (double)py;
        az += (double)pz;
    }
    if (bad && status && blockIdx.x == 0) atomicOr(status, 1);
    if (active) {
        const double vx = Gq * ax, vy = Gq * ay, vz = Gq * az;
        if (g) {
            double *o = g + ((int64_t)b * M + j) * 3;
            o[0] = vx;
            o[1] = vy;
            o[2] = vz;
        }
        if (gz) gz[(int64_t)b * M + j] = vz;
    }
}

// ---------------------------------------------------------------- FMM set-up
struct PtGeo {
    double lo[3], inv_s;
    int64_t slo[3], sn[3];         // dense block of source leaves
    float lof[3], isf;             // FP32 copies for the fast key path
    int fixk;                      // fixed-point frame of the tree (< 0: not used)
    long long lofix[3], halfleaf_fix;
    float fix_to_leaf;
};

// Leaf coordinate of a source along one axis: floor((x - lo) / s) as
// evaluated in FP64 with one rounded subtraction and one rounded
// multiplication, clamped to the block.  FP32 gives the same floor unless
// the value is within a few FP32 roundings of an integer; FP64 is used only
// there.
__device__ __forceinline__ int64_t leaf_coord(double v, const PtGeo &g, int a) {
    float xf;
    const bool fin = trunc_f32(v, xf);
    const float qf = (xf - g.lof[a]) * g.isf;
    const float fl = floorf(qf);
    const float dist = fminf(qf - fl, fl + 1.f - qf);
    const float tol = ((fabsf(xf) + fabsf(g.lof[a])) * fabsf(g.isf) + fabsf(qf) + 1.f) * 2e-6f;
    int64_t c;
    if (!fin || !(dist > tol)) {
        const double f = floor(__dmul_rn(__dsub_rn(v, g.lo[a]), g.inv_s));
        c = (int64_t)fmin(fmax(f, (double)g.slo[a]), (double)(g.slo[a] + g.sn[a] - 1));
    } else {
        c = (int64_t)fl;
    }
    return min(max(c, g.slo[a]), g.slo[a] + g.sn[a] - 1);
}

// Linear index of each source's leaf in the dense block.
__global__ void point_keys(const double *__restrict__ x, int64_t S, PtGeo g, uint64_t *__restrict__ keys,
                           int32_t *__restrict__ vals, int *__restrict__ status) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    int64_t c[3];
    for (int a = 0; a < 3; ++a) {
        const double v = x[3 * s + a];
        if ((((unsigned long long)__double_as_longlong(v) >> 52) & 0x7ff) == 0x7ff) atomicOr(status + 2, 1);
        c[a] = leaf_coord(v, g, a);
    }
    keys[s] = (uint64_t)(((c[2] - g.slo[2]) * g.sn[1] + (c[1] - g.slo[1])) * g.sn[0] + (c[0] - g.slo[0]));
    vals[s] = (int32_t)s;
}

// Sorted sources: offset from the own leaf's centre and volume, leaf units.
// The leaf comes from the sorted key.  FP32: the offset as an exact
// fixed-point difference (the frame of the observers' offsets) scaled to
// leaf units; FP64: (x - lo) / s - (c + 1/2).
template <class T>
__global__ void point_gather(const double *__restrict__ x, const double *__restrict__ wt,
                             const int32_t *__restrict__ perm, const uint64_t *__restrict__ keys, int64_t S, PtGeo g,
                             double inv_s3, T *__restrict__ loc, int *__restrict__ status) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S) return;
    const int64_t s = perm[i];
    const uint64_t key = keys[i];
    const uint64_t sxy = (uint64_t)(g.sn[0] * g.sn[1]);
    const int64_t c[3] = {g.slo[0] + (int64_t)(key % (uint64_t)g.sn[0]),
                          g.slo[1] + (int64_t)((key / (uint64_t)g.sn[0]) % (uint64_t)g.sn[1]),
                          g.slo[2] + (int64_t)(key / sxy)};
    for (int a = 0; a < 3; ++a) {
        if constexpr (sizeof(T) == 4) {
            if (g.fixk >= 0) {
                const long long d = to_fix(x[3 * s + a], g.fixk) - (g.lofix[a] + (2 * c[a] + 1) * g.halfleaf_fix);
                loc[4 * i + a] = fix_to_f32(d) * g.fix_to_leaf;
                continue;
            }
        }
        const double u = (x[3 * s + a] - g.lo[a]) * g.inv_s;
        loc[4 * i + a] = (T)(u - ((double)c[a] + 0.5));
    }
    const double v = wt[s] * inv_s3;
    if (!isfinite(v)) atomicOr(status + 3, 1);
    if constexpr (sizeof(T) == 4) {
        float f;
        trunc_f32(v, f);
        loc[4 * i + 3] = f;
    } else {
        loc[4 * i + 3] = v;
    }
}

// First sorted source of every dense leaf: leaf_beg[l] = number of sources
// whose key is below l (keys sorted), by a binary search per leaf.
__global__ void point_leaf_beg(const uint64_t *__restrict__ keys, int64_t S, int64_t nleaf,
                               int64_t *__restrict__ beg) {
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l > nleaf) return;
    int64_t lo = 0, hi = S;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (keys[mid] < (uint64_t)l)
            lo = mid + 1;
        else
            hi = mid;
    }
    beg[l] = lo;
}

// ---------------------------------------------------------------- FMM forward
template <class T>
__device__ __forceinline__ void ld_loc(const T *loc, int64_t i, T &x, T &y, T &z, T &w) {
    if constexpr (sizeof(T) == 4) {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(loc) + i);
        x = v.x;
        y = v.y;
        z = v.z;
        w = v.w;
    } else {
        const double2 a = __ldg(reinterpret_cast<const double2 *>(loc) + 2 * i);
        const double2 b = __ldg(reinterpret_cast<const double2 *>(loc) + 2 * i + 1);
        x = a.x;
        y = a.y;
        z = b.x;
        w = b.y;
    }
}

// Sorted masses in leaf units: m_i = rho_{c(perm_i)} v_i, [B][S].
template <class T>
__global__ void point_masses(const void *__restrict__ rho, int rho_f32, const int32_t *__restrict__ perm,
                             const T *__restrict__ loc, int64_t S, int per_cell, int64_t ncell, int B,
                             T *__restrict__ m, int *__restrict__ status) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= S * B) return;
    const int b = (int)(e / S);
    const int64_t i = e - (int64_t)b * S;
    const double r = load_rho_p(rho, rho_f32, (int64_t)b * ncell + perm[i] / per_cell);
    if (!isfinite(r)) atomicOr(status, 1);
    m[e] = (T)(r * (double)loc[4 * i + 3]);
}

// Recursion coefficients of the regular harmonics (the recursion of
// fmm_math.cuh) for the point P2M, n <= kMaxP: for m < n, t = n (n + 1) / 2 + m,
//   c_pa[t] = (2n - 1) / sqrt((n + m)(n - m)),
//   c_pb[t] = sqrt((n - 1 + m)(n - 1 - m)) / sqrt((n + m)(n - m))  (0 for n = m + 1),
// and c_pf[n] = -sqrt((2n - 1) / (2n)), the sectoral step into R_n^n; in
// FP64 and rounded to FP32.
constexpr int kPT = (kMaxP + 1) * (kMaxP + 2) / 2;
__constant__ double c_pa[kPT], c_pb[kPT], c_pf[kMaxP + 1];
__constant__ float c_paf[kPT], c_pbf[kPT], c_pff[kMaxP + 1];

template <class T>
__device__ __forceinline__ T coef(const double *d, const float *f, int i) {
    if constexpr (sizeof(T) == 4)
        return f[i];
    else
        return d[i];
}

// P2M over the points of each leaf: ME_n^m = sum_i m_i conj(R_n^m(x_i - c)),
// x_i - c the point's offset from the leaf centre (leaf units).  One warp
// per leaf, 64 points per round: each lane runs the recursion for two
// points at once (the sectoral steps R_m^m, then the upward steps in n for
// each order m, the coefficients uniform across the warp) and writes the
// two points' mass-weighted harmonics, summed, into its own row of the
// warp's shared-memory block ([32][K], odd row stride); the lanes then sum
// the 32 rows column by column into the expansion.
constexpr int kP2MRound = 64;

template <class T>
constexpr int p2m_warps() {
    return sizeof(T) == 4 ? 4 : 2;
}

inline int p2m_stride(int K) { return K | 1; }

template <class T>
__global__ void __launch_bounds__(p2m_warps<T>() * 32)
point_p2m(const T *__restrict__ loc, const T *__restrict__ mass, const int64_t *__restrict__ leaf_beg,
          int64_t nleaf, int64_t S, int p, int B, int ldk, int stride, T *__restrict__ me) {
    extern __shared__ unsigned char shraw[];
    constexpr int W = p2m_warps<T>();
    constexpr int kMaxCols = (kMaxP + 1) * (kMaxP + 1) / 32 + 2;   // ceil(ldk / 32) for ldk <= 320
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T *rows = reinterpret_cast<T *>(shraw) + (size_t)warp * 32 * stride;
    T *row = rows + lane * stride;
    const int K = (p + 1) * (p + 1);
    for (int64_t leaf = (int64_t)blockIdx.x * W + warp; leaf < nleaf; leaf += (int64_t)gridDim.x * W) {
        const int64_t i0 = leaf_beg[leaf], i1 = leaf_beg[leaf + 1];
        for (int bb = 0; bb < B; ++bb) {
            T acc[kMaxCols];
#pragma unroll
            for (int j = 0; j < kMaxCols; ++j) acc[j] = T(0);
            for (int64_t r0 = i0; r0 < i1; r0 += kP2MRound) {
                const int64_t ia = r0 + lane, ib = r0 + 32 + lane;
                T xa = T(0), ya = T(0), za = T(0), qa = T(0), xb = T(0), yb = T(0), zb = T(0), qb = T(0), w;
                if (ia < i1) {
                    ld_loc(loc, ia, xa, ya, za, w);
                    qa = mass[(int64_t)bb * S + ia];
                }
                if (ib < i1) {
                    ld_loc(loc, ib, xb, yb, zb, w);
                    qb = mass[(int64_t)bb * S + ib];
                }
                const T r2a = xa * xa + ya * ya + za * za, r2b = xb * xb + yb * yb + zb * zb;
                T sra = T(1), sia = T(0), srb = T(1), sib = T(0);   // R_m^m of both points
                for (int m = 0; m <= p; ++m) {
                    if (m > 0) {
                        const T f = coef<T>(c_pf, c_pff, m);
                        const T fxa = f * xa, fya = f * ya, fxb = f * xb, fyb = f * yb;
                        const T nra = fxa * sra - fya * sia, nia = fxa * sia + fya * sra;
                        const T nrb = fxb * srb - fyb * sib, nib = fxb * sib + fyb * srb;
                        sra = nra;
                        sia = nia;
                        srb = nrb;
                        sib = nib;
                    }
                    T cra = sra, cia = sia, crb = srb, cib = sib;
                    T pra = T(0), pia = T(0), prb = T(0), pib = T(0);
                    int k = m * m + (m == 0 ? 0 : 2 * m - 1);   // R_m^m's real index
                    for (int n = m;; ++n) {
                        // the two points' mass-weighted conj(R_n^m), summed
                        const T vr = qa * cra + qb * crb, vi = qa * cia + qb * cib;
                        if (m == 0) {
                            row[k] = vr;
                        } else {
                            row[k] = vr;
                            row[k + 1] = -vi;
                        }
                        if (n == p) break;
                        k += 2 * n + 1;   // the same order one degree up: (n + 1)^2 - n^2
                        const int t = (n + 1) * (n + 2) / 2 + m;
                        const T av = coef<T>(c_pa, c_paf, t), bv = coef<T>(c_pb, c_pbf, t);
                        const T aza = av * za, brea = bv * r2a, azb = av * zb, breb = bv * r2b;
                        const T nra = aza * cra - brea * pra, nia = aza * cia - brea * pia;
                        const T nrb = azb * crb - breb * prb, nib = azb * cib - breb * pib;
                        pra = cra;
                        pia = cia;
                        prb = crb;
                        pib = cib;
                        cra = nra;
                        cia = nia;
                        crb = nrb;
                        cib = nib;
                    }
                }
                __syncwarp();
#pragma unroll
                for (int j = 0; j < kMaxCols; ++j) {
                    const int kk = lane + 32 * j;
                    if (kk < K) {
                        T sum = T(0);
#pragma unroll 8
                        for (int r = 0; r < 32; ++r) sum += rows[r * stride + kk];
                        acc[j] += sum;
                    }
                }
                __syncwarp();
            }
            T *dst = me + (leaf * B + bb) * ldk;
#pragma unroll
            for (int j = 0; j < kMaxCols; ++j) {
                const int kk = lane + 32 * j;
                if (kk < ldk) dst[kk] = kk < K ? acc[j] : T(0);
            }
        }
    }
}

// The FP32 P2M, the same sums in packed pairs: a lane's two points form
// one f32x2 value and one packed instruction advances both recursions (the
// coefficients are stored as duplicated pairs).  The harmonics are made in
// groups of consecutive orders m holding at most kGrpEnt real entries; a
// group's entries go to the warp's [32][kGrpEnt + 1] block and are summed
// over the rows before the next group starts (the sectoral steps below the
// group's first order are redone, a few complex products), so a warp needs
// 8 KB of shared memory and many warps fit an SM.  In each order the upward
// recursion overwrites the older of its two values (no register moves).
constexpr int kGrpEnt = 64;
constexpr int kMaxGroups = 12;
constexpr int kGrpStride = kGrpEnt + 1;
constexpr int kP2MWarpsF = 4;

struct P2MGroups {
    int ng;
    int m_lo[kMaxGroups + 1];   // group g: orders [m_lo[g], m_lo[g + 1])
    int ent0[kMaxGroups + 1];   // its entries [ent0[g], ent0[g + 1]) in generation order
};
__constant__ float2 c_a2[kPT], c_nb2[kPT], c_f2[kMaxP + 1], c_nf2[kMaxP + 1];
__constant__ P2MGroups c_grp[kMaxP + 1];
__constant__ short c_ktab[kMaxP + 1][(kMaxP + 1) * (kMaxP + 1)];   // real index of each generated entry

__device__ __forceinline__ uint64_t ldc2(const float2 &v) { return pk2(v.x, v.y); }

__global__ void __launch_bounds__(kP2MWarpsF * 32)
point_p2m_f32(const float *__restrict__ loc, const float *__restrict__ mass, const int64_t *__restrict__ leaf_beg,
              int64_t nleaf, int64_t S, int p, int B, int ldk, float *__restrict__ me) {
    __shared__ float rows_all[kP2MWarpsF][32 * kGrpStride];
    __shared__ short kt[(kMaxP + 1) * (kMaxP + 1)];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int K = (p + 1) * (p + 1);
    for (int i = threadIdx.x; i < K; i += blockDim.x) kt[i] = c_ktab[p][i];
    __syncthreads();
    float *rows = rows_all[warp];
    float *row = rows + lane * kGrpStride;
    const int ng = c_grp[p].ng;
    for (int64_t leaf = (int64_t)blockIdx.x * kP2MWarpsF + warp; leaf < nleaf;
         leaf += (int64_t)gridDim.x * kP2MWarpsF) {
        const int64_t i0 = leaf_beg[leaf], i1 = leaf_beg[leaf + 1];
        for (int bb = 0; bb < B; ++bb) {
            float *dst = me + (leaf * B + bb) * ldk;
            for (int k = K + lane; k < ldk; k += 32) dst[k] = 0.f;
            for (int g = 0; g < ng; ++g) {
                const int mlo = c_grp[p].m_lo[g], mhi = c_grp[p].m_lo[g + 1];
                const int ne = c_grp[p].ent0[g + 1] - c_grp[p].ent0[g];
                float acc0 = 0.f, acc1 = 0.f;
                for (int64_t r0 = i0; r0 < i1; r0 += kP2MRound) {
                    const int64_t ia = r0 + lane, ib = r0 + 32 + lane;
                    float xa = 0.f, ya = 0.f, za = 0.f, qa = 0.f, xb = 0.f, yb = 0.f, zb = 0.f, qb = 0.f, w;
                    if (ia < i1) {
                        ld_loc(loc, ia, xa, ya, za, w);
                        qa = mass[(int64_t)bb * S + ia];
                    }
                    if (ib < i1) {
                        ld_loc(loc, ib, xb, yb, zb, w);
                        qb = mass[(int64_t)bb * S + ib];
                    }
                    const uint64_t X = pk2(xa, xb), Y = pk2(ya, yb), Z = pk2(za, zb), Q = pk2(qa, qb);
                    const uint64_t R2 = fma2(Z, Z, fma2(Y, Y, mul2(X, X)));
                    uint64_t SR = pk2(1.f, 1.f), SI = 0;   // R_m^m of both points
                    auto sectoral = [&](int m) {
                        const uint64_t FX = mul2(ldc2(c_f2[m]), X), FY = mul2(ldc2(c_f2[m]), Y),
                                       NFY = mul2(ldc2(c_nf2[m]), Y);
                        const uint64_t nr = fma2(FX, SR, mul2(NFY, SI)), ni = fma2(FX, SI, mul2(FY, SR));
                        SR = nr;
                        SI = ni;
                    };
                    for (int m = 1; m < mlo; ++m) sectoral(m);
                    int j = 0;
                    auto put = [&](uint64_t vr, uint64_t vi, bool re_only) {
                        float l, h;
                        up2(mul2(Q, vr), l, h);
                        row[j] = l + h;
                        if (!re_only) {
                            up2(mul2(Q, vi), l, h);
                            row[j + 1] = -(l + h);   // conj
                        }
                        j += re_only ? 1 : 2;
                    };
                    for (int m = mlo; m < mhi; ++m) {
                        if (m > 0) sectoral(m);
                        const bool m0 = m == 0;
                        uint64_t Cr = SR, Ci = SI, Pr = 0, Pi = 0;   // R_n^m, R_{n-1}^m
                        put(Cr, Ci, m0);
                        int t = (m + 1) * (m + 2) / 2 + m;      // coefficient index of (n + 1, m), n = m
                        for (int n = m; n < p; n += 2) {
                            {   // P <- R_{n+1}^m
                                const uint64_t AZ = mul2(ldc2(c_a2[t]), Z), NB = mul2(ldc2(c_nb2[t]), R2);
                                Pr = fma2(AZ, Cr, mul2(NB, Pr));
                                Pi = fma2(AZ, Ci, mul2(NB, Pi));
                                put(Pr, Pi, m0);
                                t += n + 2;
                            }
                            if (n + 1 == p) break;
                            {   // C <- R_{n+2}^m
                                const uint64_t AZ = mul2(ldc2(c_a2[t]), Z), NB = mul2(ldc2(c_nb2[t]), R2);
                                Cr = fma2(AZ, Pr, mul2(NB, Cr));
                                Ci = fma2(AZ, Pi, mul2(NB, Ci));
                                put(Cr, Ci, m0);
                                t += n + 3;
                            }
                        }
                    }
                    __syncwarp();
                    if (lane < ne) {
                        float sum = 0.f;
#pragma unroll 8
                        for (int r = 0; r < 32; ++r) sum += rows[r * kGrpStride + lane];
                        acc0 += sum;
                    }
                    if (lane + 32 < ne) {
                        float sum = 0.f;
#pragma unroll 8
                        for (int r = 0; r < 32; ++r) sum += rows[r * kGrpStride + lane + 32];
                        acc1 += sum;
                    }
                    __syncwarp();
                }
                const int e0 = c_grp[p].ent0[g];
                if (lane < ne) dst[kt[e0 + lane]] = acc0;
                if (lane + 32 < ne) dst[kt[e0 + lane + 32]] = acc1;
            }
        }
    }
}

// Near field over the points of the 27 neighbour leaves + the L2P gradient
// of the leaf's local expansion + near + far in FP64, scattered to caller
// order.  One warp per work item (at most 64 observers of one leaf), two
// observers per lane.  A neighbour leaf's points are staged 64 at a time in
// the warp's shared-memory slice, as offsets from the item's leaf centre
// with their masses.  FP32: pairs of points as {x0,x1, y0,y1, z0,z1, m0,m1}
// and each observer duplicated, so one packed instruction does two pairs;
// the L2P evaluates the lane's two observers as one packed pair.
constexpr int kPtWarps = 4;
constexpr int kPtChunk = 64;

// Elements of a warp's slice (a multiple of 8): staged points, the three
// gradient expansions (FP32: duplicated pairs), 27 neighbour leaves (int64).
inline __host__ __device__ int pt_slice(int P2, int tsize) {
    const int dmul = tsize == 4 ? 2 : 1;
    return (4 * kPtChunk + 3 * dmul * P2 + 27 * (8 / tsize) + 7) & ~7;
}

struct PtEvalArgs {
    const int4 *items;
    int64_t n_items;
    const uint64_t *tkey;
    const int32_t *perm;
    const void *tloc;
    const void *loc;           // [S][4] sorted sources: offset from own leaf centre, volume
    const void *mass;          // [B][S] sorted masses (leaf units)
    const int64_t *leaf_beg;   // [nleaf + 1]
    const void *le;
    PtGeo g;
    int L, B, p, ldk;
    int64_t S, M;
    uint32_t part_lo, part_hi;
    double scale, eps2;
    double *gout, *gz;
};

template <class T>
__global__ void __launch_bounds__(kPtWarps * 32) point_eval(PtEvalArgs a) {
    extern __shared__ unsigned char shraw[];
    constexpr bool kF32 = sizeof(T) == 4;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int P2 = a.p * a.p;
    T *wsh = reinterpret_cast<T *>(shraw) + (size_t)warp * pt_slice(P2, sizeof(T));
    T *Dx = wsh + 4 * kPtChunk, *Dy = Dx + (kF32 ? 2 : 1) * P2, *Dz = Dy + (kF32 ? 2 : 1) * P2;
    int64_t *nbl = reinterpret_cast<int64_t *>(Dz + (kF32 ? 2 : 1) * P2);
    const T *tloc = reinterpret_cast<const T *>(a.tloc);
    const T *loc = reinterpret_cast<const T *>(a.loc);
    const T *mass = reinterpret_cast<const T *>(a.mass);
    const T *le = reinterpret_cast<const T *>(a.le);
    const T eps2 = (T)a.eps2;
    for (int64_t it = (int64_t)blockIdx.x * kPtWarps + warp; it < a.n_items; it += (int64_t)gridDim.x * kPtWarps) {
        const int4 item = a.items[it];
        const int leaf = item.x;
        const uint64_t key = a.tkey[leaf];
        int64_t lc[3] = {0, 0, 0};
        for (int bit = 0; bit < 21; ++bit) {
            lc[0] |= (int64_t)((key >> (3 * bit)) & 1) << bit;
            lc[1] |= (int64_t)((key >> (3 * bit + 1)) & 1) << bit;
            lc[2] |= (int64_t)((key >> (3 * bit + 2)) & 1) << bit;
        }
        T tx[2], ty[2], tz[2];
        int tid[2];
        for (int w = 0; w < 2; ++w) {
            const int r = lane + 32 * w;
            tid[w] = r < item.z ? item.y + r : -1;
            const int64_t i = tid[w] >= 0 ? tid[w] : item.y;
            tx[w] = tloc[3 * i];
            ty[w] = tloc[3 * i + 1];
            tz[w] = tloc[3 * i + 2];
        }
        __syncwarp();
        if (lane < 27) {
            const int dx = lane % 3 - 1, dy = (lane / 3) % 3 - 1, dz = lane / 9 - 1;
            const int64_t sx_ = lc[0] + dx - a.g.slo[0], sy_ = lc[1] + dy - a.g.slo[1], sz_ = lc[2] + dz - a.g.slo[2];
            const bool in = sx_ >= 0 && sy_ >= 0 && sz_ >= 0 && sx_ < a.g.sn[0] && sy_ < a.g.sn[1] && sz_ < a.g.sn[2] &&
                            in_source_part(lc[0] + dx, lc[1] + dy, lc[2] + dz, a.L - 2, a.part_lo, a.part_hi);
            nbl[lane] = in ? (sz_ * a.g.sn[1] + sy_) * a.g.sn[0] + sx_ : -1;
        }
        __syncwarp();
        for (int bb = 0; bb < a.B; ++bb) {
            T hx[2] = {T(0), T(0)}, hy[2] = {T(0), T(0)}, hz[2] = {T(0), T(0)};
            T lx[2] = {T(0), T(0)}, ly[2] = {T(0), T(0)}, lz[2] = {T(0), T(0)};
            for (int nb = 0; nb < 27; ++nb) {
                const int64_t sl = nbl[nb];
                if (sl < 0) continue;
                const T ox = T(nb % 3 - 1), oy = T((nb / 3) % 3 - 1), oz = T(nb / 9 - 1);
                const int64_t i0 = a.leaf_beg[sl], i1 = a.leaf_beg[sl + 1];
                T px[2] = {T(0), T(0)}, py[2] = {T(0), T(0)}, pz[2] = {T(0), T(0)};
                uint64_t qx[2] = {0, 0}, qy[2] = {0, 0}, qz[2] = {0, 0};   // packed sums (FP32)
                for (int64_t c0 = i0; c0 < i1; c0 += kPtChunk) {
                    const int cnt = (int)min((int64_t)kPtChunk, i1 - c0);
                    __syncwarp();
                    for (int s = lane; s < cnt; s += 32) {
                        const int64_t i = c0 + s;
                        T x, y, z, w;
                        ld_loc(loc, i, x, y, z, w);
                        const T mq = mass[(int64_t)bb * a.S + i];
                        if constexpr (kF32) {
                            T *rec = wsh + (s >> 1) * 8 + (s & 1);
                            rec[0] = x + ox;
                            rec[2] = y + oy;
                            rec[4] = z + oz;
                            rec[6] = mq;
                        } else {
                            T *rec = wsh + 4 * s;
                            rec[0] = x + ox;
                            rec[1] = y + oy;
                            rec[2] = z + oz;
                            rec[3] = mq;
                        }
                    }
                    if constexpr (kF32) {
                        // an odd chunk ends with a massless point far away
                        if ((cnt & 1) && lane == 0) {
                            T *rec = wsh + (cnt >> 1) * 8 + 1;
                            rec[0] = rec[2] = rec[4] = T(1.0e4);
                            rec[6] = T(0);
                        }
                        __syncwarp();
                        uint64_t TX[2], TY[2], TZ[2];
#pragma unroll
                        for (int w = 0; w < 2; ++w) {
                            TX[w] = pk2(tx[w], tx[w]);
                            TY[w] = pk2(ty[w], ty[w]);
                            TZ[w] = pk2(tz[w], tz[w]);
                        }
                        const int npair = (cnt + 1) >> 1;
#pragma unroll 2
                        for (int q = 0; q < npair; ++q) {
                            const ulonglong2 xy = *reinterpret_cast<const ulonglong2 *>(wsh + q * 8);
                            const ulonglong2 zw = *reinterpret_cast<const ulonglong2 *>(wsh + q * 8 + 4);
#pragma unroll
                            for (int w = 0; w < 2; ++w) {
                                const uint64_t DX = sub2(TX[w], xy.x), DY = sub2(TY[w], xy.y), DZ = sub2(TZ[w], zw.x);
                                const uint64_t R2 = fma2(DZ, DZ, fma2(DY, DY, mul2(DX, DX)));
                                float r0, r1;
                                up2(R2, r0, r1);
                                // a point on the observer contributes nothing
                                const float i0f = r0 > (float)eps2 ? rsqrt_ftz(r0) : 0.f;
                                const float i1f = r1 > (float)eps2 ? rsqrt_ftz(r1) : 0.f;
                                const uint64_t RI = pk2(i0f, i1f);
                                const uint64_t K3 = mul2(mul2(mul2(RI, RI), RI), zw.y);
                                qx[w] = fma2(K3, DX, qx[w]);
                                qy[w] = fma2(K3, DY, qy[w]);
                                qz[w] = fma2(K3, DZ, qz[w]);
                            }
                        }
                    } else {
                        __syncwarp();
                        for (int s = 0; s < cnt; ++s) {
                            const T ux = wsh[4 * s], uy = wsh[4 * s + 1], uz = wsh[4 * s + 2], mq = wsh[4 * s + 3];
#pragma unroll
                            for (int w = 0; w < 2; ++w) {
                                const T dx = tx[w] - ux, dy = ty[w] - uy, dz = tz[w] - uz;
                                const T r2 = dx * dx + dy * dy + dz * dz;
                                const T ri = r2 > eps2 ? rsqrt(r2) : T(0);
                                const T k3 = mq * ri * ri * ri;
                                px[w] += k3 * dx;
                                py[w] += k3 * dy;
                                pz[w] += k3 * dz;
                            }
                        }
                    }
                }
                if constexpr (kF32) {
#pragma unroll
                    for (int w = 0; w < 2; ++w) {
                        float a0, a1;
                        up2(qx[w], a0, a1);
                        px[w] = a0 + a1;
                        up2(qy[w], a0, a1);
                        py[w] = a0 + a1;
                        up2(qz[w], a0, a1);
                        pz[w] = a0 + a1;
                    }
                }
#pragma unroll
                for (int w = 0; w < 2; ++w) {
                    two_sum(hx[w], lx[w], px[w]);
                    two_sum(hy[w], ly[w], py[w]);
                    two_sum(hz[w], lz[w], pz[w]);
                }
            }
            // far field: gradient of the leaf's local expansion
            __syncwarp();
            const T *Lc = le + ((int64_t)leaf * a.B + bb) * a.ldk;
            T fx[2], fy[2], fz[2];
            if constexpr (kF32) {
                float2 *Dx2 = reinterpret_cast<float2 *>(Dx), *Dy2 = reinterpret_cast<float2 *>(Dy),
                       *Dz2 = reinterpret_cast<float2 *>(Dz);
                for (int e = lane; e < P2; e += 32) {
                    float vx, vy, vz;
                    grad_coeff<float>(Lc, e, vx, vy, vz);
                    int n = 0;
                    while ((n + 1) * (n + 1) <= e) ++n;
                    const float f2 = e == n * n ? 1.f : 2.f;
                    Dx2[e] = make_float2(f2 * vx, f2 * vx);
                    Dy2[e] = make_float2(f2 * vy, f2 * vy);
                    Dz2[e] = make_float2(f2 * vz, f2 * vz);
                }
                __syncwarp();
                uint64_t FX, FY, FZ;
                l2p_sum2(a.p, Dx2, Dy2, Dz2, pk2(tx[0], tx[1]), pk2(ty[0], ty[1]), pk2(tz[0], tz[1]), FX, FY, FZ);
                up2(FX, fx[0], fx[1]);
                up2(FY, fy[0], fy[1]);
                up2(FZ, fz[0], fz[1]);
            } else {
                for (int e = lane; e < P2; e += 32) grad_coeff<T>(Lc, e, Dx[e], Dy[e], Dz[e]);
                __syncwarp();
                for (int w = 0; w < 2; ++w) l2p_sum<T>(a.p, Dx, Dy, Dz, tx[w], ty[w], tz[w], fx[w], fy[w], fz[w]);
            }
            for (int w = 0; w < 2; ++w) {
                if (tid[w] < 0) continue;
                const double gx = ((double)hx[w] + (double)lx[w] - (double)fx[w]) * a.scale;
                const double gy = ((double)hy[w] + (double)ly[w] - (double)fy[w]) * a.scale;
                const double gzv = ((double)hz[w] + (double)lz[w] - (double)fz[w]) * a.scale;
                const int64_t j = a.perm[tid[w]];
                if (a.gout) {
                    double *o = a.gout + ((int64_t)bb * a.M + j) * 3;
                    o[0] = gx;
                    o[1] = gy;
                    o[2] = gzv;
                }
                if (a.gz) a.gz[(int64_t)bb * a.M + j] = gzv;
            }
            __syncwarp();
        }
    }
}

// Near (observer, source) pairs of the FMM: observers of each observer leaf
// times the points of its neighbour leaves.
__global__ void point_count_near(const uint64_t *__restrict__ tkey, const int32_t *__restrict__ leaf_obs,
                                 int64_t ntl, const int64_t *__restrict__ leaf_beg, PtGeo g,
                                 unsigned long long *__restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntl) return;
    const uint64_t key = tkey[t];
    int64_t lc[3] = {0, 0, 0};
    for (int bit = 0; bit < 21; ++bit) {
        lc[0] |= (int64_t)((key >> (3 * bit)) & 1) << bit;
        lc[1] |= (int64_t)((key >> (3 * bit + 1)) & 1) << bit;
        lc[2] |= (int64_t)((key >> (3 * bit + 2)) & 1) << bit;
    }
    unsigned long long src = 0;
    for (int nb = 0; nb < 27; ++nb) {
        const int64_t x = lc[0] + nb % 3 - 1 - g.slo[0], y = lc[1] + (nb / 3) % 3 - 1 - g.slo[1],
                      z = lc[2] + nb / 9 - 1 - g.slo[2];
        if (x < 0 || y < 0 || z < 0 || x >= g.sn[0] || y >= g.sn[1] || z >= g.sn[2]) continue;
        const int64_t l = (z * g.sn[1] + y) * g.sn[0] + x;
        src += (unsigned long long)(leaf_beg[l + 1] - leaf_beg[l]);
    }
    atomicAdd(out, src * (unsigned long long)(leaf_obs[t + 1] - leaf_obs[t]));
}

PtGeo pt_geo(const gf_plan_s *plan) {
    const FmmPlan *F = plan->fmm;
    PtGeo g;
    memset(&g, 0, sizeof(g));
    for (int a = 0; a < 3; ++a) {
        g.lo[a] = F->lo[a];
        g.lof[a] = (float)F->lo[a];
        g.slo[a] = F->lev[F->L].slo[a];
        g.sn[a] = F->lev[F->L].sn[a];
    }
    g.inv_s = F->inv_s;
    g.isf = (float)F->inv_s;
    g.fixk = -1;
    return g;
}

// The recursion tables of this file's kernels on the current device.
gf_status upload_point_tables(int device) {
    static std::mutex mu;
    static unsigned long long done = 0;
    std::lock_guard<std::mutex> lk(mu);
    if (device >= 0 && device < 64 && ((done >> device) & 1ull)) return GF_OK;
    double pa[kPT] = {}, pb[kPT] = {}, pf[kMaxP + 1] = {};
    for (int n = 1; n <= kMaxP; ++n) {
        for (int m = 0; m < n; ++m) {
            const int t = n * (n + 1) / 2 + m;
            const double inv = 1.0 / std::sqrt((double)((n + m) * (n - m)));
            pa[t] = (2 * n - 1) * inv;
            pb[t] = n - 1 > m ? std::sqrt((double)((n - 1 + m) * (n - 1 - m))) * inv : 0.0;
        }
        pf[n] = -std::sqrt((2.0 * n - 1.0) / (2.0 * n));
    }
    float paf[kPT], pbf[kPT], pff[kMaxP + 1];
    for (int t = 0; t < kPT; ++t) {
        paf[t] = (float)pa[t];
        pbf[t] = (float)pb[t];
    }
    for (int n = 0; n <= kMaxP; ++n) pff[n] = (float)pf[n];
    GF_CUDA(cudaMemcpyToSymbol(c_pa, pa, sizeof(pa)));
    GF_CUDA(cudaMemcpyToSymbol(c_pb, pb, sizeof(pb)));
    GF_CUDA(cudaMemcpyToSymbol(c_pf, pf, sizeof(pf)));
    {
        // packed pairs, and the order groups and entry order of the FP32 P2M
        float2 a2[kPT], nb2[kPT], f2[kMaxP + 1], nf2[kMaxP + 1];
        for (int t = 0; t < kPT; ++t) {
            a2[t] = make_float2(paf[t], paf[t]);
            nb2[t] = make_float2(-pbf[t], -pbf[t]);
        }
        for (int n = 0; n <= kMaxP; ++n) {
            f2[n] = make_float2(pff[n], pff[n]);
            nf2[n] = make_float2(-pff[n], -pff[n]);
        }
        static P2MGroups grp[kMaxP + 1];
        static short ktab[kMaxP + 1][(kMaxP + 1) * (kMaxP + 1)];
        memset(grp, 0, sizeof(grp));
        memset(ktab, 0, sizeof(ktab));
        for (int pp = 1; pp <= kMaxP; ++pp) {
            P2MGroups &G = grp[pp];
            int e = 0, cur = 0;
            G.ng = 0;
            G.m_lo[0] = 0;
            G.ent0[0] = 0;
            for (int m = 0; m <= pp; ++m) {
                const int em = m == 0 ? pp + 1 : 2 * (pp + 1 - m);
                if (cur + em > kGrpEnt) {   // close the group before order m
                    ++G.ng;
                    G.m_lo[G.ng] = m;
                    G.ent0[G.ng] = e;
                    cur = 0;
                }
                for (int n = m; n <= pp; ++n) {
                    if (m == 0) {
                        ktab[pp][e++] = (short)(n * n);
                    } else {
                        ktab[pp][e++] = (short)(n * n + 2 * m - 1);
                        ktab[pp][e++] = (short)(n * n + 2 * m);
                    }
                }
                cur += em;
            }
            ++G.ng;
            G.m_lo[G.ng] = pp + 1;
            G.ent0[G.ng] = e;
            if (G.ng > kMaxGroups || e != (pp + 1) * (pp + 1)) {
                set_error("internal: P2M order groups for p = %d", pp);
                return GF_ERR_CUDA;
            }
        }
        GF_CUDA(cudaMemcpyToSymbol(c_a2, a2, sizeof(a2)));
        GF_CUDA(cudaMemcpyToSymbol(c_nb2, nb2, sizeof(nb2)));
        GF_CUDA(cudaMemcpyToSymbol(c_f2, f2, sizeof(f2)));
        GF_CUDA(cudaMemcpyToSymbol(c_nf2, nf2, sizeof(nf2)));
        GF_CUDA(cudaMemcpyToSymbol(c_grp, grp, sizeof(grp)));
        GF_CUDA(cudaMemcpyToSymbol(c_ktab, ktab, sizeof(ktab)));
    }
    GF_CUDA(cudaMemcpyToSymbol(c_paf, paf, sizeof(paf)));
    GF_CUDA(cudaMemcpyToSymbol(c_pbf, pbf, sizeof(pbf)));
    GF_CUDA(cudaMemcpyToSymbol(c_pff, pff, sizeof(pff)));
    GF_TRY(upload_l2p_coefs());
    if (device >= 0 && device < 64) done |= 1ull << device;
    return GF_OK;
}

}  // namespace

// ---------------------------------------------------------------- host side
gf_status hex_sources_run(const double *verts, int64_t ncell, const QuadRule &qr, int precision, double *x,
                          double *a, cudaStream_t st) {
    const int64_t n = ncell * qr.nq;
    if (n == 0) return GF_OK;
    if (precision == GF_PREC_MIXED) {
        HexRuleF rf;
        memset(&rf, 0, sizeof(rf));
        rf.nq = qr.nq;
        for (int q = 0; q < qr.nq; ++q) {
            for (int d = 0; d < 3; ++d) rf.xi[q][d] = (float)qr.xi[q][d];
            rf.w8[q] = (float)(8.0 * qr.wn[q]);
        }
        hex_sources_fix<<<ceil_div(ncell, 128), 128, 0, st>>>(verts, ncell, rf, x, a);
    } else {
        hex_sources_kernel<<<ceil_div(n, 256), 256, 0, st>>>(verts, ncell, qr, x, a);
    }
    GF_KERNEL_DONE();
    return GF_OK;
}

gf_status points_prepare_direct(gf_plan_s *plan, const double *src, const double *wt, const double *obs,
                                cudaStream_t st) {
    PointSet &P = plan->pts;
    DeviceArena &A = plan->arena;
    const int64_t S = P.S, M = plan->M;
    GF_TRY(A.alloc_n(&P.x, std::max<int64_t>(3 * S, 1)));
    GF_TRY(A.alloc_n(&P.a, std::max<int64_t>(S, 1)));
    GF_TRY(A.alloc_n(&plan->d_obs, std::max<int64_t>(3 * M, 1)));
    if (S > 0) {
        GF_CUDA(cudaMemcpyAsync(P.x, src, sizeof(double) * 3 * S, cudaMemcpyDeviceToDevice, st));
        GF_CUDA(cudaMemcpyAsync(P.a, wt, sizeof(double) * S, cudaMemcpyDeviceToDevice, st));
    }
    if (M > 0) GF_CUDA(cudaMemcpyAsync(plan->d_obs, obs, sizeof(double) * 3 * M, cudaMemcpyDeviceToDevice, st));
    if (plan->opt.precision == GF_PREC_MIXED && S > 0 && M > 0) {
        // one quantum for sources and observers: 2^-22 of the joint extent
        double bs[12], bo[12], lo[3], hi[3];
        double *d_bb;
        GF_TRY(A.alloc_n(&d_bb, 24));
        GF_TRY(bbox3(P.x, S, d_bb, st));
        GF_TRY(bbox3(plan->d_obs, M, d_bb + 12, st));
        GF_CUDA(cudaMemcpyAsync(bs, d_bb, sizeof(bs), cudaMemcpyDeviceToHost, st));
        GF_CUDA(cudaMemcpyAsync(bo, d_bb + 12, sizeof(bo), cudaMemcpyDeviceToHost, st));
        GF_CUDA(cudaStreamSynchronize(st));
        double ext = 0.0;
        for (int d = 0; d < 3; ++d) {
            lo[d] = std::min(bs[d], bo[d]);
            hi[d] = std::max(bs[3 + d], bo[3 + d]);
            if (!isfinite(lo[d]) || !isfinite(hi[d])) {
                set_error("source and observer coordinates must be finite");
                return GF_ERR_INVALID_ARG;
            }
            ext = std::max(ext, hi[d] - lo[d]);
        }
        int e = 0;
        frexp(std::max(ext, 1e-300), &e);   // ext < 2^e
        P.q = ldexp(1.0, e - 22);
        GF_TRY(A.alloc_n(&P.xi, 3 * S));
        GF_TRY(A.alloc_n(&P.xf, 3 * S));
        GF_TRY(A.alloc_n(&P.oi, 3 * M));
        GF_TRY(A.alloc_n(&P.of, 3 * M));
        split_points<<<ceil_div(S, 256), 256, 0, st>>>(P.x, S, lo[0], lo[1], lo[2], 1.0 / P.q, P.xi, P.xf);
        GF_KERNEL_DONE();
        split_points<<<ceil_div(M, 256), 256, 0, st>>>(plan->d_obs, M, lo[0], lo[1], lo[2], 1.0 / P.q, P.oi,
                                                       P.of);
        GF_KERNEL_DONE();
    }
    return GF_OK;
}

gf_status points_direct_forward(gf_plan_s *plan, const void *rho, int rho_dtype, int B, double *g, double *gz,
                                cudaStream_t st) {
    const PointSet &P = plan->pts;
    const int64_t M = plan->M;
    if (M == 0) return GF_OK;
    const dim3 grid(ceil_div(M, kPtTile), B);
    const int f32 = rho_dtype == GF_DTYPE_F32;
    if (plan->opt.precision == GF_PREC_FP64 || P.S == 0) {
        direct_points_f64<<<grid, kPtTile, 0, st>>>(plan->d_obs, M, P.x, P.a, P.S, P.per_cell, P.ncell, rho, f32,
                                                   plan->G, g, gz, plan->d_status);
    } else {
        // mass and separations in quanta: g = G / q^2 * (quantum-unit sum)
        direct_points_mixed<<<grid, kPtTile, 0, st>>>(P.oi, P.of, M, P.xi, P.xf, P.a, P.S, P.per_cell,
                                                     P.ncell, rho, f32, (float)P.q, plan->G * P.q, g, gz,
                                                     plan->d_status);
    }
    GF_KERNEL_DONE();
    return GF_OK;
}

gf_status points_fmm_create(gf_plan_s *plan, const double *src, const double *wt, const double *obs,
                            cudaStream_t st) {
    FmmPlan *F = new (std::nothrow) FmmPlan();
    if (!F) {
        set_error("host allocation failed");
        return GF_ERR_OOM;
    }
    plan->fmm = F;
    PointSet &P = plan->pts;
    const int64_t S = P.S, M = plan->M;
    F->p = plan->opt.p;
    F->K = (F->p + 1) * (F->p + 1);
    F->B = plan->opt.max_batch;
    F->nq = 1;
    F->mixed = plan->opt.precision == GF_PREC_MIXED;
    F->m2l_tc64 = !F->mixed && (plan->opt.reserved0 & GF_FLAG_M2L_TENSOR);
    F->b = 1;
    F->points = true;
    DeviceArena &A = plan->arena;
    // ---- extents of the sources and of the observers
    double bs[6] = {0, 0, 0, 0, 0, 0}, bo[6] = {0, 0, 0, 0, 0, 0};
    {
        double *d_bb;
        GF_TRY(A.alloc_n(&d_bb, 24));
        if (S > 0) GF_TRY(bbox3(src, S, d_bb, st));
        if (M > 0) GF_TRY(bbox3(obs, M, d_bb + 12, st));
        double h[24];
        GF_CUDA(cudaMemcpyAsync(h, d_bb, sizeof(h), cudaMemcpyDeviceToHost, st));
        GF_CUDA(cudaStreamSynchronize(st));
        for (int d = 0; d < 6; ++d) {
            if (S > 0) bs[d] = h[d];
            if (M > 0) bo[d] = h[12 + d];
            if (!isfinite(bs[d]) || !isfinite(bo[d])) {
                set_error("source and observer coordinates must be finite");
                return GF_ERR_INVALID_ARG;
            }
        }
        if (S == 0)
            for (int d = 0; d < 6; ++d) bs[d] = bo[d];
        if (M == 0)
            for (int d = 0; d < 6; ++d) bo[d] = bs[d];
    }
    // ---- leaf side: about kPointsPerLeaf sources per leaf of their extent
    double ext_s[3], ext_max = 0.0, vol = 1.0;
    for (int d = 0; d < 3; ++d) {
        ext_s[d] = bs[3 + d] - bs[d];
        ext_max = std::max(ext_max, ext_s[d]);
    }
    if (ext_max <= 0.0) ext_max = 1.0;
    int flat = 0;
    for (int d = 0; d < 3; ++d) {
        if (ext_s[d] > 1e-6 * ext_max)
            vol *= ext_s[d];
        else
            ++flat;
    }
    const double nleaf_want = std::max(1.0, (double)S / kPointsPerLeaf);
    double side = flat == 0 ? cbrt(vol / nleaf_want) : (flat == 1 ? sqrt(vol / nleaf_want) : vol / nleaf_want);
    side = std::max(side, ext_max * 1e-6);
    double bb[6];
    for (int d = 0; d < 3; ++d) {
        bb[d] = std::min(bs[d], bo[d]);
        bb[3 + d] = std::max(bs[3 + d], bo[3 + d]);
    }
    double root_ext = 0.0;
    for (int d = 0; d < 3; ++d) root_ext = std::max(root_ext, bb[3 + d] - bb[d]);
    // the root spans the joint extent plus the shift of its corner below
    const double span = root_ext + 1e-6 * side;
    int L = 2;
    while (L < kMaxLevels - 1 && side * (double)((int64_t)1 << L) < span) ++L;
    if (side * (double)((int64_t)1 << L) < span) side = span / (double)((int64_t)1 << L) * (1.0 + 1e-9);
    F->L = L;
    F->h = side;   // the plan's length unit is the leaf side
    F->s_leaf = side;
    F->inv_s = 1.0 / side;
    for (int d = 0; d < 3; ++d) {
        F->lo[d] = bb[d] - 1e-7 * side;   // strictly inside the root
        F->voff[d] = 0;
    }
    const int64_t top = ((int64_t)1 << L) - 1;
    int64_t slo[3], shi[3];
    for (int d = 0; d < 3; ++d) {
        slo[d] = std::min<int64_t>(top, std::max<int64_t>(0, (int64_t)floor((bs[d] - F->lo[d]) * F->inv_s)));
        shi[d] = std::min<int64_t>(top, std::max<int64_t>(slo[d], (int64_t)floor((bs[3 + d] - F->lo[d]) * F->inv_s)));
    }
    for (int l = 0; l <= L; ++l) {
        FmmLevel &lv = F->lev[l];
        lv.ns = 1;
        for (int d = 0; d < 3; ++d) {
            lv.slo[d] = slo[d] >> (L - l);
            lv.sn[d] = (shi[d] >> (L - l)) - lv.slo[d] + 1;
            lv.ns *= lv.sn[d];
        }
    }
    const int64_t nleaf = F->lev[L].ns;
    if (nleaf > ((int64_t)1 << 31)) {
        set_error("the sources' leaf block is too large (%lld leaves)", (long long)nleaf);
        return GF_ERR_UNSUPPORTED;
    }
    // ---- sources sorted by leaf, each leaf's first source
    GF_TRY(upload_point_tables(plan->device));
    PtGeo g = pt_geo(plan);
    double bb_root[6];
    for (int d = 0; d < 6; ++d) bb_root[d] = bb[d];
    g.fixk = fixed_point_frame(F, bb_root, g.lofix, &g.halfleaf_fix, &g.fix_to_leaf);
    const size_t rs = F->mixed ? sizeof(float) : sizeof(double);
    GF_TRY(A.alloc(&P.loc, rs * 4 * (size_t)std::max<int64_t>(S, 1)));
    GF_TRY(A.alloc_n(&P.perm, std::max<int64_t>(S, 1)));
    GF_TRY(A.alloc_n(&P.leaf_beg, nleaf + 1));
    if (S > 0) {
        uint64_t *keys, *keys2;
        int32_t *vals2;
        GF_TRY(A.alloc_n(&keys, S));
        GF_TRY(A.alloc_n(&keys2, S));
        GF_TRY(A.alloc_n(&vals2, S));
        void *scratch;
        GF_TRY(A.alloc(&scratch, sort_scratch_bytes(S)));
        point_keys<<<ceil_div(S, 256), 256, 0, st>>>(src, S, g, keys, P.perm, plan->d_status);
        GF_KERNEL_DONE();
        int bits = 1;
        while (bits < 63 && ((int64_t)1 << bits) < nleaf) ++bits;
        GF_TRY(radix_sort_u64(keys, P.perm, keys2, vals2, S, bits, scratch, st));
        const double inv_s3 = F->inv_s * F->inv_s * F->inv_s;
        if (F->mixed)
            point_gather<float><<<ceil_div(S, 256), 256, 0, st>>>(src, wt, P.perm, keys, S, g, inv_s3,
                                                                  (float *)P.loc, plan->d_status);
        else
            point_gather<double><<<ceil_div(S, 256), 256, 0, st>>>(src, wt, P.perm, keys, S, g, inv_s3,
                                                                   (double *)P.loc, plan->d_status);
        GF_KERNEL_DONE();
        point_leaf_beg<<<ceil_div(nleaf + 1, 256), 256, 0, st>>>(keys, S, nleaf, P.leaf_beg);
        GF_KERNEL_DONE();
    } else {
        GF_CUDA(cudaMemsetAsync(P.leaf_beg, 0, sizeof(int64_t) * (nleaf + 1), st));
    }
    double oz[2] = {bo[2], bo[5]}, olo[3] = {bo[0], bo[1], bo[2]}, ohi[3] = {bo[3], bo[4], bo[5]};
    return fmm_observer_tree(plan, obs, oz, olo, ohi, bb, st);
}

template <class T>
gf_status points_masses(gf_plan_s *plan, const void *rho, int rho_dtype, int B, cudaStream_t st) {
    FmmPlan *F = plan->fmm;
    const PointSet &P = plan->pts;
    if (P.S == 0) return GF_OK;
    point_masses<T><<<ceil_div(P.S * B, 256), 256, 0, st>>>(rho, rho_dtype == GF_DTYPE_F32, P.perm,
                                                           (const T *)P.loc, P.S, P.per_cell, P.ncell, B,
                                                           (T *)F->mass, plan->d_status);
    GF_KERNEL_DONE();
    return GF_OK;
}

template <class T>
gf_status points_p2m(gf_plan_s *plan, int B, cudaStream_t st) {
    FmmPlan *F = plan->fmm;
    const PointSet &P = plan->pts;
    const FmmLevel &lv = F->lev[F->L];
    if constexpr (sizeof(T) == 4) {
        const unsigned grid = (unsigned)std::min<int64_t>((lv.ns + kP2MWarpsF - 1) / kP2MWarpsF, 152 * 64);
        point_p2m_f32<<<grid, kP2MWarpsF * 32, 0, st>>>((const float *)P.loc, (const float *)F->mass, P.leaf_beg,
                                                        lv.ns, P.S, F->p, B, F->KS, (float *)lv.me);
        GF_KERNEL_DONE();
        return GF_OK;
    }
    constexpr int W = p2m_warps<T>();
    const int stride = p2m_stride(F->K);
    const size_t shm = sizeof(T) * W * 32 * (size_t)stride;
    GF_TRY(ensure_smem(point_p2m<T>, shm));
    const unsigned grid = (unsigned)std::min<int64_t>((lv.ns + W - 1) / W, 152 * 64);
    point_p2m<T><<<grid, W * 32, shm, st>>>((const T *)P.loc, (const T *)F->mass, P.leaf_beg, lv.ns, P.S, F->p, B,
                                            F->KS, stride, (T *)lv.me);
    GF_KERNEL_DONE();
    return GF_OK;
}

template <class T>
gf_status points_eval(gf_plan_s *plan, int B, double *g, double *gz, cudaStream_t st) {
    FmmPlan *F = plan->fmm;
    const PointSet &P = plan->pts;
    if (F->n_items == 0) return GF_OK;
    PtEvalArgs a;
    a.items = F->items;
    a.n_items = F->n_items;
    a.tkey = F->lev[F->L].tkey;
    a.perm = F->perm;
    a.tloc = sizeof(T) == 8 ? (const void *)F->tloc_d : (const void *)F->tloc_f;
    a.loc = P.loc;
    a.mass = F->mass;
    a.leaf_beg = P.leaf_beg;
    a.le = F->lev[F->L].le;
    a.g = pt_geo(plan);
    a.L = F->L;
    a.B = B;
    a.p = F->p;
    a.ldk = F->KS;
    a.S = P.S;
    a.M = plan->M;
    a.part_lo = plan->part_lo;
    a.part_hi = plan->part_hi;
    a.scale = plan->G * F->h;
    a.eps2 = sizeof(T) == 8 ? 1e-24 : 1e-14;
    a.gout = g;
    a.gz = gz;
    const size_t shm = sizeof(T) * kPtWarps * (size_t)pt_slice(F->p * F->p, (int)sizeof(T));
    GF_TRY(ensure_smem(point_eval<T>, shm));
    const unsigned grid = (unsigned)std::min<int64_t>((F->n_items + kPtWarps - 1) / kPtWarps, 152 * 64);
    point_eval<T><<<grid, kPtWarps * 32, shm, st>>>(a);
    GF_KERNEL_DONE();
    return GF_OK;
}

template gf_status points_masses<float>(gf_plan_s *, const void *, int, int, cudaStream_t);
template gf_status points_masses<double>(gf_plan_s *, const void *, int, int, cudaStream_t);
template gf_status points_p2m<float>(gf_plan_s *, int, cudaStream_t);
template gf_status points_p2m<double>(gf_plan_s *, int, cudaStream_t);
template gf_status points_eval<float>(gf_plan_s *, int, double *, double *, cudaStream_t);
template gf_status points_eval<double>(gf_plan_s *, int, double *, double *, cudaStream_t);

gf_status points_count_near(gf_plan_s *plan, unsigned long long *d_out, cudaStream_t st) {
    FmmPlan *F = plan->fmm;
    const FmmLevel &leaf = F->lev[F->L];
    if (leaf.nt == 0) return GF_OK;
    point_count_near<<<ceil_div(leaf.nt, 256), 256, 0, st>>>(leaf.tkey, F->leaf_beg, leaf.nt, plan->pts.leaf_beg,
                                                            pt_geo(plan), d_out);
    GF_KERNEL_DONE();
    return GF_OK;
}

}  // namespace gf
