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
#include <new>
#include <vector>

#include "fmm_math.cuh"
#include "gf_fmm.cuh"
#include "gf_prim.cuh"

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
    int64_t top;                 // 2^L - 1
    int64_t slo[3], sn[3];       // dense block of source leaves
};

// Linear index of each source's leaf in the dense block (leaf = floor((x -
// lo) / s), clamped to the block), and the source's position in leaf units
// from the root corner.
__global__ void point_keys(const double *__restrict__ x, int64_t S, PtGeo g, uint64_t *__restrict__ keys,
                           int32_t *__restrict__ vals, int *__restrict__ status) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    int64_t c[3];
    for (int a = 0; a < 3; ++a) {
        const double v = x[3 * s + a];
        if (!isfinite(v)) atomicOr(status + 2, 1);
        double f = floor(__dmul_rn(__dsub_rn(v, g.lo[a]), g.inv_s));
        f = fmin(fmax(f, (double)g.slo[a]), (double)(g.slo[a] + g.sn[a] - 1));
        c[a] = (int64_t)f;
    }
    keys[s] = (uint64_t)(((c[2] - g.slo[2]) * g.sn[1] + (c[1] - g.slo[1])) * g.sn[0] + (c[0] - g.slo[0]));
    vals[s] = (int32_t)s;
}

// Sorted copies: positions in leaf units from the root corner, weights.
__global__ void point_gather(const double *__restrict__ x, const double *__restrict__ wt,
                             const int32_t *__restrict__ perm, int64_t S, PtGeo g, double *__restrict__ u,
                             double *__restrict__ a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S) return;
    const int64_t s = perm[i];
    for (int d = 0; d < 3; ++d) u[3 * i + d] = (x[3 * s + d] - g.lo[d]) * g.inv_s;
    a[i] = wt[s];
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
// Sorted masses in leaf units: m_i = rho_{c(perm_i)} a_i / s^3, [B][S].
template <class T>
__global__ void point_masses(const void *__restrict__ rho, int rho_f32, const int32_t *__restrict__ perm,
                             const double *__restrict__ a, int64_t S, int per_cell, int64_t ncell, int B,
                             double inv_s3, T *__restrict__ m, int *__restrict__ status) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= S * B) return;
    const int b = (int)(e / S);
    const int64_t i = e - (int64_t)b * S;
    const double r = load_rho_p(rho, rho_f32, (int64_t)b * ncell + perm[i] / per_cell);
    if (!isfinite(r)) atomicOr(status, 1);
    m[e] = (T)(r * a[i] * inv_s3);
}

// P2M over the points of each dense leaf: ME_n^m = sum_i m_i conj(R_n^m(u_i
// - c)), u in leaf units, c the leaf centre.  One warp per leaf; lane m < =
// p runs the recursion of order m (fmm_math.cuh) for each point in turn and
// adds into its coefficients, so the lanes never touch the same entry.
template <class T>
__global__ void __launch_bounds__(128)
point_p2m(const double *__restrict__ u, const T *__restrict__ mass, const int64_t *__restrict__ leaf_beg,
          int64_t nleaf, int64_t S, PtGeo g, int p, int B, int ldk, T *__restrict__ me) {
    extern __shared__ unsigned char shraw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int K = (p + 1) * (p + 1);
    T *acc = reinterpret_cast<T *>(shraw) + (size_t)warp * ((K + 7) & ~7);
    for (int64_t leaf = (int64_t)blockIdx.x * 4 + warp; leaf < nleaf; leaf += (int64_t)gridDim.x * 4) {
        const int64_t lx = leaf % g.sn[0], ly = (leaf / g.sn[0]) % g.sn[1], lz = leaf / (g.sn[0] * g.sn[1]);
        const double cx = (double)(g.slo[0] + lx) + 0.5, cy = (double)(g.slo[1] + ly) + 0.5,
                     cz = (double)(g.slo[2] + lz) + 0.5;
        const int64_t i0 = leaf_beg[leaf], i1 = leaf_beg[leaf + 1];
        for (int bb = 0; bb < B; ++bb) {
            for (int k = lane; k < K; k += 32) acc[k] = T(0);
            __syncwarp();
            const int m = lane;
            if (m <= p) {
                // the normalisation of the sectoral and the upward recursions
                for (int64_t i = i0; i < i1; ++i) {
                    const T x = (T)(u[3 * i] - cx), y = (T)(u[3 * i + 1] - cy), z = (T)(u[3 * i + 2] - cz);
                    const T q = mass[(int64_t)bb * S + i];
                    const T r2 = x * x + y * y + z * z;
                    // R_m^m by the sectoral recursion
                    T sr = T(1), si = T(0);
                    for (int n = 1; n <= m; ++n) {
                        const T f = -sqrt(T(2 * n - 1) / T(2 * n));
                        const T nr = f * (x * sr - y * si), ni = f * (x * si + y * sr);
                        sr = nr;
                        si = ni;
                    }
                    // R_n^m for n = m .. p, adding q conj(R) into the real storage
                    T pr = T(0), pi = T(0), cr = sr, ci = si;
                    for (int n = m; n <= p; ++n) {
                        if (n > m) {
                            const T inv = T(1) / sqrt(T((n + m) * (n - m)));
                            const T a = T(2 * n - 1) * inv;
                            const T bcoef = n - 1 > m ? sqrt(T((n - 1 + m) * (n - 1 - m))) * inv * r2 : T(0);
                            const T nr = a * z * cr - bcoef * pr, ni = a * z * ci - bcoef * pi;
                            pr = cr;
                            pi = ci;
                            cr = nr;
                            ci = ni;
                        }
                        if (m == 0) {
                            acc[n * n] += q * cr;
                        } else {
                            acc[n * n + 2 * m - 1] += q * cr;
                            acc[n * n + 2 * m] -= q * ci;
                        }
                    }
                }
            }
            __syncwarp();
            T *dst = me + (leaf * B + bb) * ldk;
            for (int k = lane; k < ldk; k += 32) dst[k] = k < K ? acc[k] : T(0);
            __syncwarp();
        }
    }
}

// Near field over the points of the 27 neighbour leaves + the L2P gradient
// of the leaf's local expansion + near + far in FP64, scattered to caller
// order.  One warp per work item, two observers per lane; each neighbour
// leaf's points are staged 64 at a time (position from the item's leaf
// centre, mass) in the warp's shared-memory slice.
constexpr int kPtWarps = 4;
constexpr int kPtChunk = 64;

inline __host__ __device__ int pt_slice(int P2) { return (4 * kPtChunk + 3 * P2 + 27 * 2 + 7) & ~7; }

struct PtEvalArgs {
    const int4 *items;
    int64_t n_items;
    const uint64_t *tkey;
    const int32_t *perm;
    const void *tloc;
    const double *u;           // sorted point positions, leaf units from the root corner
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
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int P2 = a.p * a.p;
    T *wsh = reinterpret_cast<T *>(shraw) + (size_t)warp * pt_slice(P2);
    T *sx = wsh, *sy = sx + kPtChunk, *sz = sy + kPtChunk, *sm = sz + kPtChunk;
    T *Dx = wsh + 4 * kPtChunk, *Dy = Dx + P2, *Dz = Dy + P2;
    int64_t *nbl = reinterpret_cast<int64_t *>(Dz + P2 + ((3 * P2) & 1));
    const T *tloc = reinterpret_cast<const T *>(a.tloc);
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
        const double cx = (double)lc[0] + 0.5, cy = (double)lc[1] + 0.5, cz = (double)lc[2] + 0.5;
        for (int bb = 0; bb < a.B; ++bb) {
            double nx_[2] = {0.0, 0.0}, ny_[2] = {0.0, 0.0}, nz_[2] = {0.0, 0.0};
            for (int nb = 0; nb < 27; ++nb) {
                const int64_t sl = nbl[nb];
                if (sl < 0) continue;
                const int64_t i0 = a.leaf_beg[sl], i1 = a.leaf_beg[sl + 1];
                T px[2] = {T(0), T(0)}, py[2] = {T(0), T(0)}, pz[2] = {T(0), T(0)};
                for (int64_t c0 = i0; c0 < i1; c0 += kPtChunk) {
                    const int cnt = (int)min((int64_t)kPtChunk, i1 - c0);
                    __syncwarp();
                    for (int s = lane; s < cnt; s += 32) {
                        const int64_t i = c0 + s;
                        sx[s] = (T)(a.u[3 * i] - cx);
                        sy[s] = (T)(a.u[3 * i + 1] - cy);
                        sz[s] = (T)(a.u[3 * i + 2] - cz);
                        sm[s] = mass[(int64_t)bb * a.S + i];
                    }
                    __syncwarp();
                    for (int s = 0; s < cnt; ++s) {
                        const T ux = sx[s], uy = sy[s], uz = sz[s], m = sm[s];
#pragma unroll
                        for (int w = 0; w < 2; ++w) {
                            const T dx = tx[w] - ux, dy = ty[w] - uy, dz = tz[w] - uz;
                            const T r2 = dx * dx + dy * dy + dz * dz;
                            const T ri = r2 > eps2 ? T(1) / sqrt(r2) : T(0);
                            const T k3 = m * ri * ri * ri;
                            px[w] += k3 * dx;
                            py[w] += k3 * dy;
                            pz[w] += k3 * dz;
                        }
                    }
                }
                for (int w = 0; w < 2; ++w) {
                    nx_[w] += (double)px[w];
                    ny_[w] += (double)py[w];
                    nz_[w] += (double)pz[w];
                }
            }
            // far field: gradient of the leaf's local expansion
            __syncwarp();
            const T *Lc = le + ((int64_t)leaf * a.B + bb) * a.ldk;
            for (int e = lane; e < P2; e += 32) grad_coeff<T>(Lc, e, Dx[e], Dy[e], Dz[e]);
            __syncwarp();
            for (int w = 0; w < 2; ++w) {
                if (tid[w] < 0) continue;
                T fx, fy, fz;
                l2p_sum<T>(a.p, Dx, Dy, Dz, tx[w], ty[w], tz[w], fx, fy, fz);
                const double gx = (nx_[w] - (double)fx) * a.scale;
                const double gy = (ny_[w] - (double)fy) * a.scale;
                const double gzv = (nz_[w] - (double)fz) * a.scale;
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
    for (int a = 0; a < 3; ++a) {
        g.lo[a] = F->lo[a];
        g.slo[a] = F->lev[F->L].slo[a];
        g.sn[a] = F->lev[F->L].sn[a];
    }
    g.inv_s = F->inv_s;
    g.top = ((int64_t)1 << F->L) - 1;
    return g;
}

}  // namespace

// ---------------------------------------------------------------- host side
gf_status hex_sources_run(const double *verts, int64_t ncell, const QuadRule &qr, double *x, double *a,
                          cudaStream_t st) {
    const int64_t n = ncell * qr.nq;
    if (n == 0) return GF_OK;
    hex_sources_kernel<<<ceil_div(n, 256), 256, 0, st>>>(verts, ncell, qr, x, a);
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
    PtGeo g = pt_geo(plan);
    GF_TRY(A.alloc_n(&P.x, std::max<int64_t>(3 * S, 1)));   // positions in leaf units, sorted
    GF_TRY(A.alloc_n(&P.a, std::max<int64_t>(S, 1)));
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
        point_gather<<<ceil_div(S, 256), 256, 0, st>>>(src, wt, P.perm, S, g, P.x, P.a);
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
    const double inv_s3 = F->inv_s * F->inv_s * F->inv_s;
    point_masses<T><<<ceil_div(P.S * B, 256), 256, 0, st>>>(rho, rho_dtype == GF_DTYPE_F32, P.perm, P.a, P.S,
                                                           P.per_cell, P.ncell, B, inv_s3, (T *)F->mass,
                                                           plan->d_status);
    GF_KERNEL_DONE();
    return GF_OK;
}

template <class T>
gf_status points_p2m(gf_plan_s *plan, int B, cudaStream_t st) {
    FmmPlan *F = plan->fmm;
    const PointSet &P = plan->pts;
    const FmmLevel &lv = F->lev[F->L];
    const size_t shm = sizeof(T) * 4 * (size_t)((F->K + 7) & ~7);
    GF_TRY(ensure_smem(point_p2m<T>, shm));
    const unsigned grid = (unsigned)std::min<int64_t>((lv.ns + 3) / 4, 152 * 32);
    point_p2m<T><<<grid, 128, shm, st>>>(P.x, (const T *)F->mass, P.leaf_beg, lv.ns, P.S, pt_geo(plan), F->p, B,
                                         F->KS, (T *)lv.me);
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
    a.u = P.x;
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
    const size_t shm = sizeof(T) * kPtWarps * (size_t)pt_slice(F->p * F->p) + 64;
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
