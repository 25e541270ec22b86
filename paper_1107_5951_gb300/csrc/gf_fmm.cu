// gf_fmm.cu -- the FMM of Sec. 2.3 on the GPU: operator tables, upward sweep
// (P2M, M2M), downward sweep (M2L over the interaction list, L2L) and field
// evaluation (L2P plus the near-field direct sum, Eq. 10).
//
// Every kernel here works in voxel units (h = 1); see gf_fmm.cuh.  The
// evaluation kernel fuses the near-field sum over the nearest-neighbour
// leaves, the local-expansion gradient, the near+far sum in FP64 and the
// scatter back to the caller's observer order.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <type_traits>
#include <vector>

#include "fmm_math.cuh"
#include "gf_fmm.cuh"
#include "gf_m2l.cuh"
#include "gf_simd.cuh"
#include "gf_sum_an.cuh"

namespace gf {

namespace {

struct LogFact {
    double v[kLogFactN];
};

LogFact host_logfact() {
    LogFact lf;
    for (int i = 0; i < kLogFactN; ++i) lf.v[i] = lgamma((double)i + 1.0);
    return lf;
}

// One block per operator: 343 M2L slots (the 27 near offsets stay unused),
// then 8 M2M and 8 L2L octants.  Entries are written transposed
// (input component major).
__global__ void build_ops(int p, int K, LogFact lf, double *__restrict__ m2l_d, float *__restrict__ m2l_f,
                          double *__restrict__ m2m_d, float *__restrict__ m2m_f, double *__restrict__ l2l_d,
                          float *__restrict__ l2l_f) {
    extern __shared__ double sh[];
    const int op = blockIdx.x;
    int kind;
    double d[3];
    double *od;
    float *of;
    int H;
    if (op < 343) {
        const int dx = op % 7 - 3, dy = (op / 7) % 7 - 3, dz = op / 49 - 3;
        if (max(abs(dx), max(abs(dy), abs(dz))) <= 1) return;
        kind = OP_M2L;
        d[0] = dx;
        d[1] = dy;
        d[2] = dz;
        H = 2 * p;
        od = m2l_d + (size_t)op * K * K;
        of = m2l_f + (size_t)op * K * K;
    } else {
        const int oct = (op - 343) & 7;
        kind = op < 351 ? OP_M2M : OP_L2L;
        d[0] = ((oct & 1) - 0.5) * 0.5;
        d[1] = (((oct >> 1) & 1) - 0.5) * 0.5;
        d[2] = (((oct >> 2) & 1) - 0.5) * 0.5;
        H = p;
        od = (kind == OP_M2M ? m2m_d : l2l_d) + (size_t)oct * K * K;
        of = (kind == OP_M2M ? m2m_f : l2l_f) + (size_t)oct * K * K;
    }
    const int nt = (H + 1) * (H + 2) / 2;
    double *re = sh, *im = sh + nt;
    if (threadIdx.x == 0) {
        if (kind == OP_M2L)
            irregular_harmonics<double>(H, d[0], d[1], d[2], re, im);
        else
            regular_harmonics<double>(H, d[0], d[1], d[2], re, im);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
        const int c = e / K, k = e - c * K;
        const double v = op_entry(kind, p, k, c, re, im, lf.v);
        od[e] = v;
        of[e] = (float)v;
    }
}

// P2M matrix with the quadrature folded in: P[v][k] = sum_q wn_q *
// (k-th real component of conj R((x_vq - c)/b)), x_vq - c in voxel units.
__global__ void build_p2m(int p, int K, int b, const QuadRule *__restrict__ qr, double *__restrict__ pd,
                          float *__restrict__ pf) {
    extern __shared__ double sh[];
    const int v = blockIdx.x;
    const int lx = v % b, ly = (v / b) % b, lz = v / (b * b);
    const int nt = (p + 1) * (p + 2) / 2;
    double *re = sh, *im = sh + nt, *acc = sh + 2 * nt;
    for (int k = threadIdx.x; k < K; k += blockDim.x) acc[k] = 0.0;
    __syncthreads();
    for (int q = 0; q < qr->nq; ++q) {
        if (threadIdx.x == 0) {
            const double y0 = (lx + 0.5 + 0.5 * qr->xi[q][0] - 0.5 * b) / b;
            const double y1 = (ly + 0.5 + 0.5 * qr->xi[q][1] - 0.5 * b) / b;
            const double y2 = (lz + 0.5 + 0.5 * qr->xi[q][2] - 0.5 * b) / b;
            regular_harmonics<double>(p, y0, y1, y2, re, im);
        }
        __syncthreads();
        const double w = qr->wn[q];
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
            int n = (int)sqrt((double)k);
            while (n * n > k) --n;
            while ((n + 1) * (n + 1) <= k) ++n;
            const int ro = k - n * n, m = (ro + 1) / 2;
            const bool isim = ro > 0 && (ro % 2 == 0);
            acc[k] += isim ? -w * im[tri(n, m)] : w * re[tri(n, m)];
        }
        __syncthreads();
    }
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        pd[(size_t)v * K + k] = acc[k];
        pf[(size_t)v * K + k] = (float)acc[k];
    }
}

// P2M into the parent level: Q[o][v][k] = sum_i P[v][i] T_o[i][k] for the
// 8 child positions o (T_o the M2M operator, input component major), i.e.
// the parent expansion contributed by unit mass at voxel v of child o.
// Grid (8, b3), one thread per output component.
__global__ void compose_p2m_up(const double *__restrict__ P, const double *__restrict__ m2m, int K, int b3,
                               double *__restrict__ Q) {
    const int o = blockIdx.x, v = blockIdx.y;
    const double *pv = P + (size_t)v * K;
    const double *T = m2m + (size_t)o * K * K;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < K; ++i) s += pv[i] * T[(size_t)i * K + k];
        Q[((size_t)o * b3 + v) * K + k] = s;
    }
}

// P2M matrix of closed-form voxels (SUM-AN): P[v][k] = the k-th real component
// of conj R((x - c)/b) integrated over voxel v (unit volume in voxel units),
// by a Gauss-Legendre rule of m nodes per axis, exact for every regular solid
// harmonic of degree <= 2m - 1.
struct GaussLeg {
    int m;
    double x[16], w[16];   // nodes on [-1, 1], weights summing to 2
};

__global__ void build_p2m_exact(int p, int K, int b, GaussLeg gl, double *__restrict__ pd,
                                float *__restrict__ pf) {
    extern __shared__ double sh[];
    const int v = blockIdx.x;
    const int lx = v % b, ly = (v / b) % b, lz = v / (b * b);
    const int nt = (p + 1) * (p + 2) / 2;
    double *re = sh, *im = sh + nt, *acc = sh + 2 * nt;
    for (int k = threadIdx.x; k < K; k += blockDim.x) acc[k] = 0.0;
    __syncthreads();
    const int m = gl.m;
    for (int q = 0; q < m * m * m; ++q) {
        const int qi = q % m, qj = (q / m) % m, qk = q / (m * m);
        if (threadIdx.x == 0) {
            const double y0 = (lx + 0.5 + 0.5 * gl.x[qi] - 0.5 * b) / b;
            const double y1 = (ly + 0.5 + 0.5 * gl.x[qj] - 0.5 * b) / b;
            const double y2 = (lz + 0.5 + 0.5 * gl.x[qk] - 0.5 * b) / b;
            regular_harmonics<double>(p, y0, y1, y2, re, im);
        }
        __syncthreads();
        const double w = 0.125 * gl.w[qi] * gl.w[qj] * gl.w[qk];
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
            int n = (int)sqrt((double)k);
            while (n * n > k) --n;
            while ((n + 1) * (n + 1) <= k) ++n;
            const int ro = k - n * n, mm = (ro + 1) / 2;
            const bool isim = ro > 0 && (ro % 2 == 0);
            acc[k] += isim ? -w * im[tri(n, mm)] : w * re[tri(n, mm)];
        }
        __syncthreads();
    }
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        pd[(size_t)v * K + k] = acc[k];
        pf[(size_t)v * K + k] = (float)acc[k];
    }
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton's method on the
// three-term recurrence of the Legendre polynomials).
GaussLeg gauss_legendre(int m) {
    GaussLeg g;
    g.m = m;
    for (int i = 0; i < m; ++i) {
        double x = cos(M_PI * (i + 0.75) / (m + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int n = 2; n <= m; ++n) {
                const double pn = ((2.0 * n - 1.0) * x * p1 - (n - 1.0) * p0) / n;
                p0 = p1;
                p1 = pn;
            }
            const double pm = m == 1 ? x : p1, pm1 = m == 1 ? 1.0 : p0;
            dp = m * (x * pm - pm1) / (x * x - 1.0);
            const double dx = pm / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        g.x[i] = x;
        g.w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    return g;
}

// ---------------------------------------------------------------- sources
struct Block3 {
    int64_t lo[3], n[3];
};

Block3 block_of(const FmmLevel &lv) {
    Block3 b;
    for (int a = 0; a < 3; ++a) {
        b.lo[a] = lv.slo[a];
        b.n[a] = lv.sn[a];
    }
    return b;
}

// Leaf-blocked densities: mass[leaf][bb][v] = rho of the grid voxel that
// sits at local position v of the leaf (0 outside the grid).  Flags any
// non-finite density in status[0].
template <class Tm>
__global__ void block_densities(const void *__restrict__ rho, int rho_f32, int64_t nx, int64_t ny, int64_t nz,
                                int64_t vx, int64_t vy, int64_t vz, Block3 blk, int b, int B,
                                Tm *__restrict__ mass, int *__restrict__ status) {
    const int64_t b3 = (int64_t)b * b * b;
    const int64_t total = blk.n[0] * blk.n[1] * blk.n[2] * B * b3;
    const int64_t nvox = nx * ny * nz;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = e % b3;
        const int64_t rest = e / b3;
        const int bb = (int)(rest % B);
        const int64_t leaf = rest / B;
        const int64_t Lx = blk.lo[0] + leaf % blk.n[0];
        const int64_t Ly = blk.lo[1] + (leaf / blk.n[0]) % blk.n[1];
        const int64_t Lz = blk.lo[2] + leaf / (blk.n[0] * blk.n[1]);
        const int64_t i = Lx * b + v % b - vx;
        const int64_t j = Ly * b + (v / b) % b - vy;
        const int64_t k = Lz * b + v / ((int64_t)b * b) - vz;
        Tm m = Tm(0);
        if (i >= 0 && i < nx && j >= 0 && j < ny && k >= 0 && k < nz) {
            const int64_t idx = (int64_t)bb * nvox + (k * ny + j) * nx + i;
            const double r = rho_f32 ? (double)reinterpret_cast<const float *>(rho)[idx]
                                     : reinterpret_cast<const double *>(rho)[idx];
            if (!isfinite(r)) atomicOr(status, 1);
            m = (Tm)r;
        }
        mass[e] = m;
    }
}

// P2M: ME[leaf][bb][k] = sum_v P[v][k] mass[leaf][bb][v].  A block handles
// kP2MLeaves leaves; each thread owns coefficients k, k + blockDim, ...
constexpr int kP2MLeaves = 4;

template <class T>
__global__ void __launch_bounds__(128)
p2m_kernel(const T *__restrict__ mass, const T *__restrict__ P, int64_t nleaf, int b3, int B, int K,
           int ldk, T *__restrict__ me) {
    extern __shared__ unsigned char shraw[];
    T *ms = reinterpret_cast<T *>(shraw);  // [kP2MLeaves*B][b3]
    const int64_t leaf0 = (int64_t)blockIdx.x * kP2MLeaves;
    const int nl = (int)std::min<int64_t>(kP2MLeaves, nleaf - leaf0);
    const int ncol = nl * B;
    for (int e = threadIdx.x; e < ncol * b3; e += blockDim.x) ms[e] = mass[leaf0 * B * b3 + e];
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        T acc[kP2MLeaves * 4];
        for (int c0 = 0; c0 < ncol; c0 += kP2MLeaves * 4) {
            const int cn = std::min(kP2MLeaves * 4, ncol - c0);
#pragma unroll
            for (int c = 0; c < kP2MLeaves * 4; ++c) acc[c] = T(0);
            for (int v = 0; v < b3; ++v) {
                const T pv = P[(size_t)v * K + k];
#pragma unroll
                for (int c = 0; c < kP2MLeaves * 4; ++c)
                    if (c < cn) acc[c] += pv * ms[(c0 + c) * b3 + v];
            }
#pragma unroll
            for (int c = 0; c < kP2MLeaves * 4; ++c)
                if (c < cn) me[(leaf0 * B + c0 + c) * ldk + k] = acc[c];
        }
    }
}

// Fused a0 + a3 for leaves of at most 4^3 voxels: a block takes a 4x4x4
// tile of leaves for one batch member, reads their densities straight from
// the caller's grid (rows of 4b contiguous voxels), writes the leaf-blocked
// copy used by the near field, and multiplies the 64 leaves' masses by the
// P2M matrix held in shared memory: ME[leaf][k] = sum_v P[v][k] mass[leaf][v].
// Thread (tl, tk) of 16 x 16 owns leaves 4tl..4tl+3 and coefficients
// tk + 16j, j < RPT.
constexpr int kFTile = 4;                       // leaves per tile edge
constexpr int kFLeaves = kFTile * kFTile * kFTile;
constexpr int kFPitch = kFLeaves + 4;           // padded row of the mass tile (bank spread)

__host__ __device__ inline int p2m_fused_pitch(int K) { return (K + 15) & ~15; }

template <class T>
__host__ __device__ inline size_t p2m_fused_smem(int b3, int K, int ldk) {
    const size_t in = (size_t)b3 * p2m_fused_pitch(K) + (size_t)b3 * kFPitch;
    const size_t out = (size_t)kFLeaves * ldk;
    return sizeof(T) * (in > out ? in : out);
}

template <class T, int BV, int RPT>
__global__ void __launch_bounds__(256)
p2m_fused(const void *__restrict__ rho, int rho_f32, int64_t nx, int64_t ny, int64_t nz, int64_t vx, int64_t vy,
          int64_t vz, Block3 blk, int B, const T *__restrict__ P, int K, int ldk, T *__restrict__ mass,
          T *__restrict__ me, int *__restrict__ status) {
    extern __shared__ unsigned char shraw[];
    constexpr int b3 = BV * BV * BV;
    constexpr int e4 = kFTile * BV;   // voxels per tile edge
    const int KP = p2m_fused_pitch(K);
    T *Ps = reinterpret_cast<T *>(shraw);   // [b3][KP]
    T *ms = Ps + (size_t)b3 * KP;           // [b3][kFPitch]: voxel-major, leaf-minor
    T *os = reinterpret_cast<T *>(shraw);   // [64][ldk] (after the product)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int bb = blockIdx.y;
    const int64_t ntx = (blk.n[0] + kFTile - 1) / kFTile, nty = (blk.n[1] + kFTile - 1) / kFTile;
    const int64_t tile = blockIdx.x;
    const int64_t l0x = (tile % ntx) * kFTile, l0y = ((tile / ntx) % nty) * kFTile, l0z = tile / (ntx * nty) * kFTile;
    for (int v = warp; v < b3; v += 8)
        for (int k = lane; k < KP; k += 32) Ps[v * KP + k] = k < K ? P[(size_t)v * K + k] : T(0);
    // densities of the tile's (4b)^3 voxels, x fastest (coalesced rows)
    const int64_t nvox = nx * ny * nz;
    const int64_t gx0 = (blk.lo[0] + l0x) * BV - vx, gy0 = (blk.lo[1] + l0y) * BV - vy,
                  gz0 = (blk.lo[2] + l0z) * BV - vz;
    bool bad = false;
    for (int e = tid; e < e4 * e4 * e4; e += 256) {
        const int ix = e % e4, iy = (e / e4) % e4, iz = e / (e4 * e4);
        const int64_t i = gx0 + ix, j = gy0 + iy, k = gz0 + iz;
        T m = T(0);
        if (i >= 0 && i < nx && j >= 0 && j < ny && k >= 0 && k < nz) {
            const int64_t idx = (int64_t)bb * nvox + (k * ny + j) * nx + i;
            const double r = rho_f32 ? (double)reinterpret_cast<const float *>(rho)[idx]
                                     : reinterpret_cast<const double *>(rho)[idx];
            bad |= !isfinite(r);
            m = (T)r;
        }
        const int leaf = ((iz / BV) * kFTile + iy / BV) * kFTile + ix / BV;
        const int v = ((iz % BV) * BV + iy % BV) * BV + ix % BV;
        ms[v * kFPitch + leaf] = m;
    }
    if (bad) atomicOr(status, 1);
    __syncthreads();
    // leaf-blocked masses for the near field: mass[leaf][bb][v]
    for (int e = tid; e < kFLeaves * b3; e += 256) {
        const int leaf = e / b3, v = e % b3;
        const int64_t gx = l0x + leaf % kFTile, gy = l0y + (leaf / kFTile) % kFTile, gz = l0z + leaf / (kFTile * kFTile);
        if (gx >= blk.n[0] || gy >= blk.n[1] || gz >= blk.n[2]) continue;
        const int64_t gl = (gz * blk.n[1] + gy) * blk.n[0] + gx;
        mass[(gl * B + bb) * b3 + v] = ms[v * kFPitch + leaf];
    }
    const int tl = tid & 15, tk = tid >> 4;
    T acc[4][RPT];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < RPT; ++j) acc[i][j] = T(0);
#pragma unroll 4
    for (int v = 0; v < b3; ++v) {
        T m4[4];
        if constexpr (sizeof(T) == 4) {
            const float4 t4 = *reinterpret_cast<const float4 *>(ms + v * kFPitch + 4 * tl);
            m4[0] = t4.x;
            m4[1] = t4.y;
            m4[2] = t4.z;
            m4[3] = t4.w;
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) m4[i] = ms[v * kFPitch + 4 * tl + i];
        }
        const T *pr = Ps + (size_t)v * KP + tk;
#pragma unroll
        for (int j = 0; j < RPT; ++j) {
            const T pv = (tk + 16 * j < KP) ? pr[16 * j] : T(0);
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[i][j] += pv * m4[i];
        }
    }
    __syncthreads();   // Ps and ms are reused as the output staging area
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < RPT; ++j) {
            const int k = tk + 16 * j;
            if (k < ldk) os[(4 * tl + i) * ldk + k] = k < K ? acc[i][j] : T(0);
        }
    __syncthreads();
    for (int leaf = warp; leaf < kFLeaves; leaf += 8) {
        const int64_t gx = l0x + leaf % kFTile, gy = l0y + (leaf / kFTile) % kFTile, gz = l0z + leaf / (kFTile * kFTile);
        if (gx >= blk.n[0] || gy >= blk.n[1] || gz >= blk.n[2]) continue;
        const int64_t gl = (gz * blk.n[1] + gy) * blk.n[0] + gx;
        T *dst = me + (gl * B + bb) * ldk;
        for (int k = lane; k < ldk; k += 32) dst[k] = os[leaf * ldk + k];
    }
}

template <class T, int BV>
gf_status launch_p2m_fused_b(gf_plan_s *plan, const void *rho, int rho_f32, int B, cudaStream_t st) {
    FmmPlan *F = plan->fmm;
    const FmmLevel &lv = F->lev[F->L];
    const int K = F->K;
    const Block3 blk = block_of(lv);
    const int64_t tiles = ((blk.n[0] + kFTile - 1) / kFTile) * ((blk.n[1] + kFTile - 1) / kFTile) *
                          ((blk.n[2] + kFTile - 1) / kFTile);
    const size_t shm = p2m_fused_smem<T>(BV * BV * BV, K, F->KS);
    const T *P = sizeof(T) == 8 ? (const T *)F->p2m_d : (const T *)F->p2m_f;
    const dim3 grid((unsigned)tiles, (unsigned)B);
#define GF_P2M_LAUNCH(R)                                                                                    \
    do {                                                                                                    \
        GF_TRY(ensure_smem(p2m_fused<T, BV, R>, shm));                                                      \
        p2m_fused<T, BV, R><<<grid, 256, shm, st>>>(rho, rho_f32, plan->grid.n[0], plan->grid.n[1],          \
                                                    plan->grid.n[2], F->voff[0], F->voff[1], F->voff[2], blk, B, \
                                                    P, K, F->KS, (T *)F->mass, (T *)lv.me, plan->d_status); \
    } while (0)
    const int rpt = (p2m_fused_pitch(K) + 15) / 16;
    if (rpt <= 4)
        GF_P2M_LAUNCH(4);
    else if (rpt <= 8)
        GF_P2M_LAUNCH(8);
    else if (rpt <= 12)
        GF_P2M_LAUNCH(12);
    else
        GF_P2M_LAUNCH(20);
#undef GF_P2M_LAUNCH
    GF_KERNEL_DONE();
    return GF_OK;
}

// Leaf-blocked densities only (the P2M then runs on the tensor cores):
// thread x of block (y, z) copies the BV voxels of row (y, z) of leaf x --
// consecutive threads read consecutive voxels of the grid row and each
// writes one BV-wide piece of its leaf's mass row.  Grid: (ceil(nLx/128),
// nLy*BV, nLz*BV*B).
template <class T, int BV>
__global__ void __launch_bounds__(128)
block_rows(const void *__restrict__ rho, int rho_f32, int64_t nx, int64_t ny, int64_t nz, int64_t vx, int64_t vy,
           int64_t vz, Block3 blk, int64_t lz0, int64_t nlz, int B, T *__restrict__ mass, int *__restrict__ status) {
    constexpr int b3 = BV * BV * BV;
    const int64_t lx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (lx >= blk.n[0]) return;
    const int yv = blockIdx.y;
    const int64_t zb = blockIdx.z;
    const int64_t nzv = nlz * BV;
    const int zv = (int)(lz0 * BV + zb % nzv);   // voxel layer within the block
    const int bb = (int)(zb / nzv);
    const int64_t j = blk.lo[1] * BV + yv - vy, k = blk.lo[2] * BV + zv - vz;
    const int64_t i0 = (blk.lo[0] + lx) * BV - vx;
    const bool row_in = j >= 0 && j < ny && k >= 0 && k < nz;
    const int64_t base = (int64_t)bb * nx * ny * nz + (k * ny + j) * nx;
    T m[BV];
    bool bad = false;
#pragma unroll
    for (int x = 0; x < BV; ++x) {
        const int64_t i = i0 + x;
        T v = T(0);
        if (row_in && i >= 0 && i < nx) {
            const double r = rho_f32 ? (double)reinterpret_cast<const float *>(rho)[base + i]
                                     : reinterpret_cast<const double *>(rho)[base + i];
            bad |= !isfinite(r);
            v = (T)r;
        }
        m[x] = v;
    }
    if (bad) atomicOr(status, 1);
    const int64_t leaf = ((int64_t)(zv / BV) * blk.n[1] + yv / BV) * blk.n[0] + lx;
    T *dst = mass + (leaf * B + bb) * b3 + ((zv % BV) * BV + yv % BV) * BV;
    if constexpr (BV == 4 && sizeof(T) == 4) {
        *reinterpret_cast<float4 *>(dst) = make_float4(m[0], m[1], m[2], m[3]);
    } else {
#pragma unroll
        for (int x = 0; x < BV; ++x) dst[x] = m[x];
    }
}

template <class T, int BV>
gf_status launch_blocking(gf_plan_s *plan, const void *rho, int rho_f32, int B, int64_t lz0, int64_t nlz,
                          cudaStream_t st) {
    FmmPlan *F = plan->fmm;
    const Block3 blk = block_of(F->lev[F->L]);
    if (nlz <= 0) return GF_OK;
    const int64_t gz = nlz * BV * B;
    if (blk.n[1] * BV > 65535 || gz > 65535) {
        set_error("leaf block too large for the density re-blocking grid");
        return GF_ERR_UNSUPPORTED;
    }
    const dim3 grid(ceil_div(blk.n[0], 128), (unsigned)(blk.n[1] * BV), (unsigned)gz);
    block_rows<T, BV><<<grid, 128, 0, st>>>(rho, rho_f32, plan->grid.n[0], plan->grid.n[1], plan->grid.n[2],
                                            F->voff[0], F->voff[1], F->voff[2], blk, lz0, nlz, B, (T *)F->mass,
                                            plan->d_status);
    GF_KERNEL_DONE();
    return GF_OK;
}

template <class T>
gf_status launch_p2m_fused(gf_plan_s *plan, const void *rho, int rho_f32, int B, cudaStream_t st) {
    switch (plan->fmm->b) {
        case 1: return launch_p2m_fused_b<T, 1>(plan, rho, rho_f32, B, st);
        case 2: return launch_p2m_fused_b<T, 2>(plan, rho, rho_f32, B, st);
        case 3: return launch_p2m_fused_b<T, 3>(plan, rho, rho_f32, B, st);
        default: return launch_p2m_fused_b<T, 4>(plan, rho, rho_f32, B, st);
    }
}

// Whether the fused kernel applies (leaves of at most 4^3 voxels, tables
// that fit one block's shared memory).
template <class T>
bool p2m_fused_ok(const FmmPlan *F) {
    const int b3 = F->b * F->b * F->b;
    return F->b <= 4 && p2m_fused_pitch(F->K) <= 320 && p2m_fused_smem<T>(b3, F->K, F->KS) <= 200 * 1024;
}

// Top-level translations in FP64 (mixed precision keeps the M2M into
// level 2 and the L2L out of it in double).  The work is small but FP64 is
// slow, so each block computes 32 output coefficients of one box and its 8
// warps split the input coefficients; the partial sums meet in shared
// memory.  Grid: (boxes, ceil(K / 32)), 256 threads.
constexpr int kTopWarps = 8;

// Batch members [b0, b0 + nb) of B are handled by one launch (nb bounded by
// shared memory).
// sum_{i0 <= i < i1} t[i K] x[i] with four partial sums, so that four
// table loads are in flight at once (the FP64 top-level translations are
// bound by the latency of these loads, not by arithmetic)
template <class Tc>
__device__ __forceinline__ Tc dot_strided(const Tc *__restrict__ t, const Tc *x, int i0, int i1, int K) {
    Tc a0 = Tc(0), a1 = Tc(0), a2 = Tc(0), a3 = Tc(0);
    int i = i0;
    for (; i + 3 < i1; i += 4) {
        const Tc t0 = t[(size_t)i * K], t1 = t[(size_t)(i + 1) * K], t2 = t[(size_t)(i + 2) * K],
                 t3 = t[(size_t)(i + 3) * K];
        a0 += t0 * x[i];
        a1 += t1 * x[i + 1];
        a2 += t2 * x[i + 2];
        a3 += t3 * x[i + 3];
    }
    for (; i < i1; ++i) a0 += t[(size_t)i * K] * x[i];
    return (a0 + a1) + (a2 + a3);
}

__host__ __device__ inline size_t top_smem(int nexp, int nb, int K) {
    return sizeof(double) * ((size_t)nexp * nb * K + (size_t)kTopWarps * nb * 32);
}

// M2M: parent ME[k] = sum over existing children c, inputs i of
// T_oct(c)[i][k] * child ME[i].  amax (may be null): the largest |ME[k]|
// written into parents [alo, ahi), as float bits with atomicMax.
template <class Ts, class Tc>
__global__ void __launch_bounds__(kTopWarps * 32)
m2m_kernel(const Ts *__restrict__ me_c, Block3 bc, Ts *__restrict__ me_p, Block3 bp, int B, int b0, int nb, int K,
           int ldk, const Tc *__restrict__ tab, uint32_t *amax = nullptr, int64_t alo = 0, int64_t ahi = 0) {
    extern __shared__ unsigned char shraw[];
    Tc *xs = reinterpret_cast<Tc *>(shraw);   // [8][nb][K] child expansions
    Tc *red = xs + 8 * nb * K;                // [kTopWarps][nb][32] partial sums
    __shared__ int present[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t pi = blockIdx.x;
    const int k = blockIdx.y * 32 + lane;
    const int64_t px = bp.lo[0] + pi % bp.n[0], py = bp.lo[1] + (pi / bp.n[0]) % bp.n[1],
                  pz = bp.lo[2] + pi / (bp.n[0] * bp.n[1]);
    for (int e = threadIdx.x; e < 8 * nb * K; e += blockDim.x) {
        const int oct = e / (nb * K), r = e - oct * nb * K;
        const int64_t cx = 2 * px + (oct & 1) - bc.lo[0], cy = 2 * py + ((oct >> 1) & 1) - bc.lo[1],
                      cz = 2 * pz + ((oct >> 2) & 1) - bc.lo[2];
        const bool in = cx >= 0 && cx < bc.n[0] && cy >= 0 && cy < bc.n[1] && cz >= 0 && cz < bc.n[2];
        const int rb = r / K, rk = r - rb * K;
        xs[e] = in ? (Tc)me_c[(((cz * bc.n[1] + cy) * bc.n[0] + cx) * B + b0 + rb) * ldk + rk] : Tc(0);
        if (r == 0) present[oct] = in;
    }
    __syncthreads();
    const int per = (K + kTopWarps - 1) / kTopWarps;
    const int i0 = warp * per, i1 = min(K, i0 + per);
    for (int bb = 0; bb < nb; ++bb) {
        Tc acc = Tc(0);
        if (k < K)
            for (int oct = 0; oct < 8; ++oct) {
                if (!present[oct]) continue;
                const Tc *t = tab + (size_t)oct * K * K + k;
                const Tc *x = xs + (oct * nb + bb) * K;
                acc += dot_strided(t, x, i0, i1, K);
            }
        red[(warp * nb + bb) * 32 + lane] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nb * 32; e += blockDim.x) {
        const int bb = e / 32, kk = blockIdx.y * 32 + (e & 31);
        if (kk >= K) continue;
        Tc acc = Tc(0);
        for (int w = 0; w < kTopWarps; ++w) acc += red[(w * nb + bb) * 32 + (e & 31)];
        const Ts v = (Ts)acc;
        me_p[(pi * B + b0 + bb) * ldk + kk] = v;
        if (amax && pi >= alo && pi < ahi && v != Ts(0) && v == v)   // NaN is skipped, as fmaxf does
            atomicMax(amax, __float_as_uint(fabsf((float)v)));
    }
}

// L2L: child LE[k] += sum_i T_oct[i][k] * parent LE[i], one block per
// (observer box of level l, 32 outputs).
template <class Ts, class Tc>
__global__ void __launch_bounds__(kTopWarps * 32)
l2l_kernel(const Ts *__restrict__ le_p, const uint64_t *__restrict__ tkey, const int32_t *__restrict__ tparent,
           Ts *__restrict__ le_c, int B, int b0, int nb, int K, int ldk, const Tc *__restrict__ tab) {
    extern __shared__ unsigned char shraw[];
    Tc *xs = reinterpret_cast<Tc *>(shraw);   // [nb][K]
    Tc *red = xs + nb * K;                    // [kTopWarps][nb][32]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t t = blockIdx.x;
    const int k = blockIdx.y * 32 + lane;
    const int oct = (int)(tkey[t] & 7);
    const int64_t par = tparent[t];
    for (int e = threadIdx.x; e < nb * K; e += blockDim.x) {
        const int rb = e / K, rk = e - rb * K;
        xs[e] = (Tc)le_p[(par * B + b0 + rb) * ldk + rk];
    }
    __syncthreads();
    const int per = (K + kTopWarps - 1) / kTopWarps;
    const int i0 = warp * per, i1 = min(K, i0 + per);
    const Tc *tb = tab + (size_t)oct * K * K + k;
    for (int bb = 0; bb < nb; ++bb) {
        Tc acc = Tc(0);
        if (k < K) acc = dot_strided(tb, xs + bb * K, i0, i1, K);
        red[(warp * nb + bb) * 32 + lane] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nb * 32; e += blockDim.x) {
        const int bb = e / 32, kk = blockIdx.y * 32 + (e & 31);
        if (kk >= K) continue;
        Tc acc = Tc(0);
        for (int w = 0; w < kTopWarps; ++w) acc += red[(w * nb + bb) * 32 + (e & 31)];
        Ts *o = le_c + (t * B + b0 + bb) * ldk + kk;
        *o = (Ts)((Tc)*o + acc);
    }
}

// Largest batch chunk whose shared memory fits one block.
inline int top_batch_chunk(int nexp, int B, int K) {
    int nb = B;
    while (nb > 1 && top_smem(nexp, nb, K) > 200 * 1024) nb = (nb + 1) / 2;
    return nb;
}

// ---------------------------------------------------------------- evaluation
constexpr int kEvalWarps = 4;
constexpr int kEvalChunk = 64;
constexpr int kTPL = 2;            // targets per lane: a work item has <= 64 targets
constexpr int kSrcTable = 512;     // per-block table of a leaf's source offsets
constexpr int kMaxLat = 8;         // lattice planes per axis of a leaf (lattice near field)

constexpr int kLatGroups = 4;      // lattice form: lane groups sharing a small item

// Elements of one warp's shared-memory slice of the evaluation kernel
// (a multiple of 8): 4 kEvalChunk staged source values (FP32: 8, the
// duplicated lattice weights of up to kLatGroups leaves), three gradient
// expansions of P2 coefficients (FP32: duplicated pairs) and 27
// neighbour-leaf entries (int64).
inline __host__ __device__ int eval_stage(int tsize) { return (tsize == 4 ? 2 : 1) * 4 * kEvalChunk; }
inline __host__ __device__ int eval_slice(int P2, int tsize) {
    const int dmul = tsize == 4 ? 2 : 1;
    return (eval_stage(tsize) + 3 * dmul * P2 + 27 * 8 / tsize + 7) & ~7;
}

struct EvalArgs {
    int L;                       // leaf level
    uint32_t part_lo, part_hi;   // source partition (in_source_part)
    const int4 *items;
    int64_t n_items;
    unsigned long long *queue; // [0]: next item, [1]: warps done (zero between launches)
    int mode;                  // 0: near + far field; 1: near field only, sums to nsum;
                               // 2: far field, near sums from nsum
    void *nsum;                // [B][M][6] T: (hi, lo) of x, y, z per observer (key order)
    const uint64_t *tkey;      // leaf keys
    const int32_t *perm;
    const void *tloc;          // [M][3] T
    const void *mass;          // [ns_L][B][b3] T
    const void *le;            // [nt_L][B][ldk] T
    const QuadRule *qr;
    Block3 blk;                // leaf source block
    int b, nq, B, K, ldk, p;
    int64_t M;
    double scale;              // G * h
    double eps2;               // coincidence radius^2 (voxel units)
    int guard_all;             // quadrature nodes on voxel faces: every leaf may hold
                               // a source coincident with an observer (else only
                               // the observer's own leaf can)
    double *g, *gz;
    // Lattice form of a leaf's sources (rules that are tensor products of m
    // nodes per axis): the b^3 nq sources sit on N1^3 lattice points, N1 =
    // b m.  lat_c[a][i]: coordinate of lattice plane i along axis a from the
    // leaf centre (voxel units); lat_q[(ia % m) + m ((ib % m) + m (ic % m))]
    // is the rule's node at lattice point (ia, ib, ic).
    int lat_m;
    float lat_c[3][kMaxLat];
    int lat_q[kMaxQuad];
};

// Near field + far field of the observers of one leaf, one warp per work
// item; warps take items from a queue (one atomic per item), so a warp that
// drew a short item takes the next one at once.  The sources of each
// neighbouring leaf are staged in the warp's shared-memory slice in chunks
// of 64 (position relative to the target leaf's centre, mass times
// quadrature weight) and every lane sweeps them for its two observers.
// Per-leaf partial sums are merged with TwoSum.  N1 > 0 (FP32, sources on
// an N1^3 lattice per leaf): the lattice form of the near field below; an
// item of at most 32 observers there splits its neighbour leaves over 2 or
// 4 groups of lanes that hold the same observers, and the groups' sums are
// merged by shuffles.
template <class T, int N1>
__global__ void __launch_bounds__(kEvalWarps * 32, sizeof(T) == 4 ? 5 : 1)   // FP32: 5 blocks (20 warps, 96 registers) per SM
eval_kernel(EvalArgs a) {
    extern __shared__ unsigned char shraw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int P2 = a.p * a.p;
    const int b3 = a.b * a.b * a.b;
    const int nsrc = b3 * a.nq;
    // block-wide table: offset of source u (voxel u / nq, node u % nq) from
    // its leaf's centre, quadrature weight, voxel index
    Vec4<T> *tab = reinterpret_cast<Vec4<T> *>(shraw);
    int *tvox = reinterpret_cast<int *>(tab + kSrcTable);
    // per-warp slice, a multiple of 8 elements so every slice keeps the
    // alignment of the vector type: staged sources, the gradient expansions
    // (FP32: duplicated pairs), the item's neighbour leaves
    constexpr bool kF32 = std::is_same<T, float>::value;
    const int wstride = eval_slice(P2, sizeof(T));
    T *wsh = reinterpret_cast<T *>(tvox + kSrcTable) + (size_t)warp * wstride;
    Vec4<T> *src = reinterpret_cast<Vec4<T> *>(wsh);
    T *Dx = wsh + eval_stage(sizeof(T)), *Dy = Dx + (kF32 ? 2 : 1) * P2, *Dz = Dy + (kF32 ? 2 : 1) * P2;
    int64_t *nbl = reinterpret_cast<int64_t *>(Dz + (kF32 ? 2 : 1) * P2);
    const T *tloc = reinterpret_cast<const T *>(a.tloc);
    const T *mass = reinterpret_cast<const T *>(a.mass);
    const T *le = reinterpret_cast<const T *>(a.le);
    const T half_b = T(0.5) * T(a.b);
    const T inv_b = T(1) / T(a.b);
    const T eps2 = (T)a.eps2;
    const bool use_tab = nsrc <= kSrcTable;
    if (N1 > 0) {
        // lattice point n = i + N1 (j + N1 k): its voxel and the rule's weight
        const int m = a.lat_m;
        for (int n = threadIdx.x; n < N1 * N1 * N1; n += blockDim.x) {
            const int i = n % N1, j = (n / N1) % N1, k = n / (N1 * N1);
            const int v = i / m + a.b * (j / m + a.b * (k / m));
            const int q = a.lat_q[i % m + m * (j % m + m * (k % m))];
            tab[n].w = (T)a.qr->wn[q];
            tvox[n] = v;
        }
    } else if (use_tab) {
        for (int u = threadIdx.x; u < nsrc; u += blockDim.x) {
            const int v = u / a.nq, q = u - v * a.nq;
            Vec4<T> e;
            e.x = T(v % a.b) + (T)(0.5 + 0.5 * a.qr->xi[q][0]) - half_b;
            e.y = T((v / a.b) % a.b) + (T)(0.5 + 0.5 * a.qr->xi[q][1]) - half_b;
            e.z = T(v / (a.b * a.b)) + (T)(0.5 + 0.5 * a.qr->xi[q][2]) - half_b;
            e.w = (T)a.qr->wn[q];
            tab[u] = e;
            tvox[u] = v;
        }
    }
    __syncthreads();
    // far-field scale of the L2P gradient (voxel units)
    const double far_s = -1.0 / ((double)a.b * (double)a.b);
    const float far_sf = (float)far_s;
    // lattice form: this lane's two lattice points (weight, voxel)
    float lw0 = 0.f, lw1 = 0.f;
    int lv0 = 0, lv1 = 0;
    if (N1 > 0) {
        lw0 = (float)tab[lane].w;
        lw1 = (float)tab[lane + 32].w;
        lv0 = tvox[lane];
        lv1 = tvox[lane + 32];
    }
    for (;;) {
        int64_t it = 0;
        if (lane == 0) it = (int64_t)atomicAdd(a.queue, 1ull);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= a.n_items) break;
        const int4 item = a.items[it];
        const int leaf = item.x;
        // lattice form: lanes per group (gs) and groups (ns) for this item;
        // lane = grp * gs + r0 holds observers r0 and r0 + gs of the item
        int gs = 32;
        if constexpr (N1 > 0 && kF32) {
            const int np = (item.z + 1) >> 1;
            if (a.mode != 2) gs = np > 16 ? 32 : np > 8 ? 16 : 32 / kLatGroups;
        }
        const int ns = 32 / gs, grp = lane / gs, r0 = lane - grp * gs;
        int64_t lc[3] = {0, 0, 0};   // the leaf's box coordinates (near field only)
        if (a.mode != 2) {
            const uint64_t k = a.tkey[leaf];
            for (int bit = 0; bit < 21; ++bit) {
                lc[0] |= (int64_t)((k >> (3 * bit)) & 1) << bit;
                lc[1] |= (int64_t)((k >> (3 * bit + 1)) & 1) << bit;
                lc[2] |= (int64_t)((k >> (3 * bit + 2)) & 1) << bit;
            }
        }
        T tx[kTPL], ty[kTPL], tz[kTPL];
        int tid[kTPL];
#pragma unroll
        for (int u = 0; u < kTPL; ++u) {
            const int r = r0 + gs * u;
            tid[u] = r < item.z ? item.y + r : -1;
            const int64_t i = tid[u] >= 0 ? tid[u] : item.y;
            tx[u] = tloc[3 * i + 0];
            ty[u] = tloc[3 * i + 1];
            tz[u] = tloc[3 * i + 2];
        }
        // the item's neighbour leaves inside the source block, in the order of
        // nb = (dx + 1) + 3 (dy + 1) + 9 (dz + 1): source-block index * 32 + nb
        __syncwarp();
        int nv = 0;
        if (a.mode != 2) {
            bool in = false;
            int64_t sidx = 0;
            if (lane < 27) {
                const int dx = lane % 3 - 1, dy = (lane / 3) % 3 - 1, dz = lane / 9 - 1;
                const int64_t sx = lc[0] + dx - a.blk.lo[0], sy = lc[1] + dy - a.blk.lo[1],
                              sz = lc[2] + dz - a.blk.lo[2];
                in = sx >= 0 && sy >= 0 && sz >= 0 && sx < a.blk.n[0] && sy < a.blk.n[1] && sz < a.blk.n[2] &&
                     in_source_part(lc[0] + dx, lc[1] + dy, lc[2] + dz, a.L - 2, a.part_lo, a.part_hi);
                sidx = (sz * a.blk.n[1] + sy) * a.blk.n[0] + sx;
            }
            const unsigned vm = __ballot_sync(0xffffffffu, in);
            if (in) nbl[__popc(vm & ((1u << lane) - 1u))] = sidx * 32 + lane;
            nv = __popc(vm);
        }
        __syncwarp();
        for (int bb = 0; bb < a.B; ++bb) {
            T hx[kTPL], hy[kTPL], hz[kTPL], lx[kTPL], ly[kTPL], lz[kTPL];
#pragma unroll
            for (int u = 0; u < kTPL; ++u) hx[u] = hy[u] = hz[u] = lx[u] = ly[u] = lz[u] = T(0);
            // ---- near field: the leaf itself and its nearest neighbours (in the
            // lattice form, group grp takes entries grp, grp + ns, ...; a group
            // past the end computes entry c0's leaf and drops the result)
            for (int c0 = 0; c0 < nv; c0 += ns) {
                const bool act = c0 + grp < nv;
                const int64_t ent = nbl[act ? c0 + grp : c0];
                const int64_t sl = ent >> 5;
                const int nb = (int)(ent & 31);
                const int dx = nb % 3 - 1, dy = (nb / 3) % 3 - 1, dz = nb / 9 - 1;
                const T *ms = mass + (sl * a.B + bb) * b3;
                const T ox = T(dx * a.b), oy = T(dy * a.b), oz = T(dz * a.b);
                if constexpr (N1 > 0 && std::is_same<T, float>::value) {
                    // Lattice form.  With d = t - s and the sources on the planes
                    // x = X_i, y = Y_j, z = Z_k, the leaf's sum of w d / |d|^3 is
                    //   (sum_i dx_i Sx_i, sum_j dy_j Sy_j, sum_k dz_k Sz_k),
                    //   Sx_i = sum_{j,k} w_ijk |d_ijk|^-3  (Sy_j, Sz_k alike),
                    // so a source costs one add (|d|^2 from the squared plane
                    // distances), the reciprocal square root, three multiplies and
                    // three adds; the lane's two observers form one packed pair.
                    constexpr int N3 = N1 * N1 * N1;
                    __syncwarp();
                    float2 *wl = reinterpret_cast<float2 *>(wsh) + grp * N3;
                    static_assert(N1 == 4, "two lattice points per lane, rows of four");
                    if (gs == 32) {
                        const float w0 = lw0 * ms[lv0], w1 = lw1 * ms[lv1];
                        wl[lane] = make_float2(w0, w0);
                        wl[lane + 32] = make_float2(w1, w1);
                    } else {
                        for (int n = r0; n < N3; n += gs) {
                            const float w = (float)tab[n].w * ms[tvox[n]];
                            wl[n] = make_float2(w, w);
                        }
                    }
                    __syncwarp();
                    const uint64_t PX = pk2(tx[0], tx[1]), PY = pk2(ty[0], ty[1]), PZ = pk2(tz[0], tz[1]);
                    uint64_t X2[N1], Y2[N1], SX[N1], SY[N1];
#pragma unroll
                    for (int i = 0; i < N1; ++i) {
                        const float cx = a.lat_c[0][i] + ox, cy = a.lat_c[1][i] + oy;
                        const uint64_t ex = sub2(PX, pk2(cx, cx)), ey = sub2(PY, pk2(cy, cy));
                        X2[i] = mul2(ex, ex);
                        Y2[i] = mul2(ey, ey);
                        SX[i] = SY[i] = 0;
                    }
                    uint64_t QZ = 0;
                    // one z-plane of the lattice at a time (Sz_k is a single sum)
                    auto lattice = [&](auto guarded) {
                        constexpr bool kGuard = decltype(guarded)::value;
#pragma unroll 1
                        for (int k = 0; k < N1; ++k) {
                            const float cz = a.lat_c[2][k] + oz;
                            const uint64_t ez = sub2(PZ, pk2(cz, cz));
                            const uint64_t Z2 = mul2(ez, ez);
                            const uint64_t *wk = reinterpret_cast<const uint64_t *>(wl + N1 * N1 * k);
                            uint64_t SZ = 0;
#pragma unroll
                            for (int j = 0; j < N1; ++j) {
                                const uint64_t YZ = add2(Y2[j], Z2);
                                // the row's four terms: each into its Sx_i, their
                                // pairwise sum once into Sy_j and Sz (short chains)
                                uint64_t K3v[N1];
#pragma unroll
                                for (int i = 0; i < N1; ++i) {
                                    const uint64_t R2 = add2(X2[i], YZ);
                                    float r0, r1;
                                    up2(R2, r0, r1);
                                    float i0 = rsqrt_ftz(r0), i1 = rsqrt_ftz(r1);
                                    if constexpr (kGuard) {
                                        i0 = r0 > (float)eps2 ? i0 : 0.f;
                                        i1 = r1 > (float)eps2 ? i1 : 0.f;
                                    }
                                    const uint64_t RI = pk2(i0, i1);
                                    K3v[i] = mul2(mul2(RI, RI), mul2(RI, wk[i + N1 * j]));
                                    SX[i] = add2(SX[i], K3v[i]);
                                }
                                const uint64_t tj = add2(add2(K3v[0], K3v[1]), add2(K3v[2], K3v[3]));
                                SY[j] = add2(SY[j], tj);
                                SZ = add2(SZ, tj);
                            }
                            QZ = fma2(SZ, ez, QZ);
                        }
                    };
                    if (a.guard_all || __any_sync(0xffffffffu, nb == 13))
                        lattice(std::true_type{});
                    else
                        lattice(std::false_type{});
                    uint64_t QX = 0, QY = 0;
#pragma unroll
                    for (int i = 0; i < N1; ++i) {
                        const float cx = a.lat_c[0][i] + ox, cy = a.lat_c[1][i] + oy;
                        QX = fma2(SX[i], sub2(PX, pk2(cx, cx)), QX);
                        QY = fma2(SY[i], sub2(PY, pk2(cy, cy)), QY);
                    }
                    float gx[2], gy[2], gz[2];
                    up2(QX, gx[0], gx[1]);
                    up2(QY, gy[0], gy[1]);
                    up2(QZ, gz[0], gz[1]);
                    if (act) {
#pragma unroll
                        for (int u = 0; u < kTPL; ++u) {
                            two_sum(hx[u], lx[u], (T)gx[u]);
                            two_sum(hy[u], ly[u], (T)gy[u]);
                            two_sum(hz[u], lz[u], (T)gz[u]);
                        }
                    }
                    continue;
                }
                T px[kTPL], py[kTPL], pz[kTPL];
#pragma unroll
                for (int u = 0; u < kTPL; ++u) px[u] = py[u] = pz[u] = T(0);
                constexpr bool kPacked = std::is_same<T, float>::value;
                uint64_t qx[kTPL], qy[kTPL], qz[kTPL];   // packed partial sums (FP32)
#pragma unroll
                for (int u = 0; u < kTPL; ++u) qx[u] = qy[u] = qz[u] = 0;
                for (int c0 = 0; c0 < nsrc; c0 += kEvalChunk) {
                    const int cnt = min(kEvalChunk, nsrc - c0);
                    __syncwarp();
                    for (int s = lane; s < cnt; s += 32) {
                        const int u = c0 + s;
                        Vec4<T> e;
                        int v;
                        if (use_tab) {
                            e = tab[u];
                            v = tvox[u];
                        } else {
                            v = u / a.nq;
                            const int q = u - v * a.nq;
                            e.x = T(v % a.b) + (T)(0.5 + 0.5 * a.qr->xi[q][0]) - half_b;
                            e.y = T((v / a.b) % a.b) + (T)(0.5 + 0.5 * a.qr->xi[q][1]) - half_b;
                            e.z = T(v / (a.b * a.b)) + (T)(0.5 + 0.5 * a.qr->xi[q][2]) - half_b;
                            e.w = (T)a.qr->wn[q];
                        }
                        e.x += ox;
                        e.y += oy;
                        e.z += oz;
                        e.w *= ms[v];
                        if constexpr (kPacked) {
                            // pairs of sources as {x0,x1, y0,y1, z0,z1, w0,w1}
                            T *rec = wsh + (s >> 1) * 8 + (s & 1);
                            rec[0] = e.x;
                            rec[2] = e.y;
                            rec[4] = e.z;
                            rec[6] = e.w;
                        } else {
                            src[s] = e;
                        }
                    }
                    if constexpr (kPacked) {
                        // an odd chunk ends with a massless source far away
                        if ((cnt & 1) && lane == 0) {
                            T *rec = wsh + (cnt >> 1) * 8 + 1;
                            rec[0] = rec[2] = rec[4] = T(1.0e4);
                            rec[6] = T(0);
                        }
                        __syncwarp();
                        uint64_t TX[kTPL], TY[kTPL], TZ[kTPL];
#pragma unroll
                        for (int u = 0; u < kTPL; ++u) {
                            TX[u] = pk2(tx[u], tx[u]);
                            TY[u] = pk2(ty[u], ty[u]);
                            TZ[u] = pk2(tz[u], tz[u]);
                        }
                        const int npair = (cnt + 1) >> 1;
                        // Only the observer's own leaf (or any leaf, when nodes lie
                        // on voxel faces) can hold a source at the observer's
                        // position; elsewhere r2 > 0 and the coincidence test is
                        // dropped from the pair loop.
                        auto sweep = [&](auto guarded) {
                            constexpr bool kGuard = decltype(guarded)::value;
#pragma unroll 2
                            for (int q = 0; q < npair; ++q) {
                                const ulonglong2 xy = *reinterpret_cast<const ulonglong2 *>(wsh + q * 8);
                                const ulonglong2 zw = *reinterpret_cast<const ulonglong2 *>(wsh + q * 8 + 4);
#pragma unroll
                                for (int u = 0; u < kTPL; ++u) {
                                    const uint64_t DX = sub2(TX[u], xy.x), DY = sub2(TY[u], xy.y),
                                                   DZ = sub2(TZ[u], zw.x);
                                    const uint64_t R2 = fma2(DZ, DZ, fma2(DY, DY, mul2(DX, DX)));
                                    float r0, r1;
                                    up2(R2, r0, r1);
                                    float i0, i1;
                                    if constexpr (kGuard) {
                                        i0 = r0 > (float)eps2 ? rsqrt_ftz(r0) : 0.f;
                                        i1 = r1 > (float)eps2 ? rsqrt_ftz(r1) : 0.f;
                                    } else {
                                        i0 = rsqrt_ftz(r0);
                                        i1 = rsqrt_ftz(r1);
                                    }
                                    const uint64_t RI = pk2(i0, i1);
                                    const uint64_t K3 = mul2(mul2(mul2(RI, RI), RI), zw.y);
                                    qx[u] = fma2(K3, DX, qx[u]);
                                    qy[u] = fma2(K3, DY, qy[u]);
                                    qz[u] = fma2(K3, DZ, qz[u]);
                                }
                            }
                        };
                        if (a.guard_all || nb == 13)
                            sweep(std::true_type{});
                        else
                            sweep(std::false_type{});
                        continue;
                    }
                    __syncwarp();
#pragma unroll 4
                    for (int s = 0; s < cnt; ++s) {
                        const Vec4<T> e = src[s];
#pragma unroll
                        for (int u = 0; u < kTPL; ++u) {
                            const T ddx = tx[u] - e.x, ddy = ty[u] - e.y, ddz = tz[u] - e.z;
                            const T r2 = ddx * ddx + ddy * ddy + ddz * ddz;
                            const T ri = r2 > eps2 ? rsqrt_t<T>(r2) : T(0);
                            const T k3 = e.w * (ri * ri * ri);
                            px[u] += k3 * ddx;
                            py[u] += k3 * ddy;
                            pz[u] += k3 * ddz;
                        }
                    }
                }
                if constexpr (kPacked) {
#pragma unroll
                    for (int u = 0; u < kTPL; ++u) {
                        float a0, a1;
                        up2(qx[u], a0, a1);
                        px[u] = a0 + a1;
                        up2(qy[u], a0, a1);
                        py[u] = a0 + a1;
                        up2(qz[u], a0, a1);
                        pz[u] = a0 + a1;
                    }
                }
#pragma unroll
                for (int u = 0; u < kTPL; ++u) {
                    two_sum(hx[u], lx[u], px[u]);
                    two_sum(hy[u], ly[u], py[u]);
                    two_sum(hz[u], lz[u], pz[u]);
                }
            }
            // the groups' sums of the same observers, merged into every group
            for (int o = gs; o < 32; o <<= 1) {
#pragma unroll
                for (int u = 0; u < kTPL; ++u) {
                    const T vx = __shfl_xor_sync(0xffffffffu, hx[u], o), wx = __shfl_xor_sync(0xffffffffu, lx[u], o);
                    const T vy = __shfl_xor_sync(0xffffffffu, hy[u], o), wy = __shfl_xor_sync(0xffffffffu, ly[u], o);
                    const T vz = __shfl_xor_sync(0xffffffffu, hz[u], o), wz = __shfl_xor_sync(0xffffffffu, lz[u], o);
                    two_sum(hx[u], lx[u], vx);
                    two_sum(hy[u], ly[u], vy);
                    two_sum(hz[u], lz[u], vz);
                    lx[u] += wx;
                    ly[u] += wy;
                    lz[u] += wz;
                }
            }
            // split evaluation: the near sums go to nsum (mode 1) or come from it (mode 2)
            if (a.mode != 0) {
                T *ns = reinterpret_cast<T *>(a.nsum);
#pragma unroll
                for (int u = 0; u < kTPL; ++u) {
                    if (tid[u] < 0 || grp != 0) continue;
                    T *q = ns + ((int64_t)bb * a.M + tid[u]) * 6;
                    if (a.mode == 1) {
                        q[0] = hx[u];
                        q[1] = lx[u];
                        q[2] = hy[u];
                        q[3] = ly[u];
                        q[4] = hz[u];
                        q[5] = lz[u];
                    } else {
                        hx[u] = q[0];
                        lx[u] = q[1];
                        hy[u] = q[2];
                        ly[u] = q[3];
                        hz[u] = q[4];
                        lz[u] = q[5];
                    }
                }
                if (a.mode == 1) continue;
            }
            // ---- far field: gradient of the leaf's local expansion
            __syncwarp();
            const T *L = le + ((int64_t)leaf * a.B + bb) * a.ldk;
            T fxa[kTPL], fya[kTPL], fza[kTPL];
            if constexpr (kF32) {
                // duplicated pairs, the factor 2 of the m > 0 terms folded in;
                // both observers of the lane in one packed sum
                float2 *Dx2 = reinterpret_cast<float2 *>(Dx), *Dy2 = reinterpret_cast<float2 *>(Dy),
                       *Dz2 = reinterpret_cast<float2 *>(Dz);
                for (int e = lane; e < P2; e += 32) {
                    float vx, vy, vz;
                    grad_coeff<float>(reinterpret_cast<const float *>(L), e, vx, vy, vz);
                    int n = 0;
                    while ((n + 1) * (n + 1) <= e) ++n;
                    const float f2 = e == n * n ? 1.f : 2.f;
                    Dx2[e] = make_float2(f2 * vx, f2 * vx);
                    Dy2[e] = make_float2(f2 * vy, f2 * vy);
                    Dz2[e] = make_float2(f2 * vz, f2 * vz);
                }
                __syncwarp();
                uint64_t FX, FY, FZ;
                l2p_sum2(a.p, Dx2, Dy2, Dz2, pk2(tx[0] * inv_b, tx[1] * inv_b), pk2(ty[0] * inv_b, ty[1] * inv_b),
                         pk2(tz[0] * inv_b, tz[1] * inv_b), FX, FY, FZ);
                float f0, f1;
                up2(FX, f0, f1);
                fxa[0] = f0;
                fxa[1] = f1;
                up2(FY, f0, f1);
                fya[0] = f0;
                fya[1] = f1;
                up2(FZ, f0, f1);
                fza[0] = f0;
                fza[1] = f1;
            } else {
                for (int e = lane; e < P2; e += 32) grad_coeff<T>(L, e, Dx[e], Dy[e], Dz[e]);
                __syncwarp();
#pragma unroll
                for (int u = 0; u < kTPL; ++u)
                    l2p_sum<T>(a.p, Dx, Dy, Dz, tx[u] * inv_b, ty[u] * inv_b, tz[u] * inv_b, fxa[u], fya[u], fza[u]);
            }
#pragma unroll
            for (int u = 0; u < kTPL; ++u) {
                if (tid[u] < 0 || grp != 0) continue;
                const T fx = fxa[u], fy = fya[u], fz = fza[u];
                double gx, gy, gzv;
                if constexpr (kF32) {
                    // near (hi + lo) + far as a compensated FP32 pair (TwoSum), then
                    // the pair's sum and the scale in FP64; the FP32 -> FP64
                    // conversions use integer operations (FP64 runs at 1/64 of
                    // the FP32 rate on this GPU)
                    float sx = hx[u], ex = lx[u], sy = hy[u], ey = ly[u], sz = hz[u], ez = lz[u];
                    two_sum(sx, ex, far_sf * fx);
                    two_sum(sy, ey, far_sf * fy);
                    two_sum(sz, ez, far_sf * fz);
                    gx = (f32_to_f64(sx) + f32_to_f64(ex)) * a.scale;
                    gy = (f32_to_f64(sy) + f32_to_f64(ey)) * a.scale;
                    gzv = (f32_to_f64(sz) + f32_to_f64(ez)) * a.scale;
                } else {
                    // near (hi + lo) + far and the scale in FP64
                    gx = ((double)hx[u] + (double)lx[u] + far_s * (double)fx) * a.scale;
                    gy = ((double)hy[u] + (double)ly[u] + far_s * (double)fy) * a.scale;
                    gzv = ((double)hz[u] + (double)lz[u] + far_s * (double)fz) * a.scale;
                }
                const int64_t j = a.perm[tid[u]];
                if (a.g) {
                    double *o = a.g + ((int64_t)bb * a.M + j) * 3;
                    o[0] = gx;
                    o[1] = gy;
                    o[2] = gzv;
                }
                if (a.gz) a.gz[(int64_t)bb * a.M + j] = gzv;
            }
        }
    }
    // the last warp out leaves the queue at zero for the next launch
    if (lane == 0) {
        __threadfence();
        if (atomicAdd(a.queue + 1, 1ull) == (unsigned long long)gridDim.x * kEvalWarps - 1) {
            a.queue[0] = 0;
            a.queue[1] = 0;
        }
    }
}

// Far field of the split evaluation in FP32 (after the near-field kernel
// has left each observer's compensated near sums in nsum): the L2P gradient
// of the leaf's local expansion, near + far, the scale and the scatter.  One
// warp takes up to 128 observers of one leaf, four per lane as two packed
// pairs that share every coefficient load; the warps take the evaluation
// items (64 observers each) from the queue and skip every second item of a
// leaf, which the warp holding the item before it covers.
constexpr int kFarWarps = 4;
constexpr int kFarTargets = 128;
static_assert(kFarTargets == 2 * kTPL * 32, "two evaluation items per far item");
inline __host__ __device__ int far_slice(int P2) { return (6 * P2 + 7) & ~7; }   // floats per warp

__global__ void __launch_bounds__(kFarWarps * 32, 6) eval_far_kernel(EvalArgs a, const int32_t *__restrict__ leaf_beg) {
    extern __shared__ float fsh[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int P2 = a.p * a.p;
    float2 *Dx2 = reinterpret_cast<float2 *>(fsh + (size_t)warp * far_slice(P2));
    float2 *Dy2 = Dx2 + P2, *Dz2 = Dy2 + P2;
    const float *tloc = reinterpret_cast<const float *>(a.tloc);
    const float *le = reinterpret_cast<const float *>(a.le);
    const float *ns = reinterpret_cast<const float *>(a.nsum);
    const float inv_b = 1.f / (float)a.b;
    const float far_sf = (float)(-1.0 / ((double)a.b * (double)a.b));
    for (;;) {
        int64_t it = 0;
        if (lane == 0) it = (int64_t)atomicAdd(a.queue, 1ull);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= a.n_items) break;
        const int4 item = a.items[it];
        const int leaf = item.x;
        const int lb = leaf_beg[leaf];
        if (((item.y - lb) / (kFarTargets / 2)) & 1) continue;   // covered with the item before it
        const int cnt = min(kFarTargets, leaf_beg[leaf + 1] - item.y);
        int tid[4];
        float tx[4], ty[4], tz[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int r = lane + 32 * u;
            tid[u] = r < cnt ? item.y + r : -1;
            const int64_t i = tid[u] >= 0 ? tid[u] : item.y;
            tx[u] = tloc[3 * i + 0] * inv_b;
            ty[u] = tloc[3 * i + 1] * inv_b;
            tz[u] = tloc[3 * i + 2] * inv_b;
        }
        for (int bb = 0; bb < a.B; ++bb) {
            const float *L = le + ((int64_t)leaf * a.B + bb) * a.ldk;
            __syncwarp();
            // duplicated pairs, the factor 2 of the m > 0 terms folded in
            for (int e = lane; e < P2; e += 32) {
                float vx, vy, vz;
                grad_coeff<float>(L, e, vx, vy, vz);
                int n = 0;
                while ((n + 1) * (n + 1) <= e) ++n;
                const float f2 = e == n * n ? 1.f : 2.f;
                Dx2[e] = make_float2(f2 * vx, f2 * vx);
                Dy2[e] = make_float2(f2 * vy, f2 * vy);
                Dz2[e] = make_float2(f2 * vz, f2 * vz);
            }
            __syncwarp();
            uint64_t G0[3], G1[3] = {0, 0, 0};
            if (cnt > kFarTargets / 2)
                l2p_sum2x2(a.p, Dx2, Dy2, Dz2, pk2(tx[0], tx[1]), pk2(ty[0], ty[1]), pk2(tz[0], tz[1]),
                           pk2(tx[2], tx[3]), pk2(ty[2], ty[3]), pk2(tz[2], tz[3]), G0, G1);
            else   // at most 64 observers: one pair per lane
                l2p_sum2(a.p, Dx2, Dy2, Dz2, pk2(tx[0], tx[1]), pk2(ty[0], ty[1]), pk2(tz[0], tz[1]), G0[0], G0[1],
                         G0[2]);
            float fx[4], fy[4], fz[4];
            up2(G0[0], fx[0], fx[1]);
            up2(G0[1], fy[0], fy[1]);
            up2(G0[2], fz[0], fz[1]);
            up2(G1[0], fx[2], fx[3]);
            up2(G1[1], fy[2], fy[3]);
            up2(G1[2], fz[2], fz[3]);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (tid[u] < 0) continue;
                // near (hi + lo) + far as a compensated FP32 pair, then the pair's
                // sum and the scale in FP64 (integer conversions)
                const float *q = ns + ((int64_t)bb * a.M + tid[u]) * 6;
                float sx = q[0], ex = q[1], sy = q[2], ey = q[3], sz = q[4], ez = q[5];
                two_sum(sx, ex, far_sf * fx[u]);
                two_sum(sy, ey, far_sf * fy[u]);
                two_sum(sz, ez, far_sf * fz[u]);
                const double gx = (f32_to_f64(sx) + f32_to_f64(ex)) * a.scale;
                const double gy = (f32_to_f64(sy) + f32_to_f64(ey)) * a.scale;
                const double gzv = (f32_to_f64(sz) + f32_to_f64(ez)) * a.scale;
                const int64_t j = a.perm[tid[u]];
                if (a.g) {
                    double *o = a.g + ((int64_t)bb * a.M + j) * 3;
                    o[0] = gx;
                    o[1] = gy;
                    o[2] = gzv;
                }
                if (a.gz) a.gz[(int64_t)bb * a.M + j] = gzv;
            }
        }
    }
    // the last warp out leaves the queue at zero for the next launch
    if (lane == 0) {
        __threadfence();
        if (atomicAdd(a.queue + 1, 1ull) == (unsigned long long)gridDim.x * kFarWarps - 1) {
            a.queue[0] = 0;
            a.queue[1] = 0;
        }
    }
}

// Near field + far field of closed-form voxels (SUM-AN in the FMM): one warp
// per work item, two observers per lane.  The densities of the item's 27
// neighbour leaves (a 12^3 voxel block, 4^3-voxel leaves) are staged in the
// warp's shared-memory slice; each observer takes the voxels within
// Chebyshev distance RAD of its own voxel in closed form on their corner
// lattice and the others by the midpoint rule with a uniform cube's l = 4
// term (an_near_block); the far field is the L2P gradient of the leaf's
// local expansion (made from exact voxel moments).
constexpr int kAnNb = 12;                          // voxels per axis of the 27-leaf block
constexpr int kAnBlock = kAnNb * kAnNb * kAnNb;

inline __host__ __device__ int eval_an_slice(int P2) { return (kAnBlock + 3 * P2 + 27 * 2 + 7) & ~7; }

template <class T, int RAD>
__global__ void __launch_bounds__(kEvalWarps * 32) eval_an_kernel(EvalArgs a) {
    extern __shared__ unsigned char shraw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int P2 = a.p * a.p;
    T *blk = reinterpret_cast<T *>(shraw) + (size_t)warp * eval_an_slice(P2);
    T *Dx = blk + kAnBlock, *Dy = Dx + P2, *Dz = Dy + P2;
    int64_t *nbl = reinterpret_cast<int64_t *>(Dz + P2 + ((P2 * 3 + kAnBlock) & 1));
    const T *tloc = reinterpret_cast<const T *>(a.tloc);
    const T *mass = reinterpret_cast<const T *>(a.mass);
    const T *le = reinterpret_cast<const T *>(a.le);
    const T inv_b = T(1) / T(a.b);
    const double far_s = -1.0 / ((double)a.b * (double)a.b);
    for (int64_t it = (int64_t)blockIdx.x * kEvalWarps + warp; it < a.n_items; it += (int64_t)gridDim.x * kEvalWarps) {
        const int4 item = a.items[it];
        const int leaf = item.x;
        const uint64_t key = a.tkey[leaf];
        int64_t lc[3] = {0, 0, 0};
        for (int bit = 0; bit < 21; ++bit) {
            lc[0] |= (int64_t)((key >> (3 * bit)) & 1) << bit;
            lc[1] |= (int64_t)((key >> (3 * bit + 1)) & 1) << bit;
            lc[2] |= (int64_t)((key >> (3 * bit + 2)) & 1) << bit;
        }
        T tx[kTPL], ty[kTPL], tz[kTPL];
        int tid[kTPL];
#pragma unroll
        for (int u = 0; u < kTPL; ++u) {
            const int r = lane + 32 * u;
            tid[u] = r < item.z ? item.y + r : -1;
            const int64_t i = tid[u] >= 0 ? tid[u] : item.y;
            tx[u] = tloc[3 * i + 0] + T(6);   // position in the block (own leaf at [4, 8))
            ty[u] = tloc[3 * i + 1] + T(6);
            tz[u] = tloc[3 * i + 2] + T(6);
        }
        __syncwarp();
        if (lane < 27) {
            const int dx = lane % 3 - 1, dy = (lane / 3) % 3 - 1, dz = lane / 9 - 1;
            const int64_t sx = lc[0] + dx - a.blk.lo[0], sy = lc[1] + dy - a.blk.lo[1], sz = lc[2] + dz - a.blk.lo[2];
            const bool in = sx >= 0 && sy >= 0 && sz >= 0 && sx < a.blk.n[0] && sy < a.blk.n[1] && sz < a.blk.n[2] &&
                            in_source_part(lc[0] + dx, lc[1] + dy, lc[2] + dz, a.L - 2, a.part_lo, a.part_hi);
            nbl[lane] = in ? (sz * a.blk.n[1] + sy) * a.blk.n[0] + sx : -1;
        }
        __syncwarp();
        for (int bb = 0; bb < a.B; ++bb) {
            for (int e = lane; e < kAnBlock; e += 32) {
                const int x = e % kAnNb, y = (e / kAnNb) % kAnNb, z = e / (kAnNb * kAnNb);
                const int64_t sl = nbl[(z >> 2) * 9 + (y >> 2) * 3 + (x >> 2)];
                blk[e] = sl >= 0 ? mass[(sl * a.B + bb) * 64 + ((z & 3) * 4 + (y & 3)) * 4 + (x & 3)] : T(0);
            }
            const T *L = le + ((int64_t)leaf * a.B + bb) * a.ldk;
            for (int e = lane; e < P2; e += 32) grad_coeff<T>(L, e, Dx[e], Dy[e], Dz[e]);
            __syncwarp();
#pragma unroll
            for (int u = 0; u < kTPL; ++u) {
                if (tid[u] < 0) continue;
                T gn[3];
                an_near_block<T>(blk, kAnNb, tx[u], ty[u], tz[u], gn, RAD);
                T fx, fy, fz;
                l2p_sum<T>(a.p, Dx, Dy, Dz, (tx[u] - T(6)) * inv_b, (ty[u] - T(6)) * inv_b, (tz[u] - T(6)) * inv_b,
                           fx, fy, fz);
                const double gx = ((double)gn[0] + far_s * (double)fx) * a.scale;
                const double gy = ((double)gn[1] + far_s * (double)fy) * a.scale;
                const double gzv = ((double)gn[2] + far_s * (double)fz) * a.scale;
                const int64_t j = a.perm[tid[u]];
                if (a.g) {
                    double *o = a.g + ((int64_t)bb * a.M + j) * 3;
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

// Adjoint tables: adj[slot][i*K + o] = fwd[mslot][o*K + i], where mslot is
// the slot of -offset for M2L and the same octant for M2M/L2L.
__global__ void transpose_ops(const double *__restrict__ fwd, double *__restrict__ adjd, float *__restrict__ adjf,
                              int K, int nslots, int negate) {
    const int slot = blockIdx.x;
    int mslot = slot;
    if (negate) {
        const int dx = slot % 7 - 3, dy = (slot / 7) % 7 - 3, dz = slot / 49 - 3;
        mslot = (-dz + 3) * 49 + (-dy + 3) * 7 + (-dx + 3);
    }
    const size_t KK = (size_t)K * K;
    for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
        const int i = e / K, o = e - i * K;
        const double v = fwd[(size_t)mslot * KK + (size_t)o * K + i];
        adjd[(size_t)slot * KK + e] = v;
        adjf[(size_t)slot * KK + e] = (float)v;
    }
    (void)nslots;
}

// ---------------------------------------------------------------- tables
std::mutex g_tab_mu;
std::vector<Tables *> g_tabs;

}  // namespace

gf_status get_tables(int device, int p, cudaStream_t st, const Tables **out) {
    std::lock_guard<std::mutex> lk(g_tab_mu);
    for (Tables *t : g_tabs)
        if (t->device == device && t->p == p) {
            *out = t;
            return GF_OK;
        }
    Tables *T = new Tables();
    T->device = device;
    T->p = p;
    T->K = (p + 1) * (p + 1);
    T->Kp = (T->K + 7) & ~7;
    const size_t KK = (size_t)T->K * T->K;
    // tables live for the life of the process: one set per (device, p)
    GF_CUDA(cudaMalloc(&T->m2l_d, 343 * KK * sizeof(double)));
    GF_CUDA(cudaMalloc(&T->m2l_f, 343 * KK * sizeof(float)));
    GF_CUDA(cudaMalloc(&T->m2m_d, 8 * KK * sizeof(double)));
    GF_CUDA(cudaMalloc(&T->l2l_d, 8 * KK * sizeof(double)));
    GF_CUDA(cudaMalloc(&T->m2m_f, 8 * KK * sizeof(float)));
    GF_CUDA(cudaMalloc(&T->l2l_f, 8 * KK * sizeof(float)));
    GF_CUDA(cudaMemsetAsync(T->m2l_d, 0, 343 * KK * sizeof(double), st));
    GF_CUDA(cudaMemsetAsync(T->m2l_f, 0, 343 * KK * sizeof(float), st));
    const int H = 2 * p;
    const size_t shm = sizeof(double) * (H + 1) * (H + 2);
    build_ops<<<343 + 16, 256, shm, st>>>(p, T->K, host_logfact(), T->m2l_d, T->m2l_f, T->m2m_d, T->m2m_f,
                                          T->l2l_d, T->l2l_f);
    GF_KERNEL_DONE();
    GF_CUDA(cudaMalloc(&T->am2l_d, 343 * KK * sizeof(double)));
    GF_CUDA(cudaMalloc(&T->am2l_f, 343 * KK * sizeof(float)));
    GF_CUDA(cudaMalloc(&T->am2m_d, 8 * KK * sizeof(double)));
    GF_CUDA(cudaMalloc(&T->am2m_f, 8 * KK * sizeof(float)));
    GF_CUDA(cudaMalloc(&T->al2l_d, 8 * KK * sizeof(double)));
    GF_CUDA(cudaMalloc(&T->al2l_f, 8 * KK * sizeof(float)));
    transpose_ops<<<343, 256, 0, st>>>(T->m2l_d, T->am2l_d, T->am2l_f, T->K, 343, 1);
    GF_KERNEL_DONE();
    transpose_ops<<<8, 256, 0, st>>>(T->m2m_d, T->am2m_d, T->am2m_f, T->K, 8, 0);
    GF_KERNEL_DONE();
    transpose_ops<<<8, 256, 0, st>>>(T->l2l_d, T->al2l_d, T->al2l_f, T->K, 8, 0);
    GF_KERNEL_DONE();
    GF_TRY(m2l_prepare_tables(T, st));
    GF_TRY(upload_l2p_coefs());
    GF_CUDA(cudaStreamSynchronize(st));
    g_tabs.push_back(T);
    *out = T;
    return GF_OK;
}

// P2M matrices, one per (device, p, leaf size, quadrature rule), cached for
// the life of the process like the operator tables: plans rebuilt for the
// same rule (a solve loop, a server) do not rebuild them.
struct P2MEntry {
    int device, p, b, nq;
    int exact;             // closed-form voxels: moments integrated exactly
    double xi[kMaxQuad][3], wn[kMaxQuad];
    double *pd;
    float *pf;
    float *tc = nullptr;   // tensor-core image (built on first use)
    float *up_tc = nullptr;   // tensor-core image of the P2M into the parent level
};
std::mutex g_p2m_mu;
std::vector<P2MEntry *> g_p2m;

gf_status get_p2m(gf_plan_s *plan, cudaStream_t st) {
    FmmPlan *F = plan->fmm;
    const QuadRule &q = plan->quad;
    std::lock_guard<std::mutex> lk(g_p2m_mu);
    const int exact = (plan->opt.reserved0 & GF_FLAG_SUM_AN) ? 1 : 0;
    for (P2MEntry *e : g_p2m)
        if (e->device == plan->device && e->p == F->p && e->b == F->b && e->nq == q.nq && e->exact == exact &&
            !memcmp(e->xi, q.xi, sizeof(double) * 3 * q.nq) && !memcmp(e->wn, q.wn, sizeof(double) * q.nq)) {
            F->p2m_d = e->pd;
            F->p2m_f = e->pf;
            return GF_OK;
        }
    P2MEntry *e = new P2MEntry();
    e->device = plan->device;
    e->p = F->p;
    e->b = F->b;
    e->nq = q.nq;
    e->exact = exact;
    memcpy(e->xi, q.xi, sizeof(double) * 3 * q.nq);
    memcpy(e->wn, q.wn, sizeof(double) * q.nq);
    const int b3 = F->b * F->b * F->b, K = F->K;
    if (cudaMalloc(&e->pd, sizeof(double) * b3 * K) != cudaSuccess ||
        cudaMalloc(&e->pf, sizeof(float) * b3 * K) != cudaSuccess) {
        cudaGetLastError();
        delete e;
        set_error("cannot allocate the P2M matrix");
        return GF_ERR_OOM;
    }
    const size_t shm = sizeof(double) * ((F->p + 1) * (F->p + 2) + K);
    if (exact) {
        // degree <= p exactly: ceil((p + 1) / 2) nodes per axis
        build_p2m_exact<<<b3, 128, shm, st>>>(F->p, K, F->b, gauss_legendre((F->p + 2) / 2), e->pd, e->pf);
    } else {
        build_p2m<<<b3, 128, shm, st>>>(F->p, K, F->b, quad_device(plan), e->pd, e->pf);
    }
    GF_KERNEL_DONE();
    GF_CUDA(cudaStreamSynchronize(st));   // other streams may use the cached matrix next
    g_p2m.push_back(e);
    F->p2m_d = e->pd;
    F->p2m_f = e->pf;
    return GF_OK;
}

gf_status get_p2m_tc(gf_plan_s *plan, cudaStream_t st) {
    FmmPlan *F = plan->fmm;
    std::lock_guard<std::mutex> lk(g_p2m_mu);
    for (P2MEntry *e : g_p2m) {
        if (e->pd != F->p2m_d) continue;
        if (!e->tc) {
            const int b3 = F->b * F->b * F->b, npad = F->tab->tc_npad;
            if (cudaMalloc(&e->tc, sizeof(float) * (size_t)(b3 / 16) * 2 * npad * 16) != cudaSuccess) {
                cudaGetLastError();
                e->tc = nullptr;
                set_error("cannot allocate the P2M tensor-core image");
                return GF_ERR_OOM;
            }
            GF_TRY(build_p2m_tc_image(e->pd, F->K, npad, b3, e->tc, st));
            GF_CUDA(cudaStreamSynchronize(st));
        }
        if (!e->up_tc) {
            const int b3 = F->b * F->b * F->b, npad = F->tab->tc_npad;
            double *q = nullptr;
            if (cudaMalloc(&q, sizeof(double) * 8 * (size_t)b3 * F->K) != cudaSuccess ||
                cudaMalloc(&e->up_tc, sizeof(float) * 8 * (size_t)(b3 / 16) * 2 * npad * 16) != cudaSuccess) {
                cudaGetLastError();
                if (q) cudaFree(q);
                e->up_tc = nullptr;
                set_error("cannot allocate the tensor-core image of the P2M into the parent level");
                return GF_ERR_OOM;
            }
            compose_p2m_up<<<dim3(8, b3), 128, 0, st>>>(e->pd, F->tab->m2m_d, F->K, b3, q);
            GF_KERNEL_DONE();
            GF_TRY(build_p2m_up_tc_image(q, F->K, npad, b3, e->up_tc, st));
            GF_CUDA(cudaStreamSynchronize(st));
            cudaFree(q);
        }
        F->p2m_tc = e->tc;
        F->p2m_up_tc = e->up_tc;
        return GF_OK;
    }
    return GF_OK;   // no cached matrix: the P2M stays on the SIMT path
}

gf_status fmm_alloc_workspaces(gf_plan_s *plan, cudaStream_t st) {
    FmmPlan *F = plan->fmm;
    DeviceArena &A = plan->arena;
    const size_t rs = F->mixed ? sizeof(float) : sizeof(double);
    const int K = F->K, B = F->B;
    F->KS = (F->mixed || F->m2l_tc64) ? (K + 31) & ~31 : K;
    for (int l = 2; l <= F->L; ++l) {
        FmmLevel &lv = F->lev[l];
        GF_TRY(A.alloc(&lv.me, (size_t)std::max<int64_t>(lv.ns, 1) * B * F->KS * rs));
        GF_TRY(A.alloc(&lv.le, (size_t)std::max<int64_t>(lv.nt, 1) * B * F->KS * rs));
    }
    const int b3 = F->b * F->b * F->b;
    const int64_t nmass = F->points ? plan->pts.S : F->lev[F->L].ns * b3;
    GF_TRY(A.alloc(&F->mass, (size_t)std::max<int64_t>(nmass, 1) * B * rs));
    if (!F->points) GF_TRY(A.alloc(&F->nsum, (size_t)std::max<int64_t>(plan->M, 1) * B * 6 * rs));
    static bool il_ready[64] = {false};
    static std::mutex il_mu;
    {
        std::lock_guard<std::mutex> lk(il_mu);
        if (!il_ready[plan->device & 63]) {
            static signed char h_il[8][189][3];
            for (int c = 0; c < 8; ++c) il_offsets_host(c, h_il[c]);
            GF_TRY(m2l_upload_offsets(h_il));
            il_ready[plan->device & 63] = true;
        }
    }
    GF_TRY(get_tables(plan->device, F->p, st, &F->tab));
    if (!F->points) GF_TRY(get_p2m(plan, st));
    return m2l_tc_prepare(plan);
}

// ---------------------------------------------------------------- forward
namespace {

// Lattice form of a leaf's sources for the near field: when the rule is a
// tensor product of m nodes per axis (the same nodes on every axis), the
// b^3 nq sources of a leaf sit on an N1^3 lattice, N1 = b m.  Fills the
// plane coordinates and the node map of `a` and returns N1, or 0 when the
// rule is not such a product or N1 is not the size the kernel handles (4).
static int lattice_of(const QuadRule &qr, int b, EvalArgs &a) {
    double nodes[kMaxQuad];
    int m = 0;
    for (int q = 0; q < qr.nq; ++q) {   // distinct x-nodes, ascending
        const double x = qr.xi[q][0];
        bool seen = false;
        for (int t = 0; t < m; ++t) seen = seen || nodes[t] == x;
        if (!seen) nodes[m++] = x;
    }
    std::sort(nodes, nodes + m);
    if (m * m * m != qr.nq || b * m != 4 || b * m > kMaxLat) return 0;
    int seen[kMaxQuad];
    for (int t = 0; t < qr.nq; ++t) seen[t] = 0;
    for (int q = 0; q < qr.nq; ++q) {
        int idx[3];
        for (int d = 0; d < 3; ++d) {
            idx[d] = -1;
            for (int t = 0; t < m; ++t)
                if (qr.xi[q][d] == nodes[t]) idx[d] = t;
            if (idx[d] < 0) return 0;
        }
        const int c = idx[0] + m * (idx[1] + m * idx[2]);
        if (seen[c]++) return 0;
        a.lat_q[c] = q;
    }
    a.lat_m = m;
    const float half_b = 0.5f * (float)b;
    for (int d = 0; d < 3; ++d)
        for (int i = 0; i < b * m; ++i)
            a.lat_c[d][i] = ((float)(i / m) + (float)(0.5 + 0.5 * nodes[i % m])) - half_b;
    return b * m;
}

// Arguments of the evaluation kernels; returns the lattice size N1 of the
// near field's lattice form (0: the generic source list).
template <class T>
int eval_setup(gf_plan_s *plan, int B, double *g, double *gz, EvalArgs &a) {
    const FmmPlan *F = plan->fmm;
    const int L = F->L;
    a.L = L;
    a.part_lo = plan->part_lo;
    a.part_hi = plan->part_hi;
    a.items = F->items;
    a.n_items = F->n_items;
    a.queue = F->eval_queue;
    a.mode = 0;
    a.nsum = F->nsum;
    a.tkey = F->lev[L].tkey;
    a.perm = F->perm;
    a.tloc = sizeof(T) == 8 ? (const void *)F->tloc_d : (const void *)F->tloc_f;
    a.mass = F->mass;
    a.le = F->lev[L].le;
    a.qr = quad_device(plan);
    a.blk = block_of(F->lev[L]);
    a.b = F->b;
    a.nq = F->nq;
    a.B = B;
    a.K = F->K;
    a.ldk = F->KS;
    a.p = F->p;
    a.M = plan->M;
    a.scale = plan->G * F->h;
    a.eps2 = sizeof(T) == 8 ? 1e-18 : 1e-12;
    a.guard_all = 0;
    for (int q = 0; q < plan->quad.nq; ++q)
        for (int d = 0; d < 3; ++d)
            if (fabs(plan->quad.xi[q][d]) >= 1.0) a.guard_all = 1;
    a.g = g;
    a.gz = gz;
    return sizeof(T) == 4 ? lattice_of(plan->quad, F->b, a) : 0;
}

// One evaluation kernel (mode 0: whole, 1: near field, 2: far field) on
// the blocks that fit the device at once; the warps drain the item queue.
template <class T>
gf_status eval_launch(gf_plan_s *plan, EvalArgs a, int n1, int mode, cudaStream_t st) {
    const FmmPlan *F = plan->fmm;
    a.mode = mode;
    const size_t shm = kSrcTable * (sizeof(Vec4<T>) + sizeof(int)) +
                       sizeof(T) * kEvalWarps * eval_slice(F->p * F->p, (int)sizeof(T));
    const unsigned grid = (unsigned)std::min<int64_t>((F->n_items + kEvalWarps - 1) / kEvalWarps, 152 * 64);
    if (sizeof(T) == 4 && mode == 2) {
        const size_t fshm = sizeof(float) * kFarWarps * far_slice(F->p * F->p);
        GF_TRY((ensure_smem(eval_far_kernel, fshm)));
        const unsigned fg = (unsigned)std::min<int64_t>((F->n_items + kFarWarps - 1) / kFarWarps, 152 * 64);
        const unsigned rg = std::min<unsigned>(fg, resident_blocks(eval_far_kernel, kFarWarps * 32, fshm));
        eval_far_kernel<<<rg, kFarWarps * 32, fshm, st>>>(a, F->leaf_beg);
    } else if (sizeof(T) == 4 && n1 == 4) {
        GF_TRY((ensure_smem(eval_kernel<float, 4>, shm)));
        const unsigned rg = std::min<unsigned>(grid, resident_blocks(eval_kernel<float, 4>, kEvalWarps * 32, shm));
        eval_kernel<float, 4><<<rg, kEvalWarps * 32, shm, st>>>(a);
    } else {
        GF_TRY((ensure_smem(eval_kernel<T, 0>, shm)));
        const unsigned rg = std::min<unsigned>(grid, resident_blocks(eval_kernel<T, 0>, kEvalWarps * 32, shm));
        eval_kernel<T, 0><<<rg, kEvalWarps * 32, shm, st>>>(a);
    }
    GF_KERNEL_DONE();
    return GF_OK;
}

template <class T>
gf_status run_forward(gf_plan_s *plan, const void *rho, int rho_dtype, int B, double *g, double *gz,
                      cudaStream_t st) {
    FmmPlan *F = plan->fmm;
    const int K = F->K, L = F->L;
    const int b3 = F->b * F->b * F->b;
    const Tables *tab = F->tab;
    const bool pts = F->points;
    const bool fused = !pts && p2m_fused_ok<T>(F);
    bool up = false;   // level L-1 expansions made straight from the leaf masses
    F->amax_fused = false;
    if (pts) {
        // a0 + a3 for point sources: masses in leaf order, P2M over each leaf's points
        GF_TRY(points_masses<T>(plan, rho, rho_dtype, B, st));
        stage_mark(plan, 1, st);
        GF_TRY(points_p2m<T>(plan, B, st));
    }
    if (fused) {
        // a0 + a3: leaf-blocked densities and P2M (timed as P2M): on the
        // tensor cores for 4^3-voxel leaves in mixed precision, else fused
        stage_mark(plan, 1, st);
        const Block3 lb = block_of(F->lev[F->L]);
        if (sizeof(T) == 4 && F->b == 4 && p2m_tc_ok(plan, B) && lb.n[1] * 4 <= 65535 &&
            lb.n[2] * 4 * B <= 65535) {
            // Leaf-blocked masses (read by the near field and the leaf P2M)
            // of every leaf, or -- when the expansions of level L-1 come
            // straight from the density grid -- of the z-slabs that the leaf
            // level's M2L (and so the near field) reaches.
            up = p2m_up_ok(plan, B);
            const bool from_grid = up && p2m_up_grid_ok(plan, rho, rho_dtype);
            // the kernels that write each level's expansions (the tensor-core
            // P2M and M2M kinds, the FP64 M2M into level 2) also take the
            // largest |input| of the slabs the M2L reads, in place of a pass
            // over those rows before the M2L
            F->amax_fused = F->tc_amax != nullptr;
            if (F->amax_fused) GF_CUDA(cudaMemsetAsync(F->tc_amax, 0, (kMaxLevels + 1) * sizeof(uint32_t), st));
            const FmmLevel &lf = F->lev[L];
            const int64_t z0 = from_grid ? lf.m2l_z0 : 0;
            const int64_t nz = from_grid ? std::max<int64_t>(0, lf.m2l_z1 - lf.m2l_z0 + 1) : lb.n[2];
            GF_TRY((launch_blocking<T, 4>(plan, rho, rho_dtype == GF_DTYPE_F32, B, z0, nz, st)));
            GF_TRY(p2m_run_tc(plan, B, st));   // every leaf, or only the slabs the M2L reads
            if (up) GF_TRY(p2m_up_run_tc(plan, B, from_grid ? (const float *)rho : nullptr, st));
        } else {
            GF_TRY(launch_p2m_fused<T>(plan, rho, rho_dtype == GF_DTYPE_F32, B, st));
        }
    }
    // a0: leaf-blocked densities
    if (!fused && !pts) {
        const FmmLevel &lv = F->lev[L];
        const int64_t total = lv.ns * B * b3;
        const unsigned grid = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 16);
        block_densities<T><<<grid, 256, 0, st>>>(rho, rho_dtype == GF_DTYPE_F32, plan->grid.n[0], plan->grid.n[1],
                                                 plan->grid.n[2], F->voff[0], F->voff[1], F->voff[2],
                                                 block_of(lv), F->b, B, (T *)F->mass, plan->d_status);
        GF_KERNEL_DONE();
    }
    if (!fused && !pts) stage_mark(plan, 1, st);
    // a3: P2M at the leaves
    if (!fused && !pts) {
        const FmmLevel &lv = F->lev[L];
        const unsigned grid = ceil_div(lv.ns, kP2MLeaves);
        const size_t shm = sizeof(T) * kP2MLeaves * B * b3;
        const T *P = sizeof(T) == 8 ? (const T *)F->p2m_d : (const T *)F->p2m_f;
        GF_TRY(ensure_smem(p2m_kernel<T>, shm));
        p2m_kernel<T><<<grid, 128, shm, st>>>((const T *)F->mass, P, lv.ns, b3, B, K, F->KS, (T *)lv.me);
        GF_KERNEL_DONE();
    }
    stage_mark(plan, 2, st);
    // a4: M2M up to level 2.  In mixed precision the translation into the
    // top level (2) is done in FP64 on the per-box kernel; the deeper levels
    // run in the batched kernel in the plan's precision.
    for (int l = up ? L - 2 : L - 1; l >= 2; --l) {
        const FmmLevel &ch = F->lev[l + 1], &pa = F->lev[l];
        if (sizeof(T) == 4 && l <= 2) {
            const int nbc = top_batch_chunk(8, B, K);
            GF_TRY((ensure_smem(m2m_kernel<T, double>, top_smem(8, nbc, K))));
            for (int b0 = 0; b0 < B; b0 += nbc) {
                const int nb = std::min(nbc, B - b0);
                const int64_t slab = pa.sn[0] * pa.sn[1];
                const bool am = F->amax_fused && pa.m2l_z1 >= pa.m2l_z0;
                m2m_kernel<T, double><<<dim3((unsigned)pa.ns, ceil_div(K, 32)), kTopWarps * 32,
                                        top_smem(8, nb, K), st>>>((const T *)ch.me, block_of(ch), (T *)pa.me,
                                                                  block_of(pa), B, b0, nb, K, F->KS, tab->m2m_d,
                                                                  am ? F->tc_amax + l : nullptr,
                                                                  am ? pa.m2l_z0 * slab : 0,
                                                                  am ? (pa.m2l_z1 + 1) * slab : 0);
                GF_KERNEL_DONE();
            }
        } else {
            GF_TRY((translate_run<T, T>(plan, l, 0, B, st)));
        }
    }
    stage_mark(plan, 3, st);
    // a7-a9 set up before the M2L: the near field of the evaluation only
    // reads the leaf masses, so it runs on the plan's second stream beside
    // the M2L and the L2L chain (from the M2L's launch on); the far field
    // (L2P, near + far in FP64, scatter) joins it once the L2L is done.
    // With stage timing on, both halves run in line on the forward's stream.
    const bool eval_on = !pts && F->n_items > 0;
    const bool an = (plan->opt.reserved0 & GF_FLAG_SUM_AN) != 0;
    EvalArgs ea;
    int n1 = 0;
    if (eval_on) n1 = eval_setup<T>(plan, B, g, gz, ea);
    const bool beside = eval_on && !an && plan->side && !plan->timing;
    // a5/a6: M2L at every level (each overwrites its level's LE), then the
    // L2L chain from level 3 down, which adds each finished parent LE.
    GF_TRY(m2l_run<T>(plan, B, false, st, beside ? plan->ev_fork : nullptr));   // marks the input split's end (4)
    if (beside) {
        GF_CUDA(cudaStreamWaitEvent(plan->side, plan->ev_fork, 0));
        GF_TRY(eval_launch<T>(plan, ea, n1, 1, plan->side));
        GF_CUDA(cudaEventRecord(plan->ev_join, plan->side));
    }
    stage_mark(plan, 5, st);
    for (int l = 3; l <= L; ++l) {
        const FmmLevel &lv = F->lev[l];
        if (lv.nt == 0) continue;
        const FmmLevel &pa = F->lev[l - 1];
        if (sizeof(T) == 4 && l - 1 <= 2) {
            const int nbc = top_batch_chunk(1, B, K);
            GF_TRY((ensure_smem(l2l_kernel<T, double>, top_smem(1, nbc, K))));
            for (int b0 = 0; b0 < B; b0 += nbc) {
                const int nb = std::min(nbc, B - b0);
                l2l_kernel<T, double><<<dim3((unsigned)lv.nt, ceil_div(K, 32)), kTopWarps * 32,
                                        top_smem(1, nb, K), st>>>((const T *)pa.le, lv.tkey, lv.tparent,
                                                                  (T *)lv.le, B, b0, nb, K, F->KS, tab->l2l_d);
                GF_KERNEL_DONE();
            }
        } else {
            GF_TRY((translate_run<T, T>(plan, l, 1, B, st)));
        }
    }
    stage_mark(plan, 6, st);
    // a7-a9: near field + L2P + combine + scatter
    if (pts) {
        GF_TRY(points_eval<T>(plan, B, g, gz, st));
    } else if (eval_on && an) {
        // closed-form voxels: radius 2 in FP32, 4 in FP64 (the closed form
        // cancels like (d/h)^3, so the precision sets how far it is used;
        // beyond it the corrected midpoint rule errs like (h/d)^6)
        const unsigned grid = (unsigned)std::min<int64_t>((F->n_items + kEvalWarps - 1) / kEvalWarps, 152 * 64);
        const size_t shan = sizeof(T) * kEvalWarps * eval_an_slice(F->p * F->p) + 64;
        if (sizeof(T) == 4) {
            GF_TRY((ensure_smem(eval_an_kernel<T, 2>, shan)));
            eval_an_kernel<T, 2><<<grid, kEvalWarps * 32, shan, st>>>(ea);
        } else {
            GF_TRY((ensure_smem(eval_an_kernel<T, 4>, shan)));
            eval_an_kernel<T, 4><<<grid, kEvalWarps * 32, shan, st>>>(ea);
        }
        GF_KERNEL_DONE();
    } else if (eval_on) {
        if (beside)
            GF_CUDA(cudaStreamWaitEvent(st, plan->ev_join, 0));
        else
            GF_TRY(eval_launch<T>(plan, ea, n1, 1, st));
        GF_TRY(eval_launch<T>(plan, ea, n1, 2, st));
    }
    stage_mark(plan, 7, st);
    return GF_OK;
}

}  // namespace

gf_status fmm_forward(gf_plan_s *plan, const void *rho, int rho_dtype, int B, double *g, double *gz,
                      cudaStream_t st) {
    if (plan->M == 0) return GF_OK;
    if (plan->fmm->mixed) return run_forward<float>(plan, rho, rho_dtype, B, g, gz, st);
    return run_forward<double>(plan, rho, rho_dtype, B, g, gz, st);
}


}  // namespace gf
