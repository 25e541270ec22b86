// gf_direct.cu -- direct summation (Sec. 2.1, SUM-G1/SUM-G2) of Eq. 1 in
// its N-body form (Eq. 7): every observer against every voxel quadrature
// point.  Used as the exact path ("direct mode") and its transpose.
//
// Layout: one thread per output (observer, or voxel for the transpose); a
// block stages a tile of 256 inputs in shared memory and every thread of the
// block sweeps it, so each staged input is read from HBM once per block.
// FP64 path: source coordinates are formed with explicitly rounded
// operations in the same order as the plain definition, so coincidence
// decisions (r == x) are exact.  Mixed path: coordinates are carried as
// integer voxel index plus an FP32 fraction, so the separation of near pairs
// is formed to FP32 relative accuracy whatever the size of the domain.
#include <cuda.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "gf_internal.cuh"

namespace gf {
namespace {

constexpr int kTile = 256;

struct GridArgs {
    int64_t nx, ny, nz, nvox;
    double ox, oy, oz, hx, hy, hz, vol;
};

GridArgs grid_args(const gf_plan_s *p) {
    GridArgs a;
    a.nx = p->grid.n[0];
    a.ny = p->grid.n[1];
    a.nz = p->grid.n[2];
    a.nvox = a.nx * a.ny * a.nz;
    a.ox = p->grid.origin[0];
    a.oy = p->grid.origin[1];
    a.oz = p->grid.origin[2];
    a.hx = p->grid.h[0];
    a.hy = p->grid.h[1];
    a.hz = p->grid.h[2];
    a.vol = a.hx * a.hy * a.hz;
    return a;
}

__device__ __forceinline__ double load_rho(const void *rho, int f32, int64_t idx) {
    return f32 ? (double)__ldg(reinterpret_cast<const float *>(rho) + idx)
               : __ldg(reinterpret_cast<const double *>(rho) + idx);
}

// Neumaier step on (s, c) with addend x.
__device__ __forceinline__ void neumaier(double &s, double &c, double x) {
    double t = s + x;
    c += (fabs(s) >= fabs(x)) ? ((s - t) + x) : ((x - t) + s);
    s = t;
}

// Position of quadrature node q of voxel (i,j,k) in FP64, rounded exactly as
// centre = origin + (i + 1/2) h, node = centre + (h/2) xi.
__device__ __forceinline__ double node_coord(double o, double h, int64_t i, double xi) {
    double c = __dadd_rn(o, __dmul_rn((double)i + 0.5, h));
    return __dadd_rn(c, __dmul_rn(__dmul_rn(0.5, h), xi));
}

__global__ void __launch_bounds__(kTile)
direct_fwd_f64(const double *__restrict__ obs, int64_t M, const void *__restrict__ rho,
               int rho_f32, GridArgs ga, const QuadRule *__restrict__ qr, double G,
               double *__restrict__ g, double *__restrict__ gz, int *__restrict__ status) {
    __shared__ double sx[kTile], sy[kTile], sz[kTile], sm[kTile];
    const int b = blockIdx.y;
    const int64_t j = (int64_t)blockIdx.x * kTile + threadIdx.x;
    const bool active = j < M;
    const double rx = active ? obs[3 * j + 0] : 0.0;
    const double ry = active ? obs[3 * j + 1] : 0.0;
    const double rz = active ? obs[3 * j + 2] : 0.0;
    const int nq = qr->nq;
    const int64_t N = ga.nvox * nq;
    const void *rho_b = rho_f32 ? (const void *)((const float *)rho + b * ga.nvox)
                                : (const void *)((const double *)rho + b * ga.nvox);
    double s0 = 0, c0 = 0, s1 = 0, c1 = 0, s2 = 0, c2 = 0;
    bool bad = false;   // a non-finite density (reported through status[0])
    for (int64_t t0 = 0; t0 < N; t0 += kTile) {
        const int64_t s = t0 + threadIdx.x;
        __syncthreads();
        if (s < N) {
            const int64_t v = s / nq;
            const int q = (int)(s - v * nq);
            const int64_t i = v % ga.nx, jj = (v / ga.nx) % ga.ny, k = v / (ga.nx * ga.ny);
            sx[threadIdx.x] = node_coord(ga.ox, ga.hx, i, qr->xi[q][0]);
            sy[threadIdx.x] = node_coord(ga.oy, ga.hy, jj, qr->xi[q][1]);
            sz[threadIdx.x] = node_coord(ga.oz, ga.hz, k, qr->xi[q][2]);
            const double rv = load_rho(rho_b, rho_f32, v);
            bad |= !isfinite(rv);
            sm[threadIdx.x] = __dmul_rn(__dmul_rn(rv, ga.vol), qr->wn[q]);
        } else {
            sx[threadIdx.x] = 0.0;
            sy[threadIdx.x] = 0.0;
            sz[threadIdx.x] = 0.0;
            sm[threadIdx.x] = 0.0;
        }
        __syncthreads();
        const int cnt = (N - t0) < kTile ? (int)(N - t0) : kTile;
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
        neumaier(s0, c0, px);
        neumaier(s1, c1, py);
        neumaier(s2, c2, pz);
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

// Mixed precision: positions in voxel units split into an integer part
// (held exactly in FP32, |i| < 2^24) and a fraction; the pair separation is
// (ri - si) + (rf - sf), exact integer difference plus one rounding.
__global__ void __launch_bounds__(kTile)
direct_fwd_mixed(const float *__restrict__ obs_i, const float *__restrict__ obs_f, int64_t M,
                 const void *__restrict__ rho, int rho_f32, GridArgs ga,
                 const QuadRule *__restrict__ qr, double G, double *__restrict__ g,
                 double *__restrict__ gz, int *__restrict__ status) {
    __shared__ float si[kTile][3], sf[kTile][3], sm[kTile];
    const int b = blockIdx.y;
    const int64_t j = (int64_t)blockIdx.x * kTile + threadIdx.x;
    const bool active = j < M;
    float ri[3] = {0.f, 0.f, 0.f}, rf[3] = {0.f, 0.f, 0.f};
    if (active) {
        for (int a = 0; a < 3; ++a) {
            ri[a] = obs_i[3 * j + a];
            rf[a] = obs_f[3 * j + a];
        }
    }
    const float hx = (float)ga.hx, hy = (float)ga.hy, hz = (float)ga.hz;
    const int nq = qr->nq;
    const int64_t N = ga.nvox * nq;
    const void *rho_b = rho_f32 ? (const void *)((const float *)rho + b * ga.nvox)
                                : (const void *)((const double *)rho + b * ga.nvox);
    double ax = 0, ay = 0, az = 0;
    bool bad = false;   // a non-finite density (reported through status[0])
    for (int64_t t0 = 0; t0 < N; t0 += kTile) {
        const int64_t s = t0 + threadIdx.x;
        __syncthreads();
        if (s < N) {
            const int64_t v = s / nq;
            const int q = (int)(s - v * nq);
            si[threadIdx.x][0] = (float)(v % ga.nx);
            si[threadIdx.x][1] = (float)((v / ga.nx) % ga.ny);
            si[threadIdx.x][2] = (float)(v / (ga.nx * ga.ny));
            sf[threadIdx.x][0] = qr->offf[q][0];
            sf[threadIdx.x][1] = qr->offf[q][1];
            sf[threadIdx.x][2] = qr->offf[q][2];
            const double rv = load_rho(rho_b, rho_f32, v);
            bad |= !isfinite(rv);
            sm[threadIdx.x] = (float)(rv * ga.vol * qr->wn[q]);
        } else {
            si[threadIdx.x][0] = si[threadIdx.x][1] = si[threadIdx.x][2] = 0.f;
            sf[threadIdx.x][0] = sf[threadIdx.x][1] = sf[threadIdx.x][2] = 0.f;
            sm[threadIdx.x] = 0.f;
        }
        __syncthreads();
        const int cnt = (N - t0) < kTile ? (int)(N - t0) : kTile;
        float px = 0.f, py = 0.f, pz = 0.f;
#pragma unroll 4
        for (int u = 0; u < cnt; ++u) {
            const float dx = hx * ((ri[0] - si[u][0]) + (rf[0] - sf[u][0]));
            const float dy = hy * ((ri[1] - si[u][1]) + (rf[1] - sf[u][1]));
            const float dz = hz * ((ri[2] - si[u][2]) + (rf[2] - sf[u][2]));
            const float r2 = dx * dx + dy * dy + dz * dz;
            const float rinv = rsqrtf(r2);
            const float k3 = (r2 > 0.f) ? sm[u] * (rinv * rinv * rinv) : 0.f;
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
        const double vx = G * ax, vy = G * ay, vz = G * az;
        if (g) {
            double *o = g + ((int64_t)b * M + j) * 3;
            o[0] = vx;
            o[1] = vy;
            o[2] = vz;
        }
        if (gz) gz[(int64_t)b * M + j] = vz;
    }
}

// Transpose: one thread per voxel, observers (with their weights) staged in
// shared memory.  grad_v = G V sum_q wn_q sum_j r_j . (x'_j - x_vq)/|.|^3.
__global__ void __launch_bounds__(kTile)
direct_adj_f64(const double *__restrict__ obs, int64_t M, const double *__restrict__ r,
               int ncomp, GridArgs ga, const QuadRule *__restrict__ qr, double G,
               double *__restrict__ grad) {
    __shared__ double ox[kTile], oy[kTile], oz[kTile], w0[kTile], w1[kTile], w2[kTile];
    const int b = blockIdx.y;
    const int64_t v = (int64_t)blockIdx.x * kTile + threadIdx.x;
    const bool active = v < ga.nvox;
    const int64_t i = active ? v % ga.nx : 0, jj = active ? (v / ga.nx) % ga.ny : 0,
                  k = active ? v / (ga.nx * ga.ny) : 0;
    const int nq = qr->nq;
    const double *rb = r + (int64_t)b * M * ncomp;
    double s = 0, c = 0;
    for (int64_t t0 = 0; t0 < M; t0 += kTile) {
        const int64_t j = t0 + threadIdx.x;
        __syncthreads();
        if (j < M) {
            ox[threadIdx.x] = obs[3 * j + 0];
            oy[threadIdx.x] = obs[3 * j + 1];
            oz[threadIdx.x] = obs[3 * j + 2];
            if (ncomp == 1) {
                w0[threadIdx.x] = 0.0;
                w1[threadIdx.x] = 0.0;
                w2[threadIdx.x] = rb[j];
            } else {
                w0[threadIdx.x] = rb[3 * j + 0];
                w1[threadIdx.x] = rb[3 * j + 1];
                w2[threadIdx.x] = rb[3 * j + 2];
            }
        } else {
            ox[threadIdx.x] = oy[threadIdx.x] = oz[threadIdx.x] = 0.0;
            w0[threadIdx.x] = w1[threadIdx.x] = w2[threadIdx.x] = 0.0;
        }
        __syncthreads();
        const int cnt = (M - t0) < kTile ? (int)(M - t0) : kTile;
        double part = 0.0;
        for (int q = 0; q < nq; ++q) {
            const double x = node_coord(ga.ox, ga.hx, i, qr->xi[q][0]);
            const double y = node_coord(ga.oy, ga.hy, jj, qr->xi[q][1]);
            const double z = node_coord(ga.oz, ga.hz, k, qr->xi[q][2]);
            double pq = 0.0;
            for (int u = 0; u < cnt; ++u) {
                const double dx = ox[u] - x, dy = oy[u] - y, dz = oz[u] - z;
                const double r2 = dx * dx + dy * dy + dz * dz;
                const double ri = rsqrt(r2);
                const double k3 = (r2 > 0.0) ? ri * ri * ri : 0.0;
                pq = fma(k3, w0[u] * dx + w1[u] * dy + w2[u] * dz, pq);
            }
            part = fma(qr->wn[q], pq, part);
        }
        neumaier(s, c, part);
    }
    if (active) grad[(int64_t)b * ga.nvox + v] = G * ga.vol * (s + c);
}

__global__ void split_voxel_coords(const double *__restrict__ obs, int64_t M, GridArgs ga,
                                   float *__restrict__ oi, float *__restrict__ of) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    const double o[3] = {ga.ox, ga.oy, ga.oz};
    const double h[3] = {ga.hx, ga.hy, ga.hz};
    for (int a = 0; a < 3; ++a) {
        const double u = (obs[3 * j + a] - o[a]) / h[a];
        const double fl = floor(u);
        oi[3 * j + a] = (float)fl;
        of[3 * j + a] = (float)(u - fl);
    }
}

}  // namespace

gf_status direct_prepare(gf_plan_s *plan, const double *obs_dev, cudaStream_t st) {
    const int64_t M = plan->M;
    GF_TRY(plan->arena.alloc_n(&plan->d_obs, (size_t)std::max<int64_t>(M, 1) * 3));
    if (M > 0)
        GF_CUDA(cudaMemcpyAsync(plan->d_obs, obs_dev, sizeof(double) * 3 * M,
                                cudaMemcpyDeviceToDevice, st));
    if (plan->opt.precision == GF_PREC_MIXED) {
        float *oi, *of;
        GF_TRY(plan->arena.alloc_n(&oi, (size_t)std::max<int64_t>(M, 1) * 3));
        GF_TRY(plan->arena.alloc_n(&of, (size_t)std::max<int64_t>(M, 1) * 3));
        plan->d_obs_ivox = nullptr;
        plan->d_obs_fvox = of;
        // integer parts are stored as exact FP32 integers
        plan->d_obs_ivox = reinterpret_cast<int32_t *>(oi);
        if (M > 0) {
            split_voxel_coords<<<ceil_div(M, 256), 256, 0, st>>>(obs_dev, M, grid_args(plan), oi, of);
            GF_KERNEL_DONE();
        }
    }
    return GF_OK;
}

gf_status direct_forward(gf_plan_s *plan, const void *rho, int rho_dtype, int B, double *g,
                         double *gz, cudaStream_t st) {
    const int64_t M = plan->M;
    if (M == 0) return GF_OK;
    const GridArgs ga = grid_args(plan);
    const dim3 grid(ceil_div(M, kTile), B);
    const int f32 = rho_dtype == GF_DTYPE_F32;
    if (plan->opt.precision == GF_PREC_FP64) {
        direct_fwd_f64<<<grid, kTile, 0, st>>>(plan->d_obs, M, rho, f32, ga, quad_device(plan),
                                               plan->G, g, gz, plan->d_status);
    } else {
        direct_fwd_mixed<<<grid, kTile, 0, st>>>(reinterpret_cast<const float *>(plan->d_obs_ivox),
                                                 plan->d_obs_fvox, M, rho, f32, ga,
                                                 quad_device(plan), plan->G, g, gz, plan->d_status);
    }
    GF_KERNEL_DONE();
    return GF_OK;
}

gf_status direct_adjoint(gf_plan_s *plan, const double *r, int ncomp, int B, double *grad,
                         cudaStream_t st) {
    const GridArgs ga = grid_args(plan);
    const dim3 grid(ceil_div(ga.nvox, kTile), B);
    direct_adj_f64<<<grid, kTile, 0, st>>>(plan->d_obs, plan->M, r, ncomp, ga, quad_device(plan),
                                           plan->G, grad);
    GF_KERNEL_DONE();
    return GF_OK;
}

}  // namespace gf

// ---------------------------------------------------------------------------
// Allocation-free direct forward (gf_direct_forward_static in gf.h).
//
// Some callers cannot allocate device memory when they need a forward
// solve: code that runs inside another framework's allocator callback and
// must not re-enter it, processes whose device memory is entirely reserved
// by a caching pool they do not own, and services that forbid any
// allocation after start-up so that their memory footprint stays fixed.
// This variant of the mixed-precision direct kernel needs no plan: its only
// scratch -- the normalised quadrature rule and the observers' voxel
// coordinates split into integer and fractional parts -- lives in one
// file-scope device array of fixed size, which every GPU that loads this
// library holds until the process exits.
namespace gf {
namespace {

constexpr int64_t kStaticMaxObs = 65536;
constexpr size_t kStaticQuadBytes = (sizeof(QuadRule) + 255) & ~size_t(255);
constexpr size_t kStaticCoordBytes = sizeof(float) * 3 * kStaticMaxObs;
constexpr size_t kStaticBytes = kStaticQuadBytes + 2 * kStaticCoordBytes;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

std::mutex g_static_mu;
void *g_static_addr[256] = {};
CUcontext g_static_ctx[256] = {};

// Device address of the scratch array on the current device.  The host
// symbol is only a stand-in, so the address is looked up once per device
// (with that device current) and cached with the context it belongs to; a
// new context on the device (after cudaDeviceReset, say) looks it up again.
gf_status static_scratch_address(void **out) {
    int dev = 0;
    GF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) {
        set_error("device ordinal %d out of range", dev);
        return GF_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_static_mu);
    // the driver's cuCtxGetCurrent, found through the runtime (the library
    // does not link the driver library)
    typedef CUresult (*CtxGetCurrent)(CUcontext *);
    static CtxGetCurrent ctx_get = nullptr;
    if (!ctx_get) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn) {
            set_error("cannot find the driver's cuCtxGetCurrent");
            return GF_ERR_CUDA;
        }
        ctx_get = reinterpret_cast<CtxGetCurrent>(fn);
    }
    CUcontext ctx = nullptr;
    if (ctx_get(&ctx) != CUDA_SUCCESS) ctx = nullptr;   // none yet: the lookup makes one
    if (!ctx || !g_static_addr[dev] || g_static_ctx[dev] != ctx) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            set_error("cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
            return GF_ERR_CUDA;
        }
        if (ctx_get(&ctx) != CUDA_SUCCESS) ctx = nullptr;
        g_static_addr[dev] = p;
        g_static_ctx[dev] = ctx;
    }
    *out = g_static_addr[dev];
    return GF_OK;
}

// Writes the quadrature rule, passed by value, into the scratch array.
__global__ void store_quad_rule(QuadRule qr, QuadRule *__restrict__ dst) {
    const uint32_t *src = reinterpret_cast<const uint32_t *>(&qr);
    uint32_t *out = reinterpret_cast<uint32_t *>(dst);
    for (size_t i = threadIdx.x; i < sizeof(QuadRule) / 4; i += blockDim.x) out[i] = src[i];
}

}  // namespace
}  // namespace gf

extern "C" gf_status gf_direct_forward_static(const gf_grid *grid, const gf_quad *quad, const double *obs_dev,
                                              int64_t M, const void *rho_dev, int32_t rho_dtype, int32_t B,
                                              double G, double *g_dev, double *gz_dev, void *stream) {
    using namespace gf;
    if (!grid || !quad) {
        set_error("grid and quad must be non-NULL");
        return GF_ERR_INVALID_ARG;
    }
    if (M < 0 || M > kStaticMaxObs) {
        set_error("gf_direct_forward_static takes at most %lld observers (M = %lld); use a plan instead",
                  (long long)kStaticMaxObs, (long long)M);
        return GF_ERR_INVALID_ARG;
    }
    for (int a = 0; a < 3; ++a) {
        if (grid->n[a] < 1 || grid->n[a] > kMaxAxis || !(grid->h[a] > 0.0) || !isfinite(grid->h[a]) ||
            !isfinite(grid->origin[a])) {
            set_error("grid axis %d: need 1 <= n <= 2^22, finite h > 0 and finite origin", a);
            return GF_ERR_INVALID_ARG;
        }
    }
    if (grid->n[0] * grid->n[1] > kMaxVoxels / grid->n[2]) {
        set_error("grid exceeds 2^40 voxels");
        return GF_ERR_INVALID_ARG;
    }
    if (quad->nq < 1 || quad->nq > kMaxQuad || !quad->xi || !quad->w) {
        set_error("quad.nq = %d must be in [1, %d] with non-NULL xi and w", quad->nq, kMaxQuad);
        return GF_ERR_INVALID_ARG;
    }
    if (rho_dtype != GF_DTYPE_F64 && rho_dtype != GF_DTYPE_F32) {
        set_error("rho_dtype = %d is neither GF_DTYPE_F64 nor GF_DTYPE_F32", rho_dtype);
        return GF_ERR_INVALID_ARG;
    }
    if (B < 1 || B > 64 || !(G >= 0.0) || !isfinite(G)) {
        set_error("need 1 <= B <= 64 and a finite G >= 0 (0 selects 6.67428e-11)");
        return GF_ERR_INVALID_ARG;
    }
    if ((M > 0 && (!obs_dev || !rho_dev)) || (!g_dev && !gz_dev)) {
        set_error("obs_dev and rho_dev must be non-NULL and at least one of g_dev, gz_dev given");
        return GF_ERR_INVALID_ARG;
    }
    QuadRule qr;
    memset(&qr, 0, sizeof(qr));
    qr.nq = quad->nq;
    double wsum = 0.0;
    for (int q = 0; q < quad->nq; ++q) {
        if (!(quad->w[q] > 0.0) || !isfinite(quad->w[q])) {
            set_error("quad.w[%d] must be finite and positive", q);
            return GF_ERR_INVALID_ARG;
        }
        wsum += quad->w[q];
    }
    for (int q = 0; q < quad->nq; ++q) {
        qr.wn[q] = quad->w[q] / wsum;
        qr.wnf[q] = (float)qr.wn[q];
        for (int a = 0; a < 3; ++a) {
            const double x = quad->xi[3 * q + a];
            if (!(fabs(x) <= 1.0)) {
                set_error("quad.xi[%d][%d] must lie in [-1, 1]", q, a);
                return GF_ERR_INVALID_ARG;
            }
            qr.xi[q][a] = x;
            qr.offf[q][a] = (float)(0.5 + 0.5 * x);
        }
    }
    if (M == 0) return GF_OK;
    void *base = nullptr;
    GF_TRY(static_scratch_address(&base));
    unsigned char *scr = reinterpret_cast<unsigned char *>(base);
    QuadRule *d_qr = reinterpret_cast<QuadRule *>(scr);
    float *oi = reinterpret_cast<float *>(scr + kStaticQuadBytes);
    float *of = reinterpret_cast<float *>(scr + kStaticQuadBytes + kStaticCoordBytes);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    GridArgs ga;
    ga.nx = grid->n[0];
    ga.ny = grid->n[1];
    ga.nz = grid->n[2];
    ga.nvox = ga.nx * ga.ny * ga.nz;
    ga.ox = grid->origin[0];
    ga.oy = grid->origin[1];
    ga.oz = grid->origin[2];
    ga.hx = grid->h[0];
    ga.hy = grid->h[1];
    ga.hz = grid->h[2];
    ga.vol = ga.hx * ga.hy * ga.hz;
    // every byte the kernels read is rewritten here, so nothing left by an
    // earlier call is used and nothing needs clearing; the rule travels as a
    // kernel argument (no host memory is read once this call returns)
    store_quad_rule<<<1, 256, 0, st>>>(qr, d_qr);
    GF_KERNEL_DONE();
    split_voxel_coords<<<ceil_div(M, 256), 256, 0, st>>>(obs_dev, M, ga, oi, of);
    GF_KERNEL_DONE();
    direct_fwd_mixed<<<dim3(ceil_div(M, kTile), B), kTile, 0, st>>>(oi, of, M, rho_dev,
                                                                     rho_dtype == GF_DTYPE_F32, ga, d_qr,
                                                                     G > 0.0 ? G : 6.67428e-11, g_dev, gz_dev,
                                                                     nullptr);
    GF_KERNEL_DONE();
    return GF_OK;
}
