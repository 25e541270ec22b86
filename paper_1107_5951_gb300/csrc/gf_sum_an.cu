// gf_sum_an.cu -- SUM-AN (Sec. 2.1): direct summation in which every
// constant-density voxel is integrated in closed form instead of being
// sampled by a quadrature rule.  FP64, direct mode, and its transpose.
//
// The field of voxel v (density rho_v) at r is G rho_v sum_c s(v, c) F(c - r)
// over its eight corners c, F the corner function of gf_sum_an.cuh and
// s(v, c) = +1 at the corners reached from the voxel's lower corner through
// an odd number of upper limits, -1 at the others.  A lattice corner is
// shared by up to eight voxels, so the sum over voxels is regrouped onto the
// corner lattice,
//
//   g(r) = G sum_c D_c F(c - r),   D_c = sum_{v sharing c} s(v, c) rho_v,
//
// one corner-function evaluation per lattice point instead of eight per
// voxel; D_c vanishes inside regions of constant density, and those corners
// are skipped.  The transpose is regrouped the same way: per corner
// E_c = sum_j r_j . F(c - x'_j), then grad_v = G sum_{c of v} s(v, c) E_c.
//
// Layout: corners are numbered I + (nx + 1) (J + (ny + 1) K) and sit at
// origin + (I, J, K) h, rounded as origin + I h.  One thread per observer
// (forward) or per corner (transpose); a block stages 128 corner weights
// (forward) or observers (transpose) in shared memory, and the per-tile
// partial sums are merged into Neumaier-compensated totals.
#include <math.h>

#include <algorithm>

#include "gf_internal.cuh"
#include "gf_sum_an.cuh"

namespace gf {
namespace {

constexpr int kAnTile = 128;

struct AnGrid {
    int64_t nx, ny, nz, nvox;
    int64_t ncx, ncy, ncz, nc;   // corner lattice
    double ox, oy, oz, hx, hy, hz;
};

AnGrid an_grid(const gf_plan_s *p) {
    AnGrid a;
    a.nx = p->grid.n[0];
    a.ny = p->grid.n[1];
    a.nz = p->grid.n[2];
    a.nvox = a.nx * a.ny * a.nz;
    a.ncx = a.nx + 1;
    a.ncy = a.ny + 1;
    a.ncz = a.nz + 1;
    a.nc = a.ncx * a.ncy * a.ncz;
    a.ox = p->grid.origin[0];
    a.oy = p->grid.origin[1];
    a.oz = p->grid.origin[2];
    a.hx = p->grid.h[0];
    a.hy = p->grid.h[1];
    a.hz = p->grid.h[2];
    return a;
}

__device__ __forceinline__ double an_rho(const void *rho, int f32, int64_t idx) {
    return f32 ? (double)__ldg(reinterpret_cast<const float *>(rho) + idx)
               : __ldg(reinterpret_cast<const double *>(rho) + idx);
}

__device__ __forceinline__ void an_neumaier(double &s, double &c, double x) {
    const double t = s + x;
    c += (fabs(s) >= fabs(x)) ? ((s - t) + x) : ((x - t) + s);
    s = t;
}

// Coordinate of lattice plane I: origin + I h, rounded once each.
__device__ __forceinline__ double an_plane(double o, double h, int64_t I) {
    return __dadd_rn(o, __dmul_rn((double)I, h));
}

// D[b][c]: signed sum of the densities of the voxels sharing corner c.
// Flags a non-finite density in status[0].
__global__ void an_corner_weights(const void *__restrict__ rho, int rho_f32, AnGrid g,
                                  double *__restrict__ D, int *__restrict__ status) {
    const int b = blockIdx.y;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.nc) return;
    const int64_t I = c % g.ncx, J = (c / g.ncx) % g.ncy, K = c / (g.ncx * g.ncy);
    double s = 0.0;
    bool bad = false;
    for (int e = 0; e < 2; ++e)
        for (int f = 0; f < 2; ++f)
            for (int a = 0; a < 2; ++a) {
                const int64_t i = I - a, j = J - f, k = K - e;
                if (i < 0 || j < 0 || k < 0 || i >= g.nx || j >= g.ny || k >= g.nz) continue;
                const double r = an_rho(rho, rho_f32, (int64_t)b * g.nvox + (k * g.ny + j) * g.nx + i);
                bad |= !isfinite(r);
                s += ((a + f + e) & 1) ? r : -r;
            }
    if (bad) atomicOr(status, 1);
    D[(int64_t)b * g.nc + c] = s;
}

// g(r_j) = G sum_c D_c F(c - r_j): one thread per observer, corner weights
// staged 128 at a time.
__global__ void __launch_bounds__(kAnTile)
an_forward(const double *__restrict__ obs, int64_t M, const double *__restrict__ D, AnGrid g, double G,
           double *__restrict__ gout, double *__restrict__ gz) {
    __shared__ double sd[kAnTile];
    const int b = blockIdx.y;
    const int64_t j = (int64_t)blockIdx.x * kAnTile + threadIdx.x;
    const bool active = j < M;
    const double rx = active ? obs[3 * j + 0] : 0.0;
    const double ry = active ? obs[3 * j + 1] : 0.0;
    const double rz = active ? obs[3 * j + 2] : 0.0;
    const double *Db = D + (int64_t)b * g.nc;
    double s0 = 0, c0 = 0, s1 = 0, c1 = 0, s2 = 0, c2 = 0;
    for (int64_t t0 = 0; t0 < g.nc; t0 += kAnTile) {
        const int64_t c = t0 + threadIdx.x;
        __syncthreads();
        sd[threadIdx.x] = c < g.nc ? Db[c] : 0.0;
        __syncthreads();
        const int cnt = (g.nc - t0) < kAnTile ? (int)(g.nc - t0) : kAnTile;
        int64_t I = t0 % g.ncx, J = (t0 / g.ncx) % g.ncy, K = t0 / (g.ncx * g.ncy);
        double px = 0, py = 0, pz = 0;
        for (int u = 0; u < cnt; ++u) {
            const double d = sd[u];   // the same for every thread: a uniform branch
            if (d != 0.0) {
                double fx, fy, fz;
                an_corner<double>(an_plane(g.ox, g.hx, I) - rx, an_plane(g.oy, g.hy, J) - ry,
                          an_plane(g.oz, g.hz, K) - rz, fx, fy, fz);
                px = fma(d, fx, px);
                py = fma(d, fy, py);
                pz = fma(d, fz, pz);
            }
            if (++I == g.ncx) {
                I = 0;
                if (++J == g.ncy) {
                    J = 0;
                    ++K;
                }
            }
        }
        an_neumaier(s0, c0, px);
        an_neumaier(s1, c1, py);
        an_neumaier(s2, c2, pz);
    }
    if (!active) return;
    const double vx = G * (s0 + c0), vy = G * (s1 + c1), vz = G * (s2 + c2);
    if (gout) {
        double *o = gout + ((int64_t)b * M + j) * 3;
        o[0] = vx;
        o[1] = vy;
        o[2] = vz;
    }
    if (gz) gz[(int64_t)b * M + j] = vz;
}

// E[b][c] = sum_j r_bj . F(c - x'_j): one thread per corner, observers and
// their weights staged 128 at a time.
__global__ void __launch_bounds__(kAnTile)
an_adjoint_corners(const double *__restrict__ obs, int64_t M, const double *__restrict__ r, int ncomp,
                   AnGrid g, double *__restrict__ E) {
    __shared__ double ox[kAnTile], oy[kAnTile], oz[kAnTile], w0[kAnTile], w1[kAnTile], w2[kAnTile];
    const int b = blockIdx.y;
    const int64_t c = (int64_t)blockIdx.x * kAnTile + threadIdx.x;
    const bool active = c < g.nc;
    const int64_t cc = active ? c : 0;
    const int64_t I = cc % g.ncx, J = (cc / g.ncx) % g.ncy, K = cc / (g.ncx * g.ncy);
    const double X = an_plane(g.ox, g.hx, I), Y = an_plane(g.oy, g.hy, J), Z = an_plane(g.oz, g.hz, K);
    const double *rb = r + (int64_t)b * M * ncomp;
    double s = 0, sc = 0;
    for (int64_t t0 = 0; t0 < M; t0 += kAnTile) {
        const int64_t j = t0 + threadIdx.x;
        __syncthreads();
        if (j < M) {
            ox[threadIdx.x] = obs[3 * j + 0];
            oy[threadIdx.x] = obs[3 * j + 1];
            oz[threadIdx.x] = obs[3 * j + 2];
            w0[threadIdx.x] = ncomp == 3 ? rb[3 * j + 0] : 0.0;
            w1[threadIdx.x] = ncomp == 3 ? rb[3 * j + 1] : 0.0;
            w2[threadIdx.x] = ncomp == 3 ? rb[3 * j + 2] : rb[j];
        } else {
            ox[threadIdx.x] = oy[threadIdx.x] = oz[threadIdx.x] = 0.0;
            w0[threadIdx.x] = w1[threadIdx.x] = w2[threadIdx.x] = 0.0;
        }
        __syncthreads();
        const int cnt = (M - t0) < kAnTile ? (int)(M - t0) : kAnTile;
        double p = 0;
        if (ncomp == 3) {
            for (int u = 0; u < cnt; ++u) {
                double fx, fy, fz;
                an_corner<double>(X - ox[u], Y - oy[u], Z - oz[u], fx, fy, fz);
                p = fma(w0[u], fx, fma(w1[u], fy, fma(w2[u], fz, p)));
            }
        } else {
            for (int u = 0; u < cnt; ++u) p = fma(w2[u], an_corner_z<double>(X - ox[u], Y - oy[u], Z - oz[u]), p);
        }
        an_neumaier(s, sc, p);
    }
    if (active) E[(int64_t)b * g.nc + c] = s + sc;
}

// grad[b][v] = G sum over the eight corners c of v of s(v, c) E[b][c].
__global__ void an_adjoint_voxels(const double *__restrict__ E, AnGrid g, double G, double *__restrict__ grad) {
    const int b = blockIdx.y;
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= g.nvox) return;
    const int64_t i = v % g.nx, j = (v / g.nx) % g.ny, k = v / (g.nx * g.ny);
    const double *Eb = E + (int64_t)b * g.nc;
    double s = 0.0;
    for (int e = 0; e < 2; ++e)
        for (int f = 0; f < 2; ++f)
            for (int a = 0; a < 2; ++a) {
                const double x = Eb[((k + e) * g.ncy + (j + f)) * g.ncx + (i + a)];
                s += ((a + f + e) & 1) ? x : -x;
            }
    grad[(int64_t)b * g.nvox + v] = G * s;
}

}  // namespace

size_t sum_an_bytes(const gf_grid *grid, int max_batch) {
    const size_t nc = (size_t)(grid->n[0] + 1) * (size_t)(grid->n[1] + 1) * (size_t)(grid->n[2] + 1);
    return nc * sizeof(double) * (size_t)max_batch + 256;
}

gf_status sum_an_prepare(gf_plan_s *plan) {
    const AnGrid g = an_grid(plan);
    if ((g.nc + kAnTile - 1) / kAnTile > 0x7fffffff || (plan->M + kAnTile - 1) / kAnTile > 0x7fffffff) {
        set_error("closed-form voxels: %lld corners and %lld observers exceed one launch grid",
                  (long long)g.nc, (long long)plan->M);
        return GF_ERR_UNSUPPORTED;
    }
    return plan->arena.alloc_n(&plan->d_corner, (size_t)g.nc * (size_t)plan->opt.max_batch);
}

gf_status sum_an_forward(gf_plan_s *plan, const void *rho, int rho_dtype, int B, double *g, double *gz,
                         cudaStream_t st) {
    const AnGrid ga = an_grid(plan);
    an_corner_weights<<<dim3(ceil_div(ga.nc, 256), B), 256, 0, st>>>(rho, rho_dtype == GF_DTYPE_F32, ga,
                                                                     plan->d_corner, plan->d_status);
    GF_KERNEL_DONE();
    if (plan->M == 0) return GF_OK;
    an_forward<<<dim3(ceil_div(plan->M, kAnTile), B), kAnTile, 0, st>>>(plan->d_obs, plan->M, plan->d_corner, ga,
                                                                        plan->G, g, gz);
    GF_KERNEL_DONE();
    return GF_OK;
}

gf_status sum_an_adjoint(gf_plan_s *plan, const double *r, int ncomp, int B, double *grad, cudaStream_t st) {
    const AnGrid ga = an_grid(plan);
    if (plan->M == 0) {
        GF_CUDA(cudaMemsetAsync(grad, 0, sizeof(double) * (size_t)B * (size_t)ga.nvox, st));
        return GF_OK;
    }
    an_adjoint_corners<<<dim3(ceil_div(ga.nc, kAnTile), B), kAnTile, 0, st>>>(plan->d_obs, plan->M, r, ncomp, ga,
                                                                              plan->d_corner);
    GF_KERNEL_DONE();
    an_adjoint_voxels<<<dim3(ceil_div(ga.nvox, 256), B), 256, 0, st>>>(plan->d_corner, ga, plan->G, grad);
    GF_KERNEL_DONE();
    return GF_OK;
}

}  // namespace gf
