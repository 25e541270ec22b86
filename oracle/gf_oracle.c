/*
 * gf_oracle.c -- FP64 CPU oracle for the voxel-gravity forward model.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * reference that the CUDA library is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or constant with the CUDA library.
 *
 * What it computes (May & Knepley, "Optimal, scalable forward models for
 * computing gravity anomalies"):
 *
 *   Eq. 1   g(r) = G * Int_Omega rho(x) (r - x) / |r - x|^3 dV
 *
 * discretised as in Sec. 2.1: a brick of Mx*My*Mz hexahedral cells, constant
 * density per cell, and a per-cell quadrature rule (1-point Gauss = SUM-G1,
 * 2x2x2 Gauss = SUM-G2).  In the N-body form of Eqs. 7-8 the sources are the
 * quadrature points x_vq of every voxel v with mass
 *
 *   m_vq = rho_v * V_v * w_q / sum_q w_q ,     x_vq = c_v + (h/2) * xi_q
 *
 * and the result is the plain double sum over observers and sources.  An
 * observer that coincides exactly with a source point receives no
 * contribution from it (the field of a uniform cube at its own centroid is
 * zero by symmetry; the direct-work count of Eq. 14 also excludes self pairs).
 *
 * Accumulation: one Neumaier-compensated sum per observer and component, so
 * the oracle's own rounding stays far below the 1e-12 parity bar even for the
 * zero-mean random densities whose terms cancel heavily.  Build with
 * -ffp-contract=off so that no fused multiply-add changes the rounding.
 *
 * Also here: the adjoint (transpose) sum, the closed-form field of a
 * constant-density rectangular prism (the SUM-AN reference of Sec. 2.1, whose
 * formula the paper cites but does not print -- restated here from the
 * mathematics), the SUM-AN sum over a voxel grid built from it, and the
 * Appendix A norm quadrature of the prism's vertical field.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- Neumaier (improved Kahan) summation ------------------------------ */
typedef struct { double s, c; } nsum;

static inline void nsum_add(nsum *a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x))
        a->c += (a->s - t) + x;
    else
        a->c += (x - t) + a->s;
    a->s = t;
}
static inline double nsum_val(const nsum *a) { return a->s + a->c; }

int gfo_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static void set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

/* Source position of quadrature point q of voxel (i,j,k), Sec. 2.1:
 * the cell centre plus the reference node scaled by half the cell size. */
static inline void source_point(const double *origin, const double *h,
                                long i, long j, long k, const double *xi_q,
                                double *x) {
    double c0 = origin[0] + ((double)i + 0.5) * h[0];
    double c1 = origin[1] + ((double)j + 0.5) * h[1];
    double c2 = origin[2] + ((double)k + 0.5) * h[2];
    x[0] = c0 + 0.5 * h[0] * xi_q[0];
    x[1] = c1 + 0.5 * h[1] * xi_q[1];
    x[2] = c2 + 0.5 * h[2] * xi_q[2];
}

/*
 * Forward sum (Eq. 1 discretised by the Sec. 2.1 quadrature, Eq. 7 form).
 *   rho : [B][nz][ny][nx] densities (kg/m^3), x fastest
 *   xi  : [nq][3] reference nodes in [-1,1]^3,  w : [nq] weights
 *   obs : [M][3] observer coordinates (m)
 *   g   : [B][M][3] output (m/s^2)
 * Returns 0 on success, -1 on bad arguments.
 */
int gfo_forward(long nx, long ny, long nz, const double *origin,
                const double *h, int nq, const double *xi, const double *w,
                const double *rho, int B, const double *obs, long M, double G,
                double *g, int nthreads) {
    if (nx < 0 || ny < 0 || nz < 0 || nq <= 0 || B <= 0 || M < 0) return -1;
    set_threads(nthreads);
    const long nvox = nx * ny * nz;
    const double vol = h[0] * h[1] * h[2];
    double wsum = 0.0;
    for (int q = 0; q < nq; ++q) wsum += w[q];

#pragma omp parallel
    {
        nsum *acc = (nsum *)malloc(sizeof(nsum) * 3 * (size_t)B);
#pragma omp for schedule(dynamic, 4)
        for (long s = 0; s < M; ++s) {
            const double r0 = obs[3 * s + 0], r1 = obs[3 * s + 1],
                         r2 = obs[3 * s + 2];
            memset(acc, 0, sizeof(nsum) * 3 * (size_t)B);
            for (long k = 0; k < nz; ++k)
                for (long j = 0; j < ny; ++j)
                    for (long i = 0; i < nx; ++i) {
                        const long v = (k * ny + j) * nx + i;
                        for (int q = 0; q < nq; ++q) {
                            double x[3];
                            source_point(origin, h, i, j, k, xi + 3 * q, x);
                            const double d0 = r0 - x[0], d1 = r1 - x[1],
                                         d2 = r2 - x[2];
                            const double rr = d0 * d0 + d1 * d1 + d2 * d2;
                            if (rr == 0.0) continue; /* coincident pair */
                            const double rinv = 1.0 / sqrt(rr);
                            const double k3 = rinv * rinv * rinv;
                            const double wq = w[q] / wsum;
                            for (int b = 0; b < B; ++b) {
                                const double m = rho[(long)b * nvox + v] * vol * wq;
                                const double c = m * k3;
                                nsum_add(&acc[3 * b + 0], c * d0);
                                nsum_add(&acc[3 * b + 1], c * d1);
                                nsum_add(&acc[3 * b + 2], c * d2);
                            }
                        }
                    }
            for (int b = 0; b < B; ++b)
                for (int a = 0; a < 3; ++a)
                    g[((long)b * M + s) * 3 + a] = G * nsum_val(&acc[3 * b + a]);
        }
        free(acc);
    }
    return 0;
}

/*
 * Adjoint (transpose) of gfo_forward.  Eq. 1 is linear in rho, so the
 * gradient of any misfit phi(g) with respect to the voxel densities is the
 * transpose of the forward matrix applied to dphi/dg.
 *   r    : weights on the outputs, [B][M][ncomp]; ncomp = 1 weights g_z
 *          only, ncomp = 3 weights all three components.
 *   grad : [B][nz][ny][nx],  grad_v = sum_s sum_c r_sc * dg_sc/drho_v
 */
int gfo_adjoint(long nx, long ny, long nz, const double *origin,
                const double *h, int nq, const double *xi, const double *w,
                const double *obs, long M, const double *r, int ncomp, int B,
                double G, double *grad, int nthreads) {
    if (nx < 0 || ny < 0 || nz < 0 || nq <= 0 || B <= 0 || M < 0) return -1;
    if (ncomp != 1 && ncomp != 3) return -1;
    set_threads(nthreads);
    const long nvox = nx * ny * nz;
    const double vol = h[0] * h[1] * h[2];
    double wsum = 0.0;
    for (int q = 0; q < nq; ++q) wsum += w[q];

#pragma omp parallel
    {
        nsum *acc = (nsum *)malloc(sizeof(nsum) * (size_t)B);
#pragma omp for schedule(dynamic, 16)
        for (long v = 0; v < nvox; ++v) {
            const long i = v % nx, j = (v / nx) % ny, k = v / (nx * ny);
            memset(acc, 0, sizeof(nsum) * (size_t)B);
            for (int q = 0; q < nq; ++q) {
                double x[3];
                source_point(origin, h, i, j, k, xi + 3 * q, x);
                const double wq = w[q] / wsum;
                for (long s = 0; s < M; ++s) {
                    const double d0 = obs[3 * s + 0] - x[0],
                                 d1 = obs[3 * s + 1] - x[1],
                                 d2 = obs[3 * s + 2] - x[2];
                    const double rr = d0 * d0 + d1 * d1 + d2 * d2;
                    if (rr == 0.0) continue;
                    const double rinv = 1.0 / sqrt(rr);
                    const double k3 = rinv * rinv * rinv * vol * wq;
                    for (int b = 0; b < B; ++b) {
                        const double *rb = r + ((long)b * M + s) * ncomp;
                        double t;
                        if (ncomp == 1)
                            t = rb[0] * d2;
                        else
                            t = rb[0] * d0 + rb[1] * d1 + rb[2] * d2;
                        nsum_add(&acc[b], t * k3);
                    }
                }
            }
            for (int b = 0; b < B; ++b)
                grad[(long)b * nvox + v] = G * nsum_val(&acc[b]);
        }
        free(acc);
    }
    return 0;
}

/*
 * The transpose sum of gfo_adjoint restricted to a list of voxels
 * (vox[nv] linear indices into [nz][ny][nx]): grad[b][i] for i < nv.  Used to
 * check large problems on a sample of voxels.
 */
int gfo_adjoint_subset(long nx, long ny, long nz, const double *origin,
                       const double *h, int nq, const double *xi,
                       const double *w, const double *obs, long M,
                       const double *r, int ncomp, int B, double G,
                       const long *vox, long nv, double *grad, int nthreads) {
    if (nx < 0 || ny < 0 || nz < 0 || nq <= 0 || B <= 0 || M < 0 || nv < 0) return -1;
    if (ncomp != 1 && ncomp != 3) return -1;
    set_threads(nthreads);
    const double vol = h[0] * h[1] * h[2];
    double wsum = 0.0;
    for (int q = 0; q < nq; ++q) wsum += w[q];
#pragma omp parallel
    {
        nsum *acc = (nsum *)malloc(sizeof(nsum) * (size_t)B);
#pragma omp for schedule(dynamic, 1)
        for (long iv = 0; iv < nv; ++iv) {
            const long v = vox[iv];
            const long i = v % nx, j = (v / nx) % ny, k = v / (nx * ny);
            memset(acc, 0, sizeof(nsum) * (size_t)B);
            for (int q = 0; q < nq; ++q) {
                double x[3];
                source_point(origin, h, i, j, k, xi + 3 * q, x);
                const double wq = w[q] / wsum;
                for (long s = 0; s < M; ++s) {
                    const double d0 = obs[3 * s + 0] - x[0],
                                 d1 = obs[3 * s + 1] - x[1],
                                 d2 = obs[3 * s + 2] - x[2];
                    const double rr = d0 * d0 + d1 * d1 + d2 * d2;
                    if (rr == 0.0) continue;
                    const double rinv = 1.0 / sqrt(rr);
                    const double k3 = rinv * rinv * rinv * vol * wq;
                    for (int b = 0; b < B; ++b) {
                        const double *rb = r + ((long)b * M + s) * ncomp;
                        double t;
                        if (ncomp == 1)
                            t = rb[0] * d2;
                        else
                            t = rb[0] * d0 + rb[1] * d1 + rb[2] * d2;
                        nsum_add(&acc[b], t * k3);
                    }
                }
            }
            for (int b = 0; b < B; ++b) grad[(long)b * nv + iv] = G * nsum_val(&acc[b]);
        }
        free(acc);
    }
    return 0;
}

/*
 * Closed-form g_z of a constant-density rectangular prism (the analytic
 * reference of Sec. 2.1 / Sec. 3, SUM-AN).  Derived here from Eq. 1:
 * with u = x - r_x, v = y - r_y, w = z - r_z (source minus observer),
 *
 *   g_z = -G rho Int Int Int w / R^3 du dv dw ,    R = |(u, v, w)|
 *
 * The w-integral of w/R^3 is -1/R and the double antiderivative of 1/R in
 * (u, v) is  u ln(v + R) + v ln(u + R) - w atan(u v / (w R)),  so
 *
 *   g_z = G rho sum_{corners} s_u s_v s_w [ u ln(v+R) + v ln(u+R)
 *                                           - w atan(u v / (w R)) ]
 *
 * with s = +1 at the upper and -1 at the lower limit of each axis.
 * The logarithms are evaluated in the cancellation-free form when the
 * argument would be a difference of nearly equal numbers.
 */
static inline double log_plus_R(double a, double b2c2, double R) {
    /* ln(a + R) with R = sqrt(a^2 + b2c2); stable for a < 0 */
    if (a >= 0.0) return log(a + R);
    return log(b2c2 / (R - a));
}

static double prism_corner(double u, double v, double w) {
    const double u2 = u * u, v2 = v * v, w2 = w * w;
    const double R = sqrt(u2 + v2 + w2);
    double t = 0.0;
    if (u != 0.0 && (u2 + w2) > 0.0) t += u * log_plus_R(v, u2 + w2, R);
    if (v != 0.0 && (v2 + w2) > 0.0) t += v * log_plus_R(u, v2 + w2, R);
    if (w != 0.0 && R > 0.0) t -= w * atan((u * v) / (w * R));
    return t;
}

double gfo_prism_gz(const double *lo, const double *hi, double rho, double G,
                    const double *r) {
    double acc = 0.0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int c = 0; c < 2; ++c) {
                const double u = (a ? hi[0] : lo[0]) - r[0];
                const double v = (b ? hi[1] : lo[1]) - r[1];
                const double w = (c ? hi[2] : lo[2]) - r[2];
                /* +1 when an even number of lower limits is taken */
                const double s = ((a + b + c) & 1) ? 1.0 : -1.0;
                acc += s * prism_corner(u, v, w);
            }
    return G * rho * acc;
}

/*
 * All three components of the prism field.  Relabelling the axes in the
 * derivation above gives g_x and g_y: the corner function keeps its form
 * with the component's own axis in the third (arctangent) slot,
 *
 *   g_x = G rho sum s [ v ln(w+R) + w ln(v+R) - u atan(v w / (u R)) ]
 *   g_y = G rho sum s [ w ln(u+R) + u ln(w+R) - v atan(w u / (v R)) ]
 *
 * with the same corner signs s.  g[2] equals gfo_prism_gz bit for bit.
 */
void gfo_prism_g(const double *lo, const double *hi, double rho, double G,
                 const double *r, double *g) {
    double ax = 0.0, ay = 0.0, az = 0.0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int c = 0; c < 2; ++c) {
                const double u = (a ? hi[0] : lo[0]) - r[0];
                const double v = (b ? hi[1] : lo[1]) - r[1];
                const double w = (c ? hi[2] : lo[2]) - r[2];
                const double s = ((a + b + c) & 1) ? 1.0 : -1.0;
                ax += s * prism_corner(v, w, u);
                ay += s * prism_corner(w, u, v);
                az += s * prism_corner(u, v, w);
            }
    g[0] = G * rho * ax;
    g[1] = G * rho * ay;
    g[2] = G * rho * az;
}

void gfo_prism_g_many(const double *lo, const double *hi, double rho, double G,
                      const double *pts, long n, double *out, int nthreads) {
    set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) gfo_prism_g(lo, hi, rho, G, pts + 3 * i, out + 3 * i);
}

/*
 * SUM-AN (Sec. 2.1): the field of the piecewise-constant density itself,
 * every voxel integrated in closed form,
 *
 *   g(r) = sum_v  prism field of voxel v = origin + [i, i+1) x [j, j+1) x
 *                 [k, k+1) * h  with density rho_v,
 *
 * with one Neumaier sum per observer, component and model.  No quadrature
 * and no coincidence rule: the closed form is finite everywhere, on voxel
 * faces, edges and corners included.
 *   rho : [B][nz][ny][nx],  obs : [M][3],  g : [B][M][3]
 */
int gfo_forward_analytic(long nx, long ny, long nz, const double *origin,
                         const double *h, const double *rho, int B,
                         const double *obs, long M, double G, double *g,
                         int nthreads) {
    if (nx < 0 || ny < 0 || nz < 0 || B <= 0 || M < 0) return -1;
    set_threads(nthreads);
    const long nvox = nx * ny * nz;
#pragma omp parallel
    {
        nsum *acc = (nsum *)malloc(sizeof(nsum) * 3 * (size_t)B);
#pragma omp for schedule(dynamic, 4)
        for (long s = 0; s < M; ++s) {
            memset(acc, 0, sizeof(nsum) * 3 * (size_t)B);
            for (long k = 0; k < nz; ++k)
                for (long j = 0; j < ny; ++j)
                    for (long i = 0; i < nx; ++i) {
                        const long v = (k * ny + j) * nx + i;
                        const double lo[3] = {origin[0] + (double)i * h[0],
                                              origin[1] + (double)j * h[1],
                                              origin[2] + (double)k * h[2]};
                        const double hi[3] = {origin[0] + (double)(i + 1) * h[0],
                                              origin[1] + (double)(j + 1) * h[1],
                                              origin[2] + (double)(k + 1) * h[2]};
                        double f[3];
                        gfo_prism_g(lo, hi, 1.0, 1.0, obs + 3 * s, f);
                        for (int b = 0; b < B; ++b) {
                            const double d = rho[(long)b * nvox + v];
                            for (int a = 0; a < 3; ++a) nsum_add(&acc[3 * b + a], d * f[a]);
                        }
                    }
            for (int b = 0; b < B; ++b)
                for (int a = 0; a < 3; ++a)
                    g[((long)b * M + s) * 3 + a] = G * nsum_val(&acc[3 * b + a]);
        }
        free(acc);
    }
    return 0;
}

/*
 * Transpose of gfo_forward_analytic: for weights r on the outputs (ncomp = 1:
 * on g_z only, r [B][M]; ncomp = 3: on g, r [B][M][3]),
 *
 *   grad_v = G sum_j r_j . (prism field of voxel v, unit density, at obs_j),
 *
 * one Neumaier sum per voxel and model.  grad : [B][nz][ny][nx].
 */
int gfo_adjoint_analytic(long nx, long ny, long nz, const double *origin,
                         const double *h, const double *obs, long M,
                         const double *r, int ncomp, int B, double G,
                         double *grad, int nthreads) {
    if (nx < 0 || ny < 0 || nz < 0 || B <= 0 || M < 0 || (ncomp != 1 && ncomp != 3)) return -1;
    set_threads(nthreads);
    const long nvox = nx * ny * nz;
#pragma omp parallel
    {
        nsum *acc = (nsum *)malloc(sizeof(nsum) * (size_t)B);
#pragma omp for schedule(dynamic, 4)
        for (long v = 0; v < nvox; ++v) {
            const long i = v % nx, j = (v / nx) % ny, k = v / (nx * ny);
            const double lo[3] = {origin[0] + (double)i * h[0], origin[1] + (double)j * h[1],
                                  origin[2] + (double)k * h[2]};
            const double hi[3] = {origin[0] + (double)(i + 1) * h[0], origin[1] + (double)(j + 1) * h[1],
                                  origin[2] + (double)(k + 1) * h[2]};
            memset(acc, 0, sizeof(nsum) * (size_t)B);
            for (long s = 0; s < M; ++s) {
                double f[3];
                gfo_prism_g(lo, hi, 1.0, 1.0, obs + 3 * s, f);
                for (int b = 0; b < B; ++b) {
                    if (ncomp == 1) {
                        nsum_add(&acc[b], r[(long)b * M + s] * f[2]);
                    } else {
                        const double *rb = r + ((long)b * M + s) * 3;
                        for (int a = 0; a < 3; ++a) nsum_add(&acc[b], rb[a] * f[a]);
                    }
                }
            }
            for (int b = 0; b < B; ++b) grad[(long)b * nvox + v] = G * nsum_val(&acc[b]);
        }
        free(acc);
    }
    return 0;
}

/* Vectorised prism field at n points. */
void gfo_prism_gz_many(const double *lo, const double *hi, double rho,
                       double G, const double *pts, long n, double *out,
                       int nthreads) {
    set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) out[i] = gfo_prism_gz(lo, hi, rho, G, pts + 3 * i);
}

/*
 * Appendix A norm quadrature: integrate |f|, f^2 and max|f| of the analytic
 * prism field over the domain box [dlo, dhi] split into Mb^3 cells, each cell
 * split into m^3 sub-cells, each sub-cell integrated with the tensor
 * Gauss-Legendre rule of ng points per axis (nodes gx in [-1,1], weights gw).
 * out[0] = Int |g_z| dV, out[1] = sqrt(Int g_z^2 dV), out[2] = max |g_z|
 * over the quadrature points.
 */
void gfo_prism_norms(const double *plo, const double *phi_, double rho,
                     double G, const double *dlo, const double *dhi, long Mb,
                     long m, int ng, const double *gx, const double *gw,
                     double *out, int nthreads) {
    set_threads(nthreads);
    const long ns = Mb * m; /* sub-cells per axis */
    double hs[3];
    for (int a = 0; a < 3; ++a) hs[a] = (dhi[a] - dlo[a]) / (double)ns;
    const double jac = 0.125 * hs[0] * hs[1] * hs[2];
    double s1 = 0.0, s2 = 0.0, mx = 0.0;
#pragma omp parallel
    {
        nsum a1 = {0, 0}, a2 = {0, 0};
        double lmx = 0.0;
#pragma omp for schedule(dynamic, 1) collapse(2)
        for (long kz = 0; kz < ns; ++kz)
            for (long ky = 0; ky < ns; ++ky)
                for (long kx = 0; kx < ns; ++kx)
                    for (int c = 0; c < ng; ++c)
                        for (int b = 0; b < ng; ++b)
                            for (int a = 0; a < ng; ++a) {
                                double p[3];
                                p[0] = dlo[0] + ((double)kx + 0.5 * (1.0 + gx[a])) * hs[0];
                                p[1] = dlo[1] + ((double)ky + 0.5 * (1.0 + gx[b])) * hs[1];
                                p[2] = dlo[2] + ((double)kz + 0.5 * (1.0 + gx[c])) * hs[2];
                                const double f = gfo_prism_gz(plo, phi_, rho, G, p);
                                const double wt = gw[a] * gw[b] * gw[c] * jac;
                                nsum_add(&a1, wt * fabs(f));
                                nsum_add(&a2, wt * f * f);
                                if (fabs(f) > lmx) lmx = fabs(f);
                            }
#pragma omp critical
        {
            s1 += nsum_val(&a1);
            s2 += nsum_val(&a2);
            if (lmx > mx) mx = lmx;
        }
    }
    out[0] = s1;
    out[1] = sqrt(s2);
    out[2] = mx;
}


/* ---- Deformed hexahedra and weighted point sources (Sec. 2.1, Sec. 4) ---- */

/*
 * Quadrature points of deformed hexahedral cells.  Sec. 2.1 allows the
 * general SUM-G1 to take arbitrarily deformed hexahedra by integrating in a
 * reference coordinate system: cell c is the trilinear image x(xi) of the
 * reference cube [-1,1]^3 through its eight corners,
 *
 *   x(xi) = sum_a N_a(xi) X_a,  N_a(xi) = (1 + s0 xi0)(1 + s1 xi1)(1 + s2 xi2) / 8,
 *
 * corner a = i + 2 j + 4 k sitting at reference signs (s0, s1, s2) =
 * (2i - 1, 2j - 1, 2k - 1), and a constant density integrates as
 *
 *   Int_cell rho K(r - x) dV = rho Int_ref K(r - x(xi)) |det dx/dxi| dxi
 *                           ~ rho sum_q (8 w_q / sum w) |det J(xi_q)| K(r - x(xi_q)).
 *
 *   verts : [ncell][8][3] corner coordinates (m)
 *   xi, w : [nq][3] reference nodes in [-1,1]^3 and [nq] weights
 *   x     : [ncell * nq][3] output source points, a : [ncell * nq] output
 *           volume weights (m^3), source s = c * nq + q
 */
int gfo_hex_sources(long ncell, const double *verts, int nq, const double *xi, const double *w,
                    double *x, double *a) {
    if (ncell < 0 || nq <= 0) return -1;
    double wsum = 0.0;
    for (int q = 0; q < nq; ++q) wsum += w[q];
    for (long c = 0; c < ncell; ++c) {
        const double *X = verts + 24 * c;
        for (int q = 0; q < nq; ++q) {
            const double *e = xi + 3 * q;
            double p[3] = {0.0, 0.0, 0.0};
            double J[3][3] = {{0.0}};   /* J[d][r] = d x_d / d xi_r */
            for (int k = 0; k < 8; ++k) {
                const double s0 = (k & 1) ? 1.0 : -1.0, s1 = (k & 2) ? 1.0 : -1.0, s2 = (k & 4) ? 1.0 : -1.0;
                const double f0 = 1.0 + s0 * e[0], f1 = 1.0 + s1 * e[1], f2 = 1.0 + s2 * e[2];
                const double N = f0 * f1 * f2 / 8.0;
                const double dN[3] = {s0 * f1 * f2 / 8.0, f0 * s1 * f2 / 8.0, f0 * f1 * s2 / 8.0};
                for (int d = 0; d < 3; ++d) {
                    p[d] += N * X[3 * k + d];
                    for (int r = 0; r < 3; ++r) J[d][r] += dN[r] * X[3 * k + d];
                }
            }
            const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                               J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                               J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
            const long s = c * nq + q;
            for (int d = 0; d < 3; ++d) x[3 * s + d] = p[d];
            a[s] = 8.0 * (w[q] / wsum) * fabs(det);
        }
    }
    return 0;
}

/*
 * Field of weighted point sources (Eq. 7 with explicit points): source s at
 * x_s carries the mass rho_{c(s)} a_s, c(s) = s / per_cell the density
 * (cell or point) it samples -- the quadrature points of deformed cells, or
 * scattered density points with their (Voronoi) volumes as Sec. 4 describes
 * for the FMM:
 *
 *   g(r) = G sum_s rho_{c(s)} a_s (r - x_s) / |r - x_s|^3
 *
 *   x   : [S][3],  a : [S],  rho : [B][S / per_cell],  obs : [M][3]
 *   g   : [B][M][3]
 * A source that coincides exactly with an observer contributes nothing to it.
 */
int gfo_forward_points(long S, const double *x, const double *a, long per_cell, const double *rho, int B,
                       const double *obs, long M, double G, double *g, int nthreads) {
    if (S < 0 || per_cell <= 0 || S % per_cell != 0 || B <= 0 || M < 0) return -1;
    set_threads(nthreads);
    const long ncell = S / per_cell;
#pragma omp parallel
    {
        nsum *acc = (nsum *)malloc(sizeof(nsum) * 3 * (size_t)B);
#pragma omp for schedule(dynamic, 4)
        for (long j = 0; j < M; ++j) {
            const double r0 = obs[3 * j + 0], r1 = obs[3 * j + 1], r2 = obs[3 * j + 2];
            memset(acc, 0, sizeof(nsum) * 3 * (size_t)B);
            for (long s = 0; s < S; ++s) {
                const double d0 = r0 - x[3 * s + 0], d1 = r1 - x[3 * s + 1], d2 = r2 - x[3 * s + 2];
                const double rr = d0 * d0 + d1 * d1 + d2 * d2;
                if (rr == 0.0) continue; /* coincident pair */
                const double rinv = 1.0 / sqrt(rr);
                const double k3 = rinv * rinv * rinv;
                const long c = s / per_cell;
                for (int b = 0; b < B; ++b) {
                    const double m = rho[(long)b * ncell + c] * a[s];
                    nsum_add(&acc[3 * b + 0], m * k3 * d0);
                    nsum_add(&acc[3 * b + 1], m * k3 * d1);
                    nsum_add(&acc[3 * b + 2], m * k3 * d2);
                }
            }
            for (int b = 0; b < B; ++b)
                for (int d = 0; d < 3; ++d) g[((long)b * M + j) * 3 + d] = G * nsum_val(&acc[3 * b + d]);
        }
        free(acc);
    }
    return 0;
}
