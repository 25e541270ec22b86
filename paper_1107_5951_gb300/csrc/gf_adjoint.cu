// gf_adjoint.cu -- the transpose of the FMM forward model.
//
// Eq. 1 is linear in the density, so the gradient of any misfit with respect
// to the voxel densities is the transpose of the forward operator applied to
// the misfit's derivative with respect to the outputs.  The forward operator
// is, per observer j,  g_j = G h (N rho + E L Mt P rho)_j  with N the near
// field, P the P2M matrix, Mt the M2M/M2L chain up to the leaf local
// expansions and E the L2P gradient.  This file applies, exactly,
//   grad = G h (N^T r + P^T Mt^T L^T E^T r):
//   E^T  -- each leaf's observers deposit r_j . grad(basis_k)(X_j) into a dual
//           local expansion (l2p_adj);
//   L^T  -- dual local expansions flow from children to parents (L2L^T);
//   M2L^T-- every source box collects T_{-o}^T times the dual local expansion
//           of the observer box at offset o, over its parity class's 189
//           offsets (the interaction-list rule is symmetric);
//   M2M^T-- dual multipole expansions flow from parents to children;
//   P^T, N^T -- per source leaf, the dual multipole expansion is expanded
//           back over its voxels and the near-field sum is taken with the
//           observers as sources (adj_eval).
// The plan's ME/LE/mass workspaces hold the dual quantities, so a plan's
// forward and adjoint calls must not overlap on the device.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "fmm_math.cuh"
#include "gf_fmm.cuh"
#include "gf_m2l.cuh"

namespace gf {
namespace {

__device__ __forceinline__ int64_t unmorton(uint64_t k, int s) {
    int64_t c = 0;
    for (int bit = 0; bit < 21; ++bit) c |= (int64_t)((k >> (3 * bit + s)) & 1) << bit;
    return c;
}

// observer box index over the widened source block of a level
__global__ void fill_imap(const uint64_t *__restrict__ tkey, int64_t nt, int64_t lo0, int64_t lo1, int64_t lo2,
                          int64_t n0, int64_t n1, int64_t n2, int32_t *__restrict__ imap) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const uint64_t k = tkey[t];
    const int64_t x = unmorton(k, 0) - lo0, y = unmorton(k, 1) - lo1, z = unmorton(k, 2) - lo2;
    if (x >= 0 && y >= 0 && z >= 0 && x < n0 && y < n1 && z < n2) imap[(z * n1 + y) * n0 + x] = (int32_t)t;
}

// child[parent][position] for the observer boxes of the next level
__global__ void fill_child(const uint64_t *__restrict__ tkey, const int32_t *__restrict__ tparent, int64_t nt,
                           int32_t *__restrict__ child) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nt) return;
    child[(int64_t)tparent[c] * 8 + (int)(tkey[c] & 7)] = (int32_t)c;
}

// ---------------------------------------------------------------- E^T
// Dual local expansion of one observer leaf:
//   LE*_k = -(1/b^2) sum_j sum_a r_ja d(phi_k)/dX_a (X_j)
// phi_k the k-th real basis function of a local expansion (R_n^0, 2 Re R_n^m,
// 2 Im R_n^m) and X_j the observer's offset from the leaf centre in leaf
// units; the harmonics of degree < p are built per observer, one column
// per thread.
template <class T>
__global__ void __launch_bounds__(128)
l2p_adj(const int32_t *__restrict__ leaf_beg, const int32_t *__restrict__ perm, const T *__restrict__ tloc,
        const double *__restrict__ r, int ncomp, int64_t M, int B, int p, int K, int ldk, int b,
        T *__restrict__ le) {
    extern __shared__ unsigned char shraw[];
    const int nh = p * (p + 1) / 2;   // harmonics of degree <= p - 1
    T *hre = reinterpret_cast<T *>(shraw), *him = hre + nh;
    T *acc = him + nh;                // [B][K]
    T *rw = acc + (size_t)B * K;      // [B][3] this observer's weights
    __shared__ T X[3];
    const int64_t t = blockIdx.x;
    const int j0 = leaf_beg[t], j1 = leaf_beg[t + 1];
    for (int e = threadIdx.x; e < B * K; e += blockDim.x) acc[e] = T(0);
    const T inv_b = T(1) / T(b);
    for (int jj = j0; jj < j1; ++jj) {
        __syncthreads();
        if (threadIdx.x < 3) X[threadIdx.x] = tloc[3 * (int64_t)jj + threadIdx.x] * inv_b;
        const int64_t cj = perm[jj];
        for (int e = threadIdx.x; e < 3 * B; e += blockDim.x) {
            const int bb = e / 3, a = e - bb * 3;
            T v = T(0);
            if (ncomp == 3)
                v = (T)r[((int64_t)bb * M + cj) * 3 + a];
            else if (a == 2)
                v = (T)r[(int64_t)bb * M + cj];
            rw[e] = v;
        }
        __syncthreads();
        const int m = threadIdx.x;
        if (m < p) {   // column m of the regular harmonics, degrees m .. p-1
            const T x = X[0], y = X[1], z = X[2];
            const T r2 = x * x + y * y + z * z;
            T sr = T(1), si = T(0);
            for (int mm = 1; mm <= m; ++mm) {
                const T f = -sqrt(T(2 * mm - 1) / T(2 * mm));
                const T nr = f * (x * sr - y * si), ni = f * (x * si + y * sr);
                sr = nr;
                si = ni;
            }
            hre[tri(m, m)] = sr;
            him[tri(m, m)] = si;
            T r1 = sr, i1 = si, r0 = T(0), i0 = T(0);
            for (int n = m + 1; n < p; ++n) {
                const T inv = T(1) / sqrt(T((n + m) * (n - m)));
                const T ca = T(2 * n - 1) * inv;
                const T cb = (n - 1 > m) ? sqrt(T((n - 1 + m) * (n - 1 - m))) * inv * r2 : T(0);
                const T cr = ca * z * r1 - cb * r0, ci = ca * z * i1 - cb * i0;
                hre[tri(n, m)] = cr;
                him[tri(n, m)] = ci;
                r0 = r1;
                i0 = i1;
                r1 = cr;
                i1 = ci;
            }
        }
        __syncthreads();
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
            int n = (int)sqrt((double)k);
            while (n * n > k) --n;
            while ((n + 1) * (n + 1) <= k) ++n;
            if (n == 0) continue;
            const int ro = k - n * n, mm = (ro + 1) / 2;
            const bool im_part = ro > 0 && (ro % 2 == 0);
            // R_{n-1}^{m-1}, R_{n-1}^m, R_{n-1}^{m+1}
            T lr = T(0), li = T(0), cr = T(0), ci = T(0), ur = T(0), ui = T(0);
            if (mm - 1 >= 0) {
                lr = hre[tri(n - 1, mm - 1)];
                li = him[tri(n - 1, mm - 1)];
            } else {   // R^{-1} = -conj(R^1)
                if (n - 1 >= 1) {
                    lr = -hre[tri(n - 1, 1)];
                    li = him[tri(n - 1, 1)];
                }
            }
            if (mm <= n - 1) {
                cr = hre[tri(n - 1, mm)];
                ci = him[tri(n - 1, mm)];
            }
            if (mm + 1 <= n - 1) {
                ur = hre[tri(n - 1, mm + 1)];
                ui = him[tri(n - 1, mm + 1)];
            }
            const T A = sqrt(T((n - mm) * (n + mm)));
            const T a = sqrt(T((n + mm) * (n + mm - 1)));
            const T bq = sqrt(T((n - mm) * (n - mm - 1)));
            // complex derivatives of R_n^m
            const T dxr = T(0.5) * (-a * lr + bq * ur), dxi = T(0.5) * (-a * li + bq * ui);
            const T sr = T(0.5) * (a * lr + bq * ur), sim = T(0.5) * (a * li + bq * ui);
            const T dyr = sim, dyi = -sr;   // -i (sr + i sim)
            const T dzr = A * cr, dzi = A * ci;
            const T f = mm == 0 ? T(1) : T(2);
            const T wx = f * (im_part ? dxi : dxr), wy = f * (im_part ? dyi : dyr), wz = f * (im_part ? dzi : dzr);
            for (int bb = 0; bb < B; ++bb)
                acc[bb * K + k] += rw[3 * bb] * wx + rw[3 * bb + 1] * wy + rw[3 * bb + 2] * wz;
        }
    }
    __syncthreads();
    const T sc = T(-1) / (T(b) * T(b));
    for (int e = threadIdx.x; e < B * K; e += blockDim.x) {
        const int bb = e / K, k = e - bb * K;
        le[(t * B + bb) * ldk + k] = sc * acc[e];
    }
}

// ---------------------------------------------------------------- N^T, P^T
// One warp per source leaf.  Each lane owns up to two voxels of the leaf;
// the observers of every neighbouring observer leaf are staged in shared
// memory (offset from this leaf's centre and the weights) and each lane
// accumulates, for its voxels' quadrature nodes, sum_j r_j . d / |d|^3 with
// d the observer minus the node.  The dual multipole expansion is then
// expanded back over the voxels with the P2M matrix.  Per-leaf partial sums
// are merged with TwoSum; the result is scaled by G h and scattered to the
// caller's grid order.
constexpr int kAdjWarps = 4;
constexpr int kAdjChunk = 32;
constexpr int kAdjMaxB = 16;

template <class T>
__device__ __forceinline__ void two_sum_a(T &hi, T &lo, T x) {
    const T s = hi + x;
    const T bp = s - hi;
    lo += (hi - (s - bp)) + (x - bp);
    hi = s;
}

struct AdjArgs {
    const int32_t *leaf_beg, *perm;
    const void *tloc;
    const double *r;
    int ncomp;
    int64_t M;
    int B, K, ldk, b, nq, p;
    const int32_t *imap;       // level L window map
    int64_t mlo[3], mn[3];
    int64_t blo[3], bn[3];     // leaf source block
    const void *me;            // dual ME at the leaves
    const void *P;             // [b^3][K]
    const QuadRule *qr;
    int64_t gn[3];             // grid voxels
    int64_t voff[3];
    double scale, eps2;
    double *grad;
};

template <class T>
__global__ void __launch_bounds__(kAdjWarps * 32)
adj_eval(AdjArgs a) {
    extern __shared__ unsigned char shraw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int B = a.B;
    // per-warp slice: observers [kAdjChunk][3 + 3 B]
    const int ostride = 3 + 3 * B;
    T *os = reinterpret_cast<T *>(shraw) + (size_t)warp * kAdjChunk * ostride;
    const T *tloc = reinterpret_cast<const T *>(a.tloc);
    const T *me = reinterpret_cast<const T *>(a.me);
    const T *P = reinterpret_cast<const T *>(a.P);
    const int b = a.b, b3 = b * b * b;
    const int64_t nleaf = a.bn[0] * a.bn[1] * a.bn[2];
    const T half_b = T(0.5) * T(b);
    const T eps2 = (T)a.eps2;
    for (int64_t sl = (int64_t)blockIdx.x * kAdjWarps + warp; sl < nleaf; sl += (int64_t)gridDim.x * kAdjWarps) {
        const int64_t lx = sl % a.bn[0], ly = (sl / a.bn[0]) % a.bn[1], lz = sl / (a.bn[0] * a.bn[1]);
        const int64_t Sx = a.blo[0] + lx, Sy = a.blo[1] + ly, Sz = a.blo[2] + lz;
        for (int v0 = 0; v0 < b3; v0 += 64) {
            int vv[2];
            vv[0] = v0 + lane;
            vv[1] = v0 + lane + 32;
            T hi[2][kAdjMaxB], lo[2][kAdjMaxB];
#pragma unroll
            for (int u = 0; u < 2; ++u)
#pragma unroll
                for (int bb = 0; bb < kAdjMaxB; ++bb) hi[u][bb] = lo[u][bb] = T(0);
            for (int nb = 0; nb < 27; ++nb) {
                const int dx = nb % 3 - 1, dy = (nb / 3) % 3 - 1, dz = nb / 9 - 1;
                const int64_t wx = Sx + dx - a.mlo[0], wy = Sy + dy - a.mlo[1], wz = Sz + dz - a.mlo[2];
                if (wx < 0 || wy < 0 || wz < 0 || wx >= a.mn[0] || wy >= a.mn[1] || wz >= a.mn[2]) continue;
                const int32_t t = a.imap[(wz * a.mn[1] + wy) * a.mn[0] + wx];
                if (t < 0) continue;
                const int j0 = a.leaf_beg[t], j1 = a.leaf_beg[t + 1];
                T part[2][kAdjMaxB];
#pragma unroll
                for (int u = 0; u < 2; ++u)
#pragma unroll
                    for (int bb = 0; bb < kAdjMaxB; ++bb) part[u][bb] = T(0);
                for (int c0 = j0; c0 < j1; c0 += kAdjChunk) {
                    const int cnt = min(kAdjChunk, j1 - c0);
                    __syncwarp();
                    if (lane < cnt) {
                        const int64_t jj = c0 + lane;
                        T *o = os + lane * ostride;
                        o[0] = tloc[3 * jj + 0] + T(dx * b);
                        o[1] = tloc[3 * jj + 1] + T(dy * b);
                        o[2] = tloc[3 * jj + 2] + T(dz * b);
                        const int64_t cj = a.perm[jj];
                        for (int bb = 0; bb < B; ++bb) {
                            if (a.ncomp == 3) {
                                o[3 + 3 * bb + 0] = (T)a.r[((int64_t)bb * a.M + cj) * 3 + 0];
                                o[3 + 3 * bb + 1] = (T)a.r[((int64_t)bb * a.M + cj) * 3 + 1];
                                o[3 + 3 * bb + 2] = (T)a.r[((int64_t)bb * a.M + cj) * 3 + 2];
                            } else {
                                o[3 + 3 * bb + 0] = T(0);
                                o[3 + 3 * bb + 1] = T(0);
                                o[3 + 3 * bb + 2] = (T)a.r[(int64_t)bb * a.M + cj];
                            }
                        }
                    }
                    __syncwarp();
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const int v = vv[u];
                        if (v >= b3) continue;
                        const int vx = v % b, vy = (v / b) % b, vz = v / (b * b);
                        for (int q = 0; q < a.nq; ++q) {
                            const T sx = T(vx) + (T)(0.5 + 0.5 * a.qr->xi[q][0]) - half_b;
                            const T sy = T(vy) + (T)(0.5 + 0.5 * a.qr->xi[q][1]) - half_b;
                            const T sz = T(vz) + (T)(0.5 + 0.5 * a.qr->xi[q][2]) - half_b;
                            const T wq = (T)a.qr->wn[q];
                            for (int s = 0; s < cnt; ++s) {
                                const T *o = os + s * ostride;
                                const T ddx = o[0] - sx, ddy = o[1] - sy, ddz = o[2] - sz;
                                const T r2 = ddx * ddx + ddy * ddy + ddz * ddz;
                                T ri = T(0);
                                if (r2 > eps2) ri = T(1) / sqrt(r2);
                                const T k3 = wq * ri * ri * ri;
#pragma unroll
                                for (int bb = 0; bb < kAdjMaxB; ++bb)
                                    if (bb < B)
                                        part[u][bb] += k3 * (o[3 + 3 * bb] * ddx + o[4 + 3 * bb] * ddy +
                                                             o[5 + 3 * bb] * ddz);
                            }
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < 2; ++u)
#pragma unroll
                    for (int bb = 0; bb < kAdjMaxB; ++bb)
                        if (bb < B) two_sum_a(hi[u][bb], lo[u][bb], part[u][bb]);
            }
            // far part and scatter
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int v = vv[u];
                if (v >= b3) continue;
                const int64_t gi = Sx * b + v % b - a.voff[0], gj = Sy * b + (v / b) % b - a.voff[1],
                              gk = Sz * b + v / (b * b) - a.voff[2];
                const bool in = gi >= 0 && gj >= 0 && gk >= 0 && gi < a.gn[0] && gj < a.gn[1] && gk < a.gn[2];
                for (int bb = 0; bb < B && bb < kAdjMaxB; ++bb) {
                    const T *mer = me + (sl * B + bb) * a.ldk;
                    double far = 0.0;
                    for (int k = 0; k < a.K; ++k) far += (double)P[(size_t)v * a.K + k] * (double)mer[k];
                    if (in) {
                        const double val = ((double)hi[u][bb] + (double)lo[u][bb] + far) * a.scale;
                        a.grad[(int64_t)bb * a.gn[0] * a.gn[1] * a.gn[2] + (gk * a.gn[1] + gj) * a.gn[0] + gi] = val;
                    }
                }
            }
        }
    }
}

}  // namespace

gf_status fmm_adjoint_prepare(gf_plan_s *plan, cudaStream_t st) {
    FmmPlan *F = plan->fmm;
    DeviceArena &A = plan->arena;
    for (int l = 2; l <= F->L; ++l) {
        FmmLevel &lv = F->lev[l];
        int64_t n = 1;
        for (int d = 0; d < 3; ++d) {
            F->mlo[l][d] = lv.slo[d] - 3;
            F->mn[l][d] = lv.sn[d] + 6;
            n *= F->mn[l][d];
        }
        GF_TRY(A.alloc_n(&F->imap[l], n));
        GF_CUDA(cudaMemsetAsync(F->imap[l], 0xff, sizeof(int32_t) * n, st));
        if (lv.nt > 0) {
            fill_imap<<<ceil_div(lv.nt, 256), 256, 0, st>>>(lv.tkey, lv.nt, F->mlo[l][0], F->mlo[l][1], F->mlo[l][2],
                                                            F->mn[l][0], F->mn[l][1], F->mn[l][2], F->imap[l]);
            GF_KERNEL_DONE();
        }
        if (l < F->L) {
            GF_TRY(A.alloc_n(&F->child[l], std::max<int64_t>(lv.nt, 1) * 8));
            GF_CUDA(cudaMemsetAsync(F->child[l], 0xff, sizeof(int32_t) * std::max<int64_t>(lv.nt, 1) * 8, st));
            const FmmLevel &ch = F->lev[l + 1];
            if (ch.nt > 0) {
                fill_child<<<ceil_div(ch.nt, 256), 256, 0, st>>>(ch.tkey, ch.tparent, ch.nt, F->child[l]);
                GF_KERNEL_DONE();
            }
        }
        // source boxes per parity class
        F->scls_off[l][0] = 0;
        for (int c = 0; c < 8; ++c) {
            int64_t cnt = 1;
            for (int d = 0; d < 3; ++d) {
                const int64_t par = (c >> d) & 1;
                const int64_t i0 = (par - (lv.slo[d] & 1) + 2) & 1;
                cnt *= lv.sn[d] > i0 ? (lv.sn[d] - i0 + 1) / 2 : 0;
            }
            F->scls_off[l][c + 1] = F->scls_off[l][c] + cnt;
        }
    }
    return GF_OK;
}

namespace {

template <class T>
gf_status run_adjoint(gf_plan_s *plan, const double *r, int ncomp, int B, double *grad, cudaStream_t st) {
    FmmPlan *F = plan->fmm;
    const int K = F->K, L = F->L;
    const FmmLevel &leaf = F->lev[L];
    // E^T: dual local expansions of the observer leaves
    if (leaf.nt > 0) {
        const int nh = F->p * (F->p + 1) / 2;
        const size_t shm = sizeof(T) * (2 * nh + (size_t)B * K + 3 * B);
        GF_TRY(ensure_smem(l2p_adj<T>, shm));
        l2p_adj<T><<<(unsigned)leaf.nt, 128, shm, st>>>(F->leaf_beg, F->perm,
                                                        sizeof(T) == 8 ? (const T *)F->tloc_d : (const T *)F->tloc_f,
                                                        r, ncomp, plan->M, B, F->p, K, F->KS, F->b, (T *)leaf.le);
        GF_KERNEL_DONE();
    }
    // L^T: children to parents (the transpose of the top FP64 translation
    // stays in FP64 in mixed precision)
    for (int l = L - 1; l >= 2; --l) {
        if (sizeof(T) == 4 && l <= 2)
            GF_TRY((translate_run<T, double>(plan, l, 3, B, st)));
        else
            GF_TRY((translate_run<T, T>(plan, l, 3, B, st)));
    }
    // M2L^T at every level (overwrites the dual multipole expansions)
    GF_TRY(m2l_run<T>(plan, B, true, st));
    // M2M^T: parents to children, top down
    for (int l = 3; l <= L; ++l) {
        if (sizeof(T) == 4 && l - 1 <= 2)
            GF_TRY((translate_run<T, double>(plan, l, 2, B, st)));
        else
            GF_TRY((translate_run<T, T>(plan, l, 2, B, st)));
    }
    // P^T and N^T, scaled by G h, scattered to grid order
    AdjArgs a;
    a.leaf_beg = F->leaf_beg;
    a.perm = F->perm;
    a.tloc = sizeof(T) == 8 ? (const void *)F->tloc_d : (const void *)F->tloc_f;
    a.r = r;
    a.ncomp = ncomp;
    a.M = plan->M;
    a.B = B;
    a.K = K;
    a.ldk = F->KS;
    a.b = F->b;
    a.nq = F->nq;
    a.p = F->p;
    a.imap = F->imap[L];
    for (int d = 0; d < 3; ++d) {
        a.mlo[d] = F->mlo[L][d];
        a.mn[d] = F->mn[L][d];
        a.blo[d] = leaf.slo[d];
        a.bn[d] = leaf.sn[d];
        a.gn[d] = plan->grid.n[d];
        a.voff[d] = F->voff[d];
    }
    a.me = leaf.me;
    a.P = sizeof(T) == 8 ? (const void *)F->p2m_d : (const void *)F->p2m_f;
    a.qr = quad_device(plan);
    a.scale = plan->G * F->h;
    a.eps2 = sizeof(T) == 8 ? 1e-18 : 1e-12;
    a.grad = grad;
    const int64_t nleaf = leaf.ns;
    const size_t shm = sizeof(T) * kAdjWarps * kAdjChunk * (3 + 3 * B);
    GF_TRY(ensure_smem(adj_eval<T>, shm));
    const unsigned grid = (unsigned)std::min<int64_t>((nleaf + kAdjWarps - 1) / kAdjWarps, 152 * 32);
    adj_eval<T><<<grid, kAdjWarps * 32, shm, st>>>(a);
    GF_KERNEL_DONE();
    return GF_OK;
}

}  // namespace

gf_status fmm_adjoint(gf_plan_s *plan, const double *r, int ncomp, int B, double *grad, cudaStream_t st) {
    if (B > kAdjMaxB) {
        set_error("the FMM adjoint takes at most %d batch members per call", kAdjMaxB);
        return GF_ERR_UNSUPPORTED;
    }
    if (plan->M == 0) {
        GF_CUDA(cudaMemsetAsync(grad, 0, sizeof(double) * B * plan->nvox, st));
        return GF_OK;
    }
    FmmPlan *F = plan->fmm;
    if (!F->adj_ready) {   // adjoint-only structures, built once per plan
        GF_TRY(fmm_adjoint_prepare(plan, plan->arena.stream));
        GF_TRY(m2l_tc_prepare_adj(plan));
        GF_CUDA(cudaStreamSynchronize(plan->arena.stream));
        F->adj_ready = true;
    }
    if (plan->fmm->mixed) return run_adjoint<float>(plan, r, ncomp, B, grad, st);
    return run_adjoint<double>(plan, r, ncomp, B, grad, st);
}

}  // namespace gf
