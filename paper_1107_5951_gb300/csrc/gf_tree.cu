// gf_tree.cu -- Morton-sorted octree of a FMM plan (Sec. 2.3, "Hierarchical
// space decomposition"): root geometry, observer keys and their stable sort,
// occupied boxes of every level, parity-grouped M2L order, observer offsets
// from their leaf centres and the evaluation work list.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "gf_fmm.cuh"
#include "gf_prim.cuh"
#include "gf_simd.cuh"

namespace gf {
namespace {

__device__ __forceinline__ uint64_t spread3(uint64_t v) {
    // insert two zero bits between the low 21 bits of v
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

__device__ __forceinline__ uint64_t compact3(uint64_t v) {
    v &= 0x1249249249249249ull;
    v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ull;
    v = (v ^ (v >> 4)) & 0x100f00f00f00f00full;
    v = (v ^ (v >> 8)) & 0x1f0000ff0000ffull;
    v = (v ^ (v >> 16)) & 0x1f00000000ffffull;
    v = (v ^ (v >> 32)) & 0x1fffffull;
    return v;
}

__device__ __forceinline__ uint64_t morton(int64_t x, int64_t y, int64_t z) {
    return spread3((uint64_t)x) | (spread3((uint64_t)y) << 1) | (spread3((uint64_t)z) << 2);
}

__device__ __forceinline__ void demorton(uint64_t k, int64_t &x, int64_t &y, int64_t &z) {
    x = (int64_t)compact3(k);
    y = (int64_t)compact3(k >> 1);
    z = (int64_t)compact3(k >> 2);
}

struct Geo {
    double lo[3];
    double inv_s, h, inv_h;
    int L, b;
    // FP32 copies for the fast paths (FP64 arithmetic and conversions are
    // slow on this GPU): lo, 1/s; and the fixed-point form of the leaf
    // centres, k fractional bits (k < 0: not used), lo and half a leaf side
    // in those units, 2^-k / h
    float lof[3], isf;
    int fixk;
    long long lofix[3], halfleaf_fix;
    float fix_to_vox;
};

// Leaf key of every observer: floor((x - lo) * inv_s) with one rounded
// subtraction and one rounded multiplication, clamped to the root.
__global__ void obs_keys(const double *__restrict__ obs, int64_t M, Geo g, uint64_t *__restrict__ keys,
                         int32_t *__restrict__ vals, int *__restrict__ status) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    const float top = (float)((1ll << g.L) - 1);
    int64_t c[3];
    for (int a = 0; a < 3; ++a) {
        const double x = obs[3 * j + a];
        if ((((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ff) == 0x7ff) atomicOr(status + 2, 1);
        // The box index is floor((x - lo) / s) evaluated in FP64 (the rounding
        // the tree is defined with).  FP32 gets it right unless the value is
        // within a few FP32 roundings of an integer, and FP64 is slow on this
        // GPU, so FP64 is used only there.
        float xf;
        const bool fin = trunc_f32(x, xf);
        const float qf = (xf - g.lof[a]) * g.isf;
        float fl = floorf(qf);
        const float dist = fminf(qf - fl, fl + 1.f - qf);
        const float tol = ((fabsf(xf) + fabsf(g.lof[a])) * fabsf(g.isf) + fabsf(qf) + 1.f) * 2e-6f;
        if (!fin || !(dist > tol))
            fl = (float)fmin(fmax(floor(__dmul_rn(__dsub_rn(x, g.lo[a]), g.inv_s)), -1.0), (double)top + 1.0);
        fl = fminf(fmaxf(fl, 0.f), top);
        c[a] = (int64_t)fl;
    }
    keys[j] = morton(c[0], c[1], c[2]);
    vals[j] = (int32_t)j;
}

// The tree is built without host round trips: counts stay on the device
// (d_n; nullptr: the host count n), kernels run over an upper bound ub and
// treat indices past the count as absent.
__device__ __forceinline__ int64_t dev_count(const int64_t *d_n, int64_t n) { return d_n ? *d_n : n; }

__global__ void mark_new(const uint64_t *__restrict__ keys, const int64_t *d_n, int64_t n, int64_t ub, int shift,
                         int64_t *__restrict__ flags) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ub) return;
    const int64_t cnt = dev_count(d_n, n);
    flags[i] = (i < cnt && (i == 0 || (keys[i] >> shift) != (keys[i - 1] >> shift))) ? 1 : 0;
}

// After an exclusive scan of the flags: write the unique (shifted) keys, the
// first index of each run, and the run index of every element.
// (also: the number of runs, excl[ub], into *runs)
__global__ void compact_runs(const uint64_t *__restrict__ keys, const int64_t *d_n, int64_t n, int64_t ub, int shift,
                             const int64_t *__restrict__ excl, uint64_t *__restrict__ ukeys,
                             int32_t *__restrict__ beg, int32_t *__restrict__ run_of, int64_t *__restrict__ runs) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *runs = excl[ub];
    if (i >= dev_count(d_n, n)) return;
    const bool nw = (i == 0 || (keys[i] >> shift) != (keys[i - 1] >> shift));
    const int64_t e = excl[i];
    if (nw) {
        ukeys[e] = keys[i] >> shift;
        if (beg) beg[e] = (int32_t)i;
    }
    if (run_of) run_of[i] = (int32_t)(nw ? e : e - 1);
}

__global__ void set_last(int32_t *__restrict__ a, const int64_t *d_idx, int32_t v) { a[*d_idx] = v; }

// Every ancestor level of the leaves in one block: for l = L-1 down to 1 the
// occupied boxes of level l are the distinct keys (child key >> 3) of the
// sorted boxes of level l+1, in order; each child records its parent's
// index.  1024 children per round, a ballot-based block scan of the "new
// parent" flags.  Used when the leaves are few (one block keeps up).
struct AncArgs {
    uint64_t *tkey[kMaxLevels + 1];
    int32_t *tparent[kMaxLevels + 1];
};

constexpr int kAncThreads = 1024;
constexpr int64_t kAncMaxLeaves = 65536;

__global__ void __launch_bounds__(kAncThreads) ancestors_small(AncArgs a, int L, int64_t *__restrict__ cnt) {
    __shared__ int warp_excl[kAncThreads / 32];
    __shared__ int64_t s_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int64_t n = cnt[L];
    for (int l = L - 1; l >= 1; --l) {
        const uint64_t *ck = a.tkey[l + 1];
        uint64_t *pk = a.tkey[l];
        int32_t *par = a.tparent[l + 1];
        if (tid == 0) s_base = 0;
        __syncthreads();
        for (int64_t c0 = 0; c0 < n; c0 += kAncThreads) {
            const int64_t i = c0 + tid;
            const bool in = i < n;
            const uint64_t key = in ? ck[i] >> 3 : 0;
            const bool nw = in && (i == 0 || (ck[i - 1] >> 3) != key);
            const unsigned bal = __ballot_sync(0xffffffffu, nw);
            const int wpre = __popc(bal & ((1u << lane) - 1u));
            if (lane == 0) warp_excl[warp] = __popc(bal);
            __syncthreads();
            if (warp == 0) {
                const int t = warp_excl[lane];
                int incl = t;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int u = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += u;
                }
                warp_excl[lane] = incl - t;
            }
            __syncthreads();
            const int64_t base = s_base;
            const int64_t e = base + warp_excl[warp] + wpre;   // parents before this child's run start
            if (nw) pk[e] = key;
            if (in) par[i] = (int32_t)(nw ? e : e - 1);
            __syncthreads();
            if (tid == kAncThreads - 1) s_base = e + (nw ? 1 : 0);
            __syncthreads();
        }
        n = s_base;
        if (tid == 0) cnt[l] = n;
        __syncthreads();
    }
}

__global__ void obs_local(const double *__restrict__ obs, const int32_t *__restrict__ perm,
                          const uint64_t *__restrict__ okey, int64_t M, Geo g, float *__restrict__ tf,
                          double *__restrict__ td) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const int64_t j = perm[i];
    int64_t c[3];
    demorton(okey[i], c[0], c[1], c[2]);
    for (int a = 0; a < 3; ++a) {
        if (tf && g.fixk >= 0) {
            // FP32 output: the offset from the leaf centre in fixed point (an
            // exact integer difference), then scaled to voxel units in FP32
            const long long d = to_fix(obs[3 * j + a], g.fixk) - (g.lofix[a] + (2 * c[a] + 1) * g.halfleaf_fix);
            tf[3 * i + a] = fix_to_f32(d) * g.fix_to_vox;
            continue;
        }
        // voxel units by a multiply (FP64 division is a long sequence on this
        // GPU); the last-bit difference from dividing stays far below the
        // coincidence radius
        const double u = (obs[3 * j + a] - g.lo[a]) * g.inv_h;
        const double loc = u - ((double)c[a] * g.b + 0.5 * g.b);
        if (td) td[3 * i + a] = loc;
        if (tf) tf[3 * i + a] = (float)loc;
    }
}

constexpr int kItemTargets = 64;   // targets per evaluation work item (2 per lane)

// ---- observer boxes of every level 2..L grouped by parity class (the M2L
// order; stable: ascending box index within a class), three launches for
// all levels: per-block class counts, one scan, a stable scatter.  Blocks
// of 1024 boxes; the counts are laid out [level][class][block] so that the
// scan gives each (level, class, block) its first position, measured from
// the level's first entry.
constexpr int kClsBlock = 1024;
struct ClsArgs {
    const uint64_t *tkey[kMaxLevels + 1];
    int32_t *order[kMaxLevels + 1];
    const int64_t *cnt;               // boxes per level (device)
    int64_t first_block[kMaxLevels + 2];   // blocks of levels 2..L, prefix
    int64_t nblk[kMaxLevels + 1];
    int64_t entry0[kMaxLevels + 2];   // first count entry of each level
    int lmin, lmax;
    int64_t *bc;                      // [entries + 1] counts, then their scan
    int *ccnt;                        // [8 l + c] boxes per class
};

__device__ __forceinline__ void cls_locate(const ClsArgs &a, int &l, int64_t &blk) {
    l = a.lmin;
    while (l < a.lmax && (int64_t)blockIdx.x >= a.first_block[l + 1]) ++l;
    blk = (int64_t)blockIdx.x - a.first_block[l];
}

__global__ void __launch_bounds__(kClsBlock) cls_count(ClsArgs a) {
    __shared__ int c8[8];
    int l;
    int64_t blk;
    cls_locate(a, l, blk);
    if (threadIdx.x < 8) c8[threadIdx.x] = 0;
    __syncthreads();
    const int64_t i = blk * kClsBlock + threadIdx.x;
    if (i < a.cnt[l]) atomicAdd(&c8[(int)(a.tkey[l][i] & 7)], 1);
    __syncthreads();
    if (threadIdx.x < 8) a.bc[a.entry0[l] + threadIdx.x * a.nblk[l] + blk] = c8[threadIdx.x];
}

__global__ void __launch_bounds__(kClsBlock) cls_scatter(ClsArgs a) {
    __shared__ int wc[kClsBlock / 32][8];
    int l;
    int64_t blk;
    cls_locate(a, l, blk);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = blk * kClsBlock + threadIdx.x;
    const bool in = i < a.cnt[l];
    const int c = in ? (int)(a.tkey[l][i] & 7) : 8;
    const unsigned peers = __match_any_sync(0xffffffffu, c);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    if (threadIdx.x < kClsBlock / 32 * 8) wc[threadIdx.x >> 3][threadIdx.x & 7] = 0;
    __syncthreads();
    if (in && rank == 0) wc[warp][c] = __popc(peers);
    __syncthreads();
    if (threadIdx.x < 8) {   // exclusive prefix over the warps, per class
        int acc = 0;
        for (int w = 0; w < kClsBlock / 32; ++w) {
            const int t = wc[w][threadIdx.x];
            wc[w][threadIdx.x] = acc;
            acc += t;
        }
    }
    __syncthreads();
    const int64_t base = a.bc[a.entry0[l]];
    if (in) a.order[l][a.bc[a.entry0[l] + c * a.nblk[l] + blk] - base + wc[warp][c] + rank] = (int32_t)i;
    if (blk == 0 && threadIdx.x < 8) {
        const int64_t e = a.entry0[l] + threadIdx.x * a.nblk[l];
        const int64_t next = threadIdx.x < 7 ? e + a.nblk[l] : a.entry0[l + 1];
        a.ccnt[8 * l + threadIdx.x] = (int)(a.bc[next] - a.bc[e]);
    }
}

__global__ void item_counts(const int32_t *__restrict__ beg, const int64_t *d_nleaf, int64_t ub,
                            int64_t *__restrict__ cnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ub) return;
    const int64_t n = i < *d_nleaf ? beg[i + 1] - beg[i] : 0;
    cnt[i] = (n + kItemTargets - 1) / kItemTargets;
}

// (also: the number of items, off[ub], into *nitems)
__global__ void item_fill(const int32_t *__restrict__ beg, const int64_t *d_nleaf, int64_t ub,
                          const int64_t *__restrict__ off, int4 *__restrict__ items, int64_t *__restrict__ nitems) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *nitems = off[ub];
    if (i >= *d_nleaf) return;
    const int b0 = beg[i], b1 = beg[i + 1];
    int64_t o = off[i];
    for (int f = b0; f < b1; f += kItemTargets) items[o++] = make_int4((int)i, f, min(kItemTargets, b1 - f), 0);
}

// Interaction list (316 offsets, dz/dy/dx ascending, max-norm >= 2) and near
// list (27 offsets) of observer boxes, as source box Morton keys or -1.
__global__ void export_lists(const uint64_t *__restrict__ tkey, int64_t nt, int level, int64_t slo0,
                             int64_t slo1, int64_t slo2, int64_t shi0, int64_t shi1, int64_t shi2,
                             int64_t *__restrict__ il, int64_t *__restrict__ nearl) {
    const int64_t t = (int64_t)blockIdx.x;
    if (t >= nt) return;
    int64_t x, y, z;
    demorton(tkey[t], x, y, z);
    for (int u = threadIdx.x; u < 343; u += blockDim.x) {
        const int dx = u % 7 - 3, dy = (u / 7) % 7 - 3, dz = u / 49 - 3;
        const int mx = max(abs(dx), max(abs(dy), abs(dz)));
        const int64_t sx = x + dx, sy = y + dy, sz = z + dz;
        const bool inblk = sx >= slo0 && sx <= shi0 && sy >= slo1 && sy <= shi1 && sz >= slo2 && sz <= shi2;
        if (mx >= 2 && il) {
            // rank of u among the 316 offsets with max-norm >= 2
            int r = 0;
            for (int w = 0; w < u; ++w) {
                const int ax = w % 7 - 3, ay = (w / 7) % 7 - 3, az = w / 49 - 3;
                if (max(abs(ax), max(abs(ay), abs(az))) >= 2) ++r;
            }
            const bool adj = level >= 2 && llabs((sx >> 1) - (x >> 1)) <= 1 && llabs((sy >> 1) - (y >> 1)) <= 1 &&
                             llabs((sz >> 1) - (z >> 1)) <= 1;
            il[t * 316 + r] = (inblk && adj && sx >= 0 && sy >= 0 && sz >= 0) ? (int64_t)morton(sx, sy, sz) : -1;
        }
        if (mx <= 1 && nearl) {
            const int r = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
            nearl[t * 27 + r] = (inblk && sx >= 0 && sy >= 0 && sz >= 0) ? (int64_t)morton(sx, sy, sz) : -1;
        }
    }
}

// Work counts for the roofline: near-field (observer, source) pairs and
// interaction-list (observer box, source box) pairs.
__global__ void count_near(const uint64_t *__restrict__ tkey, const int32_t *__restrict__ beg, int64_t nt,
                           int64_t slo0, int64_t slo1, int64_t slo2, int64_t sn0, int64_t sn1, int64_t sn2,
                           int64_t per_leaf, unsigned long long *__restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    int64_t x, y, z;
    demorton(tkey[t], x, y, z);
    int cnt = 0;
    for (int d = 0; d < 27; ++d) {
        const int64_t sx = x + d % 3 - 1 - slo0, sy = y + (d / 3) % 3 - 1 - slo1, sz = z + d / 9 - 1 - slo2;
        cnt += (sx >= 0 && sy >= 0 && sz >= 0 && sx < sn0 && sy < sn1 && sz < sn2);
    }
    const unsigned long long v = (unsigned long long)((int64_t)cnt * per_leaf * (beg[t + 1] - beg[t]));
    atomicAdd(out, v);
}

__global__ void count_il(const uint64_t *__restrict__ tkey, int64_t nt, int64_t slo0, int64_t slo1, int64_t slo2,
                         int64_t sn0, int64_t sn1, int64_t sn2, unsigned long long *__restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    int64_t x, y, z;
    demorton(tkey[t], x, y, z);
    int cnt = 0;
    for (int u = 0; u < 343; ++u) {
        const int dx = u % 7 - 3, dy = (u / 7) % 7 - 3, dz = u / 49 - 3;
        if (max(abs(dx), max(abs(dy), abs(dz))) <= 1) continue;
        const int64_t sx = x + dx, sy = y + dy, sz = z + dz;
        if (llabs((sx >> 1) - (x >> 1)) > 1 || llabs((sy >> 1) - (y >> 1)) > 1 || llabs((sz >> 1) - (z >> 1)) > 1)
            continue;
        cnt += (sx >= slo0 && sy >= slo1 && sz >= slo2 && sx < slo0 + sn0 && sy < slo1 + sn1 && sz < slo2 + sn2);
    }
    atomicAdd(out, (unsigned long long)cnt);
}

int default_leaf_vox(int nq) {
    int b = (int)lround(cbrt(64.0 / nq));
    return b < 1 ? 1 : b;
}

}  // namespace

void il_offsets_host(int cls, signed char out[189][3]) {
    const int px = cls & 1, py = (cls >> 1) & 1, pz = (cls >> 2) & 1;
    int r = 0;
    for (int dz = -3; dz <= 3; ++dz)
        for (int dy = -3; dy <= 3; ++dy)
            for (int dx = -3; dx <= 3; ++dx) {
                if (std::max(abs(dx), std::max(abs(dy), abs(dz))) <= 1) continue;
                // parent offset of (box + d) relative to the box's parent
                const int qx = (px + dx) >> 1, qy = (py + dy) >> 1, qz = (pz + dz) >> 1;
                if (abs(qx) > 1 || abs(qy) > 1 || abs(qz) > 1) continue;
                out[r][0] = (signed char)dx;
                out[r][1] = (signed char)dy;
                out[r][2] = (signed char)dz;
                ++r;
            }
}

size_t fmm_bytes_estimate(const gf_grid *grid, int nq, int64_t M, const gf_options *opt) {
    const int b = opt->leaf_vox > 0 ? opt->leaf_vox : default_leaf_vox(nq);
    const int K = (opt->p + 1) * (opt->p + 1);
    const size_t rs = opt->precision == GF_PREC_MIXED ? 4 : 8;
    double nleaf = 1.0;
    for (int a = 0; a < 3; ++a) nleaf *= (double)((grid->n[a] + b - 1) / b + 1);
    const double nsrc = nleaf * 8.0 / 7.0;
    const double ntgt = std::min<double>((double)M, nleaf * 4.0) * 8.0 / 7.0 + 64;
    double bytes = (nsrc + ntgt) * K * rs * opt->max_batch;
    bytes += nleaf * b * b * b * rs * opt->max_batch;          // blocked densities
    if (opt->precision == GF_PREC_MIXED)                         // M2L inputs split into FP16 parts
        bytes += nsrc * ((K + 31) / 32 * 32) * 4.0 * opt->max_batch;
    bytes += (double)M * (8 + 4 + 4 + 12 + 24) + ntgt * 24;       // keys, perm, locals, box tables
    bytes += (double)M * 32 + 8e6;                                // sort buffers and scratch
    return (size_t)bytes;
}

gf_status fmm_create(gf_plan_s *plan, const double *obs, cudaStream_t st) {
    FmmPlan *F = new (std::nothrow) FmmPlan();
    if (!F) {
        set_error("host allocation failed");
        return GF_ERR_OOM;
    }
    plan->fmm = F;
    const gf_grid &gr = plan->grid;
    const int64_t M = plan->M;
    F->p = plan->opt.p;
    F->K = (F->p + 1) * (F->p + 1);
    F->B = plan->opt.max_batch;
    F->nq = plan->quad.nq;
    F->mixed = plan->opt.precision == GF_PREC_MIXED;
    F->m2l_tc64 = !F->mixed && (plan->opt.reserved0 & GF_FLAG_M2L_TENSOR);
    F->b = plan->opt.leaf_vox > 0 ? plan->opt.leaf_vox : default_leaf_vox(F->nq);
    F->h = gr.h[0];
    DeviceArena &A = plan->arena;

    // ---- root geometry: observers' bounding box joined with the grid
    double bb[6];
    double obs_zlo = 0.0, obs_zhi = 0.0, obs_lo[3] = {0.0, 0.0, 0.0}, obs_hi[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < 3; ++a) {
        bb[a] = gr.origin[a];
        bb[3 + a] = gr.origin[a] + gr.n[a] * F->h;
    }
    if (M > 0) {
        double *d_bb;
        GF_TRY(A.alloc_n(&d_bb, 6 + 6 * 256));
        GF_TRY(bbox3(obs, M, d_bb, st));
        double ob[6];
        GF_CUDA(cudaMemcpyAsync(ob, d_bb, sizeof(ob), cudaMemcpyDeviceToHost, st));
        GF_CUDA(cudaStreamSynchronize(st));
        for (int a = 0; a < 3; ++a) {
            if (!isfinite(ob[a]) || !isfinite(ob[3 + a])) {
                set_error("observer coordinates must be finite");
                return GF_ERR_INVALID_ARG;
            }
            bb[a] = std::min(bb[a], ob[a]);
            bb[3 + a] = std::max(bb[3 + a], ob[3 + a]);
        }
        obs_zlo = ob[2];
        obs_zhi = ob[5];
        for (int a = 0; a < 3; ++a) {
            obs_lo[a] = ob[a];
            obs_hi[a] = ob[3 + a];
        }
    }
    int64_t need = 1;
    for (int a = 0; a < 3; ++a) {
        const double below = (gr.origin[a] - bb[a]) / F->h;
        F->voff[a] = below > 0 ? (int64_t)ceil(below) : 0;
        F->lo[a] = gr.origin[a] - (double)F->voff[a] * F->h;
        const double ext = ceil((bb[3 + a] - F->lo[a]) / F->h);
        need = std::max<int64_t>(need, std::max<int64_t>(F->voff[a] + gr.n[a], (int64_t)ext));
    }
    double oz[2] = {bb[2], bb[5]};   // observers' z extent (the grid's when M = 0)
    if (M > 0) {
        oz[0] = obs_zlo;
        oz[1] = obs_zhi;
    }
    int L = 2;
    while (((int64_t)F->b << L) < need) ++L;
    if (L > kMaxLevels - 1) {
        set_error("observers span %lld voxels: the octree would need %d levels (max %d)",
                  (long long)need, L, kMaxLevels - 1);
        return GF_ERR_UNSUPPORTED;
    }
    F->L = L;
    F->s_leaf = F->b * F->h;
    F->inv_s = 1.0 / F->s_leaf;
    for (int l = 0; l <= L; ++l) {
        FmmLevel &lv = F->lev[l];
        lv.ns = 1;
        for (int a = 0; a < 3; ++a) {
            const int64_t lo = (F->voff[a] / F->b) >> (L - l);
            const int64_t hi = ((F->voff[a] + gr.n[a] - 1) / F->b) >> (L - l);
            lv.slo[a] = lo;
            lv.sn[a] = hi - lo + 1;
            lv.ns *= lv.sn[a];
        }
    }
    return fmm_observer_tree(plan, obs, oz, obs_lo, obs_hi, bb, st);
}

int fixed_point_frame(const FmmPlan *F, const double bb[6], long long lofix[3], long long *halfleaf_fix,
                      float *fix_to_unit) {
    // k fractional bits such that every coordinate of the observers, the
    // sources and the root box stays below 2^61 in magnitude
    double xmax = 0.0;
    for (int a = 0; a < 3; ++a)
        xmax = std::max({xmax, std::fabs(bb[a]), std::fabs(bb[3 + a]), std::fabs(F->lo[a]),
                         std::fabs(F->lo[a] + std::ldexp(F->s_leaf, F->L))});
    int ex = 0;
    std::frexp(std::max(xmax, 1e-300), &ex);   // xmax < 2^ex
    const int k = std::min(80, 61 - ex);
    if (k < 0) return -1;
    const double hl = 0.5 * F->b * F->h;
    for (int a = 0; a < 3; ++a) lofix[a] = (long long)std::llround(std::ldexp(F->lo[a], k));
    *halfleaf_fix = (long long)std::llround(std::ldexp(hl, k));
    *fix_to_unit = (float)(std::ldexp(1.0, -k) / F->h);
    return k;
}

// The observer side of the tree, for a root geometry already set in the
// plan (F->lo, F->s_leaf, F->L and the source block of every level): the
// M2L's reachable source slabs, observer keys and their stable sort, the
// leaves and every ancestor level, the parity-class order, the observers'
// offsets from their leaf centres and the evaluation work items; then the
// expansion workspaces.  oz: the observers' z extent; obs_lo/obs_hi: their
// bounding box; bb: the root geometry's bounding box (observers joined with
// the sources).
gf_status fmm_observer_tree(gf_plan_s *plan, const double *obs, const double oz[2], const double obs_lo[3],
                            const double obs_hi[3], const double bb[6], cudaStream_t st) {
    FmmPlan *F = plan->fmm;
    const int64_t M = plan->M;
    const int L = F->L;
    DeviceArena &A = plan->arena;
    {
        // Source z-slabs the M2L of each level reads: observer boxes lie in
        // the leaf z-range of the observers' extent (widened by one leaf
        // against rounding at box faces), and interaction-list offsets reach
        // three boxes along each axis.
        const int64_t top = ((int64_t)1 << L) - 1;
        const int64_t iz0 = std::max<int64_t>(0, (int64_t)floor((oz[0] - F->lo[2]) * F->inv_s) - 1);
        const int64_t iz1 = std::min<int64_t>(top, (int64_t)floor((oz[1] - F->lo[2]) * F->inv_s) + 1);
        for (int l = 2; l <= L; ++l) {
            FmmLevel &lv = F->lev[l];
            lv.m2l_z0 = std::max<int64_t>(0, (iz0 >> (L - l)) - 3 - lv.slo[2]);
            lv.m2l_z1 = std::min<int64_t>(lv.sn[2] - 1, (iz1 >> (L - l)) + 3 - lv.slo[2]);
        }
    }
    Geo g;
    for (int a = 0; a < 3; ++a) g.lo[a] = F->lo[a];
    g.inv_s = F->inv_s;
    g.h = F->h;
    g.inv_h = 1.0 / F->h;
    g.L = L;
    g.b = F->b;
    for (int a = 0; a < 3; ++a) g.lof[a] = (float)F->lo[a];
    g.isf = (float)F->inv_s;
    g.fixk = fixed_point_frame(F, bb, g.lofix, &g.halfleaf_fix, &g.fix_to_vox);

    // ---- observer keys and stable sort by (key, index)
    const int64_t Mx = std::max<int64_t>(M, 1);
    uint64_t *keys, *keys2;
    int32_t *vals2;
    int64_t *flags;
    GF_TRY(A.alloc_n(&keys, Mx));
    GF_TRY(A.alloc_n(&keys2, Mx));
    GF_TRY(A.alloc_n(&F->perm, Mx));
    GF_TRY(A.alloc_n(&vals2, Mx));
    GF_TRY(A.alloc_n(&flags, Mx + 1));
    void *scratch;
    const size_t scr = std::max(sort_scratch_bytes(Mx), scan_scratch_bytes(Mx + 1));
    GF_TRY(A.alloc(&scratch, scr));
    F->okey = keys;
    if (M > 0) {
        obs_keys<<<ceil_div(M, 256), 256, 0, st>>>(obs, M, g, keys, F->perm, plan->d_status);
        GF_KERNEL_DONE();
        GF_TRY(radix_sort_u64(keys, F->perm, keys2, vals2, M, 3 * L, scratch, st));
    }

    // ---- leaves and their ancestors.  Counts stay on the device (d_cnt:
    // observer boxes per level, then the evaluation items, then boxes per
    // parity class and level) and arrays are sized by upper bounds, so the
    // whole build is one stream of launches with one read-back at the end.
    FmmLevel &leaf = F->lev[L];
    int64_t ub[kMaxLevels + 1];
    {
        // boxes of level l that can hold observers: at most M, 8^l, and the
        // boxes covering the observers' bounding box (leaf indices of its
        // corners, widened by one against rounding at box faces)
        int64_t lo_i[3] = {0, 0, 0}, hi_i[3] = {0, 0, 0};
        const int64_t top = ((int64_t)1 << L) - 1;
        for (int a = 0; a < 3; ++a) {
            const double u0 = M > 0 ? floor((obs_lo[a] - F->lo[a]) * F->inv_s) : 0.0;
            const double u1 = M > 0 ? floor((obs_hi[a] - F->lo[a]) * F->inv_s) : 0.0;
            lo_i[a] = std::min<int64_t>(top, std::max<int64_t>(0, (int64_t)std::max(-1.0, u0) - 1));
            hi_i[a] = std::min<int64_t>(top, std::max<int64_t>(0, (int64_t)std::min((double)top + 1.0, u1) + 1));
        }
        int64_t cap = std::max<int64_t>(M, 1);
        for (int l = L; l >= 0; --l) {
            const int64_t full = (int64_t)1 << std::min(62, 3 * l);
            int64_t box = 1;
            for (int a = 0; a < 3; ++a) box *= (hi_i[a] >> (L - l)) - (lo_i[a] >> (L - l)) + 1;
            cap = std::min(cap, std::min(full, box));
            ub[l] = cap;
        }
    }
    int64_t *d_cnt;   // [0, L]: boxes per level, [kMaxLevels + 1]: items, then the
                      // evaluation kernel's item queue (2 counters)
    int *d_ccnt;      // [8 (kMaxLevels + 1)]: boxes per parity class and level
    GF_TRY(A.alloc_n(&d_cnt, kMaxLevels + 4));
    GF_TRY(A.alloc_n(&d_ccnt, 8 * (kMaxLevels + 1)));
    GF_CUDA(cudaMemsetAsync(d_cnt, 0, sizeof(int64_t) * (kMaxLevels + 4), st));
    F->eval_queue = reinterpret_cast<unsigned long long *>(d_cnt + kMaxLevels + 2);
    GF_CUDA(cudaMemsetAsync(d_ccnt, 0, sizeof(int) * 8 * (kMaxLevels + 1), st));
    GF_TRY(A.alloc_n(&leaf.tkey, ub[L]));
    GF_TRY(A.alloc_n(&F->leaf_beg, ub[L] + 1));
    if (M > 0) {
        mark_new<<<ceil_div(M, 256), 256, 0, st>>>(keys, nullptr, M, M, 0, flags);
        GF_KERNEL_DONE();
        GF_TRY(exclusive_scan_i64(flags, flags, M, scratch, st));
        compact_runs<<<ceil_div(M, 256), 256, 0, st>>>(keys, nullptr, M, M, 0, flags, leaf.tkey, F->leaf_beg,
                                                      nullptr, d_cnt + L);
        GF_KERNEL_DONE();
    }
    set_last<<<1, 1, 0, st>>>(F->leaf_beg, d_cnt + L, (int32_t)M);
    GF_KERNEL_DONE();
    const bool anc_small = ub[L] <= kAncMaxLeaves;
    for (int l = L - 1; l >= 1; --l) {
        FmmLevel &ch = F->lev[l + 1], &pa = F->lev[l];
        GF_TRY(A.alloc_n(&ch.tparent, ub[l + 1]));
        GF_TRY(A.alloc_n(&pa.tkey, ub[l]));
        if (M > 0 && !anc_small) {
            const int64_t u = ub[l + 1];
            mark_new<<<ceil_div(u, 256), 256, 0, st>>>(ch.tkey, d_cnt + l + 1, 0, u, 3, flags);
            GF_KERNEL_DONE();
            GF_TRY(exclusive_scan_i64(flags, flags, u, scratch, st));
            compact_runs<<<ceil_div(u, 256), 256, 0, st>>>(ch.tkey, d_cnt + l + 1, 0, u, 3, flags, pa.tkey, nullptr,
                                                          ch.tparent, d_cnt + l);
            GF_KERNEL_DONE();
        }
    }
    if (M > 0 && anc_small && L >= 2) {
        AncArgs aa;
        memset(&aa, 0, sizeof(aa));
        for (int l = 1; l <= L; ++l) {
            aa.tkey[l] = F->lev[l].tkey;
            aa.tparent[l] = F->lev[l].tparent;
        }
        ancestors_small<<<1, kAncThreads, 0, st>>>(aa, L, d_cnt);
        GF_KERNEL_DONE();
    }

    // ---- per level: observer boxes grouped by parity class (M2L order)
    for (int l = 2; l <= L; ++l) GF_TRY(A.alloc_n(&F->lev[l].m2l_order, ub[l]));
    if (M > 0 && L >= 2) {
        ClsArgs ca;
        memset(&ca, 0, sizeof(ca));
        ca.lmin = 2;
        ca.lmax = L;
        int64_t blocks = 0, entries = 0;
        for (int l = 2; l <= L; ++l) {
            ca.tkey[l] = F->lev[l].tkey;
            ca.order[l] = F->lev[l].m2l_order;
            ca.nblk[l] = (ub[l] + kClsBlock - 1) / kClsBlock;
            ca.first_block[l] = blocks;
            ca.entry0[l] = entries;
            blocks += ca.nblk[l];
            entries += 8 * ca.nblk[l];
        }
        ca.first_block[L + 1] = blocks;
        ca.entry0[L + 1] = entries;
        ca.cnt = d_cnt;
        ca.ccnt = d_ccnt;
        ca.bc = flags;   // entries <= 8 (ub[L] / 1024 + levels) fit in the M + 1 flags
        if (entries + 1 > Mx + 1) GF_TRY(A.alloc_n(&ca.bc, entries + 1));
        cls_count<<<(unsigned)blocks, kClsBlock, 0, st>>>(ca);
        GF_KERNEL_DONE();
        GF_TRY(exclusive_scan_i64(ca.bc, ca.bc, entries, scratch, st));
        cls_scatter<<<(unsigned)blocks, kClsBlock, 0, st>>>(ca);
        GF_KERNEL_DONE();
    }

    // ---- observer offsets from their leaf centres, evaluation work list
    if (F->mixed)
        GF_TRY(A.alloc_n(&F->tloc_f, 3 * Mx));
    else
        GF_TRY(A.alloc_n(&F->tloc_d, 3 * Mx));
    if (M > 0) {
        obs_local<<<ceil_div(M, 256), 256, 0, st>>>(obs, F->perm, keys, M, g, F->tloc_f, F->tloc_d);
        GF_KERNEL_DONE();
    }
    // items: at most one per leaf plus one per kItemTargets observers
    const int64_t item_ub = ub[L] + M / kItemTargets + 1;
    GF_TRY(A.alloc_n(&F->items, item_ub));
    if (M > 0) {
        item_counts<<<ceil_div(ub[L], 256), 256, 0, st>>>(F->leaf_beg, d_cnt + L, ub[L], flags);
        GF_KERNEL_DONE();
        GF_TRY(exclusive_scan_i64(flags, flags, ub[L], scratch, st));
        item_fill<<<ceil_div(ub[L], 256), 256, 0, st>>>(F->leaf_beg, d_cnt + L, ub[L], flags, F->items,
                                                        d_cnt + kMaxLevels + 1);
        GF_KERNEL_DONE();
    }

    // ---- the one read-back: box counts, items, class counts
    int64_t hcnt[kMaxLevels + 2];
    int ccnt[8 * (kMaxLevels + 1)];
    GF_CUDA(cudaMemcpyAsync(hcnt, d_cnt, sizeof(hcnt), cudaMemcpyDeviceToHost, st));
    GF_CUDA(cudaMemcpyAsync(ccnt, d_ccnt, sizeof(ccnt), cudaMemcpyDeviceToHost, st));
    GF_CUDA(cudaStreamSynchronize(st));
    for (int l = 1; l <= L; ++l) F->lev[l].nt = M > 0 ? hcnt[l] : 0;
    F->n_items = M > 0 ? hcnt[kMaxLevels + 1] : 0;
    for (int l = 2; l <= L; ++l) {
        FmmLevel &lv = F->lev[l];
        lv.cls_off[0] = 0;
        for (int c = 0; c < 8; ++c) lv.cls_off[c + 1] = lv.cls_off[c] + ccnt[8 * l + c];
    }
    return fmm_alloc_workspaces(plan, st);
}

// Work counts (near-field pairs, interaction-list box pairs): only reported
// by gf_plan_get_info, so computed on the first request rather than at plan
// build.
gf_status fmm_work_counts(gf_plan_s *plan, cudaStream_t st) {
    FmmPlan *F = plan->fmm;
    DeviceArena &A = plan->arena;
    const int L = F->L;
    const FmmLevel &leaf = F->lev[L];
    const int64_t nleaf = leaf.nt;
    unsigned long long *d_cntw;
    GF_TRY(A.alloc_n(&d_cntw, 2));
    GF_CUDA(cudaMemsetAsync(d_cntw, 0, 2 * sizeof(unsigned long long), st));
    if (F->points) {
        GF_TRY(points_count_near(plan, d_cntw, st));
    } else if (nleaf > 0) {
        count_near<<<ceil_div(nleaf, 256), 256, 0, st>>>(leaf.tkey, F->leaf_beg, nleaf, leaf.slo[0], leaf.slo[1],
                                                         leaf.slo[2], leaf.sn[0], leaf.sn[1], leaf.sn[2],
                                                         (int64_t)F->b * F->b * F->b * F->nq, d_cntw);
        GF_KERNEL_DONE();
    }
    for (int l = 2; l <= L; ++l) {
        const FmmLevel &lv = F->lev[l];
        if (lv.nt == 0) continue;
        count_il<<<ceil_div(lv.nt, 256), 256, 0, st>>>(lv.tkey, lv.nt, lv.slo[0], lv.slo[1], lv.slo[2], lv.sn[0],
                                                       lv.sn[1], lv.sn[2], d_cntw + 1);
        GF_KERNEL_DONE();
    }
    unsigned long long hc[2];
    GF_CUDA(cudaMemcpyAsync(hc, d_cntw, sizeof(hc), cudaMemcpyDeviceToHost, st));
    GF_CUDA(cudaStreamSynchronize(st));
    plan->near_pairs = (int64_t)hc[0];
    plan->m2l_pairs = (int64_t)hc[1];
    plan->counts_done = true;
    return GF_OK;
}

void fmm_destroy(gf_plan_s *plan) {
    delete plan->fmm;
    plan->fmm = nullptr;
}

gf_status fmm_info(const gf_plan_s *plan, gf_plan_info *info) {
    const FmmPlan *F = plan->fmm;
    if (!F) return GF_OK;
    info->p = F->p;
    info->K = F->K;
    info->L = F->L;
    info->leaf_vox = F->b;
    for (int a = 0; a < 3; ++a) {
        info->voxel_offset[a] = F->voff[a];
        info->lo[a] = F->lo[a];
    }
    info->leaf_side = F->s_leaf;
    info->inv_leaf_side = F->inv_s;
    for (int l = 0; l <= F->L && l < 24; ++l) {
        info->n_target_boxes[l] = F->lev[l].nt;
        for (int a = 0; a < 3; ++a) {
            info->src_lo[l][a] = F->lev[l].slo[a];
            info->src_hi[l][a] = F->lev[l].slo[a] + F->lev[l].sn[a] - 1;
        }
    }
    return GF_OK;
}

gf_status fmm_export_tree(gf_plan_s *plan, int level, int32_t *perm, uint64_t *keys, uint64_t *box_keys,
                          int64_t *ilist, int64_t *near_) {
    FmmPlan *F = plan->fmm;
    if (level < 2 || level > F->L) {
        set_error("level %d out of range [2, %d]", level, F->L);
        return GF_ERR_INVALID_ARG;
    }
    cudaStream_t st = 0;
    const FmmLevel &lv = F->lev[level];
    if (perm && plan->M > 0)
        GF_CUDA(cudaMemcpyAsync(perm, F->perm, sizeof(int32_t) * plan->M, cudaMemcpyDeviceToHost, st));
    if (keys && plan->M > 0)
        GF_CUDA(cudaMemcpyAsync(keys, F->okey, sizeof(uint64_t) * plan->M, cudaMemcpyDeviceToHost, st));
    if (box_keys && lv.nt > 0)
        GF_CUDA(cudaMemcpyAsync(box_keys, lv.tkey, sizeof(uint64_t) * lv.nt, cudaMemcpyDeviceToHost, st));
    if ((ilist || (near_ && level == F->L)) && lv.nt > 0) {
        int64_t *d_il = nullptr, *d_near = nullptr;
        DeviceArena tmp;
        tmp.stream = st;
        gf_status s = tmp.alloc_n(&d_il, lv.nt * 316);
        if (s == GF_OK) s = tmp.alloc_n(&d_near, lv.nt * 27);
        if (s != GF_OK) {
            GF_CUDA(cudaStreamSynchronize(st));
            tmp.release();
            return s;
        }
        export_lists<<<(unsigned)lv.nt, 128, 0, st>>>(lv.tkey, lv.nt, level, lv.slo[0], lv.slo[1], lv.slo[2],
                                                      lv.slo[0] + lv.sn[0] - 1, lv.slo[1] + lv.sn[1] - 1,
                                                      lv.slo[2] + lv.sn[2] - 1, d_il, d_near);
        count_launch();
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess && ilist)
            e = cudaMemcpyAsync(ilist, d_il, sizeof(int64_t) * lv.nt * 316, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && near_ && level == F->L)
            e = cudaMemcpyAsync(near_, d_near, sizeof(int64_t) * lv.nt * 27, cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        tmp.release();
        if (e != cudaSuccess) {
            set_error("tree export failed: %s", cudaGetErrorString(e));
            return GF_ERR_CUDA;
        }
    }
    GF_CUDA(cudaStreamSynchronize(st));
    return GF_OK;
}

}  // namespace gf
