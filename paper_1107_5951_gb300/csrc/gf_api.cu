// gf_api.cu -- the C ABI of gf.h: argument validation, plan lifetime,
// dispatch to the direct and FMM paths, error reporting.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <new>
#include <vector>

#include "gf_fmm.cuh"
#include "gf_internal.cuh"

namespace gf {

static thread_local char g_errbuf[512] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_errbuf, sizeof(g_errbuf), fmt, ap);
    va_end(ap);
}

const char *get_error() { return g_errbuf; }

static std::atomic<long long> g_launches{0};
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

static void keep_pool_memory(int device) {
    static std::atomic<unsigned long long> done{0};
    if (device < 0 || device >= 64) return;
    const unsigned long long bit = 1ull << device;
    if (done.load() & bit) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    done.fetch_or(bit);
}

gf_status DeviceArena::alloc(void **p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 16;
    n = (n + 255) & ~size_t(255);
    if (n > left) {
        int dev = 0;
        cudaGetDevice(&dev);
        keep_pool_memory(dev);
        const size_t c = std::max(n, next);
        void *chunk = nullptr;
        cudaError_t e = cudaMallocAsync(&chunk, c, stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("device allocation of %zu bytes failed: %s", c, cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? GF_ERR_OOM : GF_ERR_CUDA;
        }
        blocks.push_back(chunk);
        bytes += c;
        cur = static_cast<unsigned char *>(chunk);
        left = c;
        if (c == next) next = std::min(next * 2, size_t(64) << 20);
    }
    *p = cur;
    cur += n;
    left -= n;
    return GF_OK;
}

// Called only once the device is idle (plan destruction or a failed
// build), so the blocks are returned on the legacy stream: the creation
// stream may no longer exist.
void DeviceArena::release() {
    for (void *p : blocks) cudaFreeAsync(p, 0);
    blocks.clear();
    bytes = 0;
    cur = nullptr;
    left = 0;
    next = size_t(1) << 20;
}

// Second streams of FMM plans (with their fork and join events), kept per
// device once created: a plan takes one when it is built and gives it back
// when it is freed, so building a plan creates no stream after the first.
namespace {
struct SideSet {
    cudaStream_t s;
    cudaEvent_t fork, join;
};
std::mutex g_side_mu;
std::vector<SideSet> g_side_free[64];
}  // namespace

static gf_status side_take(gf_plan_s *p) {
    {
        std::lock_guard<std::mutex> lk(g_side_mu);
        std::vector<SideSet> &v = g_side_free[p->device & 63];
        if (!v.empty()) {
            p->side = v.back().s;
            p->ev_fork = v.back().fork;
            p->ev_join = v.back().join;
            v.pop_back();
            return GF_OK;
        }
    }
    cudaError_t e = cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        set_error("cannot create the plan's second stream: %s", cudaGetErrorString(e));
        return GF_ERR_CUDA;
    }
    return GF_OK;
}

// The plan's device work has completed (its second stream is idle).
static void side_give(gf_plan_s *p) {
    if (p->side && p->ev_fork && p->ev_join) {
        std::lock_guard<std::mutex> lk(g_side_mu);
        g_side_free[p->device & 63].push_back(SideSet{p->side, p->ev_fork, p->ev_join});
    } else {
        if (p->ev_fork) cudaEventDestroy(p->ev_fork);
        if (p->ev_join) cudaEventDestroy(p->ev_join);
        if (p->side) cudaStreamDestroy(p->side);
    }
    p->side = nullptr;
    p->ev_fork = p->ev_join = nullptr;
}

// Free a plan whose device work has all completed (no device-wide wait).
void plan_release(gf_plan_s *plan) {
    fmm_destroy(plan);
    plan->arena.release();
    for (int i = 0; i <= GF_NUM_STAGES; ++i)
        if (plan->ev[i]) cudaEventDestroy(plan->ev[i]);
    side_give(plan);
    delete plan;
}

// The plan's quadrature rule lives in device memory right after the status
// word; kernels read it through this pointer.
const QuadRule *quad_device(gf_plan_s *plan) {
    return reinterpret_cast<const QuadRule *>(plan->d_status + 64);
}

static gf_status validate_options(int64_t M, const gf_options *opt);

// A quadrature rule: 1..kMaxQuad nodes in [-1, 1]^3, finite positive weights.
static gf_status validate_quad(const gf_quad *quad) {
    if (quad->nq < 1 || quad->nq > kMaxQuad || !quad->xi || !quad->w) {
        set_error("quad.nq = %d must be in [1, %d] with non-NULL xi and w", quad->nq, kMaxQuad);
        return GF_ERR_INVALID_ARG;
    }
    for (int q = 0; q < quad->nq; ++q) {
        if (!(quad->w[q] > 0.0) || !isfinite(quad->w[q])) {
            set_error("quad.w[%d] must be finite and positive", q);
            return GF_ERR_INVALID_ARG;
        }
        for (int a = 0; a < 3; ++a)
            if (!(fabs(quad->xi[3 * q + a]) <= 1.0)) {
                set_error("quad.xi[%d][%d] must lie in [-1, 1]", q, a);
                return GF_ERR_INVALID_ARG;
            }
    }
    return GF_OK;
}

// The device-side form of a validated rule.
static void fill_quad_rule(const gf_quad *quad, QuadRule &qr) {
    qr.nq = quad->nq;
    double wsum = 0.0;
    for (int q = 0; q < quad->nq; ++q) wsum += quad->w[q];
    for (int q = 0; q < quad->nq; ++q) {
        qr.wn[q] = quad->w[q] / wsum;
        qr.wnf[q] = (float)qr.wn[q];
        for (int a = 0; a < 3; ++a) {
            qr.xi[q][a] = quad->xi[3 * q + a];
            qr.offf[q][a] = (float)(0.5 + 0.5 * quad->xi[3 * q + a]);
        }
    }
}

static gf_status validate(const gf_grid *grid, const gf_quad *quad, int64_t M,
                          const gf_options *opt) {
    if (!grid || !quad || !opt) {
        set_error("grid, quad and opt must be non-NULL");
        return GF_ERR_INVALID_ARG;
    }
    for (int a = 0; a < 3; ++a) {
        if (grid->n[a] < 1 || grid->n[a] > kMaxAxis) {
            set_error("grid.n[%d] = %lld out of range [1, 2^22]", a, (long long)grid->n[a]);
            return GF_ERR_INVALID_ARG;
        }
        if (!(grid->h[a] > 0.0) || !isfinite(grid->h[a]) || !isfinite(grid->origin[a])) {
            set_error("grid.h[%d] must be finite and positive, origin finite", a);
            return GF_ERR_INVALID_ARG;
        }
    }
    // each axis is below 2^22, so the first product cannot overflow
    if (grid->n[0] * grid->n[1] > kMaxVoxels / grid->n[2]) {
        set_error("grid of %lld x %lld x %lld voxels exceeds 2^40 voxels", (long long)grid->n[0],
                  (long long)grid->n[1], (long long)grid->n[2]);
        return GF_ERR_INVALID_ARG;
    }
    GF_TRY(validate_quad(quad));
    GF_TRY(validate_options(M, opt));
    if (opt->mode == GF_MODE_FMM && !(grid->h[0] == grid->h[1] && grid->h[1] == grid->h[2])) {
        set_error("FMM mode needs cubic voxels (h[0] == h[1] == h[2])");
        return GF_ERR_UNSUPPORTED;
    }
    return GF_OK;
}

static gf_status validate_options(int64_t M, const gf_options *opt) {
    if (M < 0 || M > (int64_t(1) << 31) - 1) {
        set_error("M = %lld out of range [0, 2^31)", (long long)M);
        return GF_ERR_INVALID_ARG;
    }
    if (opt->mode != GF_MODE_DIRECT && opt->mode != GF_MODE_FMM) {
        set_error("opt.mode = %d is neither GF_MODE_DIRECT nor GF_MODE_FMM", opt->mode);
        return GF_ERR_INVALID_ARG;
    }
    if (opt->precision != GF_PREC_FP64 && opt->precision != GF_PREC_MIXED) {
        set_error("opt.precision = %d is neither GF_PREC_FP64 nor GF_PREC_MIXED", opt->precision);
        return GF_ERR_INVALID_ARG;
    }
    if (opt->max_batch < 1 || opt->max_batch > 64) {
        set_error("opt.max_batch = %d out of range [1, 64]", opt->max_batch);
        return GF_ERR_INVALID_ARG;
    }
    if (opt->G < 0.0 || !isfinite(opt->G)) {
        set_error("opt.G must be finite and >= 0 (0 selects 6.67428e-11)");
        return GF_ERR_INVALID_ARG;
    }
    if (opt->reserved0 & ~(GF_FLAG_M2L_SIMT | GF_FLAG_SUM_AN | GF_FLAG_TEST_WAIT_TIMEOUT | GF_FLAG_M2L_TENSOR)) {
        set_error("opt.reserved0 = %d holds unknown flags", opt->reserved0);
        return GF_ERR_INVALID_ARG;
    }
    if ((opt->reserved0 & GF_FLAG_M2L_TENSOR) &&
        (opt->mode != GF_MODE_FMM || opt->precision != GF_PREC_FP64 || (opt->reserved0 & GF_FLAG_M2L_SIMT))) {
        set_error("GF_FLAG_M2L_TENSOR applies to FP64 FMM plans (without GF_FLAG_M2L_SIMT)");
        return GF_ERR_UNSUPPORTED;
    }
    if ((opt->reserved0 & GF_FLAG_SUM_AN) && opt->mode == GF_MODE_DIRECT && opt->precision != GF_PREC_FP64) {
        set_error("GF_FLAG_SUM_AN (closed-form voxels) in direct mode is implemented in FP64 only");
        return GF_ERR_UNSUPPORTED;
    }
    if ((opt->reserved0 & GF_FLAG_SUM_AN) && opt->mode == GF_MODE_FMM && opt->leaf_vox != 0 && opt->leaf_vox != 4) {
        set_error("GF_FLAG_SUM_AN (closed-form voxels) in FMM mode uses leaves of 4^3 voxels (leaf_vox 0 or 4)");
        return GF_ERR_UNSUPPORTED;
    }
    if (opt->mode == GF_MODE_FMM) {
        if (opt->p < 1 || opt->p > kMaxP) {
            set_error("opt.p = %d out of range [1, %d]", opt->p, kMaxP);
            return GF_ERR_INVALID_ARG;
        }
        if (opt->leaf_vox < 0 || opt->leaf_vox > 64) {
            set_error("opt.leaf_vox = %d out of range [0, 64]", opt->leaf_vox);
            return GF_ERR_INVALID_ARG;
        }
    }
    return GF_OK;
}

// The end of a plan build: wait for the device, then hand the plan out or
// free everything it holds.
static gf_status finish_create(gf_plan_s *p, gf_status s, cudaStream_t st, gf_plan_t *out) {
    if (s == GF_OK) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            set_error("plan build failed on the device: %s", cudaGetErrorString(e));
            s = GF_ERR_CUDA;
        }
    }
    if (s != GF_OK) {
        cudaDeviceSynchronize();
        cudaGetLastError();
        char keep[512];
        snprintf(keep, sizeof(keep), "%s", get_error());
        fmm_destroy(p);
        p->arena.release();
        delete p;
        set_error("%s", keep);
        return s;
    }
    if (p->fmm && !p->fmm->points) {
        // the near field's stream (it runs beside the M2L; see the forward)
        const gf_status ss = side_take(p);
        if (ss != GF_OK) {
            plan_release(p);
            return ss;
        }
    }
    p->device_bytes = p->arena.bytes;
    *out = p;
    return GF_OK;
}

}  // namespace gf

using namespace gf;

extern "C" {

int32_t gf_version(void) { return GF_VERSION; }

int64_t gf_launch_count(void) { return (int64_t)g_launches.load(); }

const char *gf_last_error(void) { return get_error(); }

gf_status gf_plan_bytes(const gf_grid *grid, const gf_quad *quad, int64_t M,
                        const gf_options *opt, size_t *bytes) {
    GF_TRY(validate(grid, quad, M, opt));
    if (!bytes) {
        set_error("bytes must be non-NULL");
        return GF_ERR_INVALID_ARG;
    }
    size_t b = 4096 + sizeof(QuadRule) + 256;
    if (opt->mode == GF_MODE_DIRECT) {
        b += (size_t)M * 3 * sizeof(double) + 512;
        if (opt->precision == GF_PREC_MIXED) b += (size_t)M * 6 * sizeof(float) + 512;
        if (opt->reserved0 & GF_FLAG_SUM_AN) b += sum_an_bytes(grid, opt->max_batch);
    } else {
        b += fmm_bytes_estimate(grid, quad->nq, M, opt);
    }
    *bytes = b;
    return GF_OK;
}

gf_status gf_plan_create(const gf_grid *grid, const gf_quad *quad, const double *obs_dev,
                         int64_t M, const gf_options *opt, void *stream, gf_plan_t *out) {
    if (!out) {
        set_error("plan output pointer is NULL");
        return GF_ERR_INVALID_ARG;
    }
    *out = nullptr;
    GF_TRY(validate(grid, quad, M, opt));
    if (M > 0 && !obs_dev) {
        set_error("obs_dev is NULL with M = %lld", (long long)M);
        return GF_ERR_INVALID_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    gf_plan_s *p = new (std::nothrow) gf_plan_s();
    if (!p) {
        set_error("host allocation failed");
        return GF_ERR_OOM;
    }
    cudaGetDevice(&p->device);
    p->arena.stream = st;
    p->grid = *grid;
    p->opt = *opt;
    p->G = opt->G > 0.0 ? opt->G : 6.67428e-11;
    p->M = M;
    p->nvox = grid->n[0] * grid->n[1] * grid->n[2];
    QuadRule &qr = p->quad;
    memset(&qr, 0, sizeof(qr));
    if ((opt->reserved0 & GF_FLAG_SUM_AN) && opt->mode == GF_MODE_FMM) {
        // closed-form voxels in the FMM: the rule is ignored; the tree and the
        // leaf-blocked densities are those of one node per voxel
        qr.nq = 1;
        qr.wn[0] = 1.0;
        qr.wnf[0] = 1.0f;
        for (int a = 0; a < 3; ++a) qr.offf[0][a] = 0.5f;
    } else {
        fill_quad_rule(quad, qr);
    }
    gf_status s = GF_OK;
    // status word (64 ints) followed by the quadrature rule
    s = p->arena.alloc(reinterpret_cast<void **>(&p->d_status), 64 * sizeof(int) + sizeof(QuadRule));
    if (s == GF_OK) {
        cudaError_t e = cudaMemsetAsync(p->d_status, 0, 64 * sizeof(int), st);
        if (e != cudaSuccess) {
            set_error("plan setup failed: %s", cudaGetErrorString(e));
            s = GF_ERR_CUDA;
        } else {
            s = upload_small(p->d_status + 64, &qr, sizeof(QuadRule), st);
        }
    }
    if (s == GF_OK) {
        if (opt->mode == GF_MODE_DIRECT) {
            s = direct_prepare(p, obs_dev, st);
            if (s == GF_OK && (opt->reserved0 & GF_FLAG_SUM_AN)) s = sum_an_prepare(p);
            p->near_pairs = p->M * p->nvox * ((opt->reserved0 & GF_FLAG_SUM_AN) ? 1 : quad->nq);
        }
        else
            s = fmm_create(p, obs_dev, st);
    }
    return finish_create(p, s, st, out);
}

gf_status gf_hex_sources(const double *verts_dev, int64_t ncell, const gf_quad *quad, int32_t precision,
                         double *x_dev, double *a_dev, void *stream) {
    if (!quad) {
        set_error("quad must be non-NULL");
        return GF_ERR_INVALID_ARG;
    }
    if (precision != GF_PREC_FP64 && precision != GF_PREC_MIXED) {
        set_error("precision = %d is neither GF_PREC_FP64 nor GF_PREC_MIXED", precision);
        return GF_ERR_INVALID_ARG;
    }
    GF_TRY(validate_quad(quad));
    if (ncell < 0 || ncell > ((int64_t(1) << 31) - 1) / quad->nq) {
        set_error("ncell = %lld out of range: ncell * nq must be below 2^31", (long long)ncell);
        return GF_ERR_INVALID_ARG;
    }
    if (ncell > 0 && (!verts_dev || !x_dev || !a_dev)) {
        set_error("verts_dev, x_dev and a_dev must be non-NULL");
        return GF_ERR_INVALID_ARG;
    }
    QuadRule qr;
    memset(&qr, 0, sizeof(qr));
    fill_quad_rule(quad, qr);
    return hex_sources_run(verts_dev, ncell, qr, precision, x_dev, a_dev, reinterpret_cast<cudaStream_t>(stream));
}

gf_status gf_plan_create_points(const double *src_dev, const double *wt_dev, int64_t S, int32_t per_cell,
                                const double *obs_dev, int64_t M, const gf_options *opt, void *stream,
                                gf_plan_t *out) {
    if (!out) {
        set_error("plan output pointer is NULL");
        return GF_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (!opt) {
        set_error("opt must be non-NULL");
        return GF_ERR_INVALID_ARG;
    }
    GF_TRY(validate_options(M, opt));
    if (opt->reserved0 & GF_FLAG_SUM_AN) {
        set_error("GF_FLAG_SUM_AN (closed-form voxels) does not apply to point sources");
        return GF_ERR_UNSUPPORTED;
    }
    if (S < 0 || S > (int64_t(1) << 31) - 1) {
        set_error("S = %lld out of range [0, 2^31)", (long long)S);
        return GF_ERR_INVALID_ARG;
    }
    if (per_cell < 1 || S % per_cell != 0) {
        set_error("per_cell = %d must be >= 1 and divide S = %lld", per_cell, (long long)S);
        return GF_ERR_INVALID_ARG;
    }
    if ((S > 0 && (!src_dev || !wt_dev)) || (M > 0 && !obs_dev)) {
        set_error("src_dev, wt_dev (S > 0) and obs_dev (M > 0) must be non-NULL");
        return GF_ERR_INVALID_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    gf_plan_s *p = new (std::nothrow) gf_plan_s();
    if (!p) {
        set_error("host allocation failed");
        return GF_ERR_OOM;
    }
    cudaGetDevice(&p->device);
    p->arena.stream = st;
    p->opt = *opt;
    p->opt.leaf_vox = 0;
    p->G = opt->G > 0.0 ? opt->G : 6.67428e-11;
    p->M = M;
    p->pts.on = true;
    p->pts.S = S;
    p->pts.per_cell = per_cell;
    p->pts.ncell = S / per_cell;
    p->nvox = p->pts.ncell;
    QuadRule &qr = p->quad;   // one unit node: the plan's rule is not used
    memset(&qr, 0, sizeof(qr));
    qr.nq = 1;
    qr.wn[0] = 1.0;
    qr.wnf[0] = 1.0f;
    for (int a = 0; a < 3; ++a) qr.offf[0][a] = 0.5f;
    gf_status s = p->arena.alloc(reinterpret_cast<void **>(&p->d_status), 64 * sizeof(int) + sizeof(QuadRule));
    if (s == GF_OK) {
        cudaError_t e = cudaMemsetAsync(p->d_status, 0, 64 * sizeof(int), st);
        if (e != cudaSuccess) {
            set_error("plan setup failed: %s", cudaGetErrorString(e));
            s = GF_ERR_CUDA;
        } else {
            s = upload_small(p->d_status + 64, &qr, sizeof(QuadRule), st);
        }
    }
    if (s == GF_OK) {
        if (opt->mode == GF_MODE_DIRECT) {
            s = points_prepare_direct(p, src_dev, wt_dev, obs_dev, st);
            p->near_pairs = p->M * S;
        } else {
            s = points_fmm_create(p, src_dev, wt_dev, obs_dev, st);
        }
    }
    return finish_create(p, s, st, out);
}

gf_status gf_forward(gf_plan_t plan, const void *rho_dev, int32_t rho_dtype, int32_t B,
                     double *g_dev, double *gz_dev, void *stream) {
    if (!plan) {
        set_error("plan is NULL");
        return GF_ERR_INVALID_ARG;
    }
    const bool no_sources = plan->pts.on && plan->pts.S == 0;
    if ((!rho_dev && !no_sources) || (!g_dev && !gz_dev && plan->M > 0)) {
        set_error("rho_dev must be non-NULL and at least one of g_dev, gz_dev given");
        return GF_ERR_INVALID_ARG;
    }
    if (rho_dtype != GF_DTYPE_F64 && rho_dtype != GF_DTYPE_F32) {
        set_error("rho_dtype = %d is neither GF_DTYPE_F64 nor GF_DTYPE_F32", rho_dtype);
        return GF_ERR_INVALID_ARG;
    }
    if (B < 1 || B > plan->opt.max_batch) {
        set_error("B = %d out of range [1, max_batch = %d]", B, plan->opt.max_batch);
        return GF_ERR_INVALID_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    for (int i = 0; i <= GF_NUM_STAGES; ++i) plan->ev_used[i] = false;
    stage_mark(plan, 0, st);
    if (plan->opt.mode == GF_MODE_DIRECT) {
        if (plan->pts.on)
            GF_TRY(points_direct_forward(plan, rho_dev, rho_dtype, B, g_dev, gz_dev, st));
        else if (plan->opt.reserved0 & GF_FLAG_SUM_AN)
            GF_TRY(sum_an_forward(plan, rho_dev, rho_dtype, B, g_dev, gz_dev, st));
        else
            GF_TRY(direct_forward(plan, rho_dev, rho_dtype, B, g_dev, gz_dev, st));
        stage_mark(plan, 7, st);
        return GF_OK;
    }
    return fmm_forward(plan, rho_dev, rho_dtype, B, g_dev, gz_dev, st);
}

gf_status gf_adjoint(gf_plan_t plan, const double *r_dev, int32_t ncomp, int32_t B,
                     double *grad_dev, void *stream) {
    if (!plan) {
        set_error("plan is NULL");
        return GF_ERR_INVALID_ARG;
    }
    if ((!r_dev && plan->M > 0) || !grad_dev) {
        set_error("r_dev and grad_dev must be non-NULL");
        return GF_ERR_INVALID_ARG;
    }
    if (ncomp != 1 && ncomp != 3) {
        set_error("ncomp = %d must be 1 (weights on g_z) or 3 (weights on g)", ncomp);
        return GF_ERR_INVALID_ARG;
    }
    if (B < 1 || B > plan->opt.max_batch) {
        set_error("B = %d out of range [1, max_batch = %d]", B, plan->opt.max_batch);
        return GF_ERR_INVALID_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (plan->pts.on) {
        set_error("gf_adjoint of a point-source plan is not implemented");
        return GF_ERR_UNSUPPORTED;
    }
    if (plan->part_lo != 0 || plan->part_hi < 64) {
        set_error("gf_adjoint of a plan restricted to a source part is not implemented");
        return GF_ERR_UNSUPPORTED;
    }
    if ((plan->opt.reserved0 & GF_FLAG_SUM_AN) && plan->opt.mode == GF_MODE_FMM) {
        set_error("gf_adjoint of a FMM plan with closed-form voxels is not implemented (direct mode has it)");
        return GF_ERR_UNSUPPORTED;
    }
    if (plan->opt.mode == GF_MODE_DIRECT) {
        if (plan->opt.reserved0 & GF_FLAG_SUM_AN) return sum_an_adjoint(plan, r_dev, ncomp, B, grad_dev, st);
        return direct_adjoint(plan, r_dev, ncomp, B, grad_dev, st);
    }
    return fmm_adjoint(plan, r_dev, ncomp, B, grad_dev, st);
}

gf_status gf_plan_set_source_part(gf_plan_t plan, int32_t part, int32_t nparts, int32_t *code_lo,
                                  int32_t *code_hi) {
    if (!plan) {
        set_error("plan is NULL");
        return GF_ERR_INVALID_ARG;
    }
    if (nparts < 1 || nparts > 64 || part < 0 || part >= nparts) {
        set_error("need 0 <= part < nparts <= 64 (part = %d, nparts = %d)", part, nparts);
        return GF_ERR_INVALID_ARG;
    }
    if (plan->opt.mode != GF_MODE_FMM || !plan->fmm || plan->pts.on) {
        set_error("source parts are implemented for FMM plans over voxel grids only");
        return GF_ERR_UNSUPPORTED;
    }
    const FmmPlan *F = plan->fmm;
    // grid voxels under each level-2 box, by Morton code
    const int64_t side = (int64_t)F->b << (F->L - 2);   // level-2 box edge in voxels
    double w[64];
    double total = 0.0;
    for (uint32_t c = 0; c < 64; ++c) {
        const int64_t bx = (c & 1) | ((c >> 2) & 2), by = ((c >> 1) & 1) | ((c >> 3) & 2),
                      bz = ((c >> 2) & 1) | ((c >> 4) & 2);
        const int64_t bc[3] = {bx, by, bz};
        double n = 1.0;
        for (int a = 0; a < 3; ++a) {
            const int64_t v0 = std::max<int64_t>(0, bc[a] * side - F->voff[a]);
            const int64_t v1 = std::min<int64_t>(plan->grid.n[a], (bc[a] + 1) * side - F->voff[a]);
            n *= (double)std::max<int64_t>(0, v1 - v0);
        }
        w[c] = n;
        total += n;
    }
    // part k takes the codes whose cumulative count (up to the code's
    // middle) falls in [k / nparts, (k + 1) / nparts) of the total
    uint32_t lo = 64, hi = 0;
    double cum = 0.0;
    for (uint32_t c = 0; c < 64; ++c) {
        const double mid = cum + 0.5 * w[c];
        cum += w[c];
        int k = total > 0.0 ? (int)(mid / total * nparts) : 0;
        k = std::min(nparts - 1, std::max(0, k));
        if (k == part) {
            lo = std::min(lo, c);
            hi = std::max(hi, c + 1);
        }
    }
    if (lo >= hi) lo = hi = 0;   // an empty part
    if (nparts == 1) {
        lo = 0;
        hi = 64;
    }
    plan->part_lo = lo;
    plan->part_hi = hi;
    if (code_lo) *code_lo = (int32_t)lo;
    if (code_hi) *code_hi = (int32_t)hi;
    return GF_OK;
}

gf_status gf_plan_check(gf_plan_t plan, void *stream) {
    if (!plan) {
        set_error("plan is NULL");
        return GF_ERR_INVALID_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int flags[4] = {0, 0, 0, 0};
    GF_CUDA(cudaMemcpyAsync(flags, plan->d_status, sizeof(flags), cudaMemcpyDeviceToHost, st));
    GF_CUDA(cudaStreamSynchronize(st));
    if (flags[0] || flags[1] || flags[2] || flags[3]) {
        GF_CUDA(cudaMemsetAsync(plan->d_status, 0, sizeof(flags), st));
        GF_CUDA(cudaStreamSynchronize(st));
        set_error("device check failed: non-finite density %d, bounded wait %d, index %d, other %d",
                  flags[0], flags[1], flags[2], flags[3]);
        return GF_ERR_DEVICE_CHECK;
    }
    return GF_OK;
}

gf_status gf_plan_destroy(gf_plan_t plan) {
    if (!plan) return GF_OK;
    int cur = 0;
    const int dev = plan->device;
    cudaGetDevice(&cur);
    if (cur != dev) cudaSetDevice(dev);
    cudaDeviceSynchronize();
    plan_release(plan);
    if (cur != dev) cudaSetDevice(cur);
    return GF_OK;
}

gf_status gf_plan_set_timing(gf_plan_t plan, int32_t enable) {
    if (!plan) {
        set_error("plan is NULL");
        return GF_ERR_INVALID_ARG;
    }
    if (enable && !plan->ev[0]) {
        for (int i = 0; i <= GF_NUM_STAGES; ++i) GF_CUDA(cudaEventCreate(&plan->ev[i]));
    }
    plan->timing = enable != 0;
    return GF_OK;
}

gf_status gf_plan_stage_times(gf_plan_t plan, double *ms) {
    if (!plan || !ms) {
        set_error("plan and ms must be non-NULL");
        return GF_ERR_INVALID_ARG;
    }
    for (int i = 0; i < GF_NUM_STAGES; ++i) ms[i] = 0.0;
    if (!plan->ev[0] || !plan->ev_used[0]) {
        set_error("no timed forward on this plan (call gf_plan_set_timing first)");
        return GF_ERR_INVALID_ARG;
    }
    int last = 0;
    for (int i = 0; i <= GF_NUM_STAGES; ++i)
        if (plan->ev_used[i]) last = i;
    GF_CUDA(cudaEventSynchronize(plan->ev[last]));
    // boundaries: ev[0] start, ev[i+1] end of stage i; stages that did not
    // run keep their start event equal to the previous boundary
    int prev = 0;
    for (int i = 0; i < GF_NUM_STAGES - 1; ++i) {
        if (!plan->ev_used[i + 1]) continue;
        float t = 0.f;
        GF_CUDA(cudaEventElapsedTime(&t, plan->ev[prev], plan->ev[i + 1]));
        ms[i] = t;
        prev = i + 1;
    }
    float tot = 0.f;
    GF_CUDA(cudaEventElapsedTime(&tot, plan->ev[0], plan->ev[last]));
    ms[GF_NUM_STAGES - 1] = tot;
    return GF_OK;
}

gf_status gf_plan_get_info(gf_plan_t plan, gf_plan_info *info) {
    if (!plan || !info) {
        set_error("plan and info must be non-NULL");
        return GF_ERR_INVALID_ARG;
    }
    if (plan->opt.mode == GF_MODE_FMM && !plan->counts_done) {
        int cur = 0;
        cudaGetDevice(&cur);
        if (cur != plan->device) cudaSetDevice(plan->device);
        const gf_status rc = fmm_work_counts(plan, plan->arena.stream);
        if (cur != plan->device) cudaSetDevice(cur);
        if (rc != GF_OK) return rc;
    }
    memset(info, 0, sizeof(*info));
    info->mode = plan->opt.mode;
    info->precision = plan->opt.precision;
    info->M = plan->M;
    info->n_sources =
        plan->pts.on ? plan->pts.S : plan->nvox * ((plan->opt.reserved0 & GF_FLAG_SUM_AN) ? 1 : plan->quad.nq);
    info->device_bytes = plan->arena.bytes;
    info->near_pairs = plan->near_pairs;
    info->m2l_pairs = plan->m2l_pairs;
    if (plan->opt.mode == GF_MODE_FMM) return fmm_info(plan, info);
    return GF_OK;
}

gf_status gf_plan_export_tree(gf_plan_t plan, int32_t level, int32_t *perm, uint64_t *keys,
                              uint64_t *box_keys, int64_t *ilist, int64_t *near_) {
    if (!plan || plan->opt.mode != GF_MODE_FMM) {
        set_error("gf_plan_export_tree needs a FMM plan");
        return GF_ERR_INVALID_ARG;
    }
    return fmm_export_tree(plan, level, perm, keys, box_keys, ilist, near_);
}

}  // extern "C"
