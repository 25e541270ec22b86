// gf_internal.cuh -- shared declarations of the CUDA library behind gf.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "gf.h"

namespace gf {

// ----------------------------------------------------------------- errors
void set_error(const char *fmt, ...);
const char *get_error();

#define GF_TRY(expr)                                     \
    do {                                                 \
        gf_status _s = (expr);                           \
        if (_s != GF_OK) return _s;                      \
    } while (0)

#define GF_CUDA(expr)                                                        \
    do {                                                                     \
        cudaError_t _e = (expr);                                             \
        if (_e != cudaSuccess) {                                             \
            ::gf::set_error("%s failed: %s (%s:%d)", #expr,                  \
                            cudaGetErrorString(_e), __FILE__, __LINE__);     \
            return _e == cudaErrorMemoryAllocation ? GF_ERR_OOM : GF_ERR_CUDA; \
        }                                                                    \
    } while (0)

#define GF_LAUNCH_CHECK() GF_CUDA(cudaGetLastError())

constexpr int kMaxQuad = 64;
constexpr int kMaxLevels = 21;      // Morton keys use 3 bits per level in a u64
constexpr int kMaxP = 16;
constexpr int64_t kMaxAxis = int64_t(1) << 22;     // voxels along one grid axis
constexpr int64_t kMaxVoxels = int64_t(1) << 40;   // voxels in a grid (no int64 overflow)
constexpr int kNumM2LOffsets = 316; // 7^3 - 3^3 interaction-list offsets

// Quadrature rule as the kernels see it (Sec. 2.1): node offsets from the
// voxel's lower corner in voxel units (0.5 + xi/2) and normalised weights.
struct QuadRule {
    int nq;
    double xi[kMaxQuad][3];    // reference nodes in [-1,1]^3
    double wn[kMaxQuad];       // w_q / sum(w)
    float offf[kMaxQuad][3];   // 0.5 + 0.5*xi: node offset from the voxel's
                               // lower corner in voxel units
    float wnf[kMaxQuad];
};

// Bookkeeping for device memory a plan owns.
// Allocations are stream-ordered (cudaMallocAsync from the device's default
// pool, which keeps freed memory for reuse), so building and releasing a
// plan inside a timed loop costs no driver round trips after the first time.
// A plan's device memory: chunks from the stream-ordered allocator, handed
// out by bumping a pointer (256-byte alignment), all returned together when
// the plan is freed.  Chunks grow from 1 MiB by doubling up to 64 MiB; a
// larger request gets a chunk of its own size.
struct DeviceArena {
    std::vector<void *> blocks;   // chunks
    size_t bytes = 0;             // bytes held in chunks
    unsigned char *cur = nullptr; // free tail of the newest chunk
    size_t left = 0;
    size_t next = size_t(1) << 20;
    cudaStream_t stream = nullptr;
    gf_status alloc(void **p, size_t n);
    template <class T>
    gf_status alloc_n(T **p, size_t count) {
        return alloc(reinterpret_cast<void **>(p), count * sizeof(T));
    }
    void release();
};

struct FmmPlan;   // defined in gf_fmm.cuh

// Weighted point sources of a plan made by gf_plan_create_points: source s
// sits at x_s with volume weight a_s and samples density s / per_cell.
struct PointSet {
    bool on = false;
    int64_t S = 0, ncell = 0;
    int per_cell = 1;
    double *x = nullptr;          // direct: [S][3] positions, caller order
    double *a = nullptr;          // direct: [S] volume weights
    void *loc = nullptr;          // FMM: [S][4] in the plan's precision, sorted by leaf: offset from the
                                  // leaf's centre and volume, in leaf units
    int32_t *perm = nullptr;      // FMM: sorted position -> caller index
    int64_t *leaf_beg = nullptr;  // FMM: [nleaf + 1] first sorted source of each leaf of the dense block
    double q = 0.0;               // mixed direct: the length quantum
    float *xi = nullptr, *xf = nullptr;   // mixed direct: sources' integer and fractional parts (quanta)
    float *oi = nullptr, *of = nullptr;   // the same for the observers
};

}  // namespace gf

struct gf_plan_s {
    int device = 0;
    gf_grid grid{};
    gf_options opt{};
    double G = 0;
    int64_t M = 0;
    int64_t nvox = 0;
    gf::QuadRule quad{};
    gf::DeviceArena arena;
    // direct mode: observers in caller order
    double *d_obs = nullptr;     // [M][3] FP64
    int32_t *d_obs_ivox = nullptr;   // [M][3] floor of voxel coordinates (mixed)
    float *d_obs_fvox = nullptr;     // [M][3] fractional voxel coordinates (mixed)
    double *d_corner = nullptr;      // closed-form voxels: [max_batch][corners] weights
    gf::FmmPlan *fmm = nullptr;
    gf::PointSet pts;            // point-source plans only
    int *d_status = nullptr;     // device-side check word
    size_t device_bytes = 0;
    int64_t near_pairs = 0, m2l_pairs = 0;
    // FMM source partition: only the sources whose level-2 ancestor box has
    // a Morton code in [part_lo, part_hi) contribute (all: [0, 64))
    uint32_t part_lo = 0, part_hi = 64;
    bool counts_done = false;    // FMM work counts computed (on first info request)
    bool timing = false;
    cudaEvent_t ev[GF_NUM_STAGES + 1] = {};
    // FMM plans: a second stream for the near field of the evaluation, which
    // runs beside the M2L and the L2L chain, and the events that fork it from
    // the forward's stream and join it back
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool ev_used[GF_NUM_STAGES + 1] = {};
};

namespace gf {
// Record the boundary event `i` of the stage timeline when timing is on.
inline void stage_mark(gf_plan_s *p, int i, cudaStream_t st) {
    if (p->timing) {
        cudaEventRecord(p->ev[i], st);
        p->ev_used[i] = true;
    }
}
}  // namespace gf

namespace gf {

// The plan's quadrature rule in device memory.
const QuadRule *quad_device(gf_plan_s *plan);

// Direct-mode kernels (gf_direct.cu)
gf_status direct_prepare(gf_plan_s *plan, const double *obs_dev, cudaStream_t st);
gf_status direct_forward(gf_plan_s *plan, const void *rho, int rho_dtype, int B,
                         double *g, double *gz, cudaStream_t st);
gf_status direct_adjoint(gf_plan_s *plan, const double *r, int ncomp, int B,
                         double *grad, cudaStream_t st);

// Closed-form voxels, SUM-AN (gf_sum_an.cu; direct mode, FP64)
size_t sum_an_bytes(const gf_grid *grid, int max_batch);
gf_status sum_an_prepare(gf_plan_s *plan);
gf_status sum_an_forward(gf_plan_s *plan, const void *rho, int rho_dtype, int B,
                         double *g, double *gz, cudaStream_t st);
gf_status sum_an_adjoint(gf_plan_s *plan, const double *r, int ncomp, int B,
                         double *grad, cudaStream_t st);

// FMM (gf_fmm.cu)
gf_status fmm_create(gf_plan_s *plan, const double *obs_dev, cudaStream_t st);
gf_status fmm_forward(gf_plan_s *plan, const void *rho, int rho_dtype, int B,
                      double *g, double *gz, cudaStream_t st);
gf_status fmm_adjoint(gf_plan_s *plan, const double *r, int ncomp, int B,
                      double *grad, cudaStream_t st);
void fmm_destroy(gf_plan_s *plan);
// Free a plan whose device work has all completed (no device-wide wait).
void plan_release(gf_plan_s *plan);
gf_status fmm_info(const gf_plan_s *plan, gf_plan_info *info);
gf_status fmm_work_counts(gf_plan_s *plan, cudaStream_t st);
// The plan's P2M matrix as a tensor-core image, cached with the matrix.
gf_status get_p2m_tc(gf_plan_s *plan, cudaStream_t st);
gf_status fmm_export_tree(gf_plan_s *plan, int level, int32_t *perm, uint64_t *keys,
                          uint64_t *box_keys, int64_t *ilist, int64_t *near_);
size_t fmm_bytes_estimate(const gf_grid *grid, int nq, int64_t M, const gf_options *opt);

inline unsigned ceil_div(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// Weighted point sources (gf_points.cu)
gf_status hex_sources_run(const double *verts, int64_t ncell, const QuadRule &qr, int precision, double *x,
                          double *a, cudaStream_t st);
gf_status points_prepare_direct(gf_plan_s *plan, const double *src, const double *wt, const double *obs,
                                cudaStream_t st);
gf_status points_direct_forward(gf_plan_s *plan, const void *rho, int rho_dtype, int B, double *g, double *gz,
                                cudaStream_t st);
gf_status points_fmm_create(gf_plan_s *plan, const double *src, const double *wt, const double *obs,
                            cudaStream_t st);
template <class T>
gf_status points_masses(gf_plan_s *plan, const void *rho, int rho_dtype, int B, cudaStream_t st);
template <class T>
gf_status points_p2m(gf_plan_s *plan, int B, cudaStream_t st);
template <class T>
gf_status points_eval(gf_plan_s *plan, int B, double *g, double *gz, cudaStream_t st);
gf_status points_count_near(gf_plan_s *plan, unsigned long long *d_out, cudaStream_t st);

// Whether box (X, Y, Z) of level 2 + shift (absolute box coordinates) lies
// under a level-2 box whose Morton code (x -> bit 0, y -> bit 1, z -> bit 2
// per level) is in [lo, hi).  Boxes of level 2 and deeper never straddle a
// level-2 box, so a range of codes partitions the sources of every level.
__host__ __device__ __forceinline__ bool in_source_part(int64_t X, int64_t Y, int64_t Z, int shift, uint32_t lo,
                                                        uint32_t hi) {
    if (lo == 0 && hi >= 64) return true;
    const uint32_t x = (uint32_t)(X >> shift) & 3u, y = (uint32_t)(Y >> shift) & 3u, z = (uint32_t)(Z >> shift) & 3u;
    const uint32_t c = (x & 1u) | ((y & 1u) << 1) | ((z & 1u) << 2) | ((x & 2u) << 2) | ((y & 2u) << 3) | ((z & 2u) << 4);
    return c >= lo && c < hi;
}

// Opt a kernel in to more than 48 KB of dynamic shared memory.
template <class Kern>
inline gf_status ensure_smem(Kern kernel, size_t bytes) {
    if (bytes > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) {
            set_error("cannot reserve %zu bytes of shared memory: %s", bytes, cudaGetErrorString(e));
            return GF_ERR_UNSUPPORTED;
        }
    }
    return GF_OK;
}

// Copies nbytes (whole 4-byte words, dst word-aligned) of host memory to the
// device on stream st as kernel arguments rather than as a host-to-device
// copy (gf_prim.cu): the host memory may be reused once the call returns.
gf_status upload_small(void *dst, const void *src, size_t nbytes, cudaStream_t st);

// Streaming multiprocessors of the current device (cached per device).
inline int sm_count() {
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (cache[dev] == 0) {
        int n = 0;
        cache[dev] = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0 ? n : 152;
    }
    return cache[dev];
}

// Blocks of `kernel` that are resident on the current device at once, for
// grids whose warps take their work from a queue (at least 1).
template <class Kern>
inline unsigned resident_blocks(Kern kernel, int threads, size_t shm) {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, shm) != cudaSuccess)
        return 1;
    return (unsigned)(per > 0 ? per : 1) * (unsigned)(sms > 0 ? sms : 1);
}

// Number of kernels the library has launched (all plans, all threads).
void count_launch(int n = 1);
#define GF_KERNEL_DONE() \
    do {                 \
        ::gf::count_launch(); \
        GF_LAUNCH_CHECK();    \
    } while (0)

}  // namespace gf
