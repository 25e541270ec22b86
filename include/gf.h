/*
 * gf.h -- C ABI of the GB300 voxel-gravity forward model.
 *
 * The library evaluates the discretised gravity integral of Eq. 1
 *
 *     g(r) = G * Int rho(x) (r - x) / |r - x|^3 dV
 *
 * for a brick of constant-density voxels (Sec. 2.1) sampled at a per-voxel
 * quadrature rule, in the N-body form of Eqs. 7-8, at arbitrary observation
 * points -- either by direct summation (Sec. 2.1, SUM-G1/SUM-G2) or by the
 * fast multipole method of Sec. 2.3 (near/far split of Eq. 10, expansions of
 * Eq. 9, octree upward and downward sweeps).  Conventions:
 *
 *   * units are SI; g points along (r - x), i.e. from the mass to the
 *     observer, exactly as Eq. 1 is written; z is up;
 *   * a quadrature point that coincides exactly with an observer contributes
 *     nothing to that observer (the direct-work count of Eq. 14 excludes self
 *     pairs);
 *   * the mass of quadrature point q of voxel v is rho_v * V_v * w_q / sum(w).
 *
 * Memory and ownership.  Every pointer named *_dev is a device pointer owned
 * by the caller, on the device that was current when the plan was created,
 * and must stay valid until the work enqueued on `stream` has finished.
 * Host pointers (*_host and the quadrature arrays) are read during the call
 * only.  A plan owns its tree, lists, expansion workspaces and operator
 * tables; nothing a plan owns is visible to the caller except through the
 * query functions below.  `stream` is a cudaStream_t (NULL = the legacy
 * default stream).  Work is enqueued asynchronously; no call except
 * gf_plan_create, gf_plan_destroy and gf_plan_check waits for the device.
 *
 * Errors.  Every call returns a gf_status.  On failure nothing is enqueued
 * (or, for GF_ERR_CUDA, the CUDA error is reported and the plan must be
 * destroyed) and gf_last_error() returns a one-line message for the calling
 * thread.  No exception or device trap crosses the ABI.
 */
#ifndef GF_H
#define GF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GF_VERSION 1

typedef enum {
    GF_OK = 0,
    GF_ERR_INVALID_ARG = 1,   /* bad pointer, size, option or dtype          */
    GF_ERR_OOM = 2,           /* device allocation failed                    */
    GF_ERR_CUDA = 3,          /* a CUDA call failed (message has the name)   */
    GF_ERR_UNSUPPORTED = 4,   /* valid request outside what is implemented   */
    GF_ERR_TIMEOUT = 5,       /* a bounded device wait gave up               */
    GF_ERR_DEVICE_CHECK = 6,  /* a device-side check failed (e.g. NaN rho)   */
    GF_ERR_BUSY = 7           /* admission refused: not enough free memory  */
} gf_status;

/* Voxel brick of Sec. 2.1: voxel (i,j,k) spans origin + [i,i+1)*h along each
 * axis; density arrays are [nz][ny][nx] with x fastest. */
typedef struct {
    int64_t n[3];       /* nx, ny, nz in [1, 2^22], nx*ny*nz <= 2^40       */
    double origin[3];   /* lower corner of voxel (0,0,0), metres           */
    double h[3];        /* voxel edge lengths, metres, > 0                 */
} gf_grid;

/* Per-voxel quadrature rule of Sec. 2.1 (1-point Gauss = SUM-G1, 2x2x2 Gauss
 * = SUM-G2): node q sits at centre + (h/2) * xi[q] with xi in [-1,1]^3.
 * Host arrays, copied at plan creation. */
typedef struct {
    int32_t nq;         /* 1..64 nodes                                     */
    const double *xi;   /* [nq][3]                                         */
    const double *w;    /* [nq] positive weights (normalised internally)   */
} gf_quad;

enum { GF_MODE_DIRECT = 0, GF_MODE_FMM = 1 };
/* GF_PREC_FP64: every stage in FP64.  GF_PREC_MIXED: FP32 near field with
 * compensated accumulation; tensor-core M2L on FP16 high/low parts of
 * power-of-two-scaled operands (three products, FP32 accumulation) and
 * split-TF32 P2M/M2M/L2L; FP64 for the top-level translations and the final
 * near+far sum.  Results stay within a relative L2 error of about 1e-5
 * (p >= 10). */
enum { GF_PREC_FP64 = 0, GF_PREC_MIXED = 1 };
enum { GF_DTYPE_F64 = 0, GF_DTYPE_F32 = 1 };
/* Option flags (gf_options.reserved0):
 *   GF_FLAG_M2L_SIMT  FMM, mixed precision: the M2L on the SIMT cores
 *                     instead of the tensor cores.
 *   GF_FLAG_SUM_AN    every voxel integrated in closed form (SUM-AN of
 *                     Sec. 2.1, the exact field of the piecewise-constant
 *                     density, finite on voxel faces, edges and corners)
 *                     instead of sampled by the quadrature rule; the rule is
 *                     then ignored.  Direct mode: FP64 only, every voxel in
 *                     closed form.  FMM mode (4^3-voxel leaves, either
 *                     precision, forward only): the voxels within 2 (mixed)
 *                     or 4 (FP64) voxels of an observer's own voxel in closed
 *                     form, the other voxels of its leaf's 27 neighbour
 *                     leaves by the midpoint rule plus a uniform cube's
 *                     l = 4 term, the far field from multipole expansions of
 *                     the exact voxel integrals.
 *   GF_FLAG_TEST_WAIT_TIMEOUT
 *                     testing aid for the failure path of the bounded device
 *                     waits (FMM, mixed precision, tensor-core M2L): the
 *                     M2L's MMA issuer first waits, with a short bound, on a
 *                     barrier that nothing completes; the wait runs out, the
 *                     kernel's roles stop, wait for their copies in flight,
 *                     free their tensor memory and return, and the next
 *                     gf_plan_check reports GF_ERR_DEVICE_CHECK (the
 *                     forward's output is then not valid).
 *   GF_FLAG_M2L_TENSOR FMM, FP64 precision: the forward M2L on the tensor
 *                     cores as in mixed precision (the FP64 inputs scaled
 *                     and split into FP16 high/low parts, three products,
 *                     FP32 accumulation per interaction-list offset);
 *                     every other stage in FP64.  The M2L then carries
 *                     about 22 bits (relative error near 1e-7 of its
 *                     output); gf_adjoint keeps the FP64 M2L. */
enum { GF_FLAG_M2L_SIMT = 1, GF_FLAG_SUM_AN = 2, GF_FLAG_TEST_WAIT_TIMEOUT = 4, GF_FLAG_M2L_TENSOR = 8 };

typedef struct {
    int32_t mode;        /* GF_MODE_DIRECT or GF_MODE_FMM                  */
    int32_t precision;   /* GF_PREC_FP64 or GF_PREC_MIXED                  */
    int32_t p;           /* FMM expansion degree (Eq. 9 series), 1..16;    */
                         /* K = (p+1)^2 coefficients per expansion         */
    int32_t leaf_vox;    /* FMM leaf edge in voxels (leaf = leaf_vox^3     */
                         /* voxels), 0 = library default                   */
    int32_t max_batch;   /* largest B passed to gf_forward/gf_adjoint, >=1 */
    int32_t reserved0;   /* GF_FLAG_* option flags, 0 = none               */
    double G;            /* gravitational constant; 0 = 6.67428e-11        */
} gf_options;

typedef struct gf_plan_s *gf_plan_t;

/*
 * gf_plan_create -- build everything that depends on the geometry only.
 *   grid, quad : the voxel brick and its quadrature rule (Sec. 2.1)
 *   obs_dev    : [M][3] FP64 observer coordinates x'_j of Eq. 7 (device)
 *   M          : number of observers, >= 0
 *   opt        : mode, precision, expansion degree, batch capacity, G
 * In FMM mode this builds the Morton-sorted octree of Sec. 2.3 on the
 * device: observer keys and their stable sort, the occupied boxes of every
 * level, the near lists and the interaction lists (for each box: the boxes
 * one level down from its parent's neighbourhood, i.e. children of boxes
 * within Chebyshev distance 1 of the parent, minus the box's own neighbours;
 * from level 2 on), and the translation operators.
 * Waits for the device.  On success *plan receives the new plan.
 */
gf_status gf_plan_create(const gf_grid *grid, const gf_quad *quad,
                         const double *obs_dev, int64_t M,
                         const gf_options *opt, void *stream,
                         gf_plan_t *plan);

/*
 * gf_forward -- evaluate Eq. 1 (discretised, Eq. 7 form) for B densities.
 *   rho_dev   : [B][nz][ny][nx] densities, FP64 or FP32 per rho_dtype
 *               (a point-source plan: [B][S / per_cell])
 *   B         : 1..opt.max_batch
 *   g_dev     : [B][M][3] FP64 output, observers in caller order, or NULL
 *   gz_dev    : [B][M] FP64 vertical component, or NULL (not both NULL
 *               unless M = 0)
 * Enqueues on `stream` and returns; allocates nothing, so it may be captured
 * in a CUDA graph.  Direct mode sums every pair (Sec. 2.1); FMM mode runs
 * P2M, M2M, M2L, L2L, L2P and the near-field P2P (Sec. 2.3, Fig. 3) and adds
 * near and far parts (Eq. 10).  The plan's workspaces (expansions, the M2L's
 * split inputs) serve all its calls: calls on one plan whose device work
 * overlaps (different streams) race, so serialise them or use one plan per
 * stream.
 */
gf_status gf_forward(gf_plan_t plan, const void *rho_dev, int32_t rho_dtype,
                     int32_t B, double *g_dev, double *gz_dev, void *stream);

/*
 * gf_adjoint -- transpose of gf_forward (Eq. 1 is linear in rho):
 *   grad_v = sum_j sum_c r_jc * d g_c(x'_j) / d rho_v
 *   r_dev    : [B][M][ncomp] FP64 weights on the outputs; ncomp = 1 weights
 *              g_z only, ncomp = 3 weights the full vector
 *   grad_dev : [B][nz][ny][nx] FP64 output
 * In FMM mode this runs the exact algebraic transpose of the forward FMM
 * (observers act as sources, voxel quadrature points as targets), so that
 * <A x, y> = <x, A^T y> holds to rounding.  Enqueues and returns.
 */
gf_status gf_adjoint(gf_plan_t plan, const double *r_dev, int32_t ncomp,
                     int32_t B, double *grad_dev, void *stream);

/*
 * gf_direct_forward_static -- direct-mode, mixed-precision forward solve
 * (the same sum and kernels as a GF_MODE_DIRECT / GF_PREC_MIXED plan) that
 * allocates no memory.  The paper has no counterpart; this entry point is
 * for callers that cannot allocate device memory when they need a solve:
 * code running inside another framework's allocator callback (which must
 * not re-enter it), processes whose device memory is fully held by a
 * caching pool they do not own, and services that forbid allocation after
 * start-up to keep a fixed footprint.
 *   grid, quad : as for gf_plan_create (host structs, read during the call)
 *   obs_dev    : [M][3] FP64 observers (device), 0 <= M <= 65536
 *   rho_dev    : [B][nz][ny][nx] densities (device), 1 <= B <= 64
 *   G          : gravitational constant, 0 selects 6.67428e-11
 *   g_dev      : [B][M][3] FP64 output or NULL;  gz_dev : [B][M] or NULL
 * Its scratch (quadrature rule and split observer coordinates, about
 * 1.6 MB) is a fixed device array in the library that every GPU loading the
 * library holds until the process exits; M above 65536 is rejected with
 * GF_ERR_INVALID_ARG.  The first call on each device looks up the array's
 * device address (with that device current), so make that first call
 * before any stream capture.  All calls share the one array and each call
 * rewrites all of it that it reads: calls whose device work overlaps (on
 * different streams, or from different threads) race, so serialise them.
 * Enqueues on `stream` and returns.
 */
gf_status gf_direct_forward_static(const gf_grid *grid, const gf_quad *quad,
                                   const double *obs_dev, int64_t M,
                                   const void *rho_dev, int32_t rho_dtype,
                                   int32_t B, double G, double *g_dev,
                                   double *gz_dev, void *stream);

/*
 * Serving: continuous batching of forward solves (an inversion issuing
 * solves on grids of uneven size).  A server owns `max_slots` CUDA streams
 * and a cache of resident plans -- octree, expansion workspaces, input and
 * output buffers, and the forward captured once in a CUDA graph -- keyed by
 * the caller's geometry id.  A background thread admits queued requests as
 * soon as a slot is free and the device memory the request's plan needs
 * (its gf_plan_bytes estimate) fits in the budget, evicting idle cached
 * plans least-recently-used first; requests on different slots run
 * concurrently on the device.  Kernels accumulate without atomics, so a
 * request's result is the same alone and in any mix.
 */
typedef struct gf_server_s *gf_server_t;

typedef struct {
    int32_t max_slots;     /* requests on the device at once, 1..64         */
    int32_t precision;     /* GF_PREC_FP64 or GF_PREC_MIXED (FMM mode)       */
    int32_t p;             /* expansion degree                               */
    int32_t leaf_vox;      /* 0 = library default                            */
    int32_t use_graphs;    /* replay each plan's forward as a CUDA graph     */
    int32_t device;        /* CUDA device of the server                      */
    size_t mem_budget;     /* device bytes for resident plans; 0 = 70% of    */
                           /* the free memory at creation                    */
    double G;              /* 0 = 6.67428e-11                                */
} gf_server_options;

/* One forward solve.  Host arrays must stay valid until the request has
 * completed (page-locked host memory makes the copies asynchronous).
 * Requests with the same geometry_id must have the same grid, quadrature
 * and observers: the server reuses the resident plan built for the first. */
typedef struct {
    gf_grid grid;
    gf_quad quad;
    const double *obs_host;   /* [M][3]                                     */
    int64_t M;
    uint64_t geometry_id;
    const void *rho_host;     /* [nz][ny][nx] densities                     */
    int32_t rho_dtype;        /* GF_DTYPE_F64 or GF_DTYPE_F32               */
    int32_t on_device;        /* 1: rho_host/gz_host/g_host are device      */
                              /* pointers instead of host pointers          */
    double *gz_host;          /* [M] output, or NULL                        */
    double *g_host;           /* [M][3] output, or NULL                     */
} gf_request;

typedef struct {
    int64_t submitted, completed, failed;
    int64_t plans_created, plans_evicted, graph_launches;
    size_t resident_bytes, mem_budget;
    double p50_ms, p99_ms, mean_ms;   /* latency: submit -> result on host */
    double busy_s;                    /* first submit -> last completion   */
} gf_server_stats;

gf_status gf_server_create(const gf_server_options *opt, gf_server_t *server);
/* Queue a request (returns at once); *ticket identifies it. */
gf_status gf_server_submit(gf_server_t server, const gf_request *req,
                           int64_t *ticket);
/* Wait for a request (timeout_ms < 0: no limit); latency in ms. Returns
 * GF_ERR_TIMEOUT if it has not completed in time, or the request's error. */
gf_status gf_server_wait(gf_server_t server, int64_t ticket, double timeout_ms,
                         double *latency_ms);
gf_status gf_server_stats_get(gf_server_t server, gf_server_stats *stats);
/* Wait for all requests, then release every resident plan and stream. */
gf_status gf_server_destroy(gf_server_t server);

/*
 * gf_plan_set_source_part -- restrict a FMM plan's forward to one part of
 * its sources, for a source-partitioned solve over several devices.  Eq. 1
 * is linear in the sources, so the field is the sum over parts of each
 * part's field, as the summation method of Sec. 2.1 splits the voxels over
 * processes and sums the station vector; one sum all-reduce of the outputs
 * of the nparts plans (one per device, each with its own part) gives the
 * whole field.
 *   part, nparts : 0 <= part < nparts <= 64; nparts = 1 restores all sources
 *   code_lo, code_hi : if not NULL, receive the part as a range [lo, hi) of
 *                  Morton codes (x -> bit 0, y -> bit 1, z -> bit 2 per level)
 *                  of the 64 boxes of octree level 2
 * A part is a range of level-2 boxes (every box of level 2 and deeper lies
 * under exactly one of them), cut so that the parts hold nearly equal
 * numbers of grid voxels.  The plan's near field and M2L then skip the
 * source boxes of the other parts.  FMM mode only (GF_ERR_UNSUPPORTED in
 * direct mode); gf_adjoint of a partitioned plan returns GF_ERR_UNSUPPORTED.
 * Host-side only: enqueues nothing.
 */
gf_status gf_plan_set_source_part(gf_plan_t plan, int32_t part, int32_t nparts, int32_t *code_lo,
                                  int32_t *code_hi);

/*
 * gf_hex_sources -- quadrature points of deformed hexahedral cells (the
 * general summation of Sec. 2.1: each cell is the trilinear image of the
 * reference cube [-1, 1]^3 and its integral is the rule's weighted sum of
 * the integrand times |det dx/dxi| at the rule's nodes).
 *   verts_dev : [ncell][8][3] FP64 corners (device); corner a = i + 2 j + 4 k
 *               sits at reference coordinates (2i - 1, 2j - 1, 2k - 1)
 *   quad      : nq nodes in [-1, 1]^3 and positive weights (host)
 *   precision : GF_PREC_FP64: every step in FP64.  GF_PREC_MIXED (for
 *               mixed-precision plans): the corners as 64-bit fixed point,
 *               the image relative to the cell's first corner and the
 *               Jacobian in FP32 -- positions within about 1e-6 of the
 *               cell's extent, weights within about 1e-6 relative.
 *   x_dev     : [ncell * nq][3] FP64 output, the trilinear image of node q
 *               of cell c at source s = c * nq + q
 *   a_dev     : [ncell * nq] FP64 output, the volume weight
 *               8 (w_q / sum w) |det dx/dxi(xi_q)| (the cell volume for a
 *               rule exact on the Jacobian)
 * The outputs feed gf_plan_create_points with per_cell = nq.  Enqueues on
 * `stream` and returns; ncell = 0 enqueues nothing.
 */
gf_status gf_hex_sources(const double *verts_dev, int64_t ncell, const gf_quad *quad, int32_t precision,
                         double *x_dev, double *a_dev, void *stream);

/*
 * gf_plan_create_points -- a plan over weighted point sources: source s at
 * x_s with volume weight a_s samples the density of cell s / per_cell, so
 *     g(r) = G sum_s rho_{s / per_cell} a_s (r - x_s) / |r - x_s|^3,
 * the N-body form of Eq. 7 for any source layout: the quadrature points of
 * deformed cells (gf_hex_sources) or a random point distribution whose
 * points carry the volumes of their Voronoi cells (Sec. 4).
 *   src_dev : [S][3] FP64 source positions (device, copied by the plan)
 *   wt_dev  : [S] FP64 volume weights (device, copied by the plan)
 *   S       : 0 <= S < 2^31, a multiple of per_cell
 *   per_cell: sources per density cell, >= 1; gf_forward then takes
 *             rho_dev as [B][S / per_cell]
 *   obs_dev : [M][3] FP64 observers (device)
 *   opt     : as for gf_plan_create; leaf_vox and GF_FLAG_SUM_AN do not
 *             apply (GF_ERR_UNSUPPORTED for the flag)
 * Direct mode sums every pair (FP64 with compensated sums, or mixed:
 * positions split into an exact integer number of quanta of 2^-22 of the
 * joint extent plus an FP32 fraction, FP32 pair terms, FP64 tile sums).
 * FMM mode builds a uniform octree whose leaf side makes about 48 sources
 * per leaf of the sources' extent; the sources are sorted by leaf, their
 * multipole expansions come from the points themselves, and the near field
 * sums the points of the 27 neighbour leaves.  An exact coincidence of an
 * observer and a source contributes nothing.  gf_adjoint and
 * gf_plan_set_source_part return GF_ERR_UNSUPPORTED on such plans.  Waits
 * for the device.
 */
gf_status gf_plan_create_points(const double *src_dev, const double *wt_dev, int64_t S, int32_t per_cell,
                                const double *obs_dev, int64_t M, const gf_options *opt, void *stream,
                                gf_plan_t *plan);

/* Release a plan and everything it owns (waits for its device work). */
gf_status gf_plan_destroy(gf_plan_t plan);

/* Wait for the plan's device work and report any device-side check that
 * failed since the last call (GF_ERR_DEVICE_CHECK, e.g. a non-finite
 * density or a bounded wait that gave up), then clear it. */
gf_status gf_plan_check(gf_plan_t plan, void *stream);

/* One-line message describing the calling thread's last failure. */
const char *gf_last_error(void);

/* Device bytes a plan with these inputs would hold (upper bound), without
 * allocating; used for admission by memory footprint. */
gf_status gf_plan_bytes(const gf_grid *grid, const gf_quad *quad, int64_t M,
                        const gf_options *opt, size_t *bytes);

/* Octree geometry chosen by a FMM plan (zeros in direct mode). */
typedef struct {
    int32_t mode, precision, p, K;    /* K = (p+1)^2                       */
    int32_t L;                        /* leaf level; 2^L leaves per axis   */
    int32_t leaf_vox;                 /* voxels per leaf edge              */
    int64_t voxel_offset[3];          /* voxel (0,0,0) sits at tree voxel  */
                                      /* coordinates voxel_offset          */
    double lo[3];                     /* root cube lower corner, metres    */
    double leaf_side;                 /* leaf edge, metres                 */
    double inv_leaf_side;             /* 1/leaf_side used for the keys     */
    int64_t n_target_boxes[24];       /* occupied observer boxes per level */
    int64_t src_lo[24][3];            /* source boxes per level: inclusive */
    int64_t src_hi[24][3];            /* integer bounds of the dense block */
    int64_t M, n_sources;             /* observers; quadrature points (or  */
                                      /* voxels, with GF_FLAG_SUM_AN; the  */
                                      /* S points of a point-source plan)  */
    int64_t near_pairs;               /* (observer, source) pairs summed   */
                                      /* directly in the near field        */
    int64_t m2l_pairs;                /* (observer box, source box) pairs  */
                                      /* of all interaction lists          */
    size_t device_bytes;
} gf_plan_info;

gf_status gf_plan_get_info(gf_plan_t plan, gf_plan_info *info);

/*
 * Copy a FMM plan's tree to host buffers (verification aid; waits):
 *   perm_host  : [M] int32, observers in (Morton key, original index) order
 *   keys_host  : [M] uint64 leaf key of each sorted observer
 *   level      : 2..L
 *   box_keys_host : [n_target_boxes[level]] uint64 occupied boxes, ascending
 *   ilist_host : [n_target_boxes[level]][316] int64 source box per
 *                interaction-list offset (offset order: dz, dy, dx each
 *                ascending over -3..3, skipping max-norm <= 1), as the
 *                source box's Morton key, or -1 when that offset is not in
 *                the box's list or falls outside the source block
 *   near_host  : [n_target_boxes[L]][27] int64 (only for level == L): the
 *                near-list source leaf key per offset (dz,dy,dx ascending
 *                over -1..1), or -1
 * Any pointer may be NULL to skip that array.
 */
gf_status gf_plan_export_tree(gf_plan_t plan, int32_t level, int32_t *perm_host,
                              uint64_t *keys_host, uint64_t *box_keys_host,
                              int64_t *ilist_host, int64_t *near_host);

/* Stage timing (verification and profiling aid).  When enabled, each
 * gf_forward records CUDA events between its stages on its stream;
 * gf_plan_stage_times waits for the last forward and returns the device
 * time of each stage in milliseconds:
 *   [0] leaf-blocked densities  [1] P2M  [2] M2M
 *   [3] M2L input split (mixed precision: scaled FP16 parts of every level's
 *       multipole expansions)  [4] M2L  [5] L2L
 *   [6] evaluation (near field + L2P + combine)  [7] whole forward
 * (direct mode: only [6] and [7]).  Without timing, an FMM plan runs the
 * evaluation's near field on a second stream of its own beside the M2L and
 * the L2L (forked from and joined back into the forward's stream); with
 * timing on it runs in line, so that every stage is timed alone (the field
 * is the same bit for bit).  Timing must be off while a forward is
 * captured in a CUDA graph. */
#define GF_NUM_STAGES 8
gf_status gf_plan_set_timing(gf_plan_t plan, int32_t enable);
gf_status gf_plan_stage_times(gf_plan_t plan, double *ms);

int32_t gf_version(void);

/* Number of CUDA kernels this library has launched since it was loaded
 * (all plans and threads); lets a caller count the library's launches in a
 * timed region. */
int64_t gf_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* GF_H */
