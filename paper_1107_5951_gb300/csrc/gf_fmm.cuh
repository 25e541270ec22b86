// gf_fmm.cuh -- octree and expansion workspaces of a FMM plan (Sec. 2.3).
//
// The tree has uniform depth L.  Leaves are cubes of b^3 voxels aligned to
// the voxel grid, so every box that overlaps the grid holds sources and the
// source boxes of each level form a dense integer block; their multipole
// expansions (ME) are stored densely over that block.  Observers are sorted
// by Morton key; the boxes that contain observers (and their ancestors) are
// listed per level in ascending key order and carry the local expansions
// (LE).  All FMM arithmetic is done in voxel units (h = 1): sources carry
// q = rho * w_q / sum(w), and the result is scaled by G*h at the end.
#pragma once

#include "gf_internal.cuh"

namespace gf {

struct FmmLevel {
    int64_t slo[3] = {0, 0, 0};   // source block: lowest box coordinate
    int64_t sn[3] = {0, 0, 0};    // source block extent (boxes per axis)
    int64_t ns = 0;               // number of source boxes
    int64_t nt = 0;               // number of observer boxes
    uint64_t *tkey = nullptr;     // [nt] Morton keys, ascending
    int32_t *tparent = nullptr;   // [nt] index of the parent box at level-1
    int32_t *m2l_order = nullptr; // [nt] observer boxes grouped by parity class
    int64_t cls_off[9] = {0};     // class c: m2l_order[cls_off[c] .. cls_off[c+1])
    // z-slabs [m2l_z0, m2l_z1] of the source block (relative to slo[2]) that
    // an interaction list of this level's observer boxes can reach: the
    // only multipole expansions the forward M2L reads (empty when z0 > z1)
    int64_t m2l_z0 = 0, m2l_z1 = -1;
    void *me = nullptr;           // [ns][B][KS]
    void *le = nullptr;           // [nt][B][KS]
};

// Translation operators for one expansion degree, shared by all plans on a
// device (they depend on p only, thanks to the scaled expansions).  Stored
// transposed (input component major) for the SIMT kernels:
//   m2l_*[off][c][k]  off = (dz+3)*49 + (dy+3)*7 + (dx+3)
//   m2m_*[oct][c][k], l2l_*[oct][c][k]  oct = (x&1) | (y&1)<<1 | (z&1)<<2
//                                          of the child box
struct Tables {
    int device = -1, p = 0, K = 0, Kp = 0;   // Kp = K rounded up to 8
    // Tensor-core operand images (mixed precision), one bulk copy per
    // pipeline stage, in the 64-byte-swizzled K-major shared-memory layout
    // (rows of 64 bytes):
    //   m2l_tc, am2l_tc  [343 slots][tc_nck_h chunks of 32 inputs][hi|lo][Npad][32]
    //                    FP16 parts of T_o[k_out][k_in] * colscale[k_out]
    //   m2m_tc, l2l_tc   [8][tc_nck chunks of 16 inputs][hi|lo][Npad][16]
    //                    TF32 parts of the operator
    // colscale (m2l_cs / am2l_cs: [Npad] scale, then [Npad] its inverse) is
    // the power of two that brings each output column's largest entry over
    // all offsets into (2^13, 2^14], so that both FP16 parts of every entry
    // that matters are normal numbers.
    void *m2l_tc = nullptr, *am2l_tc = nullptr;
    float *m2l_cs = nullptr, *am2l_cs = nullptr;
    int tc_npad = 0, tc_nck = 0, tc_nck_h = 0;
    double *m2l_d = nullptr;
    float *m2l_f = nullptr;
    double *m2m_d = nullptr, *l2l_d = nullptr;
    float *m2m_f = nullptr, *l2l_f = nullptr;
    // Transposed operators for the adjoint, in the same input-major layout:
    //   am2l[slot(o')] = (T_{-o'})^T, o' = observer box - source box
    //   am2m[oct] = (T_M2M,oct)^T,  al2l[oct] = (T_L2L,oct)^T
    double *am2l_d = nullptr, *am2m_d = nullptr, *al2l_d = nullptr;
    float *am2l_f = nullptr, *am2m_f = nullptr, *al2l_f = nullptr;
    float *m2m_tc = nullptr, *l2l_tc = nullptr;   // [8] operator images (tensor-core translations)
};

gf_status get_tables(int device, int p, cudaStream_t st, const Tables **out);

struct FmmPlan {
    int L = 0, b = 0, p = 0, K = 0, B = 1, nq = 1;
    int KS = 0;                   // row stride of ME/LE arrays (K padded to 32 in mixed)
    bool mixed = false;
    bool m2l_tc64 = false;        // FP64 plan whose forward M2L runs on the tensor cores
    // weighted point sources: one leaf of side s_leaf is the length unit
    // (b = 1), masses are [B][S] in leaf order, and the P2M and near field
    // read the sources' positions (gf_points.cu)
    bool points = false;
    int64_t voff[3] = {0, 0, 0};  // grid voxel (0,0,0) sits at tree voxel voff
    double lo[3] = {0, 0, 0};     // root lower corner (m)
    double h = 1, s_leaf = 1, inv_s = 1;
    FmmLevel lev[kMaxLevels + 1];
    int32_t *perm = nullptr;      // [M] sorted position -> caller index
    uint64_t *okey = nullptr;     // [M] leaf key of each sorted observer
    int32_t *leaf_beg = nullptr;  // [nt_L + 1] observer range of each leaf
    float *tloc_f = nullptr;      // [M][3] offset from own leaf centre (voxel units)
    double *tloc_d = nullptr;
    int4 *items = nullptr;        // evaluation work: (leaf, first, count <= 64, 0)
    int64_t n_items = 0;
    unsigned long long *eval_queue = nullptr;   // evaluation item queue (2 counters, zero between launches)
    void *mass = nullptr;         // [ns_L][B][b^3] voxel densities, leaf-blocked
    void *nsum = nullptr;         // [B][M][6] near-field sums (hi, lo per component) in observer-key order
    double *p2m_d = nullptr;      // [b^3][K] quadrature-folded P2M matrix
    float *p2m_f = nullptr;
    const Tables *tab = nullptr;
    void *tc_levels = nullptr;                  // tensor-core M2L level table
    // largest |input| of each level's M2L (bits of a non-negative float;
    // [0, kMaxLevels]: forward, [kMaxLevels + 1, 2 kMaxLevels + 1]: adjoint),
    // reduced on the device before each tensor-core M2L
    uint32_t *tc_amax = nullptr;
    bool amax_fused = false;      // this forward's expansion writers took the M2L input maxima
    float *m2l_part = nullptr;    // forward M2L with two CTAs per tile: [tiles][2][128][Npad] partial rows
    int *m2l_cnt = nullptr;       // [tiles][8] arrivals
    int m2l_part_tiles = 0;       // tiles m2l_part holds (0: no sharing)
    // the M2L inputs of levels 2..L split into scaled FP16 high and low
    // parts: for every input row and 32-wide chunk, 64 bytes of high parts
    // then 64 bytes of low parts (the same byte offsets as the FP32 rows)
    unsigned char *tc_split = nullptr, *tc_split_adj = nullptr;
    std::vector<unsigned char> tc_levels_host;
    // adjoint: per level, observer-box index over the source block widened
    // by 3 boxes (-1 where no observer box), the children of each observer
    // box (8 slots by position, -1 if absent), and the source boxes' count
    // per parity class (prefix sums)
    int32_t *imap[kMaxLevels + 1] = {};
    int64_t mlo[kMaxLevels + 1][3] = {}, mn[kMaxLevels + 1][3] = {};
    int32_t *child[kMaxLevels + 1] = {};
    int64_t scls_off[kMaxLevels + 1][9] = {};
    bool adj_ready = false;                      // adjoint structures built (on first adjoint)
    void *tc_levels_adj = nullptr;
    std::vector<unsigned char> tc_levels_adj_host;
    float *p2m_tc = nullptr;                     // tensor-core P2M operator image
    // tensor-core image of the P2M into level L-1: for each child position
    // o of a parent, Q_o[v][k] = sum_i P[v][i] M2M_o[i][k] (the leaf P2M
    // followed by the M2M to the parent), so a parent's expansion comes
    // straight from the masses of its 8 child leaves
    float *p2m_up_tc = nullptr;
    void *tc_xlate = nullptr;                    // tensor-core M2M / L2L / P2M level tables
    std::vector<unsigned char> tc_xlate_host;
};

// adjoint set-up and driver (gf_adjoint.cu)
gf_status fmm_adjoint_prepare(gf_plan_s *plan, cudaStream_t st);

// Interaction-list offsets of a box whose position inside its parent is
// `cls` ((x&1) | (y&1)<<1 | (z&1)<<2): the 189 vectors o with max-norm 2 or 3
// such that the parent of (box + o) neighbours the box's parent, in (dz, dy,
// dx) ascending order.
void il_offsets_host(int cls, signed char out[189][3]);

// Plan-time helpers (gf_fmm.cu)
gf_status fmm_alloc_workspaces(gf_plan_s *plan, cudaStream_t st);
// Fixed point with k fractional bits for the coordinates of a root box and
// the bounding box bb (every coordinate below 2^61 in magnitude): the root
// corner and half a leaf side in those units, and 2^-k / h.  Returns k, or
// -1 when the coordinates are too large for 64-bit fixed point (gf_tree.cu).
int fixed_point_frame(const FmmPlan *F, const double bb[6], long long lofix[3], long long *halfleaf_fix,
                      float *fix_to_unit);
// The observer side of the tree for a root geometry set in the plan, then
// the workspaces (gf_tree.cu).
gf_status fmm_observer_tree(gf_plan_s *plan, const double *obs, const double oz[2], const double obs_lo[3],
                            const double obs_hi[3], const double bb[6], cudaStream_t st);

}  // namespace gf
