// gf_m2l.cuh -- the multipole-to-local stage (Sec. 2.3: an ME is turned
// into an LE for every box of the interaction list).
#pragma once

#include "gf_fmm.cuh"

namespace gf {

gf_status m2l_upload_offsets(const signed char h_il[8][189][3]);
gf_status m2l_prepare_tables(Tables *T, cudaStream_t st);
// Tensor-core image of a P2M matrix [b3][K] (b3 a multiple of 16).
gf_status build_p2m_tc_image(const double *pd, int K, int npad, int b3, float *img, cudaStream_t st);
// Tensor-core image of the P2M into the parent level (8 operators [b3][K]).
gf_status build_p2m_up_tc_image(const double *q, int K, int npad, int b3, float *img, cudaStream_t st);

// LE_l[t] = sum over the interaction list of box t of T_o * ME_l[t + o],
// for every observer box t of every level (overwrites each LE_l).  Mixed
// precision runs on the tensor cores (tcgen05, 3xTF32) unless the plan asks
// for the SIMT kernel; FP64 runs on the SIMT kernel.
// adj: the transpose, MEdual_l[s] = sum_{o in IL(class of s)} T_{-o}^T LEdual_l[s + o]
// over every source box s (observer boxes found through the level's map).
// fork: when non-null, recorded on st right before the M2L kernels are
// launched (after the input split).
template <class T>
gf_status m2l_run(gf_plan_s *plan, int B, bool adj, cudaStream_t st, cudaEvent_t fork = nullptr);
template <class T>
gf_status m2l_level(gf_plan_s *plan, int level, int B, bool adj, cudaStream_t st);

// Batched translations (Ts = storage, Tc = arithmetic); in mixed precision
// the forward M2M / L2L run on the tensor cores (3xTF32), otherwise on the
// SIMT cores:
//   kind 0  M2M into `level` from level + 1 (store)
//   kind 1  L2L into `level` from level - 1 (update)
//   kind 2  M2M^T into `level` from level - 1 (update), over source boxes
//   kind 3  L2L^T into `level` from level + 1 (store), over observer boxes
template <class Ts, class Tc>
gf_status translate_run(gf_plan_s *plan, int level, int kind, int B, cudaStream_t st);

// Plan-time set-up of the tensor-core path (level descriptors on the device).
gf_status m2l_tc_prepare(gf_plan_s *plan);
// The adjoint's level tables (built on the plan's first adjoint call).
gf_status m2l_tc_prepare_adj(gf_plan_s *plan);

// P2M on the tensor cores (mixed precision, leaves of 16k voxels): ME of
// every leaf = P^T x its leaf-blocked masses.  p2m_tc_ok says whether the
// plan and batch size allow it.
bool p2m_tc_ok(const gf_plan_s *plan, int B);
gf_status p2m_run_tc(gf_plan_s *plan, int B, cudaStream_t st);
// Whether the parent level's expansions can come straight from the leaf
// masses (p2m_up_run_tc) instead of P2M at every leaf and the M2M out of the
// leaf level: mixed precision on the tensor cores, L - 1 > 2 (level 2 keeps
// its FP64 M2M).  The leaf expansions are then computed only for the z-slabs
// that the leaf level's M2L reads.
bool p2m_up_ok(const gf_plan_s *plan, int B);
// Whether the P2M into level L-1 can read the densities straight from the
// caller's grid (FP32, 16-byte aligned, every axis and the grid's place in
// the tree multiples of the 4-voxel leaf edge); grid NULL: the leaf-blocked
// masses of every leaf.
bool p2m_up_grid_ok(const gf_plan_s *plan, const void *rho, int rho_dtype);
gf_status p2m_up_run_tc(gf_plan_s *plan, int B, const float *grid, cudaStream_t st);

}  // namespace gf
