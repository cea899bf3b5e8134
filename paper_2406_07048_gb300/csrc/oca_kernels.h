// Host-side launchers of the CUDA kernels (one translation unit each).
#pragma once

#include "oca_common.cuh"

namespace oca {

template <typename T>
cudaError_t launch_pose(const PoseArgs<T> &a, int maxQ, cudaStream_t st);

template <typename T>
cudaError_t launch_pair(const PairArgs<T> &a, int dim, int mode, int solver, int n_tiles, int W, cudaStream_t st);

// largest warps per tile the pair kernels are compiled for (their launch bound)
int pair_max_warps(int dim, size_t es);
// dynamic shared memory of a pair-kernel launch with W warps per tile
size_t pair_smem_bytes(int dim, size_t es, int W, int mode, int solver, int FR, int FO);

template <typename T>
cudaError_t launch_scale(const ScaleArgs<T> &a, int dim, int n_tiles, int W, cudaStream_t st);

template <typename T>
cudaError_t launch_cert(const CertArgs<T> &a, int n_tiles, int W, cudaStream_t st);

template <typename T>
cudaError_t launch_riccati(const RicArgs<T> &a, bool f32, cudaStream_t st);

long long riccati_scratch_elems(int kind, int N);

// adjoint of a taped ADMM solve (oca_adjoint.cu)
template <typename T>
cudaError_t launch_adj_seed(const AdjTrajArgs<T> &a, int n_scen, cudaStream_t st);
template <typename T>
cudaError_t launch_adj_traj(const AdjTrajArgs<T> &a, int n_scen, cudaStream_t st);
template <typename T>
cudaError_t launch_adj_pair(const AdjPairArgs<T> &a, int dim, int n_tiles, int W, cudaStream_t st);
template <typename T>
cudaError_t launch_adj_alpha(const AdjAlphaArgs<T> &a, int dim, int n_tiles, int W, const int *iters,
                             const T *tape_s, long long s_slot, int NS, int n_scen, T *states_out,
                             const PoseArgs<T> &pa, int maxQ, cudaStream_t st);
// closed loop (oca_mpc.cu): stage 0 window/shift/mask, 1 pair shift, 2 plant, 3 collision
template <typename T>
cudaError_t launch_mpc(const MpcArgs<T> &a, int stage, int n_scen, int max_blk, cudaStream_t st);
// the paper's Lemke route for the pair QPs (oca_lemke.cu)
template <typename T>
cudaError_t launch_lemke(const LemkeArgs<T> &a, int dim, cudaStream_t st);
template <typename T>
cudaError_t launch_adj_finish(const double *gd, const T *obs_C, const int *obs_nf, int M_tot, int FO, int dim,
                              T *grad_d, T *grad_ctr, cudaStream_t st);

}  // namespace oca
