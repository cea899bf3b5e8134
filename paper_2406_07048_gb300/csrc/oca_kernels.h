// Host-side launchers of the CUDA kernels (one translation unit each).
#pragma once

#include "oca_common.cuh"

namespace oca {

template <typename T>
cudaError_t launch_pose(const PoseArgs<T> &a, int maxQ, cudaStream_t st);

template <typename T>
cudaError_t launch_pair(const PairArgs<T> &a, int dim, int mode, int solver, int n_tiles, int W, cudaStream_t st);

template <typename T>
cudaError_t launch_scale(const ScaleArgs<T> &a, int dim, int n_tiles, int W, cudaStream_t st);

template <typename T>
cudaError_t launch_riccati(const RicArgs<T> &a, bool f32, cudaStream_t st);

long long riccati_scratch_elems(int kind, int N);

}  // namespace oca
