// Closed-loop receding-horizon control (Sec. V-B): per control step c every
// scenario re-solves the ADMM of Sec. IV-B over the next N steps from its
// measured state, warm-started from the previous plan shifted by one step,
// with only the obstacles inside its sensing window; then the first control
// drives the plant one Euler step and the true state is checked for
// collision against every obstacle (scale LP, Sec. III-A).
#include "oca_common.cuh"
#include "oca_kernels.h"
#include "oca_models.cuh"
#include "oca_solvers.cuh"

namespace oca {

// horizon window of step c: reference rows, warm-start shift, measured
// state as s_0, sensing mask (one warp per scenario)
template <typename T, int KIND>
__global__ void __launch_bounds__(32) k_mpc_window(MpcArgs<T> a) {
    constexpr int NS = MDims<KIND>::NS, NU = MDims<KIND>::NU, D = MDims<KIND>::D;
    const int s = blockIdx.x, lane = threadIdx.x;
    const ScenMeta sm = a.meta[s];
    const int N = sm.N;
    const T *ref = a.ref + (long long)s * a.T_ref * NS;
    for (int e = lane; e < (N + 1) * NS; e += 32) {
        const int t = e / NS, i = e % NS;
        const int r = min(a.c + t, a.T_ref - 1);
        a.s_ref[(long long)(sm.state0 + t) * NS + i] = ref[(long long)r * NS + i];
    }
    if (a.c > 0) {
        // s_t <- s_{t+1} (t = 1..N-1), u_t <- u_{t+1} (t = 0..N-2); each lane
        // owns one component, so the in-place ascending copy is race-free
        if (lane < NS)
            for (int t = 1; t < N; ++t)
                a.s[(long long)(sm.state0 + t) * NS + lane] = a.s[(long long)(sm.state0 + t + 1) * NS + lane];
        if (lane < NU)
            for (int t = 0; t + 1 < N; ++t)
                a.u[(long long)(sm.ctrl0 + t) * NU + lane] = a.u[(long long)(sm.ctrl0 + t + 1) * NU + lane];
    }
    if (lane < NS) a.s[(long long)sm.state0 * NS + lane] = a.x[(long long)s * NS + lane];
    // sensing window: obstacle centres within +-win of the position
    for (int j = lane; j < sm.M; j += 32) {
        const int gm = sm.obs0 + j;
        bool in = true;
#pragma unroll
        for (int i = 0; i < D; ++i)
            if (a.win[i] > T(0)) in &= m_abs(a.obs_center[(long long)gm * D + i] - a.x[(long long)s * NS + i]) <= a.win[i];
        a.mask[gm] = in ? 1 : 0;
    }
}

// pair arrays shifted one step along t: (y, zeta, xi) at (j, part, t) <- (j, part, t + 1)
// for t = 1..N-1; one thread per (obstacle, part) block of a scenario
template <typename T>
__global__ void k_mpc_shift_pairs(MpcArgs<T> a, int D) {
    const int s = blockIdx.y;
    const ScenMeta sm = a.meta[s];
    const int blk = blockIdx.x * blockDim.x + threadIdx.x;
    if (blk >= sm.M * sm.NP) return;
    const int j = blk / sm.NP, part = blk % sm.NP;
    const int gm = sm.obs0 + j, gp = sm.part0 + part;
    const int nr = a.g.part_nf[gp], no = a.g.obs_nf[gm];
    const long long P = a.P, p0 = sm.pair0 + (long long)blk * sm.N;
    for (int t = 0; t + 1 < sm.N; ++t) {
        const long long p = p0 + t;
        for (int k = 0; k < nr; ++k) a.y[(long long)k * P + p] = a.y[(long long)k * P + p + 1];
        for (int m = 0; m < no; ++m) a.y[(long long)(a.FR + m) * P + p] = a.y[(long long)(a.FR + m) * P + p + 1];
        a.y[(long long)(a.FR + a.FO) * P + p] = a.y[(long long)(a.FR + a.FO) * P + p + 1];
        a.zeta[p] = a.zeta[p + 1];
        for (int i = 0; i < D; ++i) a.xi[(long long)i * P + p] = a.xi[(long long)i * P + p + 1];
    }
}

// plant: x <- x + dt f_c(x, u_0), u_0 the plan's first control clipped to
// the control box (zero where the solve left it non-finite); histories
template <typename T, int KIND>
__global__ void k_mpc_plant(MpcArgs<T> a, int n_scen) {
    constexpr int NS = MDims<KIND>::NS, NU = MDims<KIND>::NU;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_scen) return;
    const ScenMeta sm = a.meta[s];
    T x[NS], u0[NU], f[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) x[i] = a.x[(long long)s * NS + i];
    if (a.c == 0)
#pragma unroll
        for (int i = 0; i < NS; ++i) a.x_hist[(long long)s * (a.n_steps + 1) * NS + i] = x[i];
#pragma unroll
    for (int i = 0; i < NU; ++i) {
        T v = a.u[(long long)sm.ctrl0 * NU + i];
        if (!m_finite(v)) v = T(0);
        u0[i] = fmin(fmax(v, a.model.u_lo[i]), a.model.u_hi[i]);
        a.u_hist[((long long)s * a.n_steps + a.c) * NU + i] = u0[i];
    }
    dynamics<T, KIND>(a.model, x, u0, f, nullptr, nullptr);
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        x[i] += a.model.dt * f[i];
        a.x[(long long)s * NS + i] = x[i];
        a.x_hist[((long long)s * (a.n_steps + 1) + a.c + 1) * NS + i] = x[i];
    }
    a.iters_hist[(long long)s * a.n_steps + a.c] = a.iters[s];
}

// collision of the true state with every obstacle: alpha* < 1 for some
// (part, obstacle) marks the scenario with the first step it happened
template <typename T, int KIND>
__global__ void k_mpc_collide(MpcArgs<T> a) {
    constexpr int NS = MDims<KIND>::NS, D = MDims<KIND>::D;
    const int s = blockIdx.y;
    const ScenMeta sm = a.meta[s];
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= sm.M * sm.NP) return;
    const int j = e / sm.NP, part = e % sm.NP;
    const int gm = sm.obs0 + j, gp = sm.part0 + part;
    T x[NS], off[D];
    Lane<T, D> L;
#pragma unroll
    for (int i = 0; i < NS; ++i) x[i] = a.x[(long long)s * NS + i];
#pragma unroll
    for (int i = 0; i < D; ++i) off[i] = a.g.part_off[gp * D + i];
    part_pose<T, KIND>(a.model, a.g.part_link[gp], off, x, L.rho, L.R, nullptr, nullptr, nullptr);
    L.A = a.g.part_A + (long long)gp * a.g.FR * D;
    L.b = a.g.part_b + (long long)gp * a.g.FR;
    L.nr = a.g.part_nf[gp];
    L.C = a.g.obs_C + (long long)gm * a.g.FO * D;
    L.d = a.g.obs_d + (long long)gm * a.g.FO;
    L.no = a.g.obs_nf[gm];
    int bas[D + 1];
    T xB[D + 1], alpha;
    lp_solve<T, D>(L, bas, xB, alpha);
    if (alpha < T(1)) atomicCAS(a.collided + s, -1, a.c + 1);
}

template <typename T, int KIND>
cudaError_t mpc_launch_t(const MpcArgs<T> &a, int stage, int n_scen, int max_blk, cudaStream_t st) {
    switch (stage) {
        case 0: k_mpc_window<T, KIND><<<n_scen, 32, 0, st>>>(a); break;
        case 1: k_mpc_shift_pairs<T><<<dim3((max_blk + 63) / 64, n_scen), 64, 0, st>>>(a, MDims<KIND>::D); break;
        case 2: k_mpc_plant<T, KIND><<<(n_scen + 63) / 64, 64, 0, st>>>(a, n_scen); break;
        default: k_mpc_collide<T, KIND><<<dim3((max_blk + 63) / 64, n_scen), 64, 0, st>>>(a); break;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mpc(const MpcArgs<T> &a, int stage, int n_scen, int max_blk, cudaStream_t st) {
    if (n_scen <= 0) return cudaSuccess;
    switch (a.model.kind) {
        case 0: return mpc_launch_t<T, 0>(a, stage, n_scen, max_blk, st);
        case 1: return mpc_launch_t<T, 1>(a, stage, n_scen, max_blk, st);
        case 2: return mpc_launch_t<T, 2>(a, stage, n_scen, max_blk, st);
    }
    return cudaErrorInvalidValue;
}

template cudaError_t launch_mpc<float>(const MpcArgs<float> &, int, int, int, cudaStream_t);
template cudaError_t launch_mpc<double>(const MpcArgs<double> &, int, int, int, cudaStream_t);

}  // namespace oca
