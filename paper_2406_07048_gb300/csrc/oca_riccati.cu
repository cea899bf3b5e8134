// Trajectory step of the ADMM (Sec. IV-B eqn:ADMM_state_updates, one SQP
// QP per iteration) and the per-scenario stopping rule.  The state/control
// boxes of eqn:MPC_opt_origin are a further ADMM block: a bounded copy z of
// (s, u) with scaled dual w, so that the step stays an unconstrained LQ
// problem (Riccati) with the augmented term 0.5 rho_b |(s,u) - z + w|^2; a
// proximal term 0.5 damp |(s,u) - (s,u)^j|^2 damps the SQP step.
//
// One warp per scenario.  At launch j the warp
//   1. tests the stopping rule of iteration j-1 (Sec. IV-B):
//        r_pri  = sum dzeta^2 + |dxi|^2     (partials written by the pair kernel's head at j)
//        r_dual = sum |dlambda|^2 + |dmu|^2 (partials written by the pair kernel at j-1)
//      and retires the scenario when both are below their tolerances or j = max_iter;
//   2. otherwise assembles the LQ stage terms at (s^j, u^j): Euler dynamics
//      linearised (A_t, B_t, c_t), tracking cost of eqn:navigation_cost and
//      the Gauss-Newton model of sigma/2 sum |r_ijt(s_t)|^2 rebuilt from the
//      per-(part, t) statistics W, Wc, E through the pose Jacobians;
//   3. runs the backward Riccati recursion (factorisation precision F) and
//      the forward sweep, writing s^{j+1}, u^{j+1} and the new poses.
#include "oca_common.cuh"
#include "oca_kernels.h"
#include "oca_ric.cuh"

namespace oca {

long long riccati_scratch_elems(int kind, int N) {
    switch (kind) {
        case 0: return RicLayout<4, 2>::size(N);
        case 1: return RicLayout<5, 2>::size(N);
        default: return RicLayout<12, 4>::size(N);
    }
}

template <typename T, int KIND>
__device__ void finish_scenario(const RicArgs<T> &a, const ScenMeta &sm, int s, int status, int iters, double rp, double rd) {
    constexpr int NS = MDims<KIND>::NS, NU = MDims<KIND>::NU;
    const int lane = threadIdx.x;
    double F = 0.0;
    for (int t = lane; t <= sm.N; t += 32) {
        for (int i = 0; i < NS; ++i) {
            const double e = double(a.s[(long long)(sm.state0 + t) * NS + i]) - double(a.s_ref[(long long)(sm.state0 + t) * NS + i]);
            F += double(a.model.Qs[i]) * e * e;
        }
        if (t < sm.N)
            for (int i = 0; i < NU; ++i) {
                const double uu = double(a.u[(long long)(sm.ctrl0 + t) * NU + i]);
                F += double(a.model.Qu[i]) * uu * uu;
            }
    }
    F = warp_sum(F);
    if (lane == 0) {
        a.scen_status[s] = status;
        a.status_out[s] = status;
        a.iters_out[s] = iters;
        a.r_pri_out[s] = T(rp);
        a.r_dual_out[s] = T(rd);
        a.cost_out[s] = T(F);
        atomicSub(a.active_count, 1);
    }
}

// NT threads per scenario: warp 0 runs every phase but the Riccati
// recursion, which all NT threads share (NT > 32 for the 12-state model,
// whose per-step products have 150-200 entries).
template <typename T, typename F, int KIND, int NT>
__global__ void __launch_bounds__(NT) k_riccati(RicArgs<T> a) {
    constexpr int NS = MDims<KIND>::NS, NU = MDims<KIND>::NU, D = MDims<KIND>::D;
    const int s = blockIdx.x;
    const int lane = threadIdx.x;
    if (a.scen_status[s] != kActive) return;
    const int j = *a.iter;
    if (j > a.max_iter) return;
    const ScenMeta sm = a.meta[s];
    const int N = sm.N;
    __shared__ int s_retired;

    // ---- 1. stopping rule of iteration j-1 (warp 0)
    if (lane < 32) {
        s_retired = 0;
    if (j >= 1) {
        const double *rcur = a.res + (size_t)(j & 1) * a.n_tiles * 2;
        const double *rprev = a.res + (size_t)((j - 1) & 1) * a.n_tiles * 2;
        double rp = 0.0, rd = 0.0;
        for (int k = lane; k < sm.ntile; k += 32) {
            rp += rcur[(size_t)(sm.tile0 + k) * 2];
            rd += rprev[(size_t)(sm.tile0 + k) * 2 + 1];
        }
        rp = warp_sum(rp) + a.box_res[2 * s];      // + box-block residuals of iteration j-1
        rd = warp_sum(rd) + a.box_res[2 * s + 1];
        const bool conv = rp <= double(a.eps_pri) && rd <= double(a.eps_dual);
        if (conv || j >= a.max_iter) {
            finish_scenario<T, KIND>(a, sm, s, conv ? OCA_SCEN_CONVERGED : OCA_SCEN_MAX_ITER, j, rp, rd);
            s_retired = 1;
        }
    } else if (a.max_iter <= 0) {
        finish_scenario<T, KIND>(a, sm, s, OCA_SCEN_MAX_ITER, 0, 0.0, 0.0);
        s_retired = 1;
    }
    }
    ric_sync<NT>();
    if (s_retired) return;

    F *scr = reinterpret_cast<F *>(a.scratch) + a.scratch0[s];

    // ---- 2. stage assembly, lanes over t (in the array precision T; only
    // the factorisation below runs in F)
    StageParams<T> sp;
    sp.model = a.model;
    sp.g = a.g;
    sp.sigma = a.sigma;
    sp.rho_box = a.rho_box;
    sp.damp = a.damp;
    sp.s_ref = a.s_ref;
    sp.Qtot = a.Qtot;
    StageSrc<T> src;
    src.s = a.s;
    src.u = a.u;
    src.zs = a.box_zs;
    src.ws = a.box_ws;
    src.zu = a.box_zu;
    src.wu = a.box_wu;
    src.stats = a.stats;
    for (int t = lane; t <= N; t += NT) assemble_stage<T, F, KIND>(sp, src, sm, t, scr);
    ric_sync<NT>();

    // ---- 3. backward Riccati recursion (all NT threads), 4. forward sweep (warp 0)
    // diagonal of Ru, formed once and shared by the NT threads (a per-thread
    // copy indexed at run time gave wrong values in threads >= 32 of the
    // FP64 four-warp instantiation; the shared copy is also less work)
    __shared__ F ru_diag[NU];
    for (int i = lane; i < NU; i += NT)
        ru_diag[i] = F(2) * F(a.model.Qu[i]) + F(a.damp) +
                     (bounded(a.model.u_lo[i], a.model.u_hi[i]) ? F(a.rho_box) : F(0));
    ric_sync<NT>();
    bool ok = ric_factor<F, NS, NU, NT>(scr, N, ru_diag);
    if (lane >= 32) return;
    __shared__ F sc[NS];
    for (int i = lane; i < NS; i += 32) sc[i] = F(a.s[(long long)sm.state0 * NS + i]);
    __syncwarp();
    struct Out {
        T *s, *u;
        long long s0, c0;
        __device__ void put_u(int t, int i, F v) { u[(c0 + t) * NU + i] = T(v); }
        __device__ void put_s(int t, int i, F v) { s[(s0 + t) * NS + i] = T(v); }
    } out{a.s, a.u, (long long)sm.state0, (long long)sm.ctrl0};
    ok = ric_sweep<F, NS, NU>(scr, N, sc, out) && ok;
    if (!ok) {
        finish_scenario<T, KIND>(a, sm, s, OCA_SCEN_FAILED, j, 0.0, 0.0);
        return;
    }
    __syncwarp();
    // ---- box block: z = clip((s,u)^{j+1} + w), w += (s,u)^{j+1} - z
    double rpb = 0.0, rdb = 0.0;
    const int n_box = a.rho_box > T(0) ? N * NS + N * NU : 0;  // rho_box = 0: no box block
    for (int e = lane; e < n_box; e += 32) {
        long long k2;
        T lo, hi, x;
        T *zz, *ww;
        if (e < N * NS) {
            const int t = 1 + e / NS, i = e % NS;
            lo = a.model.s_lo[i];
            hi = a.model.s_hi[i];
            k2 = (long long)(sm.state0 + t) * NS + i;
            x = a.s[k2];
            zz = a.box_zs;
            ww = a.box_ws;
        } else {
            const int e2 = e - N * NS, t = e2 / NU, i = e2 % NU;
            lo = a.model.u_lo[i];
            hi = a.model.u_hi[i];
            k2 = (long long)(sm.ctrl0 + t) * NU + i;
            x = a.u[k2];
            zz = a.box_zu;
            ww = a.box_wu;
        }
        if (!bounded(lo, hi)) continue;
        const T zn = fmin(fmax(x + ww[k2], lo), hi);
        rdb += double(zn - zz[k2]) * double(zn - zz[k2]);
        rpb += double(x - zn) * double(x - zn);
        zz[k2] = zn;
        ww[k2] += x - zn;
    }
    rpb = warp_sum(rpb);
    rdb = warp_sum(rdb);
    if (lane == 0) {
        a.box_res[2 * s] = rpb;
        a.box_res[2 * s + 1] = rdb;
    }
    // ---- poses of s^{j+1} for the next pair kernel
    const int Q = sm.NP * N;
    for (int q = lane; q < Q; q += 32) {
        const int part = q / N, t = q % N + 1;
        const int gp = sm.part0 + part;
        T st[NS], off[D], rho[D], R[D * D];
        for (int i = 0; i < NS; ++i) st[i] = a.s[(long long)(sm.state0 + t) * NS + i];
#pragma unroll
        for (int i = 0; i < D; ++i) off[i] = a.g.part_off[gp * D + i];
        part_pose<T, KIND>(a.model, a.g.part_link[gp], off, st, rho, R, nullptr, nullptr, nullptr);
        const int col = sm.qbeg + q;
#pragma unroll
        for (int i = 0; i < D; ++i) a.pose[(long long)i * a.Qtot + col] = rho[i];
#pragma unroll
        for (int i = 0; i < D * D; ++i) a.pose[(long long)(D + i) * a.Qtot + col] = R[i];
    }
}

template <typename T, typename F>
cudaError_t launch_riccati_f(const RicArgs<T> &a, cudaStream_t st) {
    switch (a.model.kind) {
        case 0: k_riccati<T, F, 0, 32><<<a.n_scen, 32, 0, st>>>(a); break;
        case 1: k_riccati<T, F, 1, 32><<<a.n_scen, 32, 0, st>>>(a); break;
        case 2: k_riccati<T, F, 2, 128><<<a.n_scen, 128, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_riccati(const RicArgs<T> &a, bool f32, cudaStream_t st) {
    if (f32) return launch_riccati_f<T, float>(a, st);
    return launch_riccati_f<T, double>(a, st);
}

template cudaError_t launch_riccati<float>(const RicArgs<float> &, bool, cudaStream_t);
template cudaError_t launch_riccati<double>(const RicArgs<double> &, bool, cudaStream_t);

}  // namespace oca
