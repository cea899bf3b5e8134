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
#include "oca_models.cuh"

namespace oca {

template <int NS, int NU>
struct RicLayout {
    // offsets (elements) inside a scenario's scratch block for horizon N
    __host__ __device__ static long long A(int N, int t) { return (long long)t * NS * NS; }
    __host__ __device__ static long long B(int N, int t) { return (long long)N * NS * NS + (long long)t * NS * NU; }
    __host__ __device__ static long long c(int N, int t) { return (long long)N * (NS * NS + NS * NU) + (long long)t * NS; }
    __host__ __device__ static long long Q(int N, int t) { return (long long)N * (NS * NS + NS * NU + NS) + (long long)t * NS * NS; }
    __host__ __device__ static long long q(int N, int t) { return Q(N, 0) + (long long)(N + 1) * NS * NS + (long long)t * NS; }
    __host__ __device__ static long long K(int N, int t) { return q(N, 0) + (long long)(N + 1) * NS + (long long)t * NU * NS; }
    __host__ __device__ static long long k(int N, int t) { return K(N, 0) + (long long)N * NU * NS + (long long)t * NU; }
    __host__ __device__ static long long size(int N) { return k(N, 0) + (long long)N * NU; }
};

long long riccati_scratch_elems(int kind, int N) {
    switch (kind) {
        case 0: return RicLayout<4, 2>::size(N);
        case 1: return RicLayout<5, 2>::size(N);
        default: return RicLayout<12, 4>::size(N);
    }
}

template <typename T>
__device__ __forceinline__ bool bounded(T lo, T hi) { return lo > T(-1e29) || hi < T(1e29); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
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

template <typename T, typename F, int KIND>
__global__ void __launch_bounds__(32) k_riccati(RicArgs<T> a) {
    constexpr int NS = MDims<KIND>::NS, NU = MDims<KIND>::NU, D = MDims<KIND>::D, NROT = MDims<KIND>::NROT;
    constexpr int NW = StatDims<D>::NW;
    using LY = RicLayout<NS, NU>;
    const int s = blockIdx.x;
    const int lane = threadIdx.x;
    if (a.scen_status[s] != kActive) return;
    const int j = *a.iter;
    if (j > a.max_iter) return;
    const ScenMeta sm = a.meta[s];
    const int N = sm.N;

    // ---- 1. stopping rule of iteration j-1
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
            return;
        }
    } else if (a.max_iter <= 0) {
        finish_scenario<T, KIND>(a, sm, s, OCA_SCEN_MAX_ITER, 0, 0.0, 0.0);
        return;
    }

    DevModel<F> mdl;
    mdl.kind = a.model.kind;
    mdl.dt = F(a.model.dt);
#pragma unroll
    for (int i = 0; i < 8; ++i) mdl.p[i] = F(a.model.p[i]);
#pragma unroll
    for (int i = 0; i < 12; ++i) mdl.Qs[i] = F(a.model.Qs[i]);
#pragma unroll
    for (int i = 0; i < 4; ++i) mdl.Qu[i] = F(a.model.Qu[i]);
    const F rho_b = F(a.rho_box), damp = F(a.damp);
    F *scr = reinterpret_cast<F *>(a.scratch) + a.scratch0[s];

    // ---- 2. stage assembly, lanes over t
    // (in the array precision T: only the factorisation below runs in F)
    const DevModel<T> &mdt = a.model;
    for (int t = lane; t <= N; t += 32) {
        T st[NS];
#pragma unroll
        for (int i = 0; i < NS; ++i) st[i] = a.s[(long long)(sm.state0 + t) * NS + i];
        if (t < N) {
            T ut[NU], f[NS], fs[NS * NS], fu[NS * NU];
#pragma unroll
            for (int i = 0; i < NU; ++i) ut[i] = a.u[(long long)(sm.ctrl0 + t) * NU + i];
            dynamics<T, KIND>(mdt, st, ut, f, fs, fu);
            F *At = scr + LY::A(N, t), *Bt = scr + LY::B(N, t), *ct = scr + LY::c(N, t);
            for (int i = 0; i < NS; ++i) {
                T acc = st[i] + mdt.dt * f[i];
                for (int k = 0; k < NS; ++k) {
                    const T v = (i == k ? T(1) : T(0)) + mdt.dt * fs[i * NS + k];
                    At[i * NS + k] = F(v);
                    acc -= v * st[k];
                }
                for (int k = 0; k < NU; ++k) {
                    const T v = mdt.dt * fu[i * NU + k];
                    Bt[i * NU + k] = F(v);
                    acc -= v * ut[k];
                }
                ct[i] = F(acc);
            }
        }
        // stage cost accumulated in registers (T), stored once in F
        T Qr[NS * NS], qr[NS];
        for (int i = 0; i < NS * NS; ++i) Qr[i] = T(0);
        for (int i = 0; i < NS; ++i) {
            Qr[i * NS + i] = T(2) * mdt.Qs[i];
            qr[i] = -T(2) * mdt.Qs[i] * a.s_ref[(long long)(sm.state0 + t) * NS + i];
            if (t >= 1) {
                // proximal damping 0.5 damp |s - s^j|^2 and the box block's
                // augmented term 0.5 rho_b |s - z + w|^2 on bounded components
                Qr[i * NS + i] += a.damp;
                qr[i] -= a.damp * st[i];
                if (bounded(a.model.s_lo[i], a.model.s_hi[i])) {
                    const long long k2 = (long long)(sm.state0 + t) * NS + i;
                    Qr[i * NS + i] += a.rho_box;
                    qr[i] -= a.rho_box * (a.box_zs[k2] - a.box_ws[k2]);
                }
            }
        }
        if (t >= 1) {
            for (int part = 0; part < sm.NP; ++part) {
                const int gp = sm.part0 + part;
                T off[D], rho[D], R[D * D], drho[D * NS], dR[NROT][D * D];
                int ridx[NROT];
#pragma unroll
                for (int i = 0; i < D; ++i) off[i] = a.g.part_off[gp * D + i];
                part_pose<T, KIND>(mdt, a.g.part_link[gp], off, st, rho, R, drho, dR, ridx);
                const long long col = sm.qbeg + part * N + (t - 1);
                T W[D][D], Wc[D], E[D][D];
                int k = 0;
#pragma unroll
                for (int i = 0; i < D; ++i)
#pragma unroll
                    for (int jj = 0; jj <= i; ++jj) {
                        W[i][jj] = W[jj][i] = a.stats[(long long)k * a.Qtot + col];
                        ++k;
                    }
#pragma unroll
                for (int i = 0; i < D; ++i) Wc[i] = a.stats[(long long)(NW + i) * a.Qtot + col];
#pragma unroll
                for (int i = 0; i < D; ++i)
#pragma unroll
                    for (int jj = 0; jj < D; ++jj) E[i][jj] = a.stats[(long long)(NW + D + i * D + jj) * a.Qtot + col];
                // translation block: drho^T W drho, gradient -drho^T (Wc - W rho)
                T WD[D][NS], gvec[D];
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    T acc = Wc[i];
#pragma unroll
                    for (int jj = 0; jj < D; ++jj) acc -= W[i][jj] * rho[jj];
                    gvec[i] = acc;
                    for (int b2 = 0; b2 < NS; ++b2) {
                        T v = T(0);
#pragma unroll
                        for (int jj = 0; jj < D; ++jj) v += W[i][jj] * drho[jj * NS + b2];
                        WD[i][b2] = v;
                    }
                }
                T Hs[NS];
                for (int a2 = 0; a2 < NS; ++a2) {
                    for (int b2 = 0; b2 < NS; ++b2) {
                        T v = T(0);
#pragma unroll
                        for (int i = 0; i < D; ++i) v += drho[i * NS + a2] * WD[i][b2];
                        Hs[b2] = v;
                    }
                    // rotation block: tr(R_a R_b^T W), gradient tr(R_a E^T) + tr(R_a R^T W)
#pragma unroll
                    for (int ra = 0; ra < NROT; ++ra) {
                        if (ridx[ra] != a2) continue;
#pragma unroll
                        for (int rb = 0; rb < NROT; ++rb) {
                            T v = T(0);
#pragma unroll
                            for (int i = 0; i < D; ++i)
#pragma unroll
                                for (int jj = 0; jj < D; ++jj) {
                                    T m = T(0);
#pragma unroll
                                    for (int l = 0; l < D; ++l) m += dR[ra][i * D + l] * dR[rb][jj * D + l];
                                    v += m * W[i][jj];
                                }
                            Hs[ridx[rb]] += v;
                        }
                    }
                    T g = T(0);
#pragma unroll
                    for (int i = 0; i < D; ++i) g -= drho[i * NS + a2] * gvec[i];
#pragma unroll
                    for (int ra = 0; ra < NROT; ++ra) {
                        if (ridx[ra] != a2) continue;
                        T v = T(0);
#pragma unroll
                        for (int i = 0; i < D; ++i)
#pragma unroll
                            for (int jj = 0; jj < D; ++jj) {
                                T m = T(0);
#pragma unroll
                                for (int l = 0; l < D; ++l) m += dR[ra][i * D + l] * R[jj * D + l];
                                v += dR[ra][i * D + jj] * E[i][jj] + m * W[i][jj];
                            }
                        g += v;
                    }
                    T hsx = T(0);
                    for (int b2 = 0; b2 < NS; ++b2) {
                        Qr[a2 * NS + b2] += a.sigma * Hs[b2];
                        hsx += Hs[b2] * st[b2];
                    }
                    qr[a2] += a.sigma * (g - hsx);
                }
            }
        }
        F *Qt = scr + LY::Q(N, t), *qt = scr + LY::q(N, t);
        for (int i = 0; i < NS * NS; ++i) Qt[i] = F(Qr[i]);
        for (int i = 0; i < NS; ++i) qt[i] = F(qr[i]);
    }
    __syncwarp();

    // ---- 3. backward Riccati recursion
    __shared__ F P[NS * NS], pv[NS], PA[NS * NS], PB[NS * NU], wv[NS];
    __shared__ F Quu[NU * NU], Qus[NU * NS], qu[NU], Qss[NS * NS], qs[NS], Kt[NU * NS], kt[NU];
    __shared__ int bad;
    if (lane == 0) bad = 0;
    for (int e = lane; e < NS * NS; e += 32) P[e] = scr[LY::Q(N, N) + e];
    for (int e = lane; e < NS; e += 32) pv[e] = scr[LY::q(N, N) + e];
    __syncwarp();
    for (int t = N - 1; t >= 0; --t) {
        const F *At = scr + LY::A(N, t), *Bt = scr + LY::B(N, t), *ct = scr + LY::c(N, t);
        for (int e = lane; e < NS * NS; e += 32) {
            const int i = e / NS, jj = e % NS;
            F acc = F(0);
            for (int k = 0; k < NS; ++k) acc += P[i * NS + k] * At[k * NS + jj];
            PA[e] = acc;
        }
        for (int e = lane; e < NS * NU; e += 32) {
            const int i = e / NU, jj = e % NU;
            F acc = F(0);
            for (int k = 0; k < NS; ++k) acc += P[i * NS + k] * Bt[k * NU + jj];
            PB[e] = acc;
        }
        for (int i = lane; i < NS; i += 32) {
            F acc = pv[i];
            for (int k = 0; k < NS; ++k) acc += P[i * NS + k] * ct[k];
            wv[i] = acc;
        }
        __syncwarp();
        const F *Qt = scr + LY::Q(N, t), *qt = scr + LY::q(N, t);
        for (int e = lane; e < NS * NS; e += 32) {
            const int i = e / NS, jj = e % NS;
            F acc = Qt[e];
            for (int k = 0; k < NS; ++k) acc += At[k * NS + i] * PA[k * NS + jj];
            Qss[e] = acc;
        }
        for (int e = lane; e < NU * NS; e += 32) {
            const int i = e / NS, jj = e % NS;
            F acc = F(0);
            for (int k = 0; k < NS; ++k) acc += Bt[k * NU + i] * PA[k * NS + jj];
            Qus[e] = acc;
        }
        for (int e = lane; e < NU * NU; e += 32) {
            const int i = e / NU, jj = e % NU;
            F acc = (i == jj) ? F(2) * mdl.Qu[i] + damp + (bounded(a.model.u_lo[i], a.model.u_hi[i]) ? rho_b : F(0)) : F(0);
            for (int k = 0; k < NS; ++k) acc += Bt[k * NU + i] * PB[k * NU + jj];
            Quu[e] = acc;
        }
        for (int i = lane; i < NS + NU; i += 32) {
            if (i < NS) {
                F acc = qt[i];
                for (int k = 0; k < NS; ++k) acc += At[k * NS + i] * wv[k];
                qs[i] = acc;
            } else {
                const int ii = i - NS;
                const long long k2 = (long long)(sm.ctrl0 + t) * NU + ii;
                F acc = -damp * F(a.u[k2]);
                if (bounded(a.model.u_lo[ii], a.model.u_hi[ii])) acc -= rho_b * (F(a.box_zu[k2]) - F(a.box_wu[k2]));
                for (int k = 0; k < NS; ++k) acc += Bt[k * NU + ii] * wv[k];
                qu[ii] = acc;
            }
        }
        __syncwarp();
        // Cholesky of Quu (NU <= 4) by lane 0
        if (lane == 0) {
            for (int c = 0; c < NU; ++c) {
                F dg = Quu[c * NU + c];
                for (int k = 0; k < c; ++k) dg -= Quu[c * NU + k] * Quu[c * NU + k];
                if (!(dg > F(0))) {
                    bad = 1;
                    dg = F(1);
                }
                dg = m_sqrt(dg);
                Quu[c * NU + c] = dg;
                for (int r = c + 1; r < NU; ++r) {
                    F acc = Quu[r * NU + c];
                    for (int k = 0; k < c; ++k) acc -= Quu[r * NU + k] * Quu[c * NU + k];
                    Quu[r * NU + c] = acc / dg;
                }
            }
        }
        __syncwarp();
        // K = -Quu^-1 Qus (columns over lanes), k = -Quu^-1 qu (lane NS)
        for (int col = lane; col <= NS; col += 32) {
            F x[NU];
            for (int i = 0; i < NU; ++i) x[i] = -(col < NS ? Qus[i * NS + col] : qu[i]);
            for (int i = 0; i < NU; ++i) {
                F acc = x[i];
                for (int k = 0; k < i; ++k) acc -= Quu[i * NU + k] * x[k];
                x[i] = acc / Quu[i * NU + i];
            }
            for (int i = NU - 1; i >= 0; --i) {
                F acc = x[i];
                for (int k = i + 1; k < NU; ++k) acc -= Quu[k * NU + i] * x[k];
                x[i] = acc / Quu[i * NU + i];
            }
            for (int i = 0; i < NU; ++i) {
                if (col < NS) {
                    Kt[i * NS + col] = x[i];
                    scr[LY::K(N, t) + i * NS + col] = x[i];
                } else {
                    kt[i] = x[i];
                    scr[LY::k(N, t) + i] = x[i];
                }
            }
        }
        __syncwarp();
        // P = Qss + Qus^T K (symmetrised), p = qs + Qus^T k
        for (int e = lane; e < NS * NS; e += 32) {
            const int i = e / NS, jj = e % NS;
            F a1 = Qss[i * NS + jj], a2 = Qss[jj * NS + i];
            for (int k = 0; k < NU; ++k) {
                a1 += Qus[k * NS + i] * Kt[k * NS + jj];
                a2 += Qus[k * NS + jj] * Kt[k * NS + i];
            }
            P[e] = F(0.5) * (a1 + a2);
        }
        for (int i = lane; i < NS; i += 32) {
            F acc = qs[i];
            for (int k = 0; k < NU; ++k) acc += Qus[k * NS + i] * kt[k];
            pv[i] = acc;
        }
        __syncwarp();
    }

    // ---- 4. forward sweep: u_t = K_t s_t + k_t, s_{t+1} = A_t s_t + B_t u_t + c_t
    __shared__ F sc[NS], uc[NU];
    for (int i = lane; i < NS; i += 32) sc[i] = F(a.s[(long long)sm.state0 * NS + i]);
    __syncwarp();
    bool finite = true;
    for (int t = 0; t < N; ++t) {
        if (lane < NU) {
            F acc = scr[LY::k(N, t) + lane];
            for (int k = 0; k < NS; ++k) acc += scr[LY::K(N, t) + lane * NS + k] * sc[k];
            uc[lane] = acc;
            a.u[(long long)(sm.ctrl0 + t) * NU + lane] = T(acc);
            finite &= m_finite(acc);
        }
        __syncwarp();
        F nx = F(0);
        if (lane < NS) {
            nx = scr[LY::c(N, t) + lane];
            for (int k = 0; k < NS; ++k) nx += scr[LY::A(N, t) + lane * NS + k] * sc[k];
            for (int k = 0; k < NU; ++k) nx += scr[LY::B(N, t) + lane * NU + k] * uc[k];
        }
        __syncwarp();
        if (lane < NS) {
            sc[lane] = nx;
            a.s[(long long)(sm.state0 + t + 1) * NS + lane] = T(nx);
            finite &= m_finite(nx);
        }
        __syncwarp();
    }
    const bool ok = __all_sync(0xffffffffu, finite) && !bad;
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
        case 0: k_riccati<T, F, 0><<<a.n_scen, 32, 0, st>>>(a); break;
        case 1: k_riccati<T, F, 1><<<a.n_scen, 32, 0, st>>>(a); break;
        case 2: k_riccati<T, F, 2><<<a.n_scen, 32, 0, st>>>(a); break;
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
