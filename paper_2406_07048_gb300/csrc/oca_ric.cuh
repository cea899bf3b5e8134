// Trajectory step of the ADMM (Sec. IV-B eqn:ADMM_state_updates): the LQ
// stage terms and the Riccati factorisation and sweep, shared by the
// forward kernel (oca_riccati.cu) and the adjoint kernel (oca_adjoint.cu).
//
// The LQ problem of one scenario (one SQP step at the linearisation point
// (s^j, u^j)):
//   min  sum_{t=0..N} 0.5 s_t^T Q_t s_t + q_t^T s_t
//      + sum_{t<N}    0.5 u_t^T Ru u_t + r_t^T u_t
//   s.t. s_{t+1} = A_t s_t + B_t u_t + c_t,  s_0 fixed,
// with A_t, B_t, c_t the Euler dynamics linearised at (s^j_t, u^j_t), Q_t, q_t
// the tracking cost of eqn:navigation_cost plus the proximal damping, the box
// block's augmented term and the Gauss-Newton model of the pair residuals,
// and Ru = diag(2 Qu + damp + rho_b [bounded]).
#pragma once

#include "oca_common.cuh"
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
    __host__ __device__ static long long r(int N, int t) { return k(N, 0) + (long long)N * NU + (long long)t * NU; }
    // adjoint pass: solution (xs, xu) of the adjoint LQ and the costates of
    // the forward (pf) and adjoint (pa) problems
    __host__ __device__ static long long xs(int N, int t) { return r(N, 0) + (long long)N * NU + (long long)t * NS; }
    __host__ __device__ static long long xu(int N, int t) { return xs(N, 0) + (long long)(N + 1) * NS + (long long)t * NU; }
    __host__ __device__ static long long pf(int N, int t) { return xu(N, 0) + (long long)N * NU + (long long)t * NS; }
    __host__ __device__ static long long pa(int N, int t) { return pf(N, 0) + (long long)(N + 1) * NS + (long long)t * NS; }
    __host__ __device__ static long long size(int N) { return pa(N, 0) + (long long)(N + 1) * NS; }
};

template <typename T>
__device__ __forceinline__ bool bounded(T lo, T hi) { return lo > T(-1e29) || hi < T(1e29); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ----------------------------------------------------------------------------
// Gauss-Newton terms of one part at step t.  The pair residuals
// r = [T + zeta; R + xi] (Sec. IV-A) depend on s_t through the pose only:
//   T = 1 + (d - C rho)^T mu + gamma,  R = A^T lambda + R(s)^T C^T mu,
// so with w = C^T mu (world) the sums over the part's obstacles of J^T J and
// J^T r (J = dr/ds_t) follow from W = sum w w^T, Wc = sum c w and
// E = sum w e^T (c = 1 + d^T mu + gamma + zeta, e = A^T lambda + xi):
//   Hs = drho^T W drho + sum_{a,b rotation} tr(dR_a dR_b^T W)
//   g_a = -drho_a^T (Wc - W rho) + [a rotation] (tr(dR_a E^T) + tr(dR_a R^T W)).
// Wl is the lower triangle of W (row-major over i >= j).  Written over a
// number type T so that the adjoint can differentiate it (oca_dual.cuh).
// ----------------------------------------------------------------------------
template <typename T, int KIND>
__device__ void gn_part(const DevModel<T> &m, int link, const T *off, const T *st, const T *Wl, const T *Wc,
                        const T *E, T *Hs, T *g) {
    constexpr int NS = MDims<KIND>::NS, D = MDims<KIND>::D, NROT = MDims<KIND>::NROT;
    T rho[D], R[D * D], drho[D * NS], dR[NROT][D * D];
    int ridx[NROT];
    part_pose<T, KIND>(m, link, off, st, rho, R, drho, dR, ridx);
    T W[D][D];
    {
        int k = 0;
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int jj = 0; jj <= i; ++jj) {
                W[i][jj] = Wl[k];
                W[jj][i] = Wl[k];
                ++k;
            }
    }
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
    for (int a2 = 0; a2 < NS; ++a2) {
        for (int b2 = 0; b2 < NS; ++b2) {
            T v = T(0);
#pragma unroll
            for (int i = 0; i < D; ++i) v += drho[i * NS + a2] * WD[i][b2];
            Hs[a2 * NS + b2] = v;
        }
        T ga = T(0);
#pragma unroll
        for (int i = 0; i < D; ++i) ga -= drho[i * NS + a2] * gvec[i];
        g[a2] = ga;
    }
    // rotation coordinates
#pragma unroll
    for (int ra = 0; ra < NROT; ++ra) {
#pragma unroll
        for (int rb = 0; rb < NROT; ++rb) {
            T v = T(0);
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
                for (int jj = 0; jj < D; ++jj) {
                    T mm = T(0);
#pragma unroll
                    for (int l = 0; l < D; ++l) mm += dR[ra][i * D + l] * dR[rb][jj * D + l];
                    v += mm * W[i][jj];
                }
            Hs[ridx[ra] * NS + ridx[rb]] += v;
        }
        T v = T(0);
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int jj = 0; jj < D; ++jj) {
                T mm = T(0);
#pragma unroll
                for (int l = 0; l < D; ++l) mm += dR[ra][i * D + l] * R[jj * D + l];
                v += dR[ra][i * D + jj] * E[i * D + jj] + mm * W[i][jj];
            }
        g[ridx[ra]] += v;
    }
}

// Where the inputs of a stage come from: the live ADMM arrays (forward) or
// a taped iterate (adjoint).  Same row layouts as the scene's state arrays.
template <typename T>
struct StageSrc {
    const T *s, *u;          // [n_states][NS], [n_ctrls][NU]: linearisation point
    const T *zs, *ws;        // box block of the states
    const T *zu, *wu;        // box block of the controls
    const T *stats;          // [NSTAT][Qtot]
};

template <typename T>
struct StageParams {
    DevModel<T> model;
    Geom<T> g;
    T sigma, rho_box, damp;
    const T *s_ref;
    int Qtot;
};

// Stage t of one scenario into the factorisation-precision scratch:
// A_t, B_t, c_t, r_t (t < N) and Q_t, q_t (t <= N); assembled in T.
template <typename T, typename F, int KIND>
__device__ void assemble_stage(const StageParams<T> &a, const StageSrc<T> &src, const ScenMeta &sm, int t, F *scr) {
    constexpr int NS = MDims<KIND>::NS, NU = MDims<KIND>::NU, D = MDims<KIND>::D;
    constexpr int NW = StatDims<D>::NW;
    using LY = RicLayout<NS, NU>;
    const int N = sm.N;
    const DevModel<T> &mdt = a.model;
    T st[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) st[i] = src.s[(long long)(sm.state0 + t) * NS + i];
    if (t < N) {
        T ut[NU], f[NS], fs[NS * NS], fu[NS * NU];
#pragma unroll
        for (int i = 0; i < NU; ++i) ut[i] = src.u[(long long)(sm.ctrl0 + t) * NU + i];
        dynamics<T, KIND>(mdt, st, ut, f, fs, fu);
        F *At = scr + LY::A(N, t), *Bt = scr + LY::B(N, t), *ct = scr + LY::c(N, t), *rt = scr + LY::r(N, t);
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
        // control linear term: damping toward u^j, box block
#pragma unroll
        for (int i = 0; i < NU; ++i) {
            const long long k2 = (long long)(sm.ctrl0 + t) * NU + i;
            T acc = -a.damp * ut[i];
            if (bounded(mdt.u_lo[i], mdt.u_hi[i])) acc -= a.rho_box * (src.zu[k2] - src.wu[k2]);
            rt[i] = F(acc);
        }
    }
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
            if (bounded(mdt.s_lo[i], mdt.s_hi[i])) {
                const long long k2 = (long long)(sm.state0 + t) * NS + i;
                Qr[i * NS + i] += a.rho_box;
                qr[i] -= a.rho_box * (src.zs[k2] - src.ws[k2]);
            }
        }
    }
    if (t >= 1) {
        for (int part = 0; part < sm.NP; ++part) {
            const int gp = sm.part0 + part;
            T off[D], Wl[NW], Wc[D], E[D * D], Hs[NS * NS], gg[NS];
#pragma unroll
            for (int i = 0; i < D; ++i) off[i] = a.g.part_off[gp * D + i];
            const long long col = sm.qbeg + part * N + (t - 1);
#pragma unroll
            for (int k = 0; k < NW; ++k) Wl[k] = src.stats[(long long)k * a.Qtot + col];
#pragma unroll
            for (int k = 0; k < D; ++k) Wc[k] = src.stats[(long long)(NW + k) * a.Qtot + col];
#pragma unroll
            for (int k = 0; k < D * D; ++k) E[k] = src.stats[(long long)(NW + D + k) * a.Qtot + col];
            gn_part<T, KIND>(mdt, a.g.part_link[gp], off, st, Wl, Wc, E, Hs, gg);
            for (int a2 = 0; a2 < NS; ++a2) {
                T hsx = T(0);
                for (int b2 = 0; b2 < NS; ++b2) {
                    Qr[a2 * NS + b2] += a.sigma * Hs[a2 * NS + b2];
                    hsx += Hs[a2 * NS + b2] * st[b2];
                }
                qr[a2] += a.sigma * (gg[a2] - hsx);   // linear term of 0.5 sigma |r0 + J (s - s^j)|^2
            }
        }
    }
    F *Qt = scr + LY::Q(N, t), *qt = scr + LY::q(N, t);
    for (int i = 0; i < NS * NS; ++i) Qt[i] = F(Qr[i]);
    for (int i = 0; i < NS; ++i) qt[i] = F(qr[i]);
}

// ----------------------------------------------------------------------------
// Backward Riccati recursion over the scratch (one warp; every lane calls):
// P_N = Q_N, p_N = q_N; for t = N-1..0 with P+ = P_{t+1}, w = p_{t+1} + P+ c_t:
//   Quu = Ru + B^T P+ B, Qus = B^T P+ A, Qss = Q_t + A^T P+ A,
//   qu = r_t + B^T w, qs = q_t + A^T w,
//   K_t = -Quu^-1 Qus, k_t = -Quu^-1 qu  (Cholesky of Quu),
//   P_t = Qss + Qus^T K_t (symmetrised), p_t = qs + Qus^T k_t.
// ru_diag = diagonal of Ru.  Returns false if a Quu was not positive definite.
// ----------------------------------------------------------------------------
template <typename F, int NS, int NU>
__device__ bool ric_factor(F *scr, int N, const F *ru_diag) {
    using LY = RicLayout<NS, NU>;
    const int lane = threadIdx.x;
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
        const F *Qt = scr + LY::Q(N, t), *qt = scr + LY::q(N, t), *rt = scr + LY::r(N, t);
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
            F acc = (i == jj) ? ru_diag[i] : F(0);
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
                F acc = rt[ii];
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
    const int b = bad;
    __syncwarp();
    return b == 0;
}

// Forward sweep u_t = K_t s_t + k_t, s_{t+1} = A_t s_t + B_t u_t + c_t from
// s_0 = x0 (shared, NS).  out.put_u(t, i, v) and out.put_s(t + 1, i, v)
// receive the solution.  Returns false on a non-finite value.
template <typename F, int NS, int NU, class Out>
__device__ bool ric_sweep(const F *scr, int N, F *sc, Out &out) {
    using LY = RicLayout<NS, NU>;
    const int lane = threadIdx.x;
    __shared__ F uc[NU];
    bool finite = true;
    for (int t = 0; t < N; ++t) {
        if (lane < NU) {
            F acc = scr[LY::k(N, t) + lane];
            for (int k = 0; k < NS; ++k) acc += scr[LY::K(N, t) + lane * NS + k] * sc[k];
            uc[lane] = acc;
            out.put_u(t, lane, acc);
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
            out.put_s(t + 1, lane, nx);
            finite &= m_finite(nx);
        }
        __syncwarp();
    }
    return __all_sync(0xffffffffu, finite);
}

// Costates of an LQ solution x: pi_N = Q_N x_N + q_N,
// pi_t = Q_t x_t + q_t + A_t^T pi_{t+1} (t = N-1..1), into scr at LY::pf
// (ADJ = false) or LY::pa (ADJ = true).  xs(t, i) returns x_t[i].
template <typename F, int NS, int NU, bool ADJ, class Xs>
__device__ void ric_costates(F *scr, int N, const Xs &xs) {
    using LY = RicLayout<NS, NU>;
    const int lane = threadIdx.x;
    __shared__ F pi_next[NS];
    for (int t = N; t >= 1; --t) {
        F acc = F(0);
        if (lane < NS) {
            const F *Qt = scr + LY::Q(N, t);
            acc = scr[LY::q(N, t) + lane];
            for (int k = 0; k < NS; ++k) acc += Qt[lane * NS + k] * xs(t, k);
            if (t < N) {
                const F *At = scr + LY::A(N, t);
                for (int k = 0; k < NS; ++k) acc += At[k * NS + lane] * pi_next[k];
            }
        }
        __syncwarp();
        if (lane < NS) {
            pi_next[lane] = acc;
            scr[(ADJ ? LY::pa(N, t) : LY::pf(N, t)) + lane] = acc;
        }
        __syncwarp();
    }
}

}  // namespace oca
