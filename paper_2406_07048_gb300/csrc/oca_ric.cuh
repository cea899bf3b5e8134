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
// P_N = Q_N, p_N = q_N; for t = N-1..0, with G = [A_t | B_t | c_t] and
// Y = P_{t+1} G + [0 | 0 | p_{t+1}], the stage matrix
//   M = [Q_t 0 q_t; 0 Ru r_t] + G^T Y  (rows (s, u), columns (s, u, 1))
// holds Qss, Qus, Quu and qs, qu; then
//   K_t = -Quu^-1 Qus, k_t = -Quu^-1 qu,
//   P_t = Qss + Qus^T K_t, p_t = qs + Qus^T k_t.
// Only the symmetric half of M and of P is formed.  Every lane inverts the
// (small, SPD) Quu itself.  The step's data are staged in shared memory and
// the next step's are loaded while this one computes.
// ru_diag = diagonal of Ru.  Returns false if a Quu was not positive definite.
// ----------------------------------------------------------------------------
template <typename F, int NS, int NU>
__device__ __forceinline__ F ric_stage_elem(const F *scr, int N, int t, int e) {
    using LY = RicLayout<NS, NU>;
    constexpr int NX = NS + NU + 1, NG = NS * NX, NQ = NS * NS;
    if (e < NG) {
        const int k = e / NX, j = e % NX;
        if (j < NS) return scr[LY::A(N, t) + k * NS + j];
        if (j < NS + NU) return scr[LY::B(N, t) + k * NU + (j - NS)];
        return scr[LY::c(N, t) + k];
    }
    if (e < NG + NQ) return scr[LY::Q(N, t) + (e - NG)];
    if (e < NG + NQ + NS) return scr[LY::q(N, t) + (e - NG - NQ)];
    return scr[LY::r(N, t) + (e - NG - NQ - NS)];
}

// inverse of a symmetric positive-definite n x n matrix (n <= 4), in registers
template <typename F, int NU>
__device__ __forceinline__ bool spd_inverse(const F (&U)[NU][NU], F (&X)[NU][NU]) {
    if constexpr (NU == 2) {
        const F det = U[0][0] * U[1][1] - U[0][1] * U[0][1];
        if (!(U[0][0] > F(0)) || !(det > F(0))) {
            // not positive definite: X = 0 (the gains of this stage vanish; the
            // caller reports the failure), never values left from before
            X[0][0] = X[0][1] = X[1][0] = X[1][1] = F(0);
            return false;
        }
        const F id = F(1) / det;
        X[0][0] = U[1][1] * id;
        X[1][1] = U[0][0] * id;
        X[0][1] = X[1][0] = -U[0][1] * id;
        return true;
    } else {
        // U = L D L^T (L unit lower triangular: no square roots on the
        // dependent chain), then X = L^-T D^-1 L^-1; U is positive definite
        // iff every pivot d_c is positive
        F L[NU][NU], dg[NU], idg[NU];
        bool ok = true;
#pragma unroll
        for (int c = 0; c < NU; ++c) {
            F dc = U[c][c];
#pragma unroll
            for (int k = 0; k < c; ++k) dc -= L[c][k] * L[c][k] * dg[k];
            ok &= dc > F(0);
            dc = dc > F(0) ? dc : F(1);
            dg[c] = dc;
            idg[c] = F(1) / dc;
#pragma unroll
            for (int r = c + 1; r < NU; ++r) {
                F acc = U[r][c];
#pragma unroll
                for (int k = 0; k < c; ++k) acc -= L[r][k] * L[c][k] * dg[k];
                L[r][c] = acc * idg[c];
            }
        }
        // Z = L^-1 (unit lower triangular)
        F Z[NU][NU];
#pragma unroll
        for (int c = 0; c < NU; ++c)
#pragma unroll
            for (int r = 0; r < NU; ++r) {
                if (r < c) {
                    Z[r][c] = F(0);
                } else if (r == c) {
                    Z[r][c] = F(1);
                } else {
                    F acc = F(0);
#pragma unroll
                    for (int k = c; k < r; ++k) acc -= L[r][k] * Z[k][c];
                    Z[r][c] = acc;
                }
            }
#pragma unroll
        for (int i = 0; i < NU; ++i)
#pragma unroll
            for (int j = 0; j <= i; ++j) {
                F acc = F(0);
#pragma unroll
                for (int k = 0; k < NU; ++k) acc += Z[k][i] * idg[k] * Z[k][j];
                X[i][j] = X[j][i] = acc;
            }
        return ok;
    }
}

template <int NT>
__device__ __forceinline__ void ric_sync() {
    if constexpr (NT == 32) __syncwarp();
    else __syncthreads();
}

// NT threads (one warp, or the whole CTA when NT > 32) run the recursion
template <typename F, int NS, int NU, int NT = 32>
__device__ bool ric_factor(F *scr, int N, const F *ru_diag) {
    using LY = RicLayout<NS, NU>;
    constexpr int NX = NS + NU + 1;           // columns of G = [A | B | c]
    constexpr int NZ = NS + NU;               // rows of M
    constexpr int MC = NZ + 1;                // columns of M as stored
    constexpr int NG = NS * NX, NQ = NS * NS;
    constexpr int NST = NG + NQ + NS + NU;    // staged values per step
    constexpr int PF = (NST + NT - 1) / NT;   // of them per thread
    constexpr int NSYM = NZ * (NZ + 1) / 2;   // upper triangle of the Hessian part of M
    constexpr int NPS = NS * (NS + 1) / 2;    // upper triangle of P
    const int lane = threadIdx.x;  // thread of the NT
    __shared__ F P[NS * NS], pv[NS], stg[NST], Y[NS * NX], M[NZ * MC], KK[NU * (NS + 1)];
    const F *Gs = stg, *Qs = stg + NG, *qs = stg + NG + NQ, *rs = stg + NG + NQ + NS;
    for (int e = lane; e < NS * NS; e += NT) P[e] = scr[LY::Q(N, N) + e];
    for (int e = lane; e < NS; e += NT) pv[e] = scr[LY::q(N, N) + e];
    F nxt[PF];
    if (N >= 1) {
#pragma unroll
        for (int r = 0; r < PF; ++r) {
            const int e = lane + NT * r;
            if (e < NST) nxt[r] = ric_stage_elem<F, NS, NU>(scr, N, N - 1, e);
        }
    }
    // each thread's entries of the stage matrix M (upper triangle row by row,
    // then the gradient column) and of P (upper triangle, then p): their (i, j)
    // depend on the thread only.  With NT > 32 (the 12-state model: 152 and 90
    // entries per step) they are found once, before the steps; a one-warp group
    // (27-35 entries) finds them in each step, which measured faster there.
    constexpr bool HOIST = NT > 32;
    constexpr int RM = HOIST ? (NSYM + NZ + NT - 1) / NT : 1, RP = HOIST ? (NPS + NS + NT - 1) / NT : 1;
    int mi[RM], mj[RM], pi_[RP], pj[RP];
    if constexpr (HOIST) {
#pragma unroll
        for (int r = 0; r < RM; ++r) {
            const int e = lane + NT * r;
            int i = 0, j = NZ;
            if (e < NSYM) {
                int rem = e;
                while (rem >= NZ - i) {
                    rem -= NZ - i;
                    ++i;
                }
                j = i + rem;
            } else {
                i = e - NSYM;
            }
            mi[r] = i;
            mj[r] = j;
        }
#pragma unroll
        for (int r = 0; r < RP; ++r) {
            const int e = lane + NT * r;
            int i = 0, j = NS;  // j = NS marks p_i
            if (e < NPS) {
                int rem = e;
                while (rem >= NS - i) {
                    rem -= NS - i;
                    ++i;
                }
                j = i + rem;
            } else {
                i = e - NPS;
            }
            pi_[r] = i;
            pj[r] = j;
        }
    }
    bool ok = true;
    for (int t = N - 1; t >= 0; --t) {
#pragma unroll
        for (int r = 0; r < PF; ++r) {
            const int e = lane + NT * r;
            if (e < NST) stg[e] = nxt[r];
        }
        ric_sync<NT>();
        if (t >= 1) {
#pragma unroll
            for (int r = 0; r < PF; ++r) {
                const int e = lane + NT * r;
                if (e < NST) nxt[r] = ric_stage_elem<F, NS, NU>(scr, N, t - 1, e);
            }
        }
        // Y = P G + [0 | 0 | p]
        for (int e = lane; e < NS * NX; e += NT) {
            const int k = e / NX, j = e % NX;
            F acc = j == NX - 1 ? pv[k] : F(0);
#pragma unroll
            for (int l = 0; l < NS; ++l) acc += P[k * NS + l] * Gs[l * NX + j];
            Y[e] = acc;
        }
        ric_sync<NT>();
        // M: the upper triangle of the Hessian part, then the gradient column
        if constexpr (HOIST) {
#pragma unroll
            for (int r = 0; r < RM; ++r) {
                if (lane + NT * r >= NSYM + NZ) break;
                const int i = mi[r], j = mj[r];
                const int jy = j < NZ ? j : NX - 1;
                F acc;
                if (j == NZ) acc = i < NS ? qs[i] : rs[i - NS];
                else if (j < NS) acc = Qs[i * NS + j];
                else acc = (i == j) ? ru_diag[i - NS] : F(0);
#pragma unroll
                for (int k = 0; k < NS; ++k) acc += Gs[k * NX + i] * Y[k * NX + jy];
                M[i * MC + j] = acc;
                if (j < NZ && j != i) M[j * MC + i] = acc;
            }
        } else
        for (int e = lane; e < NSYM + NZ; e += NT) {
            int i, j;
            if (e < NSYM) {
                int rem = e;
                i = 0;
                while (rem >= NZ - i) {
                    rem -= NZ - i;
                    ++i;
                }
                j = i + rem;
            } else {
                i = e - NSYM;
                j = NZ;
            }
            const int jy = j < NZ ? j : NX - 1;
            F acc;
            if (j == NZ) acc = i < NS ? qs[i] : rs[i - NS];
            else if (j < NS) acc = Qs[i * NS + j];
            else acc = (i == j) ? ru_diag[i - NS] : F(0);
#pragma unroll
            for (int k = 0; k < NS; ++k) acc += Gs[k * NX + i] * Y[k * NX + jy];
            M[i * MC + j] = acc;
            if (j < NZ && j != i) M[j * MC + i] = acc;
        }
        ric_sync<NT>();
        // Quu^-1 (every lane), then [K_t | k_t] = -Quu^-1 [Qus | qu]
        F U[NU][NU], X[NU][NU];
#pragma unroll
        for (int a = 0; a < NU; ++a)
#pragma unroll
            for (int b = 0; b < NU; ++b) U[a][b] = M[(NS + a) * MC + NS + b];
        ok &= spd_inverse<F, NU>(U, X);
        for (int e = lane; e < NU * (NS + 1); e += NT) {
            const int a = e / (NS + 1), j = e % (NS + 1);
            const int cj = j < NS ? j : NZ;
            F acc = F(0);
#pragma unroll
            for (int b = 0; b < NU; ++b) acc -= X[a][b] * M[(NS + b) * MC + cj];
            KK[e] = acc;
            if (j < NS) scr[LY::K(N, t) + a * NS + j] = acc;
            else scr[LY::k(N, t) + a] = acc;
        }
        ric_sync<NT>();
        // P_t = Qss + Qus^T K_t (upper triangle, mirrored), p_t = qs + Qus^T k_t
        if constexpr (HOIST) {
#pragma unroll
            for (int r = 0; r < RP; ++r) {
                if (lane + NT * r >= NPS + NS) break;
                const int i = pi_[r], j = pj[r];
                if (j < NS) {
                    F acc = M[i * MC + j];
#pragma unroll
                    for (int a = 0; a < NU; ++a) acc += M[(NS + a) * MC + i] * KK[a * (NS + 1) + j];
                    P[i * NS + j] = acc;
                    P[j * NS + i] = acc;
                } else {
                    F acc = M[i * MC + NZ];
#pragma unroll
                    for (int a = 0; a < NU; ++a) acc += M[(NS + a) * MC + i] * KK[a * (NS + 1) + NS];
                    pv[i] = acc;
                }
            }
        } else
        for (int e = lane; e < NPS + NS; e += NT) {
            if (e < NPS) {
                int rem = e, i = 0;
                while (rem >= NS - i) {
                    rem -= NS - i;
                    ++i;
                }
                const int j = i + rem;
                F acc = M[i * MC + j];
#pragma unroll
                for (int a = 0; a < NU; ++a) acc += M[(NS + a) * MC + i] * KK[a * (NS + 1) + j];
                P[i * NS + j] = acc;
                P[j * NS + i] = acc;
            } else {
                const int i = e - NPS;
                F acc = M[i * MC + NZ];
#pragma unroll
                for (int a = 0; a < NU; ++a) acc += M[(NS + a) * MC + i] * KK[a * (NS + 1) + NS];
                pv[i] = acc;
            }
        }
        ric_sync<NT>();
    }
    if constexpr (NT == 32) return __all_sync(0xffffffffu, ok);
    else return __syncthreads_and(ok) != 0;
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
