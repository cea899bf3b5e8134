// Adjoint of a taped ADMM solve (reverse mode through the unrolled
// iterations of Sec. IV-B).  One iteration k maps
//   (s^k, u^k, y^k, zeta^{k-1}, xi^{k-1}, z^k, w^k)
// through
//   head  zeta^k = zeta^{k-1} + T(s^k, y^k),  xi^k = xi^{k-1} + R(s^k, y^k)
//   QP    y^{k+1} = pair QP at (pose(s^k), zeta^k, xi^k) with proximal centre y^k
//   stats Gauss-Newton statistics of y^{k+1}, zeta^k, xi^k per (part, t)
//   LQ    (s^{k+1}, u^{k+1}) = trajectory step linearised at (s^k, u^k)
//   box   z^{k+1} = clip((s,u)^{k+1} + w^k),  w^{k+1} = w^k + (s,u)^{k+1} - z^{k+1}
// and the reverse step k runs these backwards:
//   k_adj_traj  box and LQ adjoints (the adjoint LQ shares the Riccati
//               factorisation of the forward problem), then the chain rule
//               through the linearisation point (second derivatives of the
//               dynamics and of the part poses by dual numbers);
//   k_adj_pair  per pair: statistics, pair QP (implicit differentiation of
//               its optimality conditions in the (D+1)-dimensional dual form
//               the forward solver uses) and head adjoints, reduced to pose
//               adjoints per (part, t) and offset adjoints per obstacle face.
// The pair QP is differentiated on its active set, which is locally constant
// at strictly complementary solutions.
#include "oca_common.cuh"
#include "oca_dual.cuh"
#include "oca_kernels.h"
#include "oca_ric.cuh"
#include "oca_solvers.cuh"

namespace oca {

// ============================================================================
// chain rule through the linearisation point
// ============================================================================

// (sb, ub) += dt * d/d(s, u) [ sum At .* fs(s, u) + Bt .* fu(s, u) ]: the
// adjoint of A_t = I + dt fs, B_t = dt fu and c_t = s + dt f - A_t s - B_t u
// with respect to the linearisation point, given At = Abar - cbar s^T and
// Bt = Bbar - cbar u^T.
template <typename T, int KIND>
__device__ void dyn_vjp(const DevModel<T> &m, const T *st, const T *ut, const T *At, const T *Bt, T *sb, T *ub) {
    constexpr int NS = MDims<KIND>::NS, NU = MDims<KIND>::NU;
    const DevModel<Dual<T>> dm = dual_model(m);
    for (int e = 0; e < NS + NU; ++e) {
        Dual<T> sd[NS], ud[NU], f[NS], fs[NS * NS], fu[NS * NU];
#pragma unroll
        for (int i = 0; i < NS; ++i) sd[i] = Dual<T>(st[i], i == e ? T(1) : T(0));
#pragma unroll
        for (int i = 0; i < NU; ++i) ud[i] = Dual<T>(ut[i], i + NS == e ? T(1) : T(0));
        dynamics<Dual<T>, KIND>(dm, sd, ud, f, fs, fu);
        T acc = T(0);
        for (int i = 0; i < NS * NS; ++i) acc += At[i] * fs[i].d;
        for (int i = 0; i < NS * NU; ++i) acc += Bt[i] * fu[i].d;
        if (e < NS) sb[e] += m.dt * acc;
        else ub[e - NS] += m.dt * acc;
    }
}

// Adjoint of the Gauss-Newton stage terms sigma Hs, sigma (g - Hs s) of one
// part (gn_part) given Qbar and qbar of the stage: G = Qbar - qbar s^T.
//   sb    += d/ds  sigma [G : Hs + qbar . g] - sigma Hs^T qbar
//   statb  = d/dstats sigma [G : Hs + qbar . g]   (the terms are linear in them)
template <typename T, int KIND>
__device__ void gn_vjp(const DevModel<T> &m, int link, const T *off, const T *st, const T *Wl, const T *Wc,
                       const T *E, const T *G, const T *qb, T sigma, T *sb, T *statb) {
    constexpr int NS = MDims<KIND>::NS, D = MDims<KIND>::D;
    constexpr int NW = StatDims<D>::NW, NSTAT = StatDims<D>::NSTAT;
    const DevModel<Dual<T>> dm = dual_model(m);
    Dual<T> offd[D], sd[NS], stat[NSTAT], Hs[NS * NS], g[NS];
#pragma unroll
    for (int i = 0; i < D; ++i) offd[i] = Dual<T>(off[i]);
#pragma unroll
    for (int i = 0; i < NW; ++i) stat[i] = Dual<T>(Wl[i]);
#pragma unroll
    for (int i = 0; i < D; ++i) stat[NW + i] = Dual<T>(Wc[i]);
#pragma unroll
    for (int i = 0; i < D * D; ++i) stat[NW + D + i] = Dual<T>(E[i]);
    for (int e = 0; e < NS; ++e) {
#pragma unroll
        for (int i = 0; i < NS; ++i) sd[i] = Dual<T>(st[i], i == e ? T(1) : T(0));
        gn_part<Dual<T>, KIND>(dm, link, offd, sd, stat, stat + NW, stat + NW + D, Hs, g);
        T acc = T(0);
        for (int i = 0; i < NS * NS; ++i) acc += G[i] * Hs[i].d;
        for (int i = 0; i < NS; ++i) acc += qb[i] * (g[i].d - Hs[i * NS + e].v);
        sb[e] += sigma * acc;
    }
#pragma unroll
    for (int i = 0; i < NS; ++i) sd[i] = Dual<T>(st[i]);
    for (int kk = 0; kk < NSTAT; ++kk) {
        stat[kk].d = T(1);
        gn_part<Dual<T>, KIND>(dm, link, offd, sd, stat, stat + NW, stat + NW + D, Hs, g);
        stat[kk].d = T(0);
        T acc = T(0);
        for (int i = 0; i < NS * NS; ++i) acc += G[i] * Hs[i].d;
        for (int i = 0; i < NS; ++i) acc += qb[i] * g[i].d;
        statb[kk] = sigma * acc;
    }
}

// ============================================================================
// seed: adjoint of the trajectory cost F of eqn:navigation_cost at s^K, u^K
// ============================================================================
template <typename T, int KIND>
__global__ void __launch_bounds__(32) k_adj_seed(AdjTrajArgs<T> a) {
    constexpr int NS = MDims<KIND>::NS, NU = MDims<KIND>::NU;
    const int s = blockIdx.x, lane = threadIdx.x;
    const ScenMeta sm = a.meta[s];
    const int K = a.iters[s];
    const T *sK = a.tape.s + (long long)K * a.tape.s_slot, *uK = a.tape.u + (long long)K * a.tape.u_slot;
    const T gc = a.grad_cost[s];
    for (int t = lane; t <= sm.N; t += 32) {
        for (int i = 0; i < NS; ++i) {
            const long long k2 = (long long)(sm.state0 + t) * NS + i;
            const T v = gc * T(2) * a.model.Qs[i] * (sK[k2] - a.s_ref[k2]);
            if (t == 0) a.gs0[(long long)s * NS + i] += double(v);
            else a.sb[k2] = v;
        }
        if (t < sm.N)
            for (int i = 0; i < NU; ++i) {
                const long long k2 = (long long)(sm.ctrl0 + t) * NU + i;
                a.ub[k2] = gc * T(2) * a.model.Qu[i] * uK[k2];
            }
    }
}

// ============================================================================
// reverse step k of the trajectory side (one warp per scenario)
// ============================================================================
template <typename T, typename F, int KIND>
__global__ void __launch_bounds__(32) k_adj_traj(AdjTrajArgs<T> a) {
    constexpr int NS = MDims<KIND>::NS, NU = MDims<KIND>::NU, D = MDims<KIND>::D, NROT = MDims<KIND>::NROT;
    constexpr int NW = StatDims<D>::NW, NSTAT = StatDims<D>::NSTAT;
    using LY = RicLayout<NS, NU>;
    const int s = blockIdx.x, lane = threadIdx.x;
    const int k = a.k;
    if (k >= a.iters[s]) return;
    const ScenMeta sm = a.meta[s];
    const int N = sm.N;
    const TapeView<T> &tp = a.tape;
    const T *s_k = tp.s + (long long)k * tp.s_slot, *u_k = tp.u + (long long)k * tp.u_slot;
    const T *s_k1 = tp.s + (long long)(k + 1) * tp.s_slot, *u_k1 = tp.u + (long long)(k + 1) * tp.u_slot;
    const T *zs_k = tp.box + (long long)k * tp.box_slot;
    const T *ws_k = zs_k + tp.n_states * NS, *zu_k = ws_k + tp.n_states * NS, *wu_k = zu_k + tp.n_ctrls * NU;
    const T *stats_k = tp.stats + (long long)k * tp.stats_slot;
    F *scr = reinterpret_cast<F *>(a.scratch) + a.scratch0[s];

    // ---- 1. pose adjoints of s^{k+1} (pair side of iteration k+1) into sbar^{k+1}
    for (int t = 1 + lane; t <= N; t += 32) {
        T st[NS], acc[NS];
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            st[i] = s_k1[(long long)(sm.state0 + t) * NS + i];
            acc[i] = T(0);
        }
        for (int part = 0; part < sm.NP; ++part) {
            const int gp = sm.part0 + part;
            T off[D], rho[D], R[D * D], drho[D * NS], dR[NROT][D * D];
            int ridx[NROT];
#pragma unroll
            for (int i = 0; i < D; ++i) off[i] = a.g.part_off[gp * D + i];
            part_pose<T, KIND>(a.model, a.g.part_link[gp], off, st, rho, R, drho, dR, ridx);
            const long long col = sm.qbeg + part * N + (t - 1);
            for (int i = 0; i < D; ++i) {
                const T rb = a.poseb[(long long)i * a.Qtot + col];
                for (int e = 0; e < NS; ++e) acc[e] += rb * drho[i * NS + e];
            }
#pragma unroll
            for (int r = 0; r < NROT; ++r) {
                T v = T(0);
#pragma unroll
                for (int i = 0; i < D * D; ++i) v += a.poseb[(long long)(D + i) * a.Qtot + col] * dR[r][i];
                acc[ridx[r]] += v;
            }
        }
        for (int i = 0; i < NS; ++i) a.sb[(long long)(sm.state0 + t) * NS + i] += acc[i];
    }
    // ---- 2. box update of iteration k (z = clip(x + w), w += x - z)
    const int n_box = a.rho_box > T(0) ? N * NS + N * NU : 0;
    for (int e = lane; e < n_box; e += 32) {
        long long k2;
        T lo, hi, x, w;
        T *xb, *zb, *wb;
        if (e < N * NS) {
            const int t = 1 + e / NS, i = e % NS;
            lo = a.model.s_lo[i];
            hi = a.model.s_hi[i];
            k2 = (long long)(sm.state0 + t) * NS + i;
            x = s_k1[k2];
            w = ws_k[k2];
            xb = a.sb;
            zb = a.zsb;
            wb = a.wsb;
        } else {
            const int e2 = e - N * NS, t = e2 / NU, i = e2 % NU;
            lo = a.model.u_lo[i];
            hi = a.model.u_hi[i];
            k2 = (long long)(sm.ctrl0 + t) * NU + i;
            x = u_k1[k2];
            w = wu_k[k2];
            xb = a.ub;
            zb = a.zub;
            wb = a.wub;
        }
        if (!bounded(lo, hi)) continue;
        const T wbar = wb[k2], zp = zb[k2] - wbar, v = x + w;
        T xa = xb[k2] + wbar, wn = wbar;
        if (v > lo && v < hi) {
            xa += zp;
            wn += zp;
        }
        xb[k2] = xa;
        wb[k2] = wn;
        zb[k2] = T(0);
    }
    __syncwarp();
    // ---- 3. the LQ problem of iteration k, rebuilt from the tape
    StageParams<T> sp;
    sp.model = a.model;
    sp.g = a.g;
    sp.sigma = a.sigma;
    sp.rho_box = a.rho_box;
    sp.damp = a.damp;
    sp.s_ref = a.s_ref;
    sp.Qtot = a.Qtot;
    StageSrc<T> src;
    src.s = s_k;
    src.u = u_k;
    src.zs = zs_k;
    src.ws = ws_k;
    src.zu = zu_k;
    src.wu = wu_k;
    src.stats = stats_k;
    for (int t = lane; t <= N; t += 32) assemble_stage<T, F, KIND>(sp, src, sm, t, scr);
    __syncwarp();
    // ---- 4. costates of its solution (s^{k+1}, u^{k+1})
    {
        auto xf = [&](int t, int i) -> F { return F(s_k1[(long long)(sm.state0 + t) * NS + i]); };
        ric_costates<F, NS, NU, false>(scr, N, xf);
    }
    // ---- 5. adjoint LQ: same Q, Ru, A, B; linear terms -sbar, -ubar; c = 0; s_0 = 0
    for (int t = lane; t <= N; t += 32) {
        for (int i = 0; i < NS; ++i)
            scr[LY::q(N, t) + i] = t >= 1 ? -F(a.sb[(long long)(sm.state0 + t) * NS + i]) : F(0);
        if (t < N) {
            for (int i = 0; i < NU; ++i) scr[LY::r(N, t) + i] = -F(a.ub[(long long)(sm.ctrl0 + t) * NU + i]);
            for (int i = 0; i < NS; ++i) scr[LY::c(N, t) + i] = F(0);
        }
    }
    // sbar of the fixed initial state passes straight to the initial-state adjoint
    if (lane < NS) {
        const long long k2 = (long long)sm.state0 * NS + lane;
        a.gs0[(long long)s * NS + lane] += double(a.sb[k2]);
        a.sb[k2] = T(0);
    }
    __syncwarp();
    // diagonal of Ru in shared memory, as in the forward kernel
    __shared__ F ru_diag[NU];
    for (int i = lane; i < NU; i += 32)
        ru_diag[i] = F(2) * F(a.model.Qu[i]) + F(a.damp) +
                     (bounded(a.model.u_lo[i], a.model.u_hi[i]) ? F(a.rho_box) : F(0));
    __syncwarp();
    ric_factor<F, NS, NU>(scr, N, ru_diag);
    __shared__ F sc[NS];
    for (int i = lane; i < NS; i += 32) {
        sc[i] = F(0);
        scr[LY::xs(N, 0) + i] = F(0);
    }
    __syncwarp();
    struct Out {
        F *scr;
        int N;
        __device__ void put_u(int t, int i, F v) { scr[LY::xu(N, t) + i] = v; }
        __device__ void put_s(int t, int i, F v) { scr[LY::xs(N, t) + i] = v; }
    } out{scr, N};
    ric_sweep<F, NS, NU>(scr, N, sc, out);
    {
        auto xa = [&](int t, int i) -> F { return scr[LY::xs(N, t) + i]; };
        ric_costates<F, NS, NU, true>(scr, N, xa);
    }
    __syncwarp();
    // ---- 6. data adjoints of the LQ and the chain rule into iterate k
    //   Abar_t = -(pa_{t+1} s_t^T + pf_{t+1} xs_t^T), Bbar_t = -(pa_{t+1} u_t^T + pf_{t+1} xu_t^T),
    //   cbar_t = -pa_{t+1}, rbar_t = -xu_t, qbar_t = -xs_t, Qbar_t = -xs_t s_t^T
    // with (s, u) = (s^{k+1}, u^{k+1}), (xs, xu) the adjoint solution and
    // pf, pa the forward and adjoint costates.
    const T rho_b = a.rho_box, damp = a.damp;
    for (int t = lane; t <= N; t += 32) {
        T sbk[NS], ubk[NU], skt[NS], ukt[NU];
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            sbk[i] = T(0);
            skt[i] = s_k[(long long)(sm.state0 + t) * NS + i];
        }
#pragma unroll
        for (int i = 0; i < NU; ++i) {
            ubk[i] = T(0);
            ukt[i] = t < N ? u_k[(long long)(sm.ctrl0 + t) * NU + i] : T(0);
        }
        if (t < N) {
            F pf1[NS], pa1[NS], xt[NS], xh[NS], uh[NU], ut1[NU];
            for (int i = 0; i < NS; ++i) {
                pf1[i] = scr[LY::pf(N, t + 1) + i];
                pa1[i] = scr[LY::pa(N, t + 1) + i];
                xt[i] = F(s_k1[(long long)(sm.state0 + t) * NS + i]);
                xh[i] = scr[LY::xs(N, t) + i];
            }
            for (int i = 0; i < NU; ++i) {
                uh[i] = scr[LY::xu(N, t) + i];
                ut1[i] = F(u_k1[(long long)(sm.ctrl0 + t) * NU + i]);
            }
            T At[NS * NS], Bt[NS * NU];
            for (int i = 0; i < NS; ++i) {
                const F cb = -pa1[i];
                for (int j = 0; j < NS; ++j) At[i * NS + j] = T(-(pa1[i] * xt[j] + pf1[i] * xh[j]) - cb * F(skt[j]));
                for (int j = 0; j < NU; ++j) Bt[i * NU + j] = T(-(pa1[i] * ut1[j] + pf1[i] * uh[j]) - cb * F(ukt[j]));
            }
            dyn_vjp<T, KIND>(a.model, skt, ukt, At, Bt, sbk, ubk);
            for (int i = 0; i < NU; ++i) {
                const T rb = T(-uh[i]);
                ubk[i] -= damp * rb;
                if (rho_b > T(0) && bounded(a.model.u_lo[i], a.model.u_hi[i])) {
                    const long long k2 = (long long)(sm.ctrl0 + t) * NU + i;
                    a.zub[k2] = -rho_b * rb;
                    a.wub[k2] += rho_b * rb;
                }
            }
            if (t == 0) {
                // s_0 enters the first dynamics constraint as data: -A_0^T pa_1
                const F *A0 = scr + LY::A(N, 0);
                for (int j = 0; j < NS; ++j) {
                    F acc = F(0);
                    for (int i = 0; i < NS; ++i) acc -= A0[i * NS + j] * pa1[i];
                    sbk[j] += T(acc);
                }
            }
        }
        if (t >= 1) {
            T qb[NS], G[NS * NS];
            for (int i = 0; i < NS; ++i) {
                const F xh = scr[LY::xs(N, t) + i];
                qb[i] = T(-xh);
                for (int j = 0; j < NS; ++j)
                    G[i * NS + j] = T(-xh * F(s_k1[(long long)(sm.state0 + t) * NS + j])) - qb[i] * skt[j];
            }
            for (int i = 0; i < NS; ++i) {
                sbk[i] -= damp * qb[i];
                if (rho_b > T(0) && bounded(a.model.s_lo[i], a.model.s_hi[i])) {
                    const long long k2 = (long long)(sm.state0 + t) * NS + i;
                    a.zsb[k2] = -rho_b * qb[i];
                    a.wsb[k2] += rho_b * qb[i];
                }
            }
            for (int part = 0; part < sm.NP; ++part) {
                const int gp = sm.part0 + part;
                const long long col = sm.qbeg + part * N + (t - 1);
                T off[D], Wl[NW], Wc[D], E[D * D], statb[NSTAT];
#pragma unroll
                for (int i = 0; i < D; ++i) off[i] = a.g.part_off[gp * D + i];
#pragma unroll
                for (int i = 0; i < NW; ++i) Wl[i] = stats_k[(long long)i * a.Qtot + col];
#pragma unroll
                for (int i = 0; i < D; ++i) Wc[i] = stats_k[(long long)(NW + i) * a.Qtot + col];
#pragma unroll
                for (int i = 0; i < D * D; ++i) E[i] = stats_k[(long long)(NW + D + i) * a.Qtot + col];
                gn_vjp<T, KIND>(a.model, a.g.part_link[gp], off, skt, Wl, Wc, E, G, qb, a.sigma, sbk, statb);
#pragma unroll
                for (int i = 0; i < NSTAT; ++i) a.statsb[(long long)i * a.Qtot + col] = statb[i];
            }
        }
        if (t == 0) {
            for (int i = 0; i < NS; ++i) a.gs0[(long long)s * NS + i] += double(sbk[i]);
        } else {
            for (int i = 0; i < NS; ++i) a.sb[(long long)(sm.state0 + t) * NS + i] = sbk[i];
        }
        if (t < N)
            for (int i = 0; i < NU; ++i) a.ub[(long long)(sm.ctrl0 + t) * NU + i] = ubk[i];
    }
}

// ============================================================================
// reverse step k of the pair side.  Work decomposition of the forward pair
// kernel: a CTA owns 32 (part, t) lanes of one scenario, warp w takes the
// obstacles j = w, w+W, ...
// ============================================================================
template <typename T, int D, int NR>
__global__ void __launch_bounds__(256) k_adj_pair(AdjPairArgs<T> a) {
    constexpr int V = D + 1, NW = StatDims<D>::NW, PK = D + D * D;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *red = reinterpret_cast<T *>(smem_raw);  // [W][PK][32]
    const Tile tile = a.tiles[blockIdx.x];
    const ScenMeta sm = a.meta[tile.scen];
    const int k = a.k;
    if (k >= a.iters[tile.scen]) return;
    const int lane = threadIdx.x, warp = threadIdx.y, W = blockDim.y;
    const int Q = sm.NP * sm.N;
    const int q = tile.q0 + lane;
    const bool valid = q < Q;
    const long long P = a.P;
    const int FR = a.g.FR, FO = a.g.FO;
    const T rho_p = a.prox;
    const bool head = k >= 1;
    T pb[PK];
#pragma unroll
    for (int i = 0; i < PK; ++i) pb[i] = T(0);

    {
        // lanes past the tile's end run on the last lane's data (the warp
        // reductions below need every lane) and write nothing
        const int col = sm.qbeg + (valid ? q : Q - 1);
        T rho[D], R[D * D];
#pragma unroll
        for (int i = 0; i < D; ++i) rho[i] = a.pose[(long long)i * a.Qtot + col];
#pragma unroll
        for (int i = 0; i < D * D; ++i) R[i] = a.pose[(long long)(D + i) * a.Qtot + col];
        const int gp = sm.part0 + (valid ? q : Q - 1) / sm.N;
        const int nr = a.g.part_nf[gp];
        T ak[NR][D], bk[NR], ia2[NR];
#pragma unroll
        for (int kk = 0; kk < NR; ++kk) {
            T s2 = T(0);
#pragma unroll
            for (int i = 0; i < D; ++i) {
                ak[kk][i] = kk < nr ? a.g.part_A[((long long)gp * FR + kk) * D + i] : T(0);
                s2 += ak[kk][i] * ak[kk][i];
            }
            bk[kk] = kk < nr ? a.g.part_b[(long long)gp * FR + kk] : T(1);
            ia2[kk] = s2 > T(0) ? T(1) / s2 : T(0);
        }
        // adjoint of this lane's statistics
        T Wlb[NW], Wcb[D], Eb[D * D];
#pragma unroll
        for (int i = 0; i < NW; ++i) Wlb[i] = a.statsb[(long long)i * a.Qtot + col];
#pragma unroll
        for (int i = 0; i < D; ++i) Wcb[i] = a.statsb[(long long)(NW + i) * a.Qtot + col];
#pragma unroll
        for (int i = 0; i < D * D; ++i) Eb[i] = a.statsb[(long long)(NW + D + i) * a.Qtot + col];

        for (int j = warp; j < sm.M; j += W) {
            const int gm = sm.obs0 + j;
            const T *C = a.g.obs_C + (long long)gm * FO * D, *dd = a.g.obs_d + (long long)gm * FO;
            const int no = a.g.obs_nf[gm];
            const long long p = sm.pair0 + (long long)j * Q + (valid ? q : Q - 1);
            const T *y1 = a.y_k1 + p, *y0 = a.y_k + p, *yi = a.ybar_in + p;
            T *yo = a.ybar_out + p;
            const T zeta = a.zx_k[p];
            T xi[D];
#pragma unroll
            for (int i = 0; i < D; ++i) xi[i] = a.zx_k[(long long)(1 + i) * P + p];
            // ---- pass 1: sums of y^{k+1}
            T lp[NR], a1[D], w1w[D], Sd = T(0);
#pragma unroll
            for (int i = 0; i < D; ++i) {
                a1[i] = T(0);
                w1w[i] = T(0);
            }
#pragma unroll
            for (int kk = 0; kk < NR; ++kk) {
                lp[kk] = kk < nr ? y1[(long long)kk * P] : T(0);
#pragma unroll
                for (int i = 0; i < D; ++i) a1[i] += lp[kk] * ak[kk][i];
            }
            for (int m = 0; m < no; ++m) {
                const T mp = y1[(long long)(FR + m) * P];
#pragma unroll
                for (int i = 0; i < D; ++i) w1w[i] += mp * C[m * D + i];
                Sd += mp * dd[m];
            }
            const T gp1 = y1[(long long)(FR + FO) * P];
            // ---- statistics adjoint: W += w w^T, Wc += c w, E += w e^T
            const T cc = T(1) + Sd + gp1 + zeta;
            T e[D], w1b[D], eb[D], ccb = T(0);
#pragma unroll
            for (int i = 0; i < D; ++i) {
                e[i] = a1[i] + xi[i];
                w1b[i] = Wcb[i] * cc;
                ccb += Wcb[i] * w1w[i];
            }
            {
                int kk = 0;
#pragma unroll
                for (int i = 0; i < D; ++i)
#pragma unroll
                    for (int jj = 0; jj <= i; ++jj) {
                        if (i == jj) {
                            w1b[i] += T(2) * Wlb[kk] * w1w[i];
                        } else {
                            w1b[i] += Wlb[kk] * w1w[jj];
                            w1b[jj] += Wlb[kk] * w1w[i];
                        }
                        ++kk;
                    }
            }
#pragma unroll
            for (int jj = 0; jj < D; ++jj) {
                T acc = T(0);
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    acc += Eb[i * D + jj] * w1w[i];
                    w1b[i] += Eb[i * D + jj] * e[jj];
                }
                eb[jj] = acc;
            }
            T zb = a.zb[p] + ccb, xb[D];
#pragma unroll
            for (int i = 0; i < D; ++i) xb[i] = a.xb[(long long)i * P + p] + eb[i];
            // ---- the QP's dual point w* = K^T y^{k+1} + bq
            T wr = T(0);
#pragma unroll
            for (int i = 0; i < D; ++i) wr += w1w[i] * rho[i];
            const T w0 = T(1) + zeta + Sd - wr + gp1;
            T w1s[D], Rw1[D];
#pragma unroll
            for (int i = 0; i < D; ++i) {
                T acc = xi[i] + a1[i];
#pragma unroll
                for (int l = 0; l < D; ++l) acc += R[l * D + i] * w1w[l];
                w1s[i] = acc;
            }
#pragma unroll
            for (int i = 0; i < D; ++i) {
                T acc = T(0);
#pragma unroll
                for (int l = 0; l < D; ++l) acc += R[i * D + l] * w1s[l];
                Rw1[i] = acc;
            }
            // ---- H = rho (I - K^T dy/dw) and rr = -rho (dy/dw)^T ybar_out
            T H[V][V], rr[V];
#pragma unroll
            for (int i = 0; i < V; ++i) {
                rr[i] = T(0);
#pragma unroll
                for (int jj = 0; jj < V; ++jj) H[i][jj] = i == jj ? rho_p : T(0);
            }
            // lambda block (projection onto b^T lambda = 1 on the support S)
            T yol[NR], bb = T(0), byo = T(0), ba[D];
#pragma unroll
            for (int i = 0; i < D; ++i) ba[i] = T(0);
#pragma unroll
            for (int kk = 0; kk < NR; ++kk) {
                T v = kk < nr ? yi[(long long)kk * P] : T(0);
#pragma unroll
                for (int i = 0; i < D; ++i) v += ak[kk][i] * eb[i];
                yol[kk] = v;
                if (kk < nr && lp[kk] > T(0)) {
                    bb += bk[kk] * bk[kk] * ia2[kk];
                    byo += bk[kk] * ia2[kk] * v;
#pragma unroll
                    for (int i = 0; i < D; ++i) {
                        ba[i] += bk[kk] * ak[kk][i] * ia2[kk];
#pragma unroll
                        for (int l = 0; l < D; ++l) H[1 + i][1 + l] += ak[kk][i] * ak[kk][l] * ia2[kk];
                    }
                }
            }
            const T ibb = bb > T(0) ? T(1) / bb : T(0);
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
                for (int l = 0; l < D; ++l) H[1 + i][1 + l] -= ba[i] * ba[l] * ibb;
#pragma unroll
            for (int kk = 0; kk < NR; ++kk) {
                if (kk < nr && lp[kk] > T(0)) {
                    const T zl = yol[kk] - bk[kk] * byo * ibb;
#pragma unroll
                    for (int i = 0; i < D; ++i) rr[1 + i] += zl * ak[kk][i] * ia2[kk];
                }
            }
            // slack gamma
            const T yog = yi[(long long)(FR + FO) * P] + ccb;
            if (gp1 > T(0)) {
                H[0][0] += T(1);
                rr[0] += yog;
            }
            // ---- pass 2: active obstacle faces
            for (int m = 0; m < no; ++m) {
                const T mp = y1[(long long)(FR + m) * P];
                if (!(mp > T(0))) continue;
                T c[D], cr = T(0), c2 = T(0), Km[V];
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    c[i] = C[m * D + i];
                    cr += c[i] * rho[i];
                    c2 += c[i] * c[i];
                }
                const T dm = dd[m], dpm = dm - cr;
                Km[0] = dpm;
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    T acc = T(0);
#pragma unroll
                    for (int l = 0; l < D; ++l) acc += R[l * D + i] * c[l];
                    Km[1 + i] = acc;
                }
                T yom = yi[(long long)(FR + m) * P] + ccb * dm;
#pragma unroll
                for (int i = 0; i < D; ++i) yom += c[i] * w1b[i];
                const T iDg = T(1) / (dpm * dpm + c2);
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    rr[i] += yom * Km[i] * iDg;
#pragma unroll
                    for (int l = 0; l < V; ++l) H[i][l] += Km[i] * Km[l] * iDg;
                }
            }
            T u[V];
#pragma unroll
            for (int i = 0; i < V; ++i) u[i] = rr[i];
            if (chol_solve<T, V>(H, u, V, T(0))) {
#pragma unroll
                for (int i = 0; i < V; ++i) u[i] = -u[i];
            } else {
#pragma unroll
                for (int i = 0; i < V; ++i) u[i] = T(0);
            }
            zb += u[0];
#pragma unroll
            for (int i = 0; i < D; ++i) xb[i] += u[1 + i];
            // head of iteration k: T = 1 + d'^T mu^k + gamma^k, R = A^T lambda^k + R^T C^T mu^k
            T RRv[D];
#pragma unroll
            for (int i = 0; i < D; ++i) {
                T acc = T(0);
#pragma unroll
                for (int l = 0; l < D; ++l) acc += R[i * D + l] * xb[l];
                RRv[i] = acc;
            }
            // ---- pass 3: face outputs
            T ch[D], wk[D];
#pragma unroll
            for (int i = 0; i < D; ++i) {
                ch[i] = T(0);
                wk[i] = T(0);
            }
            for (int m = 0; m < no; ++m) {
                const T mp = y1[(long long)(FR + m) * P], mk = y0[(long long)(FR + m) * P];
                T c[D], cr = T(0), c2 = T(0), cRw = T(0), cu = T(0), cRv = T(0), cw1b = T(0);
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    c[i] = C[m * D + i];
                    cr += c[i] * rho[i];
                    c2 += c[i] * c[i];
                    cRw += c[i] * Rw1[i];
                    cRv += c[i] * RRv[i];
                    cw1b += c[i] * w1b[i];
                }
                // (R^T c) . u1
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    T acc = T(0);
#pragma unroll
                    for (int l = 0; l < D; ++l) acc += R[l * D + i] * c[l];
                    cu += acc * u[1 + i];
                }
                const T dm = dd[m], dpm = dm - cr, Dg = dpm * dpm + c2;
                T dpb = mp * u[0];   // d/dd' of (K^T y).u at fixed y
                T ybo = T(0);
                if (mp > T(0)) {
                    const T yom = yi[(long long)(FR + m) * P] + ccb * dm + cw1b;
                    const T yh = yom + dpm * u[0] + cu;
                    const T iDg = T(1) / (rho_p * Dg), h = dpm * w0 + cRw;
                    ybo = yh;
                    dpb += yh * (-w0 * iDg + T(2) * h * dpm * iDg / Dg);
#pragma unroll
                    for (int i = 0; i < D; ++i) ch[i] += yh * c[i] * iDg;
                }
                if (head) {
                    ybo += zb * dpm + cRv;
                    dpb += zb * mk;
#pragma unroll
                    for (int i = 0; i < D; ++i) wk[i] += mk * c[i];
                }
                if (valid) yo[(long long)(FR + m) * P] = ybo;
#pragma unroll
                for (int i = 0; i < D; ++i) pb[i] -= dpb * c[i];
                // offset adjoint: d' = d - c.rho, plus the statistics' c = 1 + d^T mu + ...
                T gdv = valid ? dpb + ccb * mp : T(0);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) gdv += __shfl_xor_sync(0xffffffffu, gdv, o);
                if (lane == 0) atomicAdd(a.gd + (long long)gm * FO + m, double(gdv));
            }
            // R adjoint: -sum_act yh c w1*^T / (rho Dg) + w+ u1^T + [head] w^k xi_bar^T
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
                for (int l = 0; l < D; ++l)
                    pb[D + i * D + l] += -ch[i] * w1s[l] + w1w[i] * u[1 + l] + (head ? wk[i] * xb[l] : T(0));
            // lambda outputs
            T byh = T(0);
#pragma unroll
            for (int kk = 0; kk < NR; ++kk) {
                if (kk < nr && lp[kk] > T(0)) {
                    T yh = yol[kk];
#pragma unroll
                    for (int i = 0; i < D; ++i) yh += ak[kk][i] * u[1 + i];
                    yol[kk] = yh;
                    byh += bk[kk] * ia2[kk] * yh;
                }
            }
#pragma unroll
            for (int kk = 0; kk < NR; ++kk) {
                if (kk < nr) {
                    T v = lp[kk] > T(0) ? yol[kk] - bk[kk] * byh * ibb : T(0);
                    if (head) {
#pragma unroll
                        for (int i = 0; i < D; ++i) v += ak[kk][i] * xb[i];
                    }
                    if (valid) yo[(long long)kk * P] = v;
                }
            }
            if (valid) {
                yo[(long long)(FR + FO) * P] = (gp1 > T(0) ? yog + u[0] : T(0)) + (head ? zb : T(0));
                a.zb[p] = zb;
#pragma unroll
                for (int i = 0; i < D; ++i) a.xb[(long long)i * P + p] = xb[i];
            }
        }
    }
    // ---- reduce the pose adjoints across the W warps
#pragma unroll
    for (int i = 0; i < PK; ++i) red[(warp * PK + i) * 32 + lane] = pb[i];
    __syncthreads();
    if (valid) {
        const int col = sm.qbeg + q;
        for (int i = warp; i < PK; i += W) {
            T acc = T(0);
            for (int w2 = 0; w2 < W; ++w2) acc += red[(w2 * PK + i) * 32 + lane];
            a.poseb[(long long)i * a.Qtot + col] = acc;
        }
    }
}


// ============================================================================
// alpha* of the returned trajectory (Sec. III-A eqn:scale_opt): by the LP
// envelope theorem, at the optimum (alpha*, x*; lambda*, mu*) of a pair
//   dalpha/dd_m = -mu_m,  dalpha/drho = C^T mu,  dalpha/dR = (C^T mu) x*^T
// (C' = C R, d' = d - C rho; the Lagrangian alpha + lambda^T (A x - alpha b)
// + mu^T (C' x - d') differentiated at fixed multipliers).  Writes the pose
// adjoints that seed the reverse sweep and adds the offset adjoints.
// ============================================================================
template <typename T, int D>
__global__ void __launch_bounds__(256) k_adj_alpha(AdjAlphaArgs<T> a) {
    constexpr int PK = D + D * D;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *red = reinterpret_cast<T *>(smem_raw);  // [W][PK][32]
    const Tile tile = a.tiles[blockIdx.x];
    const ScenMeta sm = a.meta[tile.scen];
    const int lane = threadIdx.x, warp = threadIdx.y, W = blockDim.y;
    const int Q = sm.NP * sm.N;
    const int q = tile.q0 + lane;
    const bool valid = q < Q;
    const int qc = valid ? q : Q - 1;
    const long long P = a.P;
    const int FR = a.g.FR, FO = a.g.FO;
    T pb[PK];
#pragma unroll
    for (int i = 0; i < PK; ++i) pb[i] = T(0);
    Lane<T, D> L;
    const int col = sm.qbeg + qc;
#pragma unroll
    for (int i = 0; i < D; ++i) L.rho[i] = a.pose[(long long)i * a.Qtot + col];
#pragma unroll
    for (int i = 0; i < D * D; ++i) L.R[i] = a.pose[(long long)(D + i) * a.Qtot + col];
    const int gp = sm.part0 + qc / sm.N;
    L.A = a.g.part_A + (long long)gp * FR * D;
    L.b = a.g.part_b + (long long)gp * FR;
    L.nr = a.g.part_nf[gp];
    for (int j = warp; j < sm.M; j += W) {
        const int gm = sm.obs0 + j;
        L.C = a.g.obs_C + (long long)gm * FO * D;
        L.d = a.g.obs_d + (long long)gm * FO;
        L.no = a.g.obs_nf[gm];
        const long long p = sm.pair0 + (long long)j * Q + qc;
        int bas[D + 1];
        T xB[D + 1], alpha, x[D];
        lp_solve<T, D>(L, bas, xB, alpha);
        const bool okx = lp_primal<T, D>(L, bas, x);
        const T ga = valid && okx ? a.grad_alpha[p] : T(0);
        T w[D];
#pragma unroll
        for (int i = 0; i < D; ++i) w[i] = T(0);
        for (int m = 0; m < L.no; ++m) {
            T mu = T(0);
#pragma unroll
            for (int i = 0; i < D + 1; ++i)
                if (bas[i] == L.nr + m) mu = xB[i];
#pragma unroll
            for (int i = 0; i < D; ++i) w[i] += mu * L.C[m * D + i];
            T gdv = -ga * mu;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) gdv += __shfl_xor_sync(0xffffffffu, gdv, o);
            if (lane == 0) atomicAdd(a.gd + (long long)gm * FO + m, double(gdv));
        }
#pragma unroll
        for (int i = 0; i < D; ++i) {
            pb[i] += ga * w[i];
#pragma unroll
            for (int l = 0; l < D; ++l) pb[D + i * D + l] += ga * w[i] * x[l];
        }
    }
#pragma unroll
    for (int i = 0; i < PK; ++i) red[(warp * PK + i) * 32 + lane] = pb[i];
    __syncthreads();
    if (valid) {
        for (int i = warp; i < PK; i += W) {
            T acc = T(0);
            for (int w2 = 0; w2 < W; ++w2) acc += red[(w2 * PK + i) * 32 + lane];
            a.poseb[(long long)i * a.Qtot + sm.qbeg + q] = acc;
        }
    }
}

// returned states of every scenario (iterate iters[s] of the tape) into one array
template <typename T>
__global__ void k_adj_final_states(const ScenMeta *meta, const int *iters, const T *tape_s, long long s_slot, int NS,
                                   T *out) {
    const int s = blockIdx.y;
    const ScenMeta sm = meta[s];
    const T *src = tape_s + (long long)iters[s] * s_slot;
    const int n = (sm.N + 1) * NS;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const long long k2 = (long long)sm.state0 * NS + e;
        out[k2] = src[k2];
    }
}

template <typename T>
cudaError_t launch_adj_alpha(const AdjAlphaArgs<T> &a, int dim, int n_tiles, int W, const int *iters,
                             const T *tape_s, long long s_slot, int NS, int n_scen, T *states_out,
                             const PoseArgs<T> &pa, int maxQ, cudaStream_t st) {
    if (n_tiles <= 0) return cudaSuccess;
    k_adj_final_states<T><<<dim3(4, n_scen), 128, 0, st>>>(a.meta, iters, tape_s, s_slot, NS, states_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    PoseArgs<T> p2 = pa;
    p2.states = states_out;
    if ((e = launch_pose<T>(p2, maxQ, st)) != cudaSuccess) return e;
    const size_t sm = (size_t)W * (dim + dim * dim) * 32 * sizeof(T);
    if (dim == 2) k_adj_alpha<T, 2><<<n_tiles, dim3(32, W), sm, st>>>(a);
    else k_adj_alpha<T, 3><<<n_tiles, dim3(32, W), sm, st>>>(a);
    return cudaGetLastError();
}

// ============================================================================
// launchers
// ============================================================================
template <typename T>
cudaError_t launch_adj_seed(const AdjTrajArgs<T> &a, int n_scen, cudaStream_t st) {
    switch (a.model.kind) {
        case 0: k_adj_seed<T, 0><<<n_scen, 32, 0, st>>>(a); break;
        case 1: k_adj_seed<T, 1><<<n_scen, 32, 0, st>>>(a); break;
        case 2: k_adj_seed<T, 2><<<n_scen, 32, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adj_traj(const AdjTrajArgs<T> &a, int n_scen, cudaStream_t st) {
    switch (a.model.kind) {
        case 0: k_adj_traj<T, double, 0><<<n_scen, 32, 0, st>>>(a); break;
        case 1: k_adj_traj<T, double, 1><<<n_scen, 32, 0, st>>>(a); break;
        case 2: k_adj_traj<T, double, 2><<<n_scen, 32, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T, int D, int NR>
cudaError_t launch_adj_pair_t(const AdjPairArgs<T> &a, int n_tiles, int W, cudaStream_t st) {
    const size_t sm = (size_t)W * (D + D * D) * 32 * sizeof(T);
    k_adj_pair<T, D, NR><<<n_tiles, dim3(32, W), sm, st>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adj_pair(const AdjPairArgs<T> &a, int dim, int n_tiles, int W, cudaStream_t st) {
    if (n_tiles <= 0) return cudaSuccess;
    if (dim == 2) {
        if (a.g.FR <= 4) return launch_adj_pair_t<T, 2, 4>(a, n_tiles, W, st);
        if (a.g.FR <= 6) return launch_adj_pair_t<T, 2, 6>(a, n_tiles, W, st);
        return launch_adj_pair_t<T, 2, 8>(a, n_tiles, W, st);
    }
    if (a.g.FR <= 6) return launch_adj_pair_t<T, 3, 6>(a, n_tiles, W, st);
    return launch_adj_pair_t<T, 3, 8>(a, n_tiles, W, st);
}

// offsets and centres from the accumulated offset adjoints: an obstacle
// translated by delta has offsets d_m + c_m . delta, so dL/ddelta = C^T dL/dd
template <typename T>
__global__ void k_adj_finish(const double *gd, const T *obs_C, const int *obs_nf, int M_tot, int FO, int dim,
                             T *grad_d, T *grad_ctr) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M_tot) return;
    const int nf = obs_nf[j];
    double ctr[3] = {0.0, 0.0, 0.0};
    for (int m = 0; m < FO; ++m) {
        const double v = m < nf ? gd[(long long)j * FO + m] : 0.0;
        if (grad_d) grad_d[(long long)j * FO + m] = T(v);
        for (int i = 0; i < dim && m < nf; ++i) ctr[i] += double(obs_C[((long long)j * FO + m) * dim + i]) * v;
    }
    if (grad_ctr)
        for (int i = 0; i < dim; ++i) grad_ctr[(long long)j * dim + i] = T(ctr[i]);
}

template <typename T>
cudaError_t launch_adj_finish(const double *gd, const T *obs_C, const int *obs_nf, int M_tot, int FO, int dim,
                              T *grad_d, T *grad_ctr, cudaStream_t st) {
    if (M_tot <= 0) return cudaSuccess;
    k_adj_finish<T><<<(M_tot + 127) / 128, 128, 0, st>>>(gd, obs_C, obs_nf, M_tot, FO, dim, grad_d, grad_ctr);
    return cudaGetLastError();
}

template cudaError_t launch_adj_seed<float>(const AdjTrajArgs<float> &, int, cudaStream_t);
template cudaError_t launch_adj_seed<double>(const AdjTrajArgs<double> &, int, cudaStream_t);
template cudaError_t launch_adj_traj<float>(const AdjTrajArgs<float> &, int, cudaStream_t);
template cudaError_t launch_adj_traj<double>(const AdjTrajArgs<double> &, int, cudaStream_t);
template cudaError_t launch_adj_pair<float>(const AdjPairArgs<float> &, int, int, int, cudaStream_t);
template cudaError_t launch_adj_pair<double>(const AdjPairArgs<double> &, int, int, int, cudaStream_t);
template cudaError_t launch_adj_alpha<float>(const AdjAlphaArgs<float> &, int, int, int, const int *, const float *,
                                             long long, int, int, float *, const PoseArgs<float> &, int, cudaStream_t);
template cudaError_t launch_adj_alpha<double>(const AdjAlphaArgs<double> &, int, int, int, const int *, const double *,
                                              long long, int, int, double *, const PoseArgs<double> &, int,
                                              cudaStream_t);
template cudaError_t launch_adj_finish<float>(const double *, const float *, const int *, int, int, int, float *, float *,
                                              cudaStream_t);
template cudaError_t launch_adj_finish<double>(const double *, const double *, const int *, int, int, int, double *,
                                               double *, cudaStream_t);

}  // namespace oca
