// Pair kernels: part poses, scale-LP collision detection and the fused
// per-pair ADMM kernel (dual update, pair QP, dual residual, Gauss-Newton
// statistics).
//
// Work decomposition ("obstacle sweep"): a CTA owns one tile = 32
// consecutive (part, t) lanes of one scenario and W warps; warp w processes
// obstacles j = w, w+W, ...  All lanes of a warp therefore work on the same
// obstacle at the same time (its halfspaces are a broadcast load and its
// face count is warp-uniform), pair arrays are read coalesced (pair index =
// j*Q + q), and the per-(part, t) sums that the trajectory step needs are
// accumulated in registers and reduced across the W warps in shared memory.
#include <cfloat>

#include "oca_common.cuh"
#include "oca_kernels.h"
#include "oca_models.cuh"
#include "oca_solvers.cuh"

namespace oca {

// ============================================================================
// poses (rho, R) of every (scenario, part, t = 1..N), Sec. IV-A
// ============================================================================
template <typename T, int KIND>
__global__ void k_pose(PoseArgs<T> a) {
    constexpr int D = MDims<KIND>::D, NS = MDims<KIND>::NS;
    const int s = blockIdx.y;
    const ScenMeta sm = a.meta[s];
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= sm.NP * sm.N) return;
    if (a.scen_status && a.scen_status[s] != kActive) return;
    const int part = q / sm.N, t = q % sm.N + 1;
    const int gp = sm.part0 + part;
    T st[NS], off[D], rho[D], R[D * D];
#pragma unroll
    for (int i = 0; i < NS; ++i) st[i] = a.states[(long long)(sm.state0 + t) * NS + i];
#pragma unroll
    for (int i = 0; i < D; ++i) off[i] = a.g.part_off[gp * D + i];
    part_pose<T, KIND>(a.model, a.g.part_link[gp], off, st, rho, R, nullptr, nullptr, nullptr);
    const int col = sm.qbeg + q;
#pragma unroll
    for (int i = 0; i < D; ++i) a.pose[(long long)i * a.Qtot + col] = rho[i];
#pragma unroll
    for (int i = 0; i < D * D; ++i) a.pose[(long long)(D + i) * a.Qtot + col] = R[i];
}

// ============================================================================
// Fused pair kernel.
//   MODE 0 (step 1 alone): y_out = QP(pose, zeta, xi, y_in); v, obj, status.
//   MODE 1 (ADMM iteration j, Gauss-Seidel):
//     head (j >= 1): zeta += T(s^j, y^j), xi += R(s^j, y^j)      [step 3 of j-1]
//                    partial r_pri += T^2 + |R|^2
//     qp   (j < max_iter): y^{j+1} = QP(s^j, zeta^j, xi^j; y^j) [step 1 of j]
//                    partial r_dual += |dlambda|^2 + |dmu|^2
//                    Gauss-Newton statistics of r = [T + zeta; R + xi] at
//                    fixed y^{j+1}: W += w w^T, Wc += c w, E += w e^T with
//                    w = C^T mu, c = 1 + d^T mu + gamma + zeta, e = A^T lambda + xi
//     y buffers alternate by the parity of j (y_in = buf[j%2], y_out = buf[(j+1)%2]).
// ============================================================================
#ifndef OCA_PAIR_MIN_BLOCKS
#define OCA_PAIR_MIN_BLOCKS 1
#endif
// Launch bound of the pair kernel: 512 threads (16 warps) at most per CTA
// for the FP32 2-D kernel, whose state fits 128 registers per thread without
// spilling (16 resident warps per SM); 384 for the FP64 2-D kernel (about 165
// registers); the 3-D kernel (4 x 4 Newton systems, up to 8 robot faces)
// needs about 245 and is bounded at 256 threads.
#ifndef OCA_PAIR_MAX_THREADS_2D
#define OCA_PAIR_MAX_THREADS_2D 512
#endif
#ifndef OCA_PAIR_MAX_THREADS_2D_F64
#define OCA_PAIR_MAX_THREADS_2D_F64 384
#endif
#ifndef OCA_PAIR_MAX_THREADS_3D
#define OCA_PAIR_MAX_THREADS_3D 256
#endif
template <typename T, int D>
struct PairBound {
    static constexpr int threads =
        D == 3 ? OCA_PAIR_MAX_THREADS_3D : (sizeof(T) == 4 ? OCA_PAIR_MAX_THREADS_2D : OCA_PAIR_MAX_THREADS_2D_F64);
};
template <typename T, int D, int MODE, int SOLVER, int NR>
__global__ void __launch_bounds__(PairBound<T, D>::threads, OCA_PAIR_MIN_BLOCKS) k_pair(PairArgs<T> a) {
    constexpr int V = D + 1, SM = D + 2, NSTAT = StatDims<D>::NSTAT, NW = StatDims<D>::NW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Tile tile = a.tiles[blockIdx.x];
    const ScenMeta sm = a.meta[tile.scen];
    int j_it = 0;
    bool head = false, do_qp = true;
    const T *y_in = a.y_in;
    T *y_out = a.y_out;
    if (MODE == 1) {
        if (a.scen_status[tile.scen] != kActive) return;
        j_it = *a.iter;
        if (j_it > a.max_iter) return;
        head = j_it >= 1;
        do_qp = j_it < a.max_iter;
        if (j_it & 1) {
            y_in = a.y_out;
            y_out = const_cast<T *>(a.y_in);
        }
    }
    const int lane = threadIdx.x, warp = threadIdx.y, W = blockDim.y;
    const int BT = 32 * W, tid = warp * 32 + lane;
    const int Q = sm.NP * sm.N;
    // a tail tile of at most 16 columns runs as 2W half-warps over the same
    // columns: half hh of warp w sweeps obstacles 2w + hh, 2w + hh + 2W, ...
    // (the face loops then cost the larger of two face counts, not their sum)
    const bool split = tile.split != 0;
    const int hh = split ? lane >> 4 : 0;
    const int q = tile.q0 + (split ? (lane & 15) : lane);
    const bool valid = q < Q;
    const int j0 = split ? 2 * warp + hh : warp, JS = split ? 2 * W : W;
    const long long P = a.P;
    const int FR = a.g.FR, FO = a.g.FO;
    // shared memory: [staged face records, BT lanes x LS] [next obstacle's pair data
    // W x NPF x 32] [halfspaces of the current and the next obstacle W x 2 x 2 x NOB]
    // [statistics W x NSTAT x 32] [residuals W x 2 (double)]; the first three with
    // SOLVER 1 only
    constexpr int NC = NrmStride<D>::N;
    const int NY = FR + FO + 1, NPF = NY + 1 + D;  // y components, zeta, xi
    const int NOB = obs_buf_elems<D>(FO);          // one obstacle's normals [FO][NC] and offsets [FO]
    T *stg = reinterpret_cast<T *>(smem_raw);
    // per-lane staged face records [d', iD, s, ybar], lane stride LS
    const int LS = face_lane_stride<T>(FO);
    T *pfb = stg + (SOLVER == 1 ? LS * BT : 0);
    T *lrec = stg + tid * LS;
    T *obb = pfb + (SOLVER == 1 ? W * NPF * 32 : 0);
    T *red = obb + (SOLVER == 1 ? W * 4 * NOB : 0);
    // this lane's column of its warp's prefetch buffer: component c at pw[c * 32]
    // (lambda_k at k, mu_m at FR + m, gamma at FR + FO, zeta at NY, xi_i at NY + 1 + i)
    T *pw = pfb + warp * NPF * 32 + lane;
    // the two halfspace buffers of this lane's (half-)warp: obstacle number c of
    // its sweep (c = 0, 1, ...) uses buffer c & 1
    T *ob2 = obb + (warp * 2 + hh) * 2 * NOB;
    // the lanes sharing that buffer: the valid lanes of this warp (or half-warp);
    // they copy it together and meet at __syncwarp(gmask) around each use
    const unsigned vmask = __ballot_sync(0xffffffffu, valid);
    const unsigned gmask = split ? (vmask & (hh ? 0xffff0000u : 0x0000ffffu)) : vmask;
    const int g_n = __popc(gmask), g_r = __popc(gmask & ((1u << lane) - 1u));

    Lane<T, D> L;
    SsnLane<T, D, NR> SL;
    // this lane's Gauss-Newton statistics, accumulated in its own slots of the
    // reduction buffer (W [NW], Wc [D], E [D*D] at rsl[k * 32])
    T *rsl = red + warp * NSTAT * 32 + lane;
    if (MODE == 1) {
#pragma unroll
        for (int k = 0; k < NSTAT; ++k) rsl[k * 32] = T(0);
    }
    double rp = 0.0, rd = 0.0;

    if (valid) {
        const int col = sm.qbeg + q;
#pragma unroll
        for (int i = 0; i < D; ++i) L.rho[i] = a.pose[(long long)i * a.Qtot + col];
#pragma unroll
        for (int i = 0; i < D * D; ++i) L.R[i] = a.pose[(long long)(D + i) * a.Qtot + col];
        const int gp = sm.part0 + q / sm.N;
        L.A = a.g.part_A + (long long)gp * FR * D;
        L.b = a.g.part_b + (long long)gp * FR;
        L.nr = a.g.part_nf[gp];
        const T rho_p = a.prox;
        const T irho = T(1) / rho_p;
        if constexpr (SOLVER == 1) {
            // robot-part constants of the lambda subproblem in its breakpoint
            // form (registers): ta_k = R a_k / (prox b_k), w_k = b_k^2 / n_k,
            // bD_k = b_k / n_k with n_k = |a_k|^2
            SL.nr = L.nr;
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                T a2 = T(0), ak[D];
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    ak[i] = k < L.nr ? ldg(L.A + k * D + i) : T(0);
                    a2 += ak[i] * ak[i];
                }
                const T bk = k < L.nr ? ldg(L.b + k) : T(1);
                if (!(a2 > T(0))) a2 = T(1);
                const T s = T(1) / (rho_p * bk);
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    T acc = T(0);
#pragma unroll
                    for (int l = 0; l < D; ++l) acc += L.R[i * D + l] * ak[l];
                    SL.ta[k][i] = acc * s;
                }
                // padding faces (k >= nr): never active, no contribution
                SL.bD[k] = k < L.nr ? bk / a2 : T(0);
                SL.w[k] = bk * SL.bD[k];
                SL.ty[k] = k < L.nr ? T(0) : T(-3.0e38);
            }
            SL.rec = lrec;
        }
        // SOLVER 1: the pair data and halfspaces of this warp's next obstacle
        // are copied to shared memory asynchronously while the current
        // obstacle is solved (halfspaces into the other of the two buffers)
        auto prefetch = [&](int jn, int buf) {
            if constexpr (SOLVER == 1) {
                if (jn >= sm.M) return;
                const int gmn = sm.obs0 + jn;
                if (a.obs_mask && !a.obs_mask[gmn]) return;
                const long long pn = sm.pair0 + (long long)jn * Q + q;
                const int non = a.g.obs_nf[gmn];
                for (int k = 0; k < L.nr; ++k) cp_async_elem(pw + k * 32, y_in + (long long)k * P + pn);
                for (int m = 0; m < non; ++m) cp_async_elem(pw + (FR + m) * 32, y_in + (long long)(FR + m) * P + pn);
                cp_async_elem(pw + (FR + FO) * 32, y_in + (long long)(FR + FO) * P + pn);
                cp_async_elem(pw + NY * 32, a.zeta + pn);
#pragma unroll
                for (int i = 0; i < D; ++i) cp_async_elem(pw + (NY + 1 + i) * 32, a.xi + (long long)i * P + pn);
                // the obstacle's halfspaces, split over the lanes sharing them:
                // normal m at [m * NC], offset m at [FO * NC + m]
                T *obn = ob2 + buf * NOB;
                const T *Cn = a.g.obs_C + (long long)gmn * FO * D;
                const T *dn = a.g.obs_d + (long long)gmn * FO;
                for (int e = g_r; e < non * (D + 1); e += g_n) {
                    if (e < non * D) cp_async_elem(obn + (e / D) * NC + e % D, Cn + e);
                    else cp_async_elem(obn + FO * NC + (e - non * D), dn + (e - non * D));
                }
                cp_async_commit();
            }
        };
        prefetch(j0, 0);

        int cnt = 0;  // obstacles of this sweep so far
        for (int j = j0; j < sm.M; j += JS, ++cnt) {
            const int gm = sm.obs0 + j;
            L.C = a.g.obs_C + (long long)gm * FO * D;
            L.d = a.g.obs_d + (long long)gm * FO;
            L.no = a.g.obs_nf[gm];
            const long long p = sm.pair0 + (long long)j * Q + q;
            const int ng = L.nr + L.no + 1;
            if (a.obs_mask && !a.obs_mask[gm]) {
                // an obstacle outside the sensing window: its pairs take no
                // part in this solve and keep their y in both buffers
                if (y_out != y_in) {
                    for (int k = 0; k < L.nr; ++k) y_out[(long long)k * P + p] = y_in[(long long)k * P + p];
                    for (int m = 0; m < L.no; ++m) y_out[(long long)(FR + m) * P + p] = y_in[(long long)(FR + m) * P + p];
                    y_out[(long long)(FR + FO) * P + p] = y_in[(long long)(FR + FO) * P + p];
                }
                // nothing was copied for this obstacle; the buffer the next copy
                // fills was read by the previous obstacle's solve, which every
                // sharing lane has finished once they meet here
                if constexpr (SOLVER == 1) __syncwarp(gmask);
                prefetch(j + JS, (cnt + 1) & 1);
                continue;
            }
            T zeta, xi[D];
            if constexpr (SOLVER == 1) {
                cp_async_wait_all();  // this obstacle's copies issued by this lane
                __syncwarp(gmask);    // ... and by the other lanes sharing its halfspaces
                zeta = pw[NY * 32];
#pragma unroll
                for (int i = 0; i < D; ++i) xi[i] = pw[(NY + 1 + i) * 32];
            } else {
                zeta = a.zeta[p];
#pragma unroll
                for (int i = 0; i < D; ++i) xi[i] = a.xi[(long long)i * P + p];
            }
            const T *yb = y_in + p;
            T *yo = y_out + p;
            // ---- one pass over y^j: compressed certificate (A^T lambda, C^T mu,
            // d^T mu + gamma), warm-start support or staged face data
            T a0[D], w0[D], del0 = T(0);
#pragma unroll
            for (int i = 0; i < D; ++i) {
                a0[i] = T(0);
                w0[i] = T(0);
            }
            Support<T, D> S;
            S.n = 0;
#pragma unroll
            for (int k = 0; k < SM; ++k) {
                S.id[k] = 0;
                S.w[k] = T(0);
            }
            bool overflow = false;
            T lam_sum = T(0);
            if constexpr (SOLVER == 1) {
                // a0 = sum lambda R a_k (world frame here); face records [d', iD, s, ybar]
                const T *obc = ob2 + (cnt & 1) * NOB;
                SL.nrm = obc;
                // (lambda_k R a_k = prox w_k (lambda_k / bD_k) ta_k; ty_k = lambda_k / bD_k)
#pragma unroll
                for (int k = 0; k < NR; ++k) {
                    if (k < L.nr) {
                        const T tv = pw[k * 32] * m_rcp(SL.bD[k]);
                        SL.ty[k] = tv;
#pragma unroll
                        for (int i = 0; i < D; ++i) a0[i] += (rho_p * SL.w[k] * tv) * SL.ta[k][i];
                    }
                }
                for (int m = 0; m < L.no; ++m) {
                    const T yv = pw[(FR + m) * 32];
                    T c[D], cr = T(0), c2 = T(0);
                    nrm_load<T, D>(obc + m * NC, c);
#pragma unroll
                    for (int i = 0; i < D; ++i) {
                        w0[i] += yv * c[i];
                        cr += c[i] * L.rho[i];
                        c2 += c[i] * c[i];
                    }
                    const T dm = obc[FO * NC + m];
                    del0 += yv * dm;
                    const T dp = dm - cr;
                    const T pD = rho_p * (dp * dp + c2);  // prox |K_m|^2
                    rec_store<T>(lrec + 4 * m, dp, m_rcp(pD), yv * pD, yv);
                }
                SL.ybg = pw[(FR + FO) * 32];
                del0 += SL.ybg;
                __syncwarp(gmask);                 // every sharing lane has read the pair data
                prefetch(j + JS, (cnt + 1) & 1);  // into the free buffers
            } else {
                for (int g = 0; g < ng; ++g) {
                    const int c = g < L.nr ? g : (g < L.nr + L.no ? FR + g - L.nr : FR + FO);
                    const T yv = yb[(long long)c * P];
                    if (g < L.nr) {
#pragma unroll
                        for (int i = 0; i < D; ++i) a0[i] += yv * ldg(L.A + g * D + i);
                    } else if (g < L.nr + L.no) {
                        const int m = g - L.nr;
#pragma unroll
                        for (int i = 0; i < D; ++i) w0[i] += yv * ldg(L.C + m * D + i);
                        del0 += yv * ldg(L.d + m);
                    } else {
                        del0 += yv;
                    }
                    if (yv > T(0)) {
                        const T wv = g < L.nr ? yv * ldg(L.b + g) : yv;
                        if (g < L.nr) lam_sum += wv;
                        if (S.n < SM) {
#pragma unroll
                            for (int k = 0; k < SM; ++k)
                                if (k == S.n) {
                                    S.id[k] = g;
                                    S.w[k] = wv;
                                }
                            S.n += 1;
                        } else {
                            overflow = true;
                        }
                    }
                }
            }
            if (head) {
                // step 3 of iteration j-1 at s^j: T = 1 + d'^T mu + gamma, R = A^T lambda + (C R)^T mu
                T wr = T(0);
#pragma unroll
                for (int i = 0; i < D; ++i) wr += w0[i] * L.rho[i];
                const T Tr = T(1) + del0 - wr;
                zeta += Tr;
                rp += double(Tr) * double(Tr);
                // (SOLVER 1 holds A^T lambda rotated to the world frame: R^T (a0 + w0))
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    T acc = SOLVER == 1 ? T(0) : a0[i];
#pragma unroll
                    for (int k = 0; k < D; ++k) acc += L.R[k * D + i] * (SOLVER == 1 ? a0[k] + w0[k] : w0[k]);
                    xi[i] += acc;
                    rp += double(acc) * double(acc);
                }
                a.zeta[p] = zeta;
#pragma unroll
                for (int i = 0; i < D; ++i) a.xi[(long long)i * P + p] = xi[i];
            }
            if (!do_qp) continue;
            T bq[V];
            bq[0] = T(1) + zeta;
#pragma unroll
            for (int i = 0; i < D; ++i) bq[1 + i] = xi[i];
            T v[V];
            int status;
            T a1[D], w1[D], del1 = T(0), dy2 = T(0);
#pragma unroll
            for (int i = 0; i < D; ++i) {
                a1[i] = T(0);
                w1[i] = T(0);
            }
            if constexpr (SOLVER == 0) {
                // ---- step 1 by the active-set method, warm-started from y^j's support
                if (overflow || S.n == 0 || !(lam_sum > T(0))) {
                    sup_cold<T, D>(L, bq, S);
                } else {
                    const T il = T(1) / lam_sum;  // renormalise the lambda weights
#pragma unroll
                    for (int k = 0; k < SM; ++k)
                        if (k < S.n && S.id[k] < L.nr) S.w[k] *= il;
                }
                status = mnp_solve<T, D>(L, S, bq, v);
                for (int g = 0; g < ng; ++g) {
                    const int c = g < L.nr ? g : (g < L.nr + L.no ? FR + g - L.nr : FR + FO);
                    T yv = T(0);
#pragma unroll
                    for (int k = 0; k < SM; ++k)
                        if (k < S.n && S.id[k] == g) yv = S.w[k];
                    if (g < L.nr) yv /= ldg(L.b + g);
                    if (g < ng - 1) {
                        const T dlt = yv - yb[(long long)c * P];
                        dy2 += dlt * dlt;
                    }
                    yo[(long long)c * P] = yv;
                    if (g < L.nr) {
#pragma unroll
                        for (int i = 0; i < D; ++i) a1[i] += yv * ldg(L.A + g * D + i);
                    } else if (g < L.nr + L.no) {
                        const int m = g - L.nr;
#pragma unroll
                        for (int i = 0; i < D; ++i) w1[i] += yv * ldg(L.C + m * D + i);
                        del1 += yv * ldg(L.d + m);
                    } else {
                        del1 += yv;
                    }
                }
            } else {
                // ---- step 1 by semismooth Newton in world coordinates (bqw = [bq0; R bq1]),
                // warm-started at K^T y^j + bqw = [bq0 + del0 - rho.w0; R bq1 + a0 + w0]
                T bqw[V], ws[V];
                bqw[0] = bq[0];
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    T acc = T(0);
#pragma unroll
                    for (int k = 0; k < D; ++k) acc += L.R[i * D + k] * bq[1 + k];
                    bqw[1 + i] = acc;
                }
                T wr = T(0);
#pragma unroll
                for (int i = 0; i < D; ++i) wr += w0[i] * L.rho[i];
                ws[0] = bqw[0] + del0 - wr;
#pragma unroll
                for (int i = 0; i < D; ++i) ws[1 + i] = bqw[1 + i] + a0[i] + w0[i];
                SL.no = L.no;
                SsnKeep<T, NR> est;
                status = ssn_solve_staged<T, D, NR>(SL, rho_p, irho, bqw, ws, est);
                T a1w[D];
#pragma unroll
                for (int i = 0; i < D; ++i) a1w[i] = T(0);
#pragma unroll
                for (int k = 0; k < NR; ++k) {
                    if (k < L.nr) {
                        const T yv = SL.bD[k] * est.x[k];
                        const T dlt = yv - SL.bD[k] * SL.ty[k];
                        dy2 += dlt * dlt;
                        yo[(long long)k * P] = yv;
#pragma unroll
                        for (int i = 0; i < D; ++i) a1w[i] += (rho_p * SL.w[k] * est.x[k]) * SL.ta[k][i];
                    }
                }
                // mu at the solution from the staged records; the sums sd = sum mu d'
                // and w1 = sum mu c (world frame) give K^T y and the statistics
                T sd = T(0);
                for (int m = 0; m < L.no; ++m) {
                    T dp, iDm, s, ybm, c[D];
                    rec_load<T>(lrec + 4 * m, dp, iDm, s, ybm);
                    nrm_load<T, D>(SL.nrm + m * NC, c);
                    T cw = T(0);
#pragma unroll
                    for (int i = 0; i < D; ++i) cw += c[i] * ws[1 + i];
                    const T yv = fmax(T(0), (s - (ws[0] * dp + cw)) * iDm);
                    const T dlt = yv - ybm;
                    dy2 += dlt * dlt;
                    yo[(long long)(FR + m) * P] = yv;
                    sd += yv * dp;
#pragma unroll
                    for (int i = 0; i < D; ++i) w1[i] += yv * c[i];
                }
                const T gv = fmax(T(0), SL.ybg - ws[0] * irho);
                yo[(long long)(FR + FO) * P] = gv;
                // v = K^T y + bq from the written y (body frame: R^T of the world sum)
                // and A^T lambda in the body frame
                v[0] = bq[0] + sd + gv;
                T wr1 = T(0);
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    T acc = T(0), acc2 = T(0);
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        acc += L.R[k * D + i] * (a1w[k] + w1[k]);
                        acc2 += L.R[k * D + i] * a1w[k];
                    }
                    v[1 + i] = bq[1 + i] + acc;
                    a1[i] = acc2;
                    wr1 += w1[i] * L.rho[i];
                }
                del1 = sd + wr1 + gv;
            }
            if (MODE == 0) {
                if (a.v_out) {
#pragma unroll
                    for (int i = 0; i < V; ++i) a.v_out[(long long)i * P + p] = v[i];
                }
                if (a.obj_out) a.obj_out[p] = T(0.5) * dotv<T, V>(v, v);
                if (a.status_out) a.status_out[p] = status;
            } else {
                rd += double(dy2);
                const T cc = T(1) + del1 + zeta;
                T e[D];
#pragma unroll
                for (int i = 0; i < D; ++i) e[i] = a1[i] + xi[i];
                int k = 0;
#pragma unroll
                for (int i = 0; i < D; ++i)
#pragma unroll
                    for (int jj = 0; jj <= i; ++jj, ++k) rsl[k * 32] += w1[i] * w1[jj];
#pragma unroll
                for (int i = 0; i < D; ++i) rsl[(NW + i) * 32] += cc * w1[i];
#pragma unroll
                for (int i = 0; i < D; ++i)
#pragma unroll
                    for (int jj = 0; jj < D; ++jj) rsl[(NW + D + i * D + jj) * 32] += w1[i] * e[jj];
            }
        }
    }
    if (MODE == 1) {
        // ---- reduce statistics and residual partials across the W warps
        // (and, in a split tile, across the two half-warps of the same columns)
        T *rs = red;  // [W][NSTAT][32]
        double *rr = reinterpret_cast<double *>(red + (size_t)W * NSTAT * 32);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            rp += __shfl_xor_sync(0xffffffffu, rp, o);
            rd += __shfl_xor_sync(0xffffffffu, rd, o);
        }
        if (lane == 0) {
            rr[2 * warp] = rp;
            rr[2 * warp + 1] = rd;
        }
        __syncthreads();
        if (do_qp && valid && hh == 0) {
            for (int k = warp; k < NSTAT; k += W) {
                T acc = T(0);
                for (int w2 = 0; w2 < W; ++w2) {
                    acc += rs[(w2 * NSTAT + k) * 32 + lane];
                    if (split) acc += rs[(w2 * NSTAT + k) * 32 + lane + 16];
                }
                a.stats[(long long)k * a.Qtot + sm.qbeg + q] = acc;
            }
        }
        if (warp == 0 && lane == 0) {
            double s1 = 0.0, s2 = 0.0;
            for (int w2 = 0; w2 < W; ++w2) {
                s1 += rr[2 * w2];
                s2 += rr[2 * w2 + 1];
            }
            const int tn = sm.tile0 + tile.q0 / 32;
            double *dst = a.res + (size_t)(j_it & 1) * a.n_tiles * 2 + (size_t)tn * 2;
            dst[0] = s1;
            dst[1] = s2;
        }
    }
}

template <typename T, int D>
__global__ void __launch_bounds__(512) k_scale(ScaleArgs<T> a) {
    constexpr int V = D + 1;
    const Tile tile = a.tiles[blockIdx.x];
    const ScenMeta sm = a.meta[tile.scen];
    const int lane = threadIdx.x, warp = threadIdx.y, W = blockDim.y;
    const int Q = sm.NP * sm.N;
    const int q = tile.q0 + lane;
    if (q >= Q) return;
    const long long P = a.P;
    const int FR = a.g.FR, FO = a.g.FO;
    Lane<T, D> L;
    const int col = sm.qbeg + q;
#pragma unroll
    for (int i = 0; i < D; ++i) L.rho[i] = a.pose[(long long)i * a.Qtot + col];
#pragma unroll
    for (int i = 0; i < D * D; ++i) L.R[i] = a.pose[(long long)(D + i) * a.Qtot + col];
    const int gp = sm.part0 + q / sm.N;
    L.A = a.g.part_A + (long long)gp * FR * D;
    L.b = a.g.part_b + (long long)gp * FR;
    L.nr = a.g.part_nf[gp];
    for (int j = warp; j < sm.M; j += W) {
        const int gm = sm.obs0 + j;
        L.C = a.g.obs_C + (long long)gm * FO * D;
        L.d = a.g.obs_d + (long long)gm * FO;
        L.no = a.g.obs_nf[gm];
        const long long p = sm.pair0 + (long long)j * Q + q;
        int bas[V];
        T xB[V], alpha;
        int st = lp_solve<T, D>(L, bas, xB, alpha);
        if (!(alpha == alpha)) st = OCA_PAIR_NONFINITE;
        a.alpha[p] = alpha;
        if (a.verdict) a.verdict[p] = alpha >= T(1) ? 1 : 0;
        if (a.status) a.status[p] = st;
        const int ART = L.nr + L.no;
        if (a.lambda) {
            for (int k = 0; k < L.nr; ++k) {
                T v = T(0);
#pragma unroll
                for (int i = 0; i < V; ++i)
                    if (bas[i] == k) v = xB[i];
                a.lambda[(long long)k * P + p] = v;
            }
        }
        if (a.mu) {
            for (int m = 0; m < L.no; ++m) {
                T v = T(0);
#pragma unroll
                for (int i = 0; i < V; ++i)
                    if (bas[i] == L.nr + m) v = xB[i];
                a.mu[(long long)m * P + p] = v;
            }
        }
        if (a.margin) {
            // FP64 weak-duality bound on alpha* from the certificate (lambda, mu)
            double rho[D], R[D * D];
#pragma unroll
            for (int i = 0; i < D; ++i) rho[i] = double(L.rho[i]);
#pragma unroll
            for (int i = 0; i < D * D; ++i) R[i] = double(L.R[i]);
            double bl = 0.0, dm = 0.0, r[D];
#pragma unroll
            for (int i = 0; i < D; ++i) r[i] = 0.0;
#pragma unroll
            for (int i = 0; i < V; ++i) {
                const int id = bas[i];
                const double x = double(xB[i]);
                if (id < L.nr) {
                    bl += double(ldg(L.b + id)) * x;
#pragma unroll
                    for (int k = 0; k < D; ++k) r[k] += double(ldg(L.A + id * D + k)) * x;
                } else if (id < ART) {
                    const int m = id - L.nr;
                    double c[D], cr = 0.0;
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        c[k] = double(ldg(L.C + m * D + k));
                        cr += c[k] * rho[k];
                    }
                    dm += (double(ldg(L.d + m)) - cr) * x;
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        double cb = 0.0;
#pragma unroll
                        for (int l = 0; l < D; ++l) cb += R[l * D + k] * c[l];
                        r[k] += cb * x;
                    }
                }
            }
            double rn = 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) rn += r[k] * r[k];
            const double den = bl + sqrt(rn) * a.part_radius[gp];
            a.margin[p] = den > 0.0 ? -dm / den : -DBL_MAX;
        }
    }
}

// ============================================================================
// FP64 weak-duality margin of given dual variables (Sec. III-B): for any
// lambda, mu >= 0 and any (alpha, x) feasible for eqn:scale_opt,
//   alpha b^T lambda >= r^T x - d'^T mu  with  r = A^T lambda + C'^T mu,
// and |x| <= alpha D (x lies in alpha P, D = the part's largest vertex norm),
// so alpha* >= -d'^T mu / (b^T lambda + |r| D).  The pose is formed in FP64
// from the stored state, so the bound holds for the geometry as stored.
// Same tile shape as k_scale: lanes over (part, t), warps over obstacles.
// ============================================================================
template <typename T, int KIND>
__global__ void __launch_bounds__(512) k_cert(CertArgs<T> a) {
    constexpr int D = MDims<KIND>::D, NS = MDims<KIND>::NS;
    const Tile tile = a.tiles[blockIdx.x];
    const ScenMeta sm = a.meta[tile.scen];
    const int lane = threadIdx.x, warp = threadIdx.y, W = blockDim.y;
    const int Q = sm.NP * sm.N;
    const int q = tile.q0 + lane;
    if (q >= Q) return;
    const long long P = a.P;
    const int FR = a.g.FR, FO = a.g.FO;
    const int part = q / sm.N, t = q % sm.N + 1;
    const int gp = sm.part0 + part;
    double st[NS], off[D], rho[D], R[D * D];
#pragma unroll
    for (int i = 0; i < NS; ++i) st[i] = double(a.states[(long long)(sm.state0 + t) * NS + i]);
#pragma unroll
    for (int i = 0; i < D; ++i) off[i] = double(a.g.part_off[gp * D + i]);
    part_pose<double, KIND>(a.model, a.g.part_link[gp], off, st, rho, R, nullptr, nullptr, nullptr);
    const T *A = a.g.part_A + (long long)gp * FR * D;
    const T *b = a.g.part_b + (long long)gp * FR;
    const int nr = a.g.part_nf[gp];
    const double Dr = a.part_radius[gp];
    for (int j = warp; j < sm.M; j += W) {
        const int gm = sm.obs0 + j;
        const T *Cw = a.g.obs_C + (long long)gm * FO * D;
        const T *dw = a.g.obs_d + (long long)gm * FO;
        const int no = a.g.obs_nf[gm];
        const long long p = sm.pair0 + (long long)j * Q + q;
        bool ok = true;
        double bl = 0.0, dm = 0.0, r[D];
#pragma unroll
        for (int i = 0; i < D; ++i) r[i] = 0.0;
        for (int k = 0; k < nr; ++k) {
            const double l = double(a.lambda[(long long)k * P + p]);
            ok = ok && l >= 0.0 && isfinite(l);
            bl += double(ldg(b + k)) * l;
#pragma unroll
            for (int i = 0; i < D; ++i) r[i] += double(ldg(A + k * D + i)) * l;
        }
        for (int m = 0; m < no; ++m) {
            const double u = double(a.mu[(long long)m * P + p]);
            ok = ok && u >= 0.0 && isfinite(u);
            double c[D], cr = 0.0;
#pragma unroll
            for (int i = 0; i < D; ++i) {
                c[i] = double(ldg(Cw + m * D + i));
                cr += c[i] * rho[i];
            }
            dm += (double(ldg(dw + m)) - cr) * u;
            // body-frame normal C'_m = c_m^T R
#pragma unroll
            for (int i = 0; i < D; ++i) {
                double cb = 0.0;
#pragma unroll
                for (int l = 0; l < D; ++l) cb += c[l] * R[l * D + i];
                r[i] += cb * u;
            }
        }
        double rn = 0.0;
#pragma unroll
        for (int i = 0; i < D; ++i) rn += r[i] * r[i];
        const double den = bl + sqrt(rn) * Dr;
        a.margin[p] = (ok && den > 0.0) ? -dm / den : -DBL_MAX;
    }
}

// ============================================================================
// launchers
// ============================================================================
template <typename T, int KIND>
cudaError_t launch_pose_t(const PoseArgs<T> &a, int maxQ, cudaStream_t st) {
    if (maxQ <= 0 || a.n_scen <= 0) return cudaSuccess;
    dim3 grid((maxQ + 127) / 128, a.n_scen);
    k_pose<T, KIND><<<grid, 128, 0, st>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pose(const PoseArgs<T> &a, int maxQ, cudaStream_t st) {
    switch (a.model.kind) {
        case 0: return launch_pose_t<T, 0>(a, maxQ, st);
        case 1: return launch_pose_t<T, 1>(a, maxQ, st);
        case 2: return launch_pose_t<T, 2>(a, maxQ, st);
    }
    return cudaErrorInvalidValue;
}

int pair_max_warps(int dim, size_t es) {
    const int t = dim == 3 ? (es == 4 ? PairBound<float, 3>::threads : PairBound<double, 3>::threads)
                           : (es == 4 ? PairBound<float, 2>::threads : PairBound<double, 2>::threads);
    return t / 32;
}

size_t pair_smem_bytes(int dim, size_t es, int W, int mode, int solver, int FR, int FO) {
    const int nstat = dim * (dim + 1) / 2 + dim + dim * dim;
    size_t b = 0;
    if (solver == 1) {
        const size_t ls = es == 4 ? face_lane_stride<float>(FO) : face_lane_stride<double>(FO);
        const size_t nob = dim == 2 ? obs_buf_elems<2>(FO) : obs_buf_elems<3>(FO);
        b += ls * 32 * W * es + (size_t)W * (FR + FO + 2 + dim) * 32 * es + (size_t)W * 4 * nob * es;
    }
    if (mode == 1) b += (size_t)W * nstat * 32 * es + (size_t)W * 2 * sizeof(double);
    return b;
}

template <typename T, int D>
size_t pair_smem(int W, int mode, int solver, int FR, int FO) {
    return pair_smem_bytes(D, sizeof(T), W, mode, solver, FR, FO);
}

template <typename T, int D, int MODE, int SOLVER, int NR>
cudaError_t launch_pair_t(const PairArgs<T> &a, int n_tiles, int W, cudaStream_t st) {
    if (n_tiles <= 0) return cudaSuccess;
    const size_t sm = pair_smem<T, D>(W, MODE, SOLVER, a.g.FR, a.g.FO);
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_pair<T, D, MODE, SOLVER, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    k_pair<T, D, MODE, SOLVER, NR><<<n_tiles, dim3(32, W), sm, st>>>(a);
    return cudaGetLastError();
}

template <typename T, int D, int MODE>
cudaError_t launch_pair_m(const PairArgs<T> &a, int solver, int n_tiles, int W, cudaStream_t st) {
    if (solver == 0) return launch_pair_t<T, D, MODE, 0, 1>(a, n_tiles, W, st);
    if (a.g.FR <= 4) return launch_pair_t<T, D, MODE, 1, 4>(a, n_tiles, W, st);
    if (a.g.FR <= 6) return launch_pair_t<T, D, MODE, 1, 6>(a, n_tiles, W, st);
    return launch_pair_t<T, D, MODE, 1, 8>(a, n_tiles, W, st);
}

template <typename T>
cudaError_t launch_pair(const PairArgs<T> &a, int dim, int mode, int solver, int n_tiles, int W, cudaStream_t st) {
    if (dim == 2) return mode == 0 ? launch_pair_m<T, 2, 0>(a, solver, n_tiles, W, st) : launch_pair_m<T, 2, 1>(a, solver, n_tiles, W, st);
    if (dim == 3) return mode == 0 ? launch_pair_m<T, 3, 0>(a, solver, n_tiles, W, st) : launch_pair_m<T, 3, 1>(a, solver, n_tiles, W, st);
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_scale(const ScaleArgs<T> &a, int dim, int n_tiles, int W, cudaStream_t st) {
    if (n_tiles <= 0) return cudaSuccess;
    if (dim == 2) k_scale<T, 2><<<n_tiles, dim3(32, W), 0, st>>>(a);
    else k_scale<T, 3><<<n_tiles, dim3(32, W), 0, st>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cert(const CertArgs<T> &a, int n_tiles, int W, cudaStream_t st) {
    if (n_tiles <= 0) return cudaSuccess;
    const dim3 blk(32, W);
    switch (a.model.kind) {
        case 0: k_cert<T, 0><<<n_tiles, blk, 0, st>>>(a); break;
        case 1: k_cert<T, 1><<<n_tiles, blk, 0, st>>>(a); break;
        case 2: k_cert<T, 2><<<n_tiles, blk, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template cudaError_t launch_pose<float>(const PoseArgs<float> &, int, cudaStream_t);
template cudaError_t launch_pose<double>(const PoseArgs<double> &, int, cudaStream_t);
template cudaError_t launch_pair<float>(const PairArgs<float> &, int, int, int, int, int, cudaStream_t);
template cudaError_t launch_pair<double>(const PairArgs<double> &, int, int, int, int, int, cudaStream_t);
template cudaError_t launch_scale<float>(const ScaleArgs<float> &, int, int, int, cudaStream_t);
template cudaError_t launch_scale<double>(const ScaleArgs<double> &, int, int, int, cudaStream_t);
template cudaError_t launch_cert<float>(const CertArgs<float> &, int, int, cudaStream_t);
template cudaError_t launch_cert<double>(const CertArgs<double> &, int, int, cudaStream_t);

}  // namespace oca
